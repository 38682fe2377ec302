"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws inputs; it holds none of the detection or precoding
arithmetic.  It implements the transmitter side of the system model of
Sec. II-A (uplink, y = H s + n) and Sec. II-B (downlink, known s, H^d = H^T):

* channel  H[w] in C^{B x U}, i.i.d. circularly-symmetric CN(0, 1) entries,
  fixed over the N OFDM symbols of one subcarrier (the channel is static over
  the symbols of a coherence block, Sec. VI-A);
* symbols  s in O^U drawn uniformly from a Gray-labelled square QAM alphabet
  O with E_s = E[|s_u|^2] = 1 (Sec. II-A, Gray mapping);
* noise    n ~ CN(0, N0) i.i.d., with N0 = U * E_s / SNR: the SNR is the
  average receive SNR per BS antenna for unit-variance channel entries.

Memory layouts (row-major, complex interleaved re/im):
    H  [W][B][U]   cluster c owns rows c*S .. c*S+S-1 (Sec. II-A.2)
    y  [W][N][B]
    s  [W][N][U]   and the integer labels of s, same shape (uint8)

Label convention (shared format, each side implements it itself): for
M = L*L points and m = log2(M) bits, label = (g(kI) << m/2) | g(kQ) with
g(k) = k ^ (k >> 1) the binary-reflected Gray code of the PAM level index
k in [0, L); the level index k maps to the amplitude (2k - (L-1)) * a with
a = sqrt(3 / (2 (M - 1))), so that E_s = 1.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "qam_alphabet",
    "noise_variance",
    "uplink_frame",
    "downlink_frame",
    "frame_seed",
]


def _gray(k: int) -> int:
    return k ^ (k >> 1)


def qam_alphabet(M: int) -> np.ndarray:
    """Transmit alphabet: point of each label 0..M-1 (complex128, E_s = 1).
    M = 2 is BPSK: label k is the real point 2k - 1."""
    if M == 2:
        return np.array([-1.0 + 0j, 1.0 + 0j])
    L = int(round(math.sqrt(M)))
    if L * L != M or M < 4 or (M & (M - 1)) != 0:
        raise ValueError(f"alphabet order must be 2 (BPSK) or a square QAM order 4, 16, 64, 256: got {M}")
    half = int(round(math.log2(M))) // 2
    a = math.sqrt(3.0 / (2.0 * (M - 1)))
    pts = np.zeros(M, dtype=np.complex128)
    for kI in range(L):
        for kQ in range(L):
            label = (_gray(kI) << half) | _gray(kQ)
            pts[label] = complex((2 * kI - (L - 1)) * a, (2 * kQ - (L - 1)) * a)
    return pts


def noise_variance(snr_db: float, U: int, Es: float = 1.0) -> float:
    """N0 for an average per-antenna receive SNR of snr_db (CN(0,1) channel)."""
    return U * Es / (10.0 ** (snr_db / 10.0))


def frame_seed(config_index: int, snr_index: int = 0) -> int:
    """Seed recipe: configuration k at SNR point i draws from seed 1000*k + i."""
    return 1000 * config_index + snr_index


def _cn(rng: np.random.Generator, shape, var: float) -> np.ndarray:
    sd = math.sqrt(var / 2.0)
    return rng.normal(0.0, sd, size=shape) + 1j * rng.normal(0.0, sd, size=shape)


def uplink_frame(W: int, N: int, B: int, U: int, M: int, snr_db: float,
                 seed: int, Es: float = 1.0, noiseless: bool = False) -> dict:
    """One uplink frame: H, y = H s + n, transmitted labels and symbols.

    Everything is returned in complex128 / uint8; callers round to the
    precision they compute in and hand the rounded values to both sides.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    H = _cn(rng, (W, B, U), 1.0)
    labels = rng.integers(0, M, size=(W, N, U), dtype=np.int64).astype(np.uint8)
    s = qam_alphabet(M)[labels] * math.sqrt(Es)
    N0 = noise_variance(snr_db, U, Es)
    noise = _cn(rng, (W, N, B), N0)
    if noiseless:
        noise[...] = 0.0
    # y[w, n, :] = H[w] @ s[w, n, :] + n[w, n, :]
    y = np.einsum("wbu,wnu->wnb", H, s) + noise
    return {"H": H, "y": y, "labels": labels, "s": s, "N0": N0, "Es": Es,
            "W": W, "N": N, "B": B, "U": U, "M": M, "snr_db": snr_db}


def at_snr(f: dict, snr_db: float, seed: int) -> dict:
    """The same uplink frame (channel and transmitted symbols) at another
    SNR: y = H s + n with fresh seeded noise of the variance snr_db gives."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N0 = noise_variance(snr_db, f["U"], f["Es"])
    clean = np.matmul(f["H"], np.swapaxes(f["s"], 1, 2)).swapaxes(1, 2)   # [W][N][B]
    out = dict(f)
    out["y"] = clean + _cn(rng, clean.shape, N0)
    out["N0"] = N0
    out["snr_db"] = snr_db
    return out


def downlink_frame(W: int, N: int, B: int, U: int, M: int, seed: int,
                   Es: float = 1.0) -> dict:
    """One downlink frame: uplink-layout channel H (H^d = H^T) and symbols s."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H = _cn(rng, (W, B, U), 1.0)
    labels = rng.integers(0, M, size=(W, N, U), dtype=np.int64).astype(np.uint8)
    s = qam_alphabet(M)[labels] * math.sqrt(Es)
    return {"H": H, "s": s, "labels": labels, "Es": Es,
            "W": W, "N": N, "B": B, "U": U, "M": M}
