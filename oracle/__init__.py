"""FP64 CPU oracle for decentralized baseband processing.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  It shares
no code with the CUDA path (``paper_1702_04458_b300``) and is never used as a
fallback for it.

The numerical core is ``oracle.c`` (plain C99 ``double complex``), which
follows Alg. 1 (decentralized ADMM detection), Alg. 2 (decentralized CG
detection) and Alg. 3 (decentralized ADMM beamforming) step by step, plus
the centralized MMSE/ZF equaliser (Sec. III-A) and ZF beamformer (Sec. IV-A).
This module adds the detection stage (hard slicing to the QAM alphabet, Sec.
III-A), max-log soft outputs (LLRs) of the linear estimate, bit-error counting
and an exhaustive maximum-likelihood search for tiny problems.

Parity status: every routine here is pinned by ``tests/test_oracle_pins.py``
(closed forms, library routines, brute force, invariants); none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB32 = os.path.join(_HERE, "liboracle32.so")

REG_ZF, REG_MMSE, REG_BOX, REG_BPSK = 0, 1, 2, 3
MODE_AUTO, MODE_UXU, MODE_SXS = 0, 1, 2

_ERRORS = {-1: "bad argument", -2: "singular matrix", -3: "out of memory"}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP over subcarriers), and
    the same source with ORACLE_REAL=float into liboracle32.so (the plain
    FP32 CPU program the benchmark times beside the oracle; never a
    reference)."""
    for lib, extra in ((_LIB, []), (_LIB32, ["-DORACLE_REAL=float"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp"] + extra + ["-o", lib, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
    return _LIB


_lib = None
_lib32 = None


def _load32():
    """The FP32 build: only Alg. 1 is bound (the CPU baseline's detector)."""
    global _lib32
    if _lib32 is None:
        build()
        lib = ctypes.CDLL(_LIB32)
        P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        lib.oracle_admm_ul.argtypes = [I, I, I, I, I, P, P, F, F, F, F, I, I, F, I, P]
        lib.oracle_admm_ul.restype = I
        _lib32 = lib
    return _lib32


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_admm_ul.argtypes = [I, I, I, I, I, P, P, D, D, D, D, I, I, D, I, P]
        lib.oracle_cg_ul.argtypes = [I, I, I, I, I, P, P, D, I, P]
        lib.oracle_admm_dl.argtypes = [I, I, I, I, I, P, P, D, D, D, I, I, P]
        lib.oracle_lmmse_ul.argtypes = [I, I, I, I, P, P, D, P]
        lib.oracle_zf_dl.argtypes = [I, I, I, I, P, P, P]
        for f in (lib.oracle_admm_ul, lib.oracle_cg_ul, lib.oracle_admm_dl,
                  lib.oracle_lmmse_ul, lib.oracle_zf_dl):
            f.restype = I
        _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.complex128)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what}: {_ERRORS.get(rc, rc)}")


def _shape_ul(H, y):
    W, B, U = H.shape
    if y.ndim != 3 or y.shape[0] != W or y.shape[2] != B:
        raise ValueError("y must be [W][N][B] matching H [W][B][U]")
    return W, y.shape[1], B, U


# ---------------------------------------------------------------------------
# Algorithms (C core)
# ---------------------------------------------------------------------------

def admm_ul(H, y, C: int, rho: float, N0: float, Es: float = 1.0, T_max: int = 3,
            gamma: float = 1.0, reg: int = REG_MMSE, box_r: float = 1.0,
            mode: int = MODE_AUTO) -> np.ndarray:
    """Alg. 1 (decentralized ADMM detection); returns s^(T_max), [W][N][U]."""
    H, y = _c128(H), _c128(y)
    W, N, B, U = _shape_ul(H, y)
    out = np.zeros((W, N, U), dtype=np.complex128)
    rc = _load().oracle_admm_ul(W, N, B, C, U, H.ctypes.data, y.ctypes.data,
                                rho, gamma, N0, Es, T_max, reg, box_r, mode,
                                out.ctypes.data)
    _check(rc, "admm_ul")
    return out


def admm_ul_fp32(H, y, C: int, rho: float, N0: float, Es: float = 1.0, T_max: int = 3,
                 gamma: float = 1.0, reg: int = REG_MMSE, box_r: float = 1.0,
                 mode: int = MODE_AUTO) -> np.ndarray:
    """Alg. 1 from the same source built in FP32 (complex64 in and out).  A
    timed CPU program for the benchmark's plain-CPU line, not a reference:
    parity is always checked against the FP64 build (admm_ul)."""
    H = np.ascontiguousarray(np.asarray(H), dtype=np.complex64)
    y = np.ascontiguousarray(np.asarray(y), dtype=np.complex64)
    W, N, B, U = _shape_ul(H, y)
    out = np.zeros((W, N, U), dtype=np.complex64)
    rc = _load32().oracle_admm_ul(W, N, B, C, U, H.ctypes.data, y.ctypes.data,
                                  rho, gamma, N0, Es, T_max, reg, box_r, mode,
                                  out.ctypes.data)
    _check(rc, "admm_ul (FP32 build)")
    return out


def cg_ul(H, y, C: int, rho: float, T_max: int) -> np.ndarray:
    """Alg. 2 (decentralized CG detection); rho = N0/Es (MMSE) or 0 (ZF)."""
    H, y = _c128(H), _c128(y)
    W, N, B, U = _shape_ul(H, y)
    out = np.zeros((W, N, U), dtype=np.complex128)
    rc = _load().oracle_cg_ul(W, N, B, C, U, H.ctypes.data, y.ctypes.data,
                              rho, T_max, out.ctypes.data)
    _check(rc, "cg_ul")
    return out


def admm_dl(H, s, C: int, rho: float = 1.0, T_max: int = 3, gamma: float = 1.0,
            eps: float = 0.0, mode: int = MODE_AUTO) -> np.ndarray:
    """Alg. 3 (decentralized ADMM beamforming, Lemma 2 with eps); [W][N][B].

    H is the uplink-layout channel [W][B][U]; the downlink matrix is H^T.
    """
    H, s = _c128(H), _c128(s)
    W, B, U = H.shape
    if s.ndim != 3 or s.shape[0] != W or s.shape[2] != U:
        raise ValueError("s must be [W][N][U]")
    N = s.shape[1]
    out = np.zeros((W, N, B), dtype=np.complex128)
    rc = _load().oracle_admm_dl(W, N, B, C, U, H.ctypes.data, s.ctypes.data,
                                rho, gamma, eps, T_max, mode, out.ctypes.data)
    _check(rc, "admm_dl")
    return out


def lmmse_ul(H, y, delta: float) -> np.ndarray:
    """Centralized equaliser (H^H H + delta I)^{-1} H^H y (delta = N0/Es or 0)."""
    H, y = _c128(H), _c128(y)
    W, N, B, U = _shape_ul(H, y)
    out = np.zeros((W, N, U), dtype=np.complex128)
    _check(_load().oracle_lmmse_ul(W, N, B, U, H.ctypes.data, y.ctypes.data,
                                   delta, out.ctypes.data), "lmmse_ul")
    return out


def zf_dl(H, s) -> np.ndarray:
    """Centralized ZF beamformer H^H (H H^H)^{-1} s with downlink H = (H^u)^T."""
    H, s = _c128(H), _c128(s)
    W, B, U = H.shape
    N = s.shape[1]
    out = np.zeros((W, N, B), dtype=np.complex128)
    _check(_load().oracle_zf_dl(W, N, B, U, H.ctypes.data, s.ctypes.data,
                                out.ctypes.data), "zf_dl")
    return out


# ---------------------------------------------------------------------------
# Detection stage (Sec. III-A): hard slicing, bits, errors
# ---------------------------------------------------------------------------

def _levels(M: int):
    L = int(round(math.sqrt(M)))
    if L * L != M or M < 4 or (M & (M - 1)):
        raise ValueError(f"unsupported QAM order {M}")
    return L, int(round(math.log2(M))) // 2


def _axis(M: int):
    """Per-axis PAM levels L, bits per axis and half-spacing a of the
    unit-energy alphabet.  M = 2 is BPSK {-1, +1}: two levels on the real
    axis only (no imaginary axis), a = 1."""
    if M == 2:
        return 2, 1, 1.0
    L, half = _levels(M)
    return L, half, math.sqrt(3.0 / (2.0 * (M - 1)))


def box_radius(M: int) -> float:
    """Radius r of the box covering the unit-energy square QAM alphabet
    (M = 2: the real segment [-1, 1] covering BPSK)."""
    L, _, a = _axis(M)
    return (L - 1) * a


def slice_labels(x, M: int, dtype=np.float64) -> np.ndarray:
    """Nearest-point hard decision per entry, returned as the Gray bit label.

    Per axis the PAM index is k = ceil(t - 1/2) clamped to [0, L-1] with
    t = (a * x + (L - 1)) / 2 and a = 1 / sqrt(3 / (2 (M - 1))): values
    beyond the outer points go to the outer points and an exact decision
    boundary goes to the lower level.  The label is (g(kI) << m/2) | g(kQ)
    with g the binary-reflected Gray code.  ``dtype`` is the precision in
    which the decision is taken (float32 to mirror a float32 kernel: the
    products and sums are rounded to float32 one operation at a time).
    """
    L, half, a = _axis(M)
    x = np.asarray(x)
    ft = np.dtype(dtype).type
    inv_a = ft(1.0 / a)
    off = ft(L - 1)

    def axis(v):
        v = np.asarray(v, dtype=dtype)
        t = (v * inv_a + off) * ft(0.5)
        k = np.ceil(t - ft(0.5))
        k = np.clip(k, 0, L - 1).astype(np.int64)
        return k ^ (k >> 1)

    gi = axis(x.real)
    if M == 2:   # BPSK: the real axis is the whole label
        return gi.astype(np.uint8)
    gq = axis(x.imag)
    return ((gi << half) | gq).astype(np.uint8)


def label_points(labels, M: int) -> np.ndarray:
    """Alphabet point of each Gray label (the slicer's own decoding)."""
    L, half, a = _axis(M)
    lab = np.asarray(labels, dtype=np.int64)
    if M == 2:   # BPSK: label k is the real point 2k - 1
        return (2.0 * lab - 1.0) + 0j

    def ungray(g):
        k = g.copy()
        shift = g >> 1
        while np.any(shift):
            k ^= shift
            shift >>= 1
        return k

    kI = ungray(lab >> half)
    kQ = ungray(lab & ((1 << half) - 1))
    return (2 * kI - (L - 1)) * a + 1j * (2 * kQ - (L - 1)) * a


def llr_stats(H, N0: float, Es: float = 1.0, reg: int = REG_MMSE):
    """Per-user bias mu and effective noise variance nu^2 of the linear
    estimate x = A H^H y with A = (G + delta I)^{-1}, G = H^H H, so that
    x_u = mu_u s_u + e_u with E|e_u|^2 = nu_u^2 (soft outputs, Sec. III-A):

      MMSE (delta = N0 / Es):  mu_u = 1 - delta A_uu,  nu_u^2 = Es mu_u (1 - mu_u)
      ZF   (delta = 0):        mu_u = 1,               nu_u^2 = N0 A_uu

    H is [W][B][U]; returns (mu, nu2), each [W][U] float64.  The inverse is a
    library routine (numpy.linalg.inv)."""
    H = _c128(H)
    W, B, U = H.shape
    G = np.einsum("wbu,wbv->wuv", H.conj(), H)
    if reg == REG_MMSE:
        delta = N0 / Es
    elif reg == REG_ZF:
        delta = 0.0
    else:
        raise ValueError("soft outputs are defined for the ZF and MMSE estimates")
    A = np.linalg.inv(G + delta * np.eye(U))
    Ad = np.real(np.diagonal(A, axis1=1, axis2=2))
    if reg == REG_MMSE:
        mu = 1.0 - delta * Ad
        nu2 = Es * mu * (1.0 - mu)
    else:
        mu = np.ones_like(Ad)
        nu2 = N0 * Ad
    return mu, nu2


def llr_maxlog(x, mu, nu2, M: int, Es: float = 1.0) -> np.ndarray:
    """Max-log LLR of every label bit, most significant bit first, positive
    when the bit is more likely 0:

      L_j = (min_{s: bit_j(s) = 1} |x - mu s|^2 - min_{s: bit_j(s) = 0} |x - mu s|^2) / nu^2

    by exhaustive search over the M alphabet points (scaled to energy Es).
    x is [W][N][U], mu and nu2 are [W][U]; returns [W][N][U][log2 M]."""
    x = _c128(x)
    m = int(round(math.log2(M)))
    pts = label_points(np.arange(M), M) * math.sqrt(Es)
    mu = np.asarray(mu, dtype=np.float64)[:, None, :, None]
    nu2 = np.asarray(nu2, dtype=np.float64)[:, None, :, None]
    d2 = np.abs(x[..., None] - mu * pts) ** 2                      # [W][N][U][M]
    out = np.empty(x.shape + (m,), dtype=np.float64)
    labels = np.arange(M)
    for j in range(m):
        bit = (labels >> (m - 1 - j)) & 1
        out[..., j] = (d2[..., bit == 1].min(axis=-1) - d2[..., bit == 0].min(axis=-1)) / nu2[..., 0]
    return out


def bit_errors(labels_a, labels_b) -> int:
    """Number of differing bits between two label arrays."""
    x = np.bitwise_xor(np.asarray(labels_a, dtype=np.uint8),
                       np.asarray(labels_b, dtype=np.uint8))
    return int(np.unpackbits(x.reshape(-1, 1), axis=1).sum())


def ml_detect(H, y, M: int) -> np.ndarray:
    """Exhaustive ML search argmin_{s in O^U} ||y - H s||^2 (tiny cases only).

    H is [B][U], y is [B]; returns the labels of the minimiser.
    """
    H, y = _c128(H), _c128(y)
    B, U = H.shape
    if M ** U > 1 << 20:
        raise ValueError("ML search too large")
    pts = label_points(np.arange(M), M)
    best, best_lab = np.inf, None
    for lab in itertools.product(range(M), repeat=U):
        s = pts[list(lab)]
        r = y - H @ s
        d = float(np.vdot(r, r).real)
        if d < best:
            best, best_lab = d, lab
    return np.array(best_lab, dtype=np.uint8)
