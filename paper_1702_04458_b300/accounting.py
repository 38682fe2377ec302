"""Algorithmic bytes and operation counts per subcarrier (the roofline units).

Operation counts are real-valued multiplications in the accounting of Table I
(one multiply-add counts as two flops, so flops = 2 x multiplications), for
the formulation each kernel executes:

* ADMM uplink, U x U form (Alg. 1 with the E1 closed form and B_c^{-1}):
  Table I's ADMM-UL U x U row, with the symbol-independent preprocessing
  (Gram 2SU^2, inverse 10/3 U^3 - U/3) counted once per subcarrier and the
  symbol-dependent terms (matched filter 4SU, regularised estimate 4U^2,
  init 2U, C(4U^2 + 4U) + 2U per later iteration) once per symbol.
* CG uplink with the precomputed Gram G_c = H_c^H H_c (the option of the
  footnote to Alg. 2): Gram 2SU^2 per cluster and subcarrier; per symbol the
  MRC 4SU per cluster, and per iteration Table I's C(8SU + 10U) + 2U with the
  two mat-vecs 8SU replaced by the Gram product 4U^2.
* ADMM downlink, U x U form with the precomputed iteration operator
  Q_c = I - rho^{-1} B_c^{-1} (m_c = H_c x_c = Q_c (z_c + lambda_c)): Gram and
  inverse as Table I's ADMM-DL U x U preprocessing, per later iteration
  C(4U^2 + 6U) + 4U (mat-vec, consensus update, dual update), and per symbol
  the output x_c = H_c^H B_c^{-1}(z_c + lambda_c), C(4U^2 + 4SU).

Bytes are what must cross HBM at least once: the channel H (once per
subcarrier, shared by its N symbols), the receive or transmit vectors, and
the outputs (equaliser outputs + one label byte per entry in the uplink; the
beamforming vectors in the downlink).
"""
from __future__ import annotations

from dataclasses import dataclass

__all__ = ["Workload", "table1_ar", "algorithmic_mults", "algorithmic_bytes",
           "detected_bits", "fp32_simt_peak_tflops"]


@dataclass(frozen=True)
class Workload:
    B: int
    C: int
    U: int
    W: int
    N: int
    M: int
    T: int
    elem_bytes: int = 8          # complex64

    @property
    def S(self) -> int:
        return self.B // self.C


def table1_ar(alg: str, mode: str, C: int, S: int, U: int) -> dict:
    """Table I, arithmetic (AR) complexity, real multiplications for one
    subcarrier and one symbol: preprocessing, first iteration, each later
    iteration."""
    c, s, u = float(C), float(S), float(U)
    if alg == "admm_dl":
        d, o = (s, u) if mode == "SxS" else (u, s)
        return {"pre": c * (2 * o * d * d + 10.0 / 3.0 * d ** 3 - d / 3.0),
                "first": c * (4 * s * u + 4 * d * d),
                "sub": c * (8 * s * u + 4 * d * d + 2 * u) + 4 * u + 1}
    if alg == "admm_ul":
        if mode == "SxS":
            return {"pre": c * (2 * u * s * s + 10.0 / 3.0 * s ** 3 + 4 * u * s + 4 * s * s - s / 3.0),
                    "first": 2 * u,
                    "sub": c * (8 * s * u + 4 * s * s + 2 * u) + 2 * u}
        return {"pre": c * (2 * s * u * u + 10.0 / 3.0 * u ** 3 + 4 * s * u + 4 * u * u - u / 3.0),
                "first": 2 * u,
                "sub": c * (4 * u * u + 4 * u) + 2 * u}
    if alg == "cg_ul":
        return {"pre": 4 * c * s * u + 2 * u,
                "first": c * (8 * s * u + 4 * u) + 2 * u,
                "sub": c * (8 * s * u + 10 * u) + 2 * u}
    raise ValueError(alg)


def algorithmic_mults(alg: str, wl: Workload) -> float:
    """Real multiplications per subcarrier (all N symbols) for the kernel's
    formulation (see the module docstring)."""
    C, S, U, N, T = wl.C, wl.S, wl.U, wl.N, wl.T
    if alg == "admm_ul":
        per_sc = C * (2 * S * U * U + 10.0 / 3.0 * U ** 3 - U / 3.0)
        per_sym = C * (4 * S * U + 4 * U * U) + 2 * U + (T - 1) * (C * (4 * U * U + 4 * U) + 2 * U)
        return per_sc + N * per_sym
    if alg == "cg_ul":
        per_sc = C * 2 * S * U * U
        per_sym = C * 4 * S * U + 2 * U + T * (C * (4 * U * U + 10 * U) + 2 * U)
        return per_sc + N * per_sym
    if alg == "admm_dl":
        per_sc = C * (2 * S * U * U + 10.0 / 3.0 * U ** 3 - U / 3.0)
        per_sym = (T - 1) * (C * (4 * U * U + 6 * U) + 4 * U) + C * (4 * U * U + 4 * S * U)
        return per_sc + N * per_sym
    raise ValueError(alg)


def algorithmic_bytes(alg: str, wl: Workload) -> float:
    """Minimum HBM bytes per subcarrier."""
    e = wl.elem_bytes                     # input element (complex64, or 2 x 16 bit)
    H = wl.B * wl.U * e
    if alg in ("admm_ul", "cg_ul"):
        return H + wl.N * wl.B * e + wl.N * wl.U * (8 + 1)   # x_hat complex64 + label
    if alg == "admm_dl":
        return H + wl.N * wl.U * e + wl.N * wl.B * 8
    raise ValueError(alg)


def detected_bits(wl: Workload) -> float:
    """Bits carried by one frame: U log2(M) per user, subcarrier and symbol."""
    m = wl.M.bit_length() - 1
    return float(wl.U * m * wl.W * wl.N)


def fp32_simt_peak_tflops(sms: int = 148, clock_mhz: float = 2032.0) -> float:
    """FP32 CUDA-core peak: 128 FMA lanes per SM, 2 flops per FMA."""
    return sms * 128 * 2 * clock_mhz * 1e6 / 1e12
