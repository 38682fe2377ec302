"""BER curves: on an SNR sweep the GPU detectors' uncoded bit error rates
agree with the oracle's on the same frames (the labels differ only at exact
decision ties), and both decrease with SNR; the FP16 path stays within the
95 % interval of the FP32 path."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbp():
    import paper_1702_04458_b300 as m
    return m


@pytest.fixture(scope="module")
def handle(dbp):
    h = dbp.dbp_create(0)
    yield h
    dbp.dbp_destroy(h)


def _wilson(k, n, z=1.96):
    p = k / n
    den = 1 + z * z / n
    c = (p + z * z / (2 * n)) / den
    hw = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return c - hw, c + hw


@pytest.mark.parametrize("algo,T", [("admm", 3), ("cg", 4)])
def test_ber_curve_matches_oracle(dbp, handle, algo, T):
    W, N, B, C, U, M = 60, 14, 64, 4, 8, 16
    bers_gpu, bers_or = [], []
    for i, snr in enumerate([0.0, 4.0, 8.0, 12.0]):
        f = synth.uplink_frame(W, N, B, U, M, snr, seed=3000 + i)
        Hd = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
        yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
        x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
        lab = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
        d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, N0=f["N0"])
        (dbp.dbp_uplink_admm if algo == "admm" else dbp.dbp_uplink_cg)(handle, d, Hd, yd, x, lab)
        torch.cuda.synchronize()
        Hr = f["H"].astype(np.complex64).astype(np.complex128)
        yr = f["y"].astype(np.complex64).astype(np.complex128)
        if algo == "admm":
            xo = oracle.admm_ul(Hr, yr, C=C, rho=1.0, N0=f["N0"], T_max=T)
        else:
            xo = oracle.cg_ul(Hr, yr, C=C, rho=f["N0"], T_max=T)
        nbits = W * N * U * 4
        eg = oracle.bit_errors(lab.cpu().numpy(), f["labels"])
        eo = oracle.bit_errors(oracle.slice_labels(xo, M), f["labels"])
        assert abs(eg - eo) <= max(2, 1e-3 * eo)          # tie decisions only
        lo, hi = _wilson(eo, nbits)
        assert lo <= eg / nbits <= hi
        bers_gpu.append(eg / nbits)
        bers_or.append(eo / nbits)
    assert all(a > b for a, b in zip(bers_gpu, bers_gpu[1:]))


def test_fp16_ber_within_fp32_interval(dbp, handle):
    W, N, B, C, U, M = 200, 14, 256, 8, 32, 64
    f = synth.uplink_frame(W, N, B, U, M, 20.0, seed=3100)
    errs = {}
    for prec, dt in (("fp32", np.complex64), ("fp16", None)):
        if prec == "fp32":
            Hd = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
            yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
            code = dbp.DBP_FP32
        else:
            Hd = torch.from_numpy(np.stack([f["H"].real, f["H"].imag], -1).astype(np.float16)).cuda()
            yd = torch.from_numpy(np.stack([f["y"].real, f["y"].imag], -1).astype(np.float16)).cuda()
            code = dbp.DBP_FP16
        x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
        lab = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
        d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3, N0=f["N0"], precision=code)
        dbp.dbp_uplink_admm(handle, d, Hd, yd, x, lab)
        torch.cuda.synchronize()
        errs[prec] = oracle.bit_errors(lab.cpu().numpy(), f["labels"])
    nbits = W * N * U * 6
    lo, hi = _wilson(errs["fp32"], nbits)
    assert lo <= errs["fp16"] / nbits <= hi, errs


@pytest.mark.parametrize("snr", [10.0, 14.0, 18.0, 22.0])
def test_16bit_ber_within_fp32_interval_over_snr(dbp, handle, snr):
    """B=256, C=8, U=32, 64-QAM on one channel at several SNRs (fresh noise
    each): FP16 and BF16 inputs give BERs inside the FP32 path's 95 %
    interval."""
    W, N, B, C, U, M = 400, 14, 256, 8, 32, 64
    base = synth.uplink_frame(W, N, B, U, M, 20.0, seed=3200)
    f = synth.at_snr(base, snr, seed=3201 + int(snr))
    errs = {}
    for prec in ("fp32", "fp16", "bf16"):
        if prec == "fp32":
            Hd = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
            yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
            code = dbp.DBP_FP32
        else:
            dt = torch.float16 if prec == "fp16" else torch.bfloat16
            Hd = torch.from_numpy(np.stack([f["H"].real, f["H"].imag], -1).astype(np.float32)).to(dt).cuda()
            yd = torch.from_numpy(np.stack([f["y"].real, f["y"].imag], -1).astype(np.float32)).to(dt).cuda()
            code = dbp.DBP_FP16 if prec == "fp16" else dbp.DBP_BF16
        x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
        lab = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
        d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3, N0=f["N0"], precision=code)
        dbp.dbp_uplink_admm(handle, d, Hd, yd, x, lab)
        torch.cuda.synchronize()
        errs[prec] = oracle.bit_errors(lab.cpu().numpy(), f["labels"])
    nbits = W * N * U * 6
    lo, hi = _wilson(errs["fp32"], nbits)
    for prec in ("fp16", "bf16"):
        assert lo <= errs[prec] / nbits <= hi, (snr, errs)
