"""Soft outputs (dbp_uplink_llr) against the oracle: the LMMSE / ZF bias and
noise statistics from the subcarrier's Gram and the max-log LLRs of the
detector's own estimate, on the same FP32 inputs."""
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


LLR_CASES = [
    # (W, N, B, C, U, M, snr_db, reg, detector)
    (37, 14, 128, 8, 8, 16, 8.0, "mmse", "admm"),      # the B=128 / C=8 / U=8 workload
    (21, 14, 128, 8, 8, 16, 8.0, "mmse", "cg"),
    (13, 5, 64, 4, 16, 64, 18.0, "mmse", "cg"),
    (9, 7, 80, 2, 5, 4, 4.0, "zf", "cg"),              # U=5 padded to 8, QPSK, ZF
    (6, 3, 256, 8, 32, 256, 25.0, "mmse", "admm"),     # U=32, 256-QAM
    (11, 6, 36, 4, 3, 4, 6.0, "mmse", "cg"),           # U=3 padded to 4
    (5, 6, 90, 3, 8, 64, 12.0, "mmse", "cg"),          # B=90: the last 4-row k-step reads zero rows
    (7, 4, 300, 4, 8, 16, 10.0, "zf", "admm"),         # B=300: three staged chunks of H
    (3, 14, 512, 8, 16, 4, 5.0, "mmse", "admm"),       # U=16 over several chunks, QPSK
    (4, 5, 150, 3, 32, 16, 15.0, "mmse", "cg"),        # U=32, B=150: a 54-row last chunk, zero rows to 56
    (3, 4, 64, 4, 20, 64, 20.0, "mmse", "admm"),       # U=20 padded to 32 (element-wise staging)
    (5, 6, 96, 4, 32, 4, 6.0, "zf", "admm"),           # U=32, ZF, B exactly one chunk
]


@pytest.mark.parametrize("W,N,B,C,U,M,snr,reg,det", LLR_CASES)
def test_llr_matches_oracle(dbp, handle, W, N, B, C, U, M, snr, reg, det):
    f = synth.uplink_frame(W, N, B, U, M, snr, seed=2100 + W + U + M)
    H32 = f["H"].astype(np.complex64)
    Hd = torch.from_numpy(H32).cuda()
    yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
    code = dbp.DBP_REG_MMSE if reg == "mmse" else dbp.DBP_REG_ZF
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3 if det == "admm" else 8, regularizer=code,
                       N0=f["N0"], Es=1.0)
    x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
    (dbp.dbp_uplink_admm if det == "admm" else dbp.dbp_uplink_cg)(handle, d, Hd, yd, x, None)
    m = int(np.log2(M))
    llr = torch.zeros((W, N, U, m), dtype=torch.float32, device="cuda")
    dbp.dbp_uplink_llr(handle, d, Hd, x, llr)
    torch.cuda.synchronize()
    mu, nu2 = oracle.llr_stats(H32.astype(np.complex128), f["N0"], 1.0,
                               oracle.REG_MMSE if reg == "mmse" else oracle.REG_ZF)
    ref = oracle.llr_maxlog(x.cpu().numpy().astype(np.complex128), mu, nu2, M)
    got = llr.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref) / (1.0 + np.abs(ref))
    assert err.max() <= 1e-3, err.max()
    # hard decisions from the LLRs agree with the oracle's wherever they are not ties
    clear = np.abs(ref) > 1e-2
    assert np.array_equal((got < 0)[clear], (ref < 0)[clear])


def test_llr_rejects_unsupported_requests(dbp, handle):
    buf = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    out = torch.zeros(4096, dtype=torch.float32, device="cuda")
    base = dict(B=32, C=4, U=4, W=3, N=2, qam_order=16, T_max=3, N0=0.1)
    for bad, status in ((dict(qam_order=0), dbp.DBP_ERR_INVALID_ARG),
                        (dict(regularizer=dbp.DBP_REG_BOX, box_r=1.0), dbp.DBP_ERR_INVALID_ARG),
                        (dict(precision=dbp.DBP_FP64), dbp.DBP_ERR_UNSUPPORTED),
                        (dict(N0=0.0), dbp.DBP_ERR_INVALID_ARG),
                        (dict(regularizer=dbp.DBP_REG_ZF, U=8, B=4, C=1), dbp.DBP_ERR_INVALID_ARG)):
        kw = dict(base)
        kw.update(bad)
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_uplink_llr(handle, dbp.frame_desc(**kw), buf, buf, out)
        assert ei.value.status == status


@pytest.mark.parametrize("h_off,l_off", [(1, 0), (0, 1), (0, 2), (1, 3)])
def test_llr_unaligned_buffers(dbp, handle, h_off, l_off):
    """H starting 8 bytes past a 16-byte boundary (element-wise staging) and
    LLR buffers 4 / 8 / 12 bytes past one (scalar and pair stores): the same
    values as the aligned buffers."""
    W, N, B, C, U, M = 9, 7, 128, 8, 8, 16
    f = synth.uplink_frame(W, N, B, U, M, 9.0, seed=2700)
    H32 = torch.from_numpy(f["H"].astype(np.complex64).reshape(-1))
    x = torch.from_numpy((f["s"] * 0.9).astype(np.complex64)).cuda()
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3, N0=f["N0"], Es=1.0)
    n = W * N * U * 4
    ref = torch.zeros(n, dtype=torch.float32, device="cuda")
    dbp.dbp_uplink_llr(handle, d, H32.cuda(), x, ref)
    hb = torch.zeros(H32.numel() + 1, dtype=torch.complex64, device="cuda")
    hb[h_off:h_off + H32.numel()] = H32.cuda()
    lb = torch.full((n + 4,), float("nan"), dtype=torch.float32, device="cuda")
    dbp.dbp_uplink_llr(handle, d, hb[h_off:], x, lb[l_off:l_off + n])
    torch.cuda.synchronize()
    assert torch.allclose(lb[l_off:l_off + n], ref, rtol=1e-5, atol=1e-5)
    assert torch.isnan(lb[:l_off]).all() and torch.isnan(lb[l_off + n:]).all()


def test_llr_full_size_sampled(dbp, handle):
    """B=128, C=8, U=8, 16-QAM, 1200 x 14 at 8 dB (the bench's soft_outputs
    line): LLRs of the whole frame's ADMM estimate; the oracle recomputes the
    statistics and LLRs of 48 sampled subcarriers from the same estimate."""
    W, N, B, C, U, M = 1200, 14, 128, 8, 8, 16
    f = synth.uplink_frame(W, N, B, U, M, 8.0, seed=synth.frame_seed(2, 4))
    H32 = f["H"].astype(np.complex64)
    Hd = torch.from_numpy(H32).cuda()
    yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3, N0=f["N0"], Es=1.0)
    x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
    dbp.dbp_uplink_admm(handle, d, Hd, yd, x, None)
    llr = torch.zeros((W, N, U, 4), dtype=torch.float32, device="cuda")
    dbp.dbp_uplink_llr(handle, d, Hd, x, llr)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(8).choice(W, size=48, replace=False))
    mu, nu2 = oracle.llr_stats(H32[idx].astype(np.complex128), f["N0"], 1.0, oracle.REG_MMSE)
    ref = oracle.llr_maxlog(x.cpu().numpy()[idx].astype(np.complex128), mu, nu2, M)
    got = llr.cpu().numpy()[idx].astype(np.float64)
    assert (np.abs(got - ref) / (1.0 + np.abs(ref))).max() <= 1e-3
    assert np.isfinite(llr.cpu().numpy()).all()


def test_llr_full_size_u32_sampled(dbp, handle):
    """B=256, C=8, U=32, 64-QAM, 3300 x 14 at 20 dB (the bench's
    mixed_vs_fp32.soft_outputs line): LLRs of the whole frame's FP32 ADMM
    estimate; the oracle recomputes 16 sampled subcarriers."""
    W, N, B, C, U, M = 3300, 14, 256, 8, 32, 64
    f = synth.uplink_frame(W, N, B, U, M, 20.0, seed=synth.frame_seed(4, 5))
    H32 = f["H"].astype(np.complex64)
    Hd = torch.from_numpy(H32).cuda()
    yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3, N0=f["N0"], Es=1.0)
    x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
    dbp.dbp_uplink_admm(handle, d, Hd, yd, x, None)
    llr = torch.zeros((W, N, U, 6), dtype=torch.float32, device="cuda")
    dbp.dbp_uplink_llr(handle, d, Hd, x, llr)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(9).choice(W, size=16, replace=False))
    mu, nu2 = oracle.llr_stats(H32[idx].astype(np.complex128), f["N0"], 1.0, oracle.REG_MMSE)
    ref = oracle.llr_maxlog(x.cpu().numpy()[idx].astype(np.complex128), mu, nu2, M)
    got = llr.cpu().numpy()[idx].astype(np.float64)
    assert (np.abs(got - ref) / (1.0 + np.abs(ref))).max() <= 1e-3
    assert np.isfinite(llr.cpu().numpy()).all()
