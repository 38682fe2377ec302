"""Degenerate inputs on the default kernels (the tcgen05 uplink at U = S = 32,
the downlink tensor-core kernel at U = 16): a symbol whose receive (or
transmit) vector is zero, a whole subcarrier of zeros, and a cluster whose
channel is zero on one subcarrier.

A zero block has no largest magnitude, so the operands' power-of-two scale
falls back to 2^0, and a zero channel leaves B_c = rho I (Alg. 1) or
rho^-1 I (Alg. 3), whose inverse is exact.  The estimates of zero inputs are
exactly zero (every product, consensus and prox of zeros is zero), and every
other vector meets the FP32 tolerance against the FP64 oracle on the same
rounded inputs."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


@pytest.fixture(scope="module")
def dbp():
    import paper_1702_04458_b300 as m
    return m


@pytest.fixture(scope="module")
def handle(dbp):
    h = dbp.dbp_create(0)
    yield h
    torch.cuda.synchronize()
    dbp.dbp_destroy(h)


def _check(x, ref, zero):
    """zero: boolean mask over (subcarrier, symbol) of vectors that must be 0."""
    assert np.all(np.isfinite(x))
    assert np.all(x[zero] == 0)
    keep = ~zero
    err = np.linalg.norm(x[keep] - ref[keep], axis=-1) / np.linalg.norm(ref[keep], axis=-1)
    assert err.max() <= FP32_TOL, err.max()


def _to16(a):
    return torch.from_numpy(np.stack([a.real, a.imag], -1).astype(np.float32)).half().cuda()


def _deq(t):
    a = t.float().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_tc5_zero_symbols_subcarrier_and_cluster(dbp, handle, prec):
    W, N, B, C, U, M = 7, 14, 256, 8, 32, 64
    f = synth.uplink_frame(W, N, B, U, M, 20.0, seed=9990)
    H, y = f["H"].copy(), f["y"].copy()
    y[2, 5] = 0.0                       # one symbol
    y[4] = 0.0                          # a whole subcarrier
    H[3, 32:64, :] = 0.0                # cluster 1's channel on subcarrier 3
    y[3, :, 32:64] = 0.0                # ... and what its antennas receive
    if prec == "fp32":
        Hd = torch.from_numpy(H.astype(np.complex64)).cuda()
        yd = torch.from_numpy(y.astype(np.complex64)).cuda()
        Hq = H.astype(np.complex64).astype(np.complex128)
        yq = y.astype(np.complex64).astype(np.complex128)
        code = dbp.DBP_FP32
    else:
        Hd, yd = _to16(H), _to16(y)
        Hq, yq = _deq(Hd), _deq(yd)
        code = dbp.DBP_FP16
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3, precision=code, N0=f["N0"])
    x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
    lab = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
    dbp.dbp_uplink_admm(handle, d, Hd, yd, x, lab)
    torch.cuda.synchronize()
    assert dbp.dbp_plan(handle, dbp.DBP_KIND_UPLINK_ADMM, d, Hd, yd, x).kernel == dbp.DBP_PATH_TC5
    ref = oracle.admm_ul(Hq, yq, C=C, rho=1.0, N0=f["N0"], Es=1.0, T_max=3)
    zero = np.zeros((W, N), dtype=bool)
    zero[2, 5] = True
    zero[4] = True
    _check(x.cpu().numpy().astype(np.complex128), ref, zero)


def test_downlink_zero_symbols_subcarrier_and_cluster(dbp, handle):
    W, N, B, C, U = 7, 14, 256, 16, 16
    f = synth.downlink_frame(W, N, B, U, 64, seed=9991)
    H, s = f["H"].copy(), f["s"].copy()
    s[2, 5] = 0.0
    s[4] = 0.0
    H[3, 16:32, :] = 0.0                # cluster 1's channel on subcarrier 3
    Hd = torch.from_numpy(H.astype(np.complex64)).cuda()
    sd = torch.from_numpy(s.astype(np.complex64)).cuda()
    d = dbp.frame_desc(B, C, U, W, N, T_max=5, rho=1.0)
    x = torch.zeros((W, N, B), dtype=torch.complex64, device="cuda")
    dbp.dbp_downlink_admm(handle, d, Hd, sd, x, None)
    torch.cuda.synchronize()
    ref = oracle.admm_dl(H.astype(np.complex64).astype(np.complex128), s.astype(np.complex64).astype(np.complex128),
                         C=C, rho=1.0, T_max=5)
    zero = np.zeros((W, N), dtype=bool)
    zero[2, 5] = True
    zero[4] = True
    xg = x.cpu().numpy().astype(np.complex128)
    _check(xg, ref, zero)
    # a cluster with no channel transmits nothing on that subcarrier
    assert np.all(xg[3, :, 16:32] == 0)
