"""Channel gain.  A frame whose channel is scaled by g, with the penalty (and
N0) scaled to match, is the unit-gain problem in other units: B_c = g^2
(G_c + rho I) in the uplink (rho -> g^2 rho, N0 -> g^2 N0, y -> g y) and
g^2 (H^d_c H^dH_c + rho^-1 I) in the downlink (rho -> rho / g^2).  The
uplink estimates and the soft outputs are unchanged and the downlink
precoder scales by 1 / g, so every kernel path must meet the FP32
tolerance against the oracle on the scaled frame itself.

This pins the Gauss-Jordan eliminations at large and small pivots: a pivot
row updated as A - (1 - 1/p) A, which equals A / p only in exact
arithmetic, kept about 2^-24 |p| of the row's relative accuracy (relative
errors 1e-2 to 0.3 at g = 30 to 1000 in the U = 16 downlink)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
GAINS = [1e3, 3e-3]


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


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), 1e-300)


def _paths(dbp, names):
    table = {"auto": dbp.DBP_PATH_AUTO, "tma": dbp.DBP_PATH_TMA, "generic": dbp.DBP_PATH_GENERIC,
             "bcast": dbp.DBP_PATH_BCAST, "mma": dbp.DBP_PATH_MMA, "tc5": dbp.DBP_PATH_TC5}
    return [(n, table[n]) for n in names]


UL_CASES = [
    # (W, N, B, C, U, M, algo, paths)
    (9, 14, 128, 8, 8, 16, "admm", ("auto", "bcast", "tma", "generic")),   # U = 8: tensor-core kernel under AUTO
    (7, 14, 256, 16, 16, 16, "admm", ("auto", "tma", "generic")),          # U = 16: broadcast kernel under AUTO
    (5, 14, 256, 8, 32, 64, "admm", ("auto", "tma")),                      # U = 32: tcgen05 kernel under AUTO
    (9, 14, 128, 8, 8, 16, "cg", ("auto", "bcast", "tma")),
]


@pytest.mark.parametrize("g", GAINS)
@pytest.mark.parametrize("W,N,B,C,U,M,algo,paths", UL_CASES)
def test_uplink_at_any_channel_gain(dbp, handle, g, W, N, B, C, U, M, algo, paths):
    f = synth.uplink_frame(W, N, B, U, M, 15.0, seed=9700 + U + B)
    H = (f["H"] * g).astype(np.complex64)
    y = (f["y"] * g).astype(np.complex64)
    N0, rho = f["N0"] * g * g, g * g
    Hq, yq = H.astype(np.complex128), y.astype(np.complex128)
    if algo == "admm":
        ref = oracle.admm_ul(Hq, yq, C=C, rho=rho, N0=N0, Es=1.0, T_max=3)
    else:
        ref = oracle.cg_ul(Hq, yq, C=C, rho=N0, T_max=6)
    fn = dbp.dbp_uplink_admm if algo == "admm" else dbp.dbp_uplink_cg
    for name, path in _paths(dbp, paths):
        dbp.dbp_set_tuning(handle, kernel=path)
        try:
            d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3 if algo == "admm" else 6, rho=rho, N0=N0, Es=1.0)
            x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
            fn(handle, d, torch.from_numpy(H).cuda(), torch.from_numpy(y).cuda(), x, None)
            torch.cuda.synchronize()
        finally:
            dbp.dbp_set_tuning(handle)
        err = _rel(x.cpu().numpy().astype(np.complex128), ref).max()
        assert err <= FP32_TOL, (name, err)


DL_CASES = [
    # (W, N, B, C, U, paths)
    (9, 14, 256, 16, 16, ("auto", "tma", "generic")),   # U = 16: downlink tensor-core kernel under AUTO
    (9, 14, 128, 8, 8, ("auto", "tma", "generic")),
]


@pytest.mark.parametrize("g", GAINS)
@pytest.mark.parametrize("W,N,B,C,U,paths", DL_CASES)
def test_downlink_at_any_channel_gain(dbp, handle, g, W, N, B, C, U, paths):
    f = synth.downlink_frame(W, N, B, U, 64, seed=9800 + U)
    H = (f["H"] * g).astype(np.complex64)
    s = f["s"].astype(np.complex64)
    rho = 1.0 / (g * g)
    ref = oracle.admm_dl(H.astype(np.complex128), s.astype(np.complex128), C=C, rho=rho, T_max=5)
    for name, path in _paths(dbp, paths):
        dbp.dbp_set_tuning(handle, kernel=path)
        try:
            d = dbp.frame_desc(B, C, U, W, N, T_max=5, rho=rho)
            x = torch.zeros((W, N, B), dtype=torch.complex64, device="cuda")
            dbp.dbp_downlink_admm(handle, d, torch.from_numpy(H).cuda(), torch.from_numpy(s).cuda(), x, None)
            torch.cuda.synchronize()
        finally:
            dbp.dbp_set_tuning(handle)
        err = _rel(x.cpu().numpy().astype(np.complex128), ref).max()
        assert err <= FP32_TOL, (name, err)


@pytest.mark.parametrize("g", GAINS)
@pytest.mark.parametrize("B,C,U,M", [(128, 8, 8, 16), (256, 16, 16, 16), (256, 8, 32, 64)])
def test_soft_outputs_at_any_channel_gain(dbp, handle, g, B, C, U, M):
    W, N = 7, 6
    f = synth.uplink_frame(W, N, B, U, M, 15.0, seed=9900 + U)
    H = (f["H"] * g).astype(np.complex64)
    N0 = f["N0"] * g * g
    # the unit-gain estimate (the soft outputs take any estimate as input)
    x0 = oracle.admm_ul(f["H"].astype(np.complex128), f["y"].astype(np.complex128), C=C, rho=1.0,
                        N0=f["N0"], T_max=3).astype(np.complex64)
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=3, N0=N0, Es=1.0)
    llr = torch.zeros((W, N, U, int(np.log2(M))), dtype=torch.float32, device="cuda")
    dbp.dbp_uplink_llr(handle, d, torch.from_numpy(H).cuda(), torch.from_numpy(x0).cuda(), llr)
    torch.cuda.synchronize()
    mu, nu2 = oracle.llr_stats(H.astype(np.complex128), N0, 1.0, oracle.REG_MMSE)
    ref = oracle.llr_maxlog(x0.astype(np.complex128), mu, nu2, M)
    got = llr.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref) / (1.0 + np.abs(ref))
    assert err.max() <= 1e-3, err.max()
