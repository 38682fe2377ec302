"""The largest and the degenerate shapes the library accepts, against the
FP64 oracle (sampled subcarriers where the frame is large):

- W = 140,000 subcarriers (grids past 65,535 CTAs, many waves of the
  persistent kernels) for every entry point;
- C = 128 clusters at U = 32 (S = 1: sixteen 8-warp CTAs per subcarrier, the
  largest thread-block cluster) for both uplink detectors and the downlink;
- N = 100 symbols (seven 16-symbol passes of the tensor-core kernel);
- one user (U = 1, padded to 4), a square system (B = U) and one antenna per
  cluster at U = 8.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


@pytest.fixture(scope="module")
def dbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_04458_b300 as p
    return p


@pytest.fixture(scope="module")
def handle(dbp):
    h = dbp.dbp_create(0)
    yield h
    torch.cuda.synchronize()
    dbp.dbp_destroy(h)


def _c64(a):
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


def _r32(a):
    """The FP32-rounded values the kernels see, in FP64 for the oracle."""
    return a.astype(np.complex64).astype(np.complex128)


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), 1e-30)


def _uplink(dbp, h, f, C, T, algo, reg=None):
    W, N, B, U = f["W"], f["N"], f["B"], f["U"]
    x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
    lab = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
    d = dbp.frame_desc(B, C, U, W, N, qam_order=f["M"], T_max=T,
                       regularizer=dbp.DBP_REG_MMSE if reg is None else reg, rho=1.0, N0=f["N0"], Es=1.0)
    (dbp.dbp_uplink_admm if algo == "admm" else dbp.dbp_uplink_cg)(h, d, _c64(f["H"]), _c64(f["y"]), x, lab)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128), lab.cpu().numpy(), d


def _oracle_ul(f, idx, C, T, algo, reg=oracle.REG_MMSE):
    H, y = _r32(f["H"][idx]), _r32(f["y"][idx])
    if algo == "admm":
        return oracle.admm_ul(H, y, C=C, rho=1.0, N0=f["N0"], Es=1.0, T_max=T, reg=reg)
    return oracle.cg_ul(H, y, C=C, rho=f["N0"] if reg == oracle.REG_MMSE else 0.0, T_max=T)


def _downlink(dbp, h, f, C, T):
    W, N, B, U = f["W"], f["N"], f["B"], f["U"]
    x = torch.zeros((W, N, B), dtype=torch.complex64, device="cuda")
    d = dbp.frame_desc(B, C, U, W, N, T_max=T, rho=1.0)
    dbp.dbp_downlink_admm(h, d, _c64(f["H"]), _c64(f["s"]), x, None)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128)


def _sample(W, k, seed):
    idx = np.random.default_rng(seed).choice(W, size=k, replace=False)
    return np.unique(np.concatenate([idx, [0, W - 1]]))   # both ends of the frame too


# ---------------------------------------------------------------------------
# W = 140,000 subcarriers
# ---------------------------------------------------------------------------

BIG_W = 140_000


@pytest.mark.parametrize("kind", ["admm", "cg", "llr"])
def test_many_subcarriers_uplink(dbp, handle, kind):
    f = synth.uplink_frame(BIG_W, 2, 16, 4, 4, 8.0, seed=4100)
    T = 4 if kind == "cg" else 3
    x, lab, d = _uplink(dbp, handle, f, 2, T, "cg" if kind == "cg" else "admm")
    idx = _sample(BIG_W, 64, 1)
    ref = _oracle_ul(f, idx, 2, T, "cg" if kind == "cg" else "admm")
    assert _rel(x[idx], ref).max() <= FP32_TOL
    assert np.array_equal(lab, oracle.slice_labels(x, 4, dtype=np.float32))
    if kind == "llr":
        llr = torch.zeros((BIG_W, 2, 4, 2), dtype=torch.float32, device="cuda")
        dbp.dbp_uplink_llr(handle, d, _c64(f["H"]), _c64(x), llr)
        torch.cuda.synchronize()
        mu, nu2 = oracle.llr_stats(_r32(f["H"][idx]), f["N0"], 1.0, oracle.REG_MMSE)
        want = oracle.llr_maxlog(x[idx].astype(np.complex64).astype(np.complex128), mu, nu2, 4)
        got = llr.cpu().numpy()[idx].astype(np.float64)
        assert (np.abs(got - want) / (1.0 + np.abs(want))).max() <= 1e-3


def test_many_subcarriers_downlink(dbp, handle):
    f = synth.downlink_frame(BIG_W, 2, 16, 4, 4, seed=4101)
    x = _downlink(dbp, handle, f, 2, 3)
    idx = _sample(BIG_W, 64, 2)
    ref = oracle.admm_dl(_r32(f["H"][idx]), _r32(f["s"][idx]), C=2, rho=1.0, T_max=3)
    assert _rel(x[idx], ref).max() <= FP32_TOL


# ---------------------------------------------------------------------------
# C = 128 clusters at U = 32: one antenna per cluster, 16-CTA clusters
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["admm", "cg", "dl"])
def test_most_clusters_at_32_users(dbp, handle, kind):
    W, N, B, C, U = 7, 3, 128, 128, 32
    if kind == "dl":
        f = synth.downlink_frame(W, N, B, U, 16, seed=4200)
        x = _downlink(dbp, handle, f, C, 3)
        ref = oracle.admm_dl(_r32(f["H"]), _r32(f["s"]), C=C, rho=1.0, T_max=3)
        assert _rel(x, ref).max() <= FP32_TOL
        return
    f = synth.uplink_frame(W, N, B, U, 16, 15.0, seed=4201)
    T = 5 if kind == "cg" else 3
    x, lab, _ = _uplink(dbp, handle, f, C, T, kind)
    ref = _oracle_ul(f, np.arange(W), C, T, kind)
    assert _rel(x, ref).max() <= FP32_TOL
    assert np.array_equal(lab, oracle.slice_labels(x, 16, dtype=np.float32))


# ---------------------------------------------------------------------------
# N = 100 symbols per subcarrier
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("algo", ["admm", "cg"])
@pytest.mark.parametrize("B,C,U", [(128, 8, 8), (256, 8, 32)])
def test_many_symbols(dbp, handle, algo, B, C, U):
    W = 37 if U == 8 else 5
    f = synth.uplink_frame(W, 100, B, U, 16, 12.0, seed=4300 + U)
    T = 8 if algo == "cg" else 3
    x, lab, _ = _uplink(dbp, handle, f, C, T, algo)
    ref = _oracle_ul(f, np.arange(W), C, T, algo)
    assert _rel(x, ref).max() <= FP32_TOL
    assert np.array_equal(lab, oracle.slice_labels(x, 16, dtype=np.float32))


def test_many_symbols_downlink(dbp, handle):
    f = synth.downlink_frame(11, 100, 256, 16, 64, seed=4310)
    x = _downlink(dbp, handle, f, 16, 5)
    ref = oracle.admm_dl(_r32(f["H"]), _r32(f["s"]), C=16, rho=1.0, T_max=5)
    assert _rel(x, ref).max() <= FP32_TOL


# ---------------------------------------------------------------------------
# Degenerate shapes: one user, a square system, one antenna per cluster
# ---------------------------------------------------------------------------

DEGENERATE = [
    # (W, N, B, C, U, M, snr)
    (50, 14, 16, 4, 1, 4, 6.0),     # one user (padded to 4)
    (40, 14, 8, 1, 8, 16, 10.0),    # B = U, one cluster: H square
    (40, 14, 16, 2, 16, 4, 10.0),   # B = U = 16 over two clusters (S = 8 < U)
    (30, 9, 8, 8, 8, 16, 10.0),     # S = 1 at U = 8: every cluster Gram has rank one
]
# (square channels are badly conditioned: 10 dB keeps N0 / Es, which loads
# the diagonal of the MMSE Gram, large enough that FP32 iterates track FP64)


@pytest.mark.parametrize("kind", ["admm", "cg", "dl"])
@pytest.mark.parametrize("W,N,B,C,U,M,snr", DEGENERATE)
def test_degenerate_shapes(dbp, handle, kind, W, N, B, C, U, M, snr):
    if kind == "dl":
        f = synth.downlink_frame(W, N, B, U, M, seed=4400 + B + U)
        x = _downlink(dbp, handle, f, C, 4)
        ref = oracle.admm_dl(_r32(f["H"]), _r32(f["s"]), C=C, rho=1.0, T_max=4)
        assert _rel(x, ref).max() <= FP32_TOL
        return
    f = synth.uplink_frame(W, N, B, U, M, snr, seed=4410 + B + U)
    T = min(U, 6) if kind == "cg" else 4
    x, lab, _ = _uplink(dbp, handle, f, C, T, kind)
    ref = _oracle_ul(f, np.arange(W), C, T, kind)
    assert _rel(x, ref).max() <= FP32_TOL
    assert np.array_equal(lab, oracle.slice_labels(x, M, dtype=np.float32))
