"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances: FP32 kernels must agree with the oracle to a relative error of
1e-4 per (subcarrier, symbol) vector, ||x_gpu - x_oracle|| / ||x_oracle||;
the FP64 kernels to 1e-12.  Sliced labels are compared bit for bit with the
oracle's slicer applied to the GPU's own outputs in the kernel's precision,
and with the oracle's labels wherever the oracle's output is not within a
small margin of a decision boundary.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
FP64_TOL = 1e-12


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


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dtype))).cuda()


def _rel_per_vector(x, ref):
    num = np.linalg.norm(x - ref, axis=-1)
    den = np.maximum(np.linalg.norm(ref, axis=-1), 1e-30)
    return num / den


def _round(a, prec):
    return a.astype(np.complex64).astype(np.complex128) if prec == "fp32" else a


def run_ul(dbp, h, f, C, T, algo, prec="fp32", reg=None, rho=1.0, M=None, box_r=0.0):
    """Run one uplink frame on the GPU; returns (x_hat, labels) on the host."""
    W, N, B, U = f["W"], f["N"], f["B"], f["U"]
    ct = np.complex64 if prec == "fp32" else np.complex128
    Hd, yd = _dev(f["H"], ct), _dev(f["y"], ct)
    xd = torch.zeros((W, N, U), dtype=torch.complex64 if prec == "fp32" else torch.complex128, device="cuda")
    ld = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
    if reg is None:
        reg = dbp.DBP_REG_MMSE
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M or f["M"], T_max=T, regularizer=reg,
                       precision=dbp.DBP_FP32 if prec == "fp32" else dbp.DBP_FP64,
                       rho=rho, N0=f["N0"], Es=f["Es"], box_r=box_r)
    fn = dbp.dbp_uplink_admm if algo == "admm" else dbp.dbp_uplink_cg
    fn(h, d, Hd, yd, xd, ld)
    torch.cuda.synchronize()
    return xd.cpu().numpy().astype(np.complex128), ld.cpu().numpy()


def run_dl(dbp, h, f, C, T, prec="fp32", rho=1.0, normalize=False, eps=0.0):
    W, N, B, U = f["W"], f["N"], f["B"], f["U"]
    ct = np.complex64 if prec == "fp32" else np.complex128
    Hd, sd = _dev(f["H"], ct), _dev(f["s"], ct)
    xd = torch.zeros((W, N, B), dtype=torch.complex64 if prec == "fp32" else torch.complex128, device="cuda")
    beta = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = dbp.frame_desc(B, C, U, W, N, T_max=T, precision=dbp.DBP_FP32 if prec == "fp32" else dbp.DBP_FP64,
                       rho=rho, flags=dbp.DBP_FLAG_NORMALIZE if normalize else 0, eps=eps)
    dbp.dbp_downlink_admm(h, d, Hd, sd, xd, beta if normalize else None)
    torch.cuda.synchronize()
    return xd.cpu().numpy().astype(np.complex128), float(beta.cpu()[0])


def oracle_ul(f, C, T, algo, prec, reg=oracle.REG_MMSE, rho=1.0, box_r=1.0):
    H, y = _round(f["H"], prec), _round(f["y"], prec)
    if algo == "admm":
        return oracle.admm_ul(H, y, C=C, rho=rho, N0=f["N0"], Es=f["Es"], T_max=T, reg=reg, box_r=box_r)
    rcg = f["N0"] / f["Es"] if reg == oracle.REG_MMSE else 0.0
    return oracle.cg_ul(H, y, C=C, rho=rcg, T_max=T)


def assert_labels(x_gpu, lab_gpu, x_or, M, dtype):
    # 1) The kernel's decision equals the oracle slicer on the kernel's output,
    #    evaluated in the kernel's precision.
    assert np.array_equal(lab_gpu, oracle.slice_labels(x_gpu, M, dtype=dtype))
    # 2) Against the oracle's own output: identical except where the oracle's
    #    value lies within a margin of a decision boundary.
    lab_or = oracle.slice_labels(x_or, M)
    a = math.sqrt(3.0 / (2.0 * (M - 1)))
    L = int(round(math.sqrt(M)))

    def margin(v):
        t = v / a + (L - 1)          # boundaries at odd integers of t
        frac = np.abs(((t + 1.0) % 2.0) - 1.0)
        return np.where(np.abs(v / a) > L, 10.0, np.abs(frac - 1.0))

    m = np.minimum(margin(x_or.real), margin(x_or.imag))
    clear = m > 1e-3
    assert np.array_equal(lab_gpu[clear], lab_or[clear])


# ---------------------------------------------------------------------------
# Uplink ADMM (Alg. 1)
# ---------------------------------------------------------------------------

UL_CASES = [
    # (W, N, B, C, U, M, T)            covers
    (37, 14, 128, 8, 8, 16, 3),        # the B=128 / C=8 / U=8 workload, ragged W
    (11, 14, 256, 8, 32, 64, 3),       # U=32: two symbol chunks, S=32 staged twice
    (9, 14, 256, 16, 16, 64, 5),       # C=16, U=16
    (13, 5, 24, 6, 8, 16, 4),          # S=4 < U=8 (Woodbury regime), ragged N
    (9, 14, 64, 8, 16, 16, 4),         # S=8 < U=16 (the paper's S < U configuration)
    (7, 15, 80, 2, 5, 16, 3),          # S=40 > stage rows, U=5 padded to 8
    (5, 1, 12, 1, 3, 4, 2),            # C=1 (centralized ADMM), N=1
    (6, 17, 64, 4, 4, 4, 6),           # U=4, two symbol chunks
]


@pytest.fixture(params=["auto", "generic", "tma"])
def path(request, dbp, handle):
    """Run a test with the automatic kernel choice (the tensor-core, broadcast
    or persistent bulk-copy kernel wherever they apply), with the generic
    kernel forced, and with the bulk-copy kernel preferred."""
    code = {"auto": dbp.DBP_PATH_AUTO, "generic": dbp.DBP_PATH_GENERIC, "tma": dbp.DBP_PATH_TMA}[request.param]
    if request.param == "tma":
        # forcing would reject shapes the bulk-copy kernel cannot take; prefer it
        # only where it applies (U a power of two, even S <= 64)
        U, B, C = request.node.callspec.params.get("U", 8), request.node.callspec.params.get("B", 32), \
            request.node.callspec.params.get("C", 4)
        S = B // C
        if U not in (4, 8, 16) or S % 2 or S > 64:   # FP32 at U = 32 does not fit its shared memory
            code = dbp.DBP_PATH_AUTO
    dbp.dbp_set_tuning(handle, kernel=code)
    yield request.param
    dbp.dbp_set_tuning(handle)


@pytest.mark.parametrize("W,N,B,C,U,M,T", UL_CASES)
def test_uplink_admm_fp32_matches_oracle(dbp, handle, path, W, N, B, C, U, M, T):
    f = synth.uplink_frame(W, N, B, U, M, 12.0, seed=W * 1000 + B + C + U)
    x, lab = run_ul(dbp, handle, f, C, T, "admm")
    ref = oracle_ul(f, C, T, "admm", "fp32")
    err = _rel_per_vector(x, ref)
    assert err.max() <= FP32_TOL, err.max()
    assert_labels(x, lab, ref, M, np.float32)


@pytest.mark.parametrize("W,N,B,C,U,M,T", UL_CASES)
def test_uplink_cg_fp32_matches_oracle(dbp, handle, path, W, N, B, C, U, M, T):
    f = synth.uplink_frame(W, N, B, U, M, 12.0, seed=W * 1000 + B + C + U + 1)
    Tcg = T + 5
    x, lab = run_ul(dbp, handle, f, C, Tcg, "cg")
    ref = oracle_ul(f, C, Tcg, "cg", "fp32")
    err = _rel_per_vector(x, ref)
    assert err.max() <= FP32_TOL, err.max()
    assert_labels(x, lab, ref, M, np.float32)


@pytest.mark.parametrize("reg", ["zf", "box"])
def test_uplink_admm_regularisers(dbp, handle, path, reg):
    f = synth.uplink_frame(23, 14, 128, 8, 16, 10.0, seed=77)
    r = oracle.box_radius(16)
    code_d = dbp.DBP_REG_ZF if reg == "zf" else dbp.DBP_REG_BOX
    code_o = oracle.REG_ZF if reg == "zf" else oracle.REG_BOX
    x, lab = run_ul(dbp, handle, f, 8, 4, "admm", reg=code_d, box_r=r)
    ref = oracle_ul(f, 8, 4, "admm", "fp32", reg=code_o, box_r=r)
    assert _rel_per_vector(x, ref).max() <= FP32_TOL


def test_uplink_cg_zf(dbp, handle):
    f = synth.uplink_frame(19, 14, 64, 8, 16, 15.0, seed=78)
    x, _ = run_ul(dbp, handle, f, 4, 6, "cg", reg=dbp.DBP_REG_ZF)
    ref = oracle_ul(f, 4, 6, "cg", "fp32", reg=oracle.REG_ZF)
    assert _rel_per_vector(x, ref).max() <= FP32_TOL


def test_uplink_fp64_small_config(dbp, handle):
    """B=32, C=2 clusters of 16, U=4, QPSK, W=64 x 1 symbol, 10 dB, rho=1,
    5 iterations, seed 0 -- in FP64."""
    f = synth.uplink_frame(64, 1, 32, 4, 4, 10.0, seed=0)
    x, lab = run_ul(dbp, handle, f, 2, 5, "admm", prec="fp64")
    ref = oracle_ul(f, 2, 5, "admm", "fp64")
    assert _rel_per_vector(x, ref).max() <= FP64_TOL
    assert_labels(x, lab, ref, 4, np.float64)
    xc, _ = run_ul(dbp, handle, f, 2, 5, "cg", prec="fp64")
    refc = oracle_ul(f, 2, 5, "cg", "fp64")
    assert _rel_per_vector(xc, refc).max() <= FP64_TOL


def test_uplink_T_edge_cases(dbp, handle):
    f = synth.uplink_frame(9, 3, 32, 4, 16, 8.0, seed=90)
    x, _ = run_ul(dbp, handle, f, 4, 1, "admm")
    assert _rel_per_vector(x, oracle_ul(f, 4, 1, "admm", "fp32")).max() <= FP32_TOL
    x0, _ = run_ul(dbp, handle, f, 4, 0, "cg")
    assert np.all(x0 == 0)


# ---------------------------------------------------------------------------
# Downlink ADMM (Alg. 3)
# ---------------------------------------------------------------------------

DL_CASES = [
    (19, 14, 256, 16, 16, 64, 5),      # the B=256 / C=16 / U=16 workload
    (13, 14, 128, 8, 8, 16, 3),
    (7, 5, 256, 8, 32, 64, 3),         # U=32
    (11, 3, 24, 6, 8, 16, 4),          # S=4 < U
    (9, 14, 64, 8, 16, 16, 4),         # S=8 < U=16 (tensor-core kernel under AUTO)
    (5, 9, 80, 2, 5, 16, 2),           # S=40, U=5
    (4, 1, 16, 1, 4, 4, 1),            # C=1, T=1 (no consensus)
]


@pytest.mark.parametrize("W,N,B,C,U,M,T", DL_CASES)
def test_downlink_admm_fp32_matches_oracle(dbp, handle, path, W, N, B, C, U, M, T):
    f = synth.downlink_frame(W, N, B, U, M, seed=W * 7 + B + C + U)
    x, _ = run_dl(dbp, handle, f, C, T)
    ref = oracle.admm_dl(_round(f["H"], "fp32"), _round(f["s"], "fp32"), C=C, rho=1.0, T_max=T)
    err = _rel_per_vector(x, ref)
    assert err.max() <= FP32_TOL, err.max()


DL_EPS_CASES = [
    # (W, N, B, C, U, T, eps)
    (19, 14, 256, 16, 16, 5, 0.3),     # the B=256 / C=16 / U=16 workload
    (13, 14, 128, 8, 8, 4, 0.2),
    (7, 5, 80, 2, 5, 3, 0.1),          # U=5 padded to 8
    (9, 3, 64, 4, 16, 6, 3.0),         # eps large enough that k = 0 for some symbols
]


@pytest.mark.parametrize("W,N,B,C,U,T,eps", DL_EPS_CASES)
def test_downlink_eps_projection_matches_oracle(dbp, handle, path, W, N, B, C, U, T, eps):
    """Lemma 2 with eps > 0: (s - w)/C scaled by max{0, 1 - eps/||s - w||}."""
    f = synth.downlink_frame(W, N, B, U, 64, seed=970 + W + B + C + U)
    x, _ = run_dl(dbp, handle, f, C, T, eps=eps)
    ref = oracle.admm_dl(_round(f["H"], "fp32"), _round(f["s"], "fp32"), C=C, rho=1.0, T_max=T, eps=eps)
    assert _rel_per_vector(x, ref).max() <= FP32_TOL
    ref0 = oracle.admm_dl(_round(f["H"], "fp32"), _round(f["s"], "fp32"), C=C, rho=1.0, T_max=T)
    assert _rel_per_vector(ref, ref0).max() > 1e-3        # the projection is active


def test_downlink_eps_fp64(dbp, handle):
    f = synth.downlink_frame(11, 4, 64, 8, 16, seed=975)
    x, _ = run_dl(dbp, handle, f, 4, 5, prec="fp64", eps=0.5)
    ref = oracle.admm_dl(f["H"], f["s"], C=4, rho=1.0, T_max=5, eps=0.5)
    assert _rel_per_vector(x, ref).max() <= FP64_TOL


def test_eps_is_validated(dbp, handle):
    buf = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    for bad in (-0.1, float("nan"), float("inf")):
        d = dbp.frame_desc(32, 4, 4, 3, 2, T_max=2, eps=bad)
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_downlink_admm(handle, d, buf, buf, buf)
        assert ei.value.status == dbp.DBP_ERR_INVALID_ARG
    d = dbp.frame_desc(32, 4, 4, 3, 2, qam_order=4, T_max=2, N0=0.1, eps=0.5)
    for fn in (dbp.dbp_uplink_admm, dbp.dbp_uplink_cg):
        with pytest.raises(dbp.DbpError) as ei:
            fn(handle, d, buf, buf, buf, None)
        assert ei.value.status == dbp.DBP_ERR_INVALID_ARG


def test_downlink_fp64(dbp, handle):
    f = synth.downlink_frame(16, 3, 64, 8, 16, seed=5)
    x, _ = run_dl(dbp, handle, f, 4, 4, prec="fp64", rho=0.7)
    ref = oracle.admm_dl(f["H"], f["s"], C=4, rho=0.7, T_max=4)
    assert _rel_per_vector(x, ref).max() <= FP64_TOL


def test_downlink_normalisation(dbp, handle, path):
    f = synth.downlink_frame(21, 14, 128, 8, 16, seed=6)
    x, beta = run_dl(dbp, handle, f, 8, 3, normalize=True)
    ref = oracle.admm_dl(_round(f["H"], "fp32"), _round(f["s"], "fp32"), C=8, rho=1.0, T_max=3)
    beta_ref = math.sqrt(ref.size / np.sum(np.abs(ref) ** 2))
    assert abs(beta - beta_ref) / beta_ref < 1e-5
    assert _rel_per_vector(x, beta_ref * ref).max() <= FP32_TOL
    assert abs(np.mean(np.abs(x) ** 2) - 1.0) < 1e-4


# ---------------------------------------------------------------------------
# Launch shapes: CTA mapping vs thread-block clusters (DSMEM consensus)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("algo", ["admm", "cg", "dl"])
@pytest.mark.parametrize("cl", [2, 4, 8])
def test_cluster_mapping_matches_cta_mapping(dbp, handle, algo, cl):
    f = synth.uplink_frame(29, 14, 128, 8, 16, 10.0, seed=400 + cl)
    try:
        dbp.dbp_set_tuning(handle, dbp.DBP_MAP_CTA)
        if algo == "dl":
            a, _ = run_dl(dbp, handle, f, 8, 4)
        else:
            a, _ = run_ul(dbp, handle, f, 8, 4, algo)
        dbp.dbp_set_tuning(handle, dbp.DBP_MAP_CLUSTER, cluster_size=cl)
        if algo == "dl":
            b, _ = run_dl(dbp, handle, f, 8, 4)
        else:
            b, _ = run_ul(dbp, handle, f, 8, 4, algo)
    finally:
        dbp.dbp_set_tuning(handle, dbp.DBP_MAP_AUTO)
    # two FP32 kernels (the CTA shape may use the bulk-copy kernel, whose
    # Gauss-Jordan step uses a rounded reciprocal): rounding-level agreement
    assert _rel_per_vector(b, a).max() <= 1e-5


@pytest.mark.parametrize("wpc", [4, 16, 32])
def test_warps_per_cta_does_not_change_results(dbp, handle, wpc):
    f = synth.uplink_frame(33, 6, 32, 4, 4, 10.0, seed=500)
    ref, _ = run_ul(dbp, handle, f, 2, 3, "admm")
    try:
        dbp.dbp_set_tuning(handle, dbp.DBP_MAP_CTA, warps_per_cta=wpc)
        x, _ = run_ul(dbp, handle, f, 2, 3, "admm")
    finally:
        dbp.dbp_set_tuning(handle, dbp.DBP_MAP_AUTO)
    assert _rel_per_vector(x, ref).max() <= 1e-6


def test_large_cluster_count_uses_cluster_mapping(dbp, handle):
    """C=16 clusters at U=32 do not fit one CTA's registers: the auto shape
    spreads each subcarrier over a thread-block cluster."""
    f = synth.uplink_frame(5, 14, 256, 32, 64, 14.0, seed=600)
    x, _ = run_ul(dbp, handle, f, 16, 3, "admm")
    ref = oracle_ul(f, 16, 3, "admm", "fp32")
    assert _rel_per_vector(x, ref).max() <= FP32_TOL


@pytest.mark.parametrize("algo", ["admm", "cg", "dl"])
def test_bulk_copy_kernel_matches_generic_kernel(dbp, handle, algo):
    """The persistent bulk-copy kernel (forced) and the generic kernel give the
    same results on a frame spanning many persistent tiles."""
    f = synth.uplink_frame(1201, 14, 128, 8, 16, 8.0, seed=450)
    runs = []
    try:
        for code in (dbp.DBP_PATH_TMA, dbp.DBP_PATH_GENERIC):
            dbp.dbp_set_tuning(handle, kernel=code)
            runs.append(run_dl(dbp, handle, f, 8, 4)[0] if algo == "dl" else run_ul(dbp, handle, f, 8, 4, algo)[0])
    finally:
        dbp.dbp_set_tuning(handle)
    assert _rel_per_vector(runs[0], runs[1]).max() <= 1e-5


@pytest.mark.parametrize("algo", ["admm", "cg"])
def test_bulk_copy_kernel_single_staging_buffer(dbp, handle, algo):
    """FP32, U=32, S=32: two staging buffers do not fit in shared memory, so the
    forced bulk-copy kernel refills one buffer after the matched filter.  301
    subcarriers take several persistent tiles per CTA (every refill path)."""
    f = synth.uplink_frame(301, 14, 256, 32, 64, 20.0, seed=452)
    try:
        dbp.dbp_set_tuning(handle, kernel=dbp.DBP_PATH_TMA)
        x, lab = run_ul(dbp, handle, f, 8, 3, algo)
    finally:
        dbp.dbp_set_tuning(handle)
    ref = oracle_ul(f, 8, 3, algo, "fp32")
    assert _rel_per_vector(x, ref).max() <= FP32_TOL
    assert_labels(x, lab, ref, 64, np.float32)


@pytest.mark.parametrize("algo", ["admm", "cg", "dl"])
@pytest.mark.parametrize("W,N,B,C", [(23, 5, 240, 8), (19, 20, 240, 8), (17, 14, 128, 4)])
def test_bulk_copy_kernel_fp32_u32_tensor_core_products(dbp, handle, algo, W, N, B, C):
    """FP32 inputs at U = 32 (Gram and matched filter as 3 x TF32 tensor-core
    products): S = 30 (rows padded to a multiple of 4), N = 5 (one partial
    8-symbol tile), N = 20 (three tiles, two chunks) and S = 32, against the
    oracle."""
    U, M, T = 32, 16, 3
    try:
        dbp.dbp_set_tuning(handle, kernel=dbp.DBP_PATH_TMA)
        if algo == "dl":
            f = synth.downlink_frame(W, N, B, U, M, seed=470 + W + N + B)
            x, _ = run_dl(dbp, handle, f, C, T)
            ref = oracle.admm_dl(_round(f["H"], "fp32"), _round(f["s"], "fp32"), C=C, rho=1.0, T_max=T)
        else:
            f = synth.uplink_frame(W, N, B, U, M, 20.0, seed=470 + W + N + B)
            x, lab = run_ul(dbp, handle, f, C, T, algo)
            ref = oracle_ul(f, C, T, algo, "fp32")
            assert_labels(x, lab, ref, M, np.float32)
    finally:
        dbp.dbp_set_tuning(handle)
    assert _rel_per_vector(x, ref).max() <= FP32_TOL


def test_forced_bulk_copy_kernel_rejects_ineligible_shapes(dbp, handle):
    f = synth.uplink_frame(3, 2, 40, 5, 16, 8.0, seed=451)      # U=5 is not a power of two
    try:
        dbp.dbp_set_tuning(handle, kernel=dbp.DBP_PATH_TMA)
        with pytest.raises(dbp.DbpError) as ei:
            run_ul(dbp, handle, f, 4, 3, "admm")
        assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED
    finally:
        dbp.dbp_set_tuning(handle)
    dbp.dbp_device_status(handle)


# ---------------------------------------------------------------------------
# U = 8 tensor-core kernel (3 x TF32 products)
# ---------------------------------------------------------------------------

MMA8_CASES = [
    # (W, N, B, C, M)
    (37, 14, 128, 8, 16),     # the B=128 / C=8 / U=8 workload, ragged W
    (9, 20, 48, 8, 16),       # S=6 (padded to a multiple of 4), N > 16 (two symbol passes)
    (5, 1, 16, 2, 4),         # S=8, N=1
    (7, 17, 64, 1, 64),       # C=1 (S=64), two symbol passes
    (11, 14, 128, 16, 16),    # C=16 clusters of 8
]


@pytest.mark.parametrize("algo", ["admm", "cg"])
@pytest.mark.parametrize("W,N,B,C,M", MMA8_CASES)
def test_mma8_kernel_matches_oracle(dbp, handle, algo, W, N, B, C, M):
    f = synth.uplink_frame(W, N, B, 8, M, 10.0, seed=800 + W + N + B + C)
    T = 3 if algo == "admm" else 8
    try:
        dbp.dbp_set_tuning(handle, kernel=dbp.DBP_PATH_MMA)
        x, lab = run_ul(dbp, handle, f, C, T, algo)
    finally:
        dbp.dbp_set_tuning(handle)
    ref = oracle_ul(f, C, T, algo, "fp32")
    err = _rel_per_vector(x, ref)
    assert err.max() <= FP32_TOL, err.max()
    assert_labels(x, lab, ref, M, np.float32)


@pytest.mark.parametrize("reg", ["zf", "box"])
def test_mma8_kernel_regularisers(dbp, handle, reg):
    f = synth.uplink_frame(21, 14, 128, 8, 16, 10.0, seed=850)
    r = oracle.box_radius(16)
    try:
        dbp.dbp_set_tuning(handle, kernel=dbp.DBP_PATH_MMA)
        x, _ = run_ul(dbp, handle, f, 8, 4, "admm", reg=dbp.DBP_REG_ZF if reg == "zf" else dbp.DBP_REG_BOX,
                      box_r=r)
    finally:
        dbp.dbp_set_tuning(handle)
    ref = oracle_ul(f, 8, 4, "admm", "fp32", reg=oracle.REG_ZF if reg == "zf" else oracle.REG_BOX, box_r=r)
    assert _rel_per_vector(x, ref).max() <= FP32_TOL


def test_mma8_fp64_retry_on_a_near_singular_cluster(dbp, handle):
    W, N, B, C = 10, 14, 128, 4                   # S = 32 > U = 8
    f = synth.uplink_frame(W, N, B, 8, 16, 20.0, seed=860)
    S = B // C
    u_, s_, vh = np.linalg.svd(f["H"][4, S:2 * S], full_matrices=False)
    s_[-1] = 1e-4 * s_[0]
    f["H"][4, S:2 * S] = (u_ * s_) @ vh
    f["y"] = np.einsum("wbu,wnu->wnb", f["H"], f["s"])
    dbp.dbp_fp64_retries(handle)
    try:
        dbp.dbp_set_tuning(handle, kernel=dbp.DBP_PATH_MMA)
        x, _ = run_ul(dbp, handle, f, C, 3, "admm", rho=1e-6)
    finally:
        dbp.dbp_set_tuning(handle)
    assert dbp.dbp_fp64_retries(handle) == 1
    ref = oracle_ul(f, C, 3, "admm", "fp32", rho=1e-6)
    good = np.arange(W) != 4
    assert np.all(np.isfinite(x))
    assert _rel_per_vector(x[good], ref[good]).max() <= FP32_TOL


def test_forced_mma8_kernel_rejects_other_shapes(dbp, handle):
    f = synth.uplink_frame(3, 2, 64, 16, 16, 8.0, seed=870)   # U = 16
    try:
        dbp.dbp_set_tuning(handle, kernel=dbp.DBP_PATH_MMA)
        with pytest.raises(dbp.DbpError) as ei:
            run_ul(dbp, handle, f, 4, 3, "admm")
        assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED
    finally:
        dbp.dbp_set_tuning(handle)


# ---------------------------------------------------------------------------
# Broadcast kernels: the consensus step once per symbol, s (Alg. 1) or p
# (Alg. 2, the first placement of Sec. III-D) broadcast to the clusters
# ---------------------------------------------------------------------------

BCAST_CASES = [
    # (W, N, B, C, U, M, T)          covers
    (37, 14, 128, 8, 8, 16, 8),      # the B=128 / C=8 / U=8 workload, ragged W
    (9, 14, 256, 16, 16, 64, 8),     # C=16 warps per CTA, U=16 (14-symbol chunk)
    (11, 20, 128, 8, 8, 16, 5),      # N > 16: two symbol chunks, the second ragged
    (7, 14, 64, 1, 8, 16, 8),        # C=1: one warp updates every symbol (4 passes of 32)
    (13, 9, 32, 2, 4, 4, 6),         # C=2: four subcarriers per CTA, U=4
    (6, 17, 64, 4, 4, 16, 3),        # U=4, 16-symbol chunks, ragged second chunk
    (5, 1, 24, 3, 8, 16, 4),         # N=1: one owner, the other warps idle in the update
    (8, 14, 96, 6, 16, 64, 16),      # T = U: CG reaches the LMMSE solution
    (3, 14, 256, 8, 16, 64, 2),      # S=32 rows of H per cluster
    (4, 14, 32, 8, 8, 16, 3),        # S=4 < U=8 (the Woodbury regime of the paper)
]


def _with_path(dbp, handle, code, fn):
    try:
        dbp.dbp_set_tuning(handle, kernel=code)
        return fn()
    finally:
        dbp.dbp_set_tuning(handle)


@pytest.mark.parametrize("algo", ["admm", "cg"])
@pytest.mark.parametrize("W,N,B,C,U,M,T", BCAST_CASES)
def test_bcast_kernels_match_oracle(dbp, handle, algo, W, N, B, C, U, M, T):
    f = synth.uplink_frame(W, N, B, U, M, 12.0, seed=900 + W + N + B + C + U)
    x, lab = _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_ul(dbp, handle, f, C, T, algo))
    ref = oracle_ul(f, C, T, algo, "fp32")
    err = _rel_per_vector(x, ref)
    assert err.max() <= FP32_TOL, err.max()
    assert_labels(x, lab, ref, M, np.float32)


@pytest.mark.parametrize("reg", ["zf", "box"])
def test_bcast_admm_kernel_regularisers(dbp, handle, reg):
    f = synth.uplink_frame(21, 14, 128, 8, 16, 10.0, seed=905)
    r = oracle.box_radius(16)
    x, _ = _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_ul(
        dbp, handle, f, 8, 4, "admm", reg=dbp.DBP_REG_ZF if reg == "zf" else dbp.DBP_REG_BOX, box_r=r))
    ref = oracle_ul(f, 8, 4, "admm", "fp32", reg=oracle.REG_ZF if reg == "zf" else oracle.REG_BOX, box_r=r)
    assert _rel_per_vector(x, ref).max() <= FP32_TOL


@pytest.mark.parametrize("U", [4, 8, 16])
def test_bcast_admm_fp64_retry_on_a_near_singular_cluster(dbp, handle, U):
    W, N, B, C = 10, 14, 128, 4                   # S = 32 > U
    f = synth.uplink_frame(W, N, B, U, 16, 20.0, seed=906 + U)
    S = B // C
    u_, s_, vh = np.linalg.svd(f["H"][4, S:2 * S], full_matrices=False)
    s_[-1] = 1e-4 * s_[0]
    f["H"][4, S:2 * S] = (u_ * s_) @ vh
    f["y"] = np.einsum("wbu,wnu->wnb", f["H"], f["s"])
    dbp.dbp_fp64_retries(handle)
    x, _ = _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_ul(dbp, handle, f, C, 3, "admm", rho=1e-6))
    assert dbp.dbp_fp64_retries(handle) == 1
    ref = oracle_ul(f, C, 3, "admm", "fp32", rho=1e-6)
    good = np.arange(W) != 4
    assert np.all(np.isfinite(x))
    assert _rel_per_vector(x[good], ref[good]).max() <= FP32_TOL


def test_bcast_cg_kernel_zf_and_T_edges(dbp, handle):
    f = synth.uplink_frame(19, 14, 64, 8, 16, 15.0, seed=910)
    x, _ = _with_path(dbp, handle, dbp.DBP_PATH_BCAST,
                      lambda: run_ul(dbp, handle, f, 4, 6, "cg", reg=dbp.DBP_REG_ZF))
    assert _rel_per_vector(x, oracle_ul(f, 4, 6, "cg", "fp32", reg=oracle.REG_ZF)).max() <= FP32_TOL
    x1, _ = _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_ul(dbp, handle, f, 4, 1, "cg"))
    assert _rel_per_vector(x1, oracle_ul(f, 4, 1, "cg", "fp32")).max() <= FP32_TOL
    x0, _ = _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_ul(dbp, handle, f, 4, 0, "cg"))
    assert np.all(x0 == 0)
    a1, _ = _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_ul(dbp, handle, f, 4, 1, "admm"))
    assert _rel_per_vector(a1, oracle_ul(f, 4, 1, "admm", "fp32")).max() <= FP32_TOL


def test_bcast_cg_kernel_stops_on_a_zero_residual(dbp, handle):
    """A symbol whose receive vector is zero has r = y_MRC = 0: its iterate
    stays x = 0 (no 0/0), and the other symbols are unaffected."""
    f = synth.uplink_frame(6, 14, 128, 8, 16, 10.0, seed=911)
    f["y"][2, 5] = 0.0
    f["y"][4] = 0.0
    x, _ = _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_ul(dbp, handle, f, 8, 8, "cg"))
    assert np.all(np.isfinite(x))
    assert np.all(x[2, 5] == 0) and np.all(x[4] == 0)
    ref = oracle_ul(f, 8, 8, "cg", "fp32")
    keep = np.ones(x.shape[:2], dtype=bool)
    keep[2, 5] = False
    keep[4] = False
    assert _rel_per_vector(x[keep], ref[keep]).max() <= FP32_TOL


@pytest.mark.parametrize("kernel", ["bcast", "mma"])
@pytest.mark.parametrize("algo", ["admm", "cg"])
def test_bcast_kernels_match_generic_kernel_over_many_tiles(dbp, handle, algo, kernel):
    f = synth.uplink_frame(1201, 14, 128, 8, 16, 8.0, seed=912)
    T = 3 if algo == "admm" else 8
    code = dbp.DBP_PATH_BCAST if kernel == "bcast" else dbp.DBP_PATH_MMA
    a, la = _with_path(dbp, handle, code, lambda: run_ul(dbp, handle, f, 8, T, algo))
    b, lb = _with_path(dbp, handle, dbp.DBP_PATH_GENERIC, lambda: run_ul(dbp, handle, f, 8, T, algo))
    # two FP32 kernels with different summation orders: rounding-level agreement
    assert _rel_per_vector(a, b).max() <= 1e-5


@pytest.mark.parametrize("algo", ["admm", "cg"])
@pytest.mark.parametrize("U", [4, 8, 16])
def test_auto_path_for_the_uplink(dbp, handle, algo, U):
    """AUTO runs the tensor-core kernel at U = 8 and the broadcast kernels at
    U = 4 and 16 (bit-identical results to forcing them)."""
    f = synth.uplink_frame(17, 14, 128, U, 16, 10.0, seed=913 + U)
    a, _ = run_ul(dbp, handle, f, 8, 8, algo)
    code = dbp.DBP_PATH_MMA if U == 8 else dbp.DBP_PATH_BCAST
    b, _ = _with_path(dbp, handle, code, lambda: run_ul(dbp, handle, f, 8, 8, algo))
    assert np.array_equal(a, b)


def test_forced_bcast_kernels_reject_other_work(dbp, handle):
    fd = synth.downlink_frame(3, 2, 64, 8, 16, seed=914)
    with pytest.raises(dbp.DbpError) as ei:
        _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_dl(dbp, handle, fd, 4, 3))
    assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED
    f32 = synth.uplink_frame(3, 2, 64, 32, 16, 8.0, seed=915)   # U = 32
    for algo in ("admm", "cg"):
        with pytest.raises(dbp.DbpError) as ei:
            _with_path(dbp, handle, dbp.DBP_PATH_BCAST, lambda: run_ul(dbp, handle, f32, 2, 3, algo))
        assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# Downlink tensor-core kernel (U = 16)
# ---------------------------------------------------------------------------

TCDL_CASES = [
    # (W, N, B, C, T)             covers
    (19, 14, 256, 16, 5),         # the B=256 / C=16 / U=16 workload, ragged W
    (9, 14, 256, 8, 5),           # S=32: four antenna m-tiles in the output product
    (11, 20, 64, 4, 3),           # two subcarriers per CTA, N > 16 (two symbol passes)
    (7, 5, 16, 2, 4),             # S=8, four subcarriers per CTA, ragged N
    (5, 1, 32, 1, 2),             # C=1 (no consensus partner), N=1
    (6, 14, 256, 16, 1),          # T=1: init and output only
]


@pytest.mark.parametrize("W,N,B,C,T", TCDL_CASES)
def test_tcdl_kernel_matches_oracle(dbp, handle, W, N, B, C, T):
    f = synth.downlink_frame(W, N, B, 16, 64, seed=950 + W + N + B + C + T)
    x, _ = _with_path(dbp, handle, dbp.DBP_PATH_MMA, lambda: run_dl(dbp, handle, f, C, T))
    ref = oracle.admm_dl(_round(f["H"], "fp32"), _round(f["s"], "fp32"), C=C, rho=1.0, T_max=T)
    err = _rel_per_vector(x, ref)
    assert err.max() <= FP32_TOL, err.max()


def test_tcdl_kernel_rho_and_normalisation(dbp, handle):
    f = synth.downlink_frame(21, 14, 128, 16, 64, seed=960)
    x, _ = _with_path(dbp, handle, dbp.DBP_PATH_MMA, lambda: run_dl(dbp, handle, f, 8, 4, rho=0.6))
    ref = oracle.admm_dl(_round(f["H"], "fp32"), _round(f["s"], "fp32"), C=8, rho=0.6, T_max=4)
    assert _rel_per_vector(x, ref).max() <= FP32_TOL
    xn, beta = _with_path(dbp, handle, dbp.DBP_PATH_MMA, lambda: run_dl(dbp, handle, f, 8, 4, rho=0.6, normalize=True))
    beta_ref = math.sqrt(ref.size / np.sum(np.abs(ref) ** 2))
    assert abs(beta - beta_ref) / beta_ref < 1e-5
    assert _rel_per_vector(xn, beta_ref * ref).max() <= FP32_TOL


def test_tcdl_fp64_retry_on_a_near_singular_cluster(dbp, handle):
    W, N, B, C = 10, 14, 128, 4                   # S = 32 > U = 16
    f = synth.downlink_frame(W, N, B, 16, 64, seed=961)
    S = B // C
    u_, s_, vh = np.linalg.svd(f["H"][4, S:2 * S], full_matrices=False)
    s_[-1] = 1e-4 * s_[0]
    f["H"][4, S:2 * S] = (u_ * s_) @ vh
    dbp.dbp_fp64_retries(handle)
    x, _ = _with_path(dbp, handle, dbp.DBP_PATH_MMA, lambda: run_dl(dbp, handle, f, C, 3, rho=1e6))
    assert dbp.dbp_fp64_retries(handle) == 1
    ref = oracle.admm_dl(_round(f["H"], "fp32"), _round(f["s"], "fp32"), C=C, rho=1e6, T_max=3)
    good = np.arange(W) != 4
    assert np.all(np.isfinite(x))
    assert _rel_per_vector(x[good], ref[good]).max() <= FP32_TOL


def test_tcdl_kernel_matches_bulk_copy_kernel_over_many_tiles(dbp, handle):
    f = synth.downlink_frame(1201, 14, 256, 16, 64, seed=962)
    a, _ = _with_path(dbp, handle, dbp.DBP_PATH_MMA, lambda: run_dl(dbp, handle, f, 16, 5))
    b, _ = _with_path(dbp, handle, dbp.DBP_PATH_TMA, lambda: run_dl(dbp, handle, f, 16, 5))
    assert _rel_per_vector(a, b).max() <= 1e-5


def test_auto_path_uses_tcdl_for_the_downlink(dbp, handle):
    f = synth.downlink_frame(17, 14, 256, 16, 64, seed=963)
    a, _ = run_dl(dbp, handle, f, 16, 5)
    b, _ = _with_path(dbp, handle, dbp.DBP_PATH_MMA, lambda: run_dl(dbp, handle, f, 16, 5))
    assert np.array_equal(a, b)
    f8 = synth.downlink_frame(5, 3, 64, 8, 16, seed=964)       # U = 8: no downlink tensor-core kernel
    with pytest.raises(dbp.DbpError) as ei:
        _with_path(dbp, handle, dbp.DBP_PATH_MMA, lambda: run_dl(dbp, handle, f8, 4, 3))
    assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# Host-buffer (end-to-end) entry points and argument errors
# ---------------------------------------------------------------------------

def test_host_variants_equal_device_variants(dbp, handle):
    f = synth.uplink_frame(17, 14, 128, 8, 16, 10.0, seed=700)
    xd, ld = run_ul(dbp, handle, f, 8, 3, "admm")
    H = np.ascontiguousarray(f["H"].astype(np.complex64))
    y = np.ascontiguousarray(f["y"].astype(np.complex64))
    xh = np.zeros((17, 14, 8), dtype=np.complex64)
    lh = np.zeros((17, 14, 8), dtype=np.uint8)
    d = dbp.frame_desc(128, 8, 8, 17, 14, qam_order=16, T_max=3, N0=f["N0"], Es=1.0)
    dbp.dbp_uplink_admm_host(handle, d, H, y, xh, lh)
    assert np.array_equal(xh.astype(np.complex128), xd) and np.array_equal(lh, ld)
    fd = synth.downlink_frame(9, 14, 256, 16, 64, seed=701)
    xdd, _ = run_dl(dbp, handle, fd, 16, 5)
    xhd = np.zeros((9, 14, 256), dtype=np.complex64)
    dd = dbp.frame_desc(256, 16, 16, 9, 14, T_max=5)
    dbp.dbp_downlink_admm_host(handle, dd, np.ascontiguousarray(fd["H"].astype(np.complex64)),
                               np.ascontiguousarray(fd["s"].astype(np.complex64)), xhd)
    assert np.array_equal(xhd.astype(np.complex128), xdd)


def test_empty_frames_are_no_ops(dbp, handle):
    for W, N in [(0, 14), (5, 0)]:
        d = dbp.frame_desc(32, 4, 4, W, N, qam_order=4, T_max=3, N0=0.1)
        dbp.dbp_uplink_admm(handle, d, 0, 0, 0, None)
        dbp.dbp_uplink_cg(handle, d, 0, 0, 0, None)
        dbp.dbp_downlink_admm(handle, d, 0, 0, 0, None)


@pytest.mark.parametrize("bad", [
    dict(B=30, C=4),            # B not a multiple of C
    dict(U=33),                 # too many users
    dict(T_max=0),              # ADMM needs at least the init
    dict(rho=0.0),
    dict(qam_order=8),
    dict(precision=7),
    dict(regularizer=9),
    dict(regularizer=2, box_r=0.0),
])
def test_invalid_descriptors_are_rejected(dbp, handle, bad):
    kw = dict(B=32, C=4, U=4, W=3, N=2, qam_order=4, T_max=2, N0=0.1)
    kw.update(bad)
    d = dbp.frame_desc(**kw)
    buf = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    with pytest.raises(dbp.DbpError) as ei:
        dbp.dbp_uplink_admm(handle, d, buf, buf, buf, None)
    assert ei.value.status in (dbp.DBP_ERR_INVALID_ARG, dbp.DBP_ERR_UNSUPPORTED)


# ---------------------------------------------------------------------------
# Full-size frames in the benchmark's launch configuration, sampled
# ---------------------------------------------------------------------------

def _sample(W, k, seed):
    return np.sort(np.random.default_rng(seed).choice(W, size=k, replace=False))


def test_full_size_uplink_sampled(dbp, handle):
    """B=128, C=8, U=8, 16-QAM, 1200 x 14 at 10 dB: ADMM (3) and CG (8) on the
    whole frame; the oracle recomputes 48 sampled subcarriers."""
    f = synth.uplink_frame(1200, 14, 128, 8, 16, 10.0, seed=synth.frame_seed(2, 5))
    idx = _sample(1200, 48, 1)
    sub = dict(f, H=f["H"][idx], y=f["y"][idx], W=len(idx))
    for algo, T in (("admm", 3), ("cg", 8)):
        x, lab = run_ul(dbp, handle, f, 8, T, algo)
        ref = oracle_ul(sub, 8, T, algo, "fp32")
        assert _rel_per_vector(x[idx], ref).max() <= FP32_TOL
        assert_labels(x[idx], lab[idx], ref, 16, np.float32)


def test_full_size_downlink_sampled(dbp, handle):
    """B=256, C=16, U=16, 64-QAM, 1200 x 14, 5 iterations: sampled parity."""
    f = synth.downlink_frame(1200, 14, 256, 16, 64, seed=synth.frame_seed(3))
    idx = _sample(1200, 24, 2)
    x, _ = run_dl(dbp, handle, f, 16, 5)
    ref = oracle.admm_dl(_round(f["H"][idx], "fp32"), _round(f["s"][idx], "fp32"), C=16, rho=1.0, T_max=5)
    assert _rel_per_vector(x[idx], ref).max() <= FP32_TOL


def test_full_size_u32_sampled(dbp, handle):
    """B=256, C=8, U=32, 64-QAM, 3300 x 14 (FP32 path): sampled parity."""
    f = synth.uplink_frame(3300, 14, 256, 32, 64, 20.0, seed=synth.frame_seed(4, 5))
    idx = _sample(3300, 16, 3)
    sub = dict(f, H=f["H"][idx], y=f["y"][idx], W=len(idx))
    x, lab = run_ul(dbp, handle, f, 8, 3, "admm")
    ref = oracle_ul(sub, 8, 3, "admm", "fp32")
    assert _rel_per_vector(x[idx], ref).max() <= FP32_TOL


def test_full_size_box_prox_sampled(dbp, handle):
    """B=128, C=8, U=8, 16-QAM, 1200 x 14 at 4 dB, ADMM T=3 with the BOX prox
    (the bench's box_prox line): sampled parity, box bound active."""
    f = synth.uplink_frame(1200, 14, 128, 8, 16, 4.0, seed=synth.frame_seed(2, 2))
    r = oracle.box_radius(16)
    idx = _sample(1200, 48, 5)
    sub = dict(f, H=f["H"][idx], y=f["y"][idx], W=len(idx))
    x, lab = run_ul(dbp, handle, f, 8, 3, "admm", reg=dbp.DBP_REG_BOX, box_r=r)
    ref = oracle_ul(sub, 8, 3, "admm", "fp32", reg=oracle.REG_BOX, box_r=r)
    assert _rel_per_vector(x[idx], ref).max() <= FP32_TOL
    assert_labels(x[idx], lab[idx], ref, 16, np.float32)
    assert np.abs(x.real).max() <= np.float32(r) and np.any(np.abs(x.real) == np.float32(r))


def test_full_size_downlink_eps_sampled(dbp, handle):
    """B=256, C=16, U=16, 64-QAM, 1200 x 14, 5 iterations with eps = 0.05 (the
    bench's downlink_eps line): sampled parity against the oracle's Lemma 2."""
    f = synth.downlink_frame(1200, 14, 256, 16, 64, seed=synth.frame_seed(3, 1))
    idx = _sample(1200, 24, 6)
    x, _ = run_dl(dbp, handle, f, 16, 5, eps=0.05)
    ref = oracle.admm_dl(_round(f["H"][idx], "fp32"), _round(f["s"][idx], "fp32"), C=16, rho=1.0, T_max=5,
                         eps=0.05)
    assert _rel_per_vector(x[idx], ref).max() <= FP32_TOL
    ref0 = oracle.admm_dl(_round(f["H"][idx], "fp32"), _round(f["s"][idx], "fp32"), C=16, rho=1.0, T_max=5)
    assert _rel_per_vector(ref, ref0).max() > 1e-3   # eps does change the result at this size
