"""The separate operator kernel (DBP_PREFACTOR_ON): B_c^{-1} of every
(subcarrier, cluster) is formed by a kernel of its own and the fused kernel
loads it.  Both kernels compute the operator with the same device code on the
same staged layout, so results must be bit-identical with and without it;
against the FP64 oracle the FP32 tolerance holds; its FP64 retry counts like
the fused kernel's; and two calls on two streams, each with its own
stream-ordered operator buffer, give the same bits as one after the other."""
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


def _dev(a, prec):
    if prec == "fp32":
        return torch.from_numpy(a.astype(np.complex64)).cuda()
    dt = torch.float16 if prec == "fp16" else torch.bfloat16
    return torch.from_numpy(np.stack([a.real, a.imag], -1).astype(np.float32)).to(dt).contiguous().cuda()


def _prec(dbp, prec):
    return {"fp32": dbp.DBP_FP32, "fp16": dbp.DBP_FP16, "bf16": dbp.DBP_BF16}[prec]


class Case:
    """One device-resident frame and its descriptor."""

    def __init__(self, dbp, kind, prec, W, N, B, C, U, M, T, seed, rho=1.0):
        self.kind, self.prec = kind, prec
        if kind == "dl":
            f = synth.downlink_frame(W, N, B, U, M, seed=seed)
            self.H, self.inp = _dev(f["H"], prec), _dev(f["s"], prec)
            self.shape = (W, N, B)
            self.d = dbp.frame_desc(B, C, U, W, N, T_max=T, precision=_prec(dbp, prec), rho=rho)
        else:
            f = synth.uplink_frame(W, N, B, U, M, 15.0, seed=seed)
            self.H, self.inp = _dev(f["H"], prec), _dev(f["y"], prec)
            self.shape = (W, N, U)
            self.d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, precision=_prec(dbp, prec),
                                    rho=rho, N0=f["N0"], Es=1.0)
        self.f, self.C, self.T, self.rho = f, C, T, rho

    def run(self, dbp, h, stream=None):
        x = torch.zeros(self.shape, dtype=torch.complex64, device="cuda")
        if self.kind == "dl":
            dbp.dbp_downlink_admm(h, self.d, self.H, self.inp, x, None, stream)
            return x, None
        lab = torch.zeros(self.shape, dtype=torch.uint8, device="cuda")
        dbp.dbp_uplink_admm(h, self.d, self.H, self.inp, x, lab, stream)
        return x, lab


def _run_with(dbp, h, case, prefactor):
    # The operator kernel serves the bulk-copy and downlink tensor-core
    # kernels; uplink ADMM at U = S = 32 would otherwise run on the tcgen05
    # kernel whenever the operator kernel is off, so its comparisons pin the
    # bulk-copy path.
    path = dbp.DBP_PATH_TMA if (case.kind == "admm" and case.shape[2] == 32) else dbp.DBP_PATH_AUTO
    try:
        dbp.dbp_set_tuning(h, kernel=path, prefactor=prefactor)
        out = case.run(dbp, h)
        torch.cuda.synchronize()
    finally:
        dbp.dbp_set_tuning(h)
    return out


CASES = [
    # (kind, prec, W, N, B, C, U, M, T)
    ("admm", "fp32", 301, 14, 256, 8, 32, 64, 3),    # bulk-copy kernel, one staging buffer
    ("admm", "fp16", 301, 14, 256, 8, 32, 64, 3),    # 16-bit inputs, Gram on the tensor cores
    ("admm", "bf16", 150, 14, 256, 8, 32, 64, 4),
    ("admm", "fp16", 97, 13, 128, 8, 16, 16, 4),     # U = 16, ragged N
    ("dl", "fp32", 301, 14, 256, 16, 16, 64, 5),     # tensor-core downlink kernel
    ("dl", "fp32", 97, 14, 128, 4, 32, 16, 3),       # bulk-copy downlink, U = 32, S = 32
    ("dl", "fp32", 61, 9, 64, 4, 16, 16, 2),         # tensor-core downlink, small frame, T = 2
]


@pytest.mark.parametrize("kind,prec,W,N,B,C,U,M,T", CASES)
def test_operator_kernel_gives_the_same_bits(dbp, handle, kind, prec, W, N, B, C, U, M, T):
    case = Case(dbp, kind, prec, W, N, B, C, U, M, T, seed=2100 + W + U)
    off = _run_with(dbp, handle, case, dbp.DBP_PREFACTOR_OFF)
    on = _run_with(dbp, handle, case, dbp.DBP_PREFACTOR_ON)
    auto = _run_with(dbp, handle, case, dbp.DBP_PREFACTOR_AUTO)
    assert torch.equal(off[0], on[0]) and torch.equal(off[0], auto[0])
    if kind != "dl":
        assert torch.equal(off[1], on[1])


def test_operator_kernel_matches_oracle(dbp, handle):
    case = Case(dbp, "admm", "fp32", 64, 14, 256, 8, 32, 64, 3, seed=2200)
    x, _ = _run_with(dbp, handle, case, dbp.DBP_PREFACTOR_ON)
    f = case.f
    H = f["H"].astype(np.complex64).astype(np.complex128)
    y = f["y"].astype(np.complex64).astype(np.complex128)
    ref = oracle.admm_ul(H, y, C=8, rho=1.0, N0=f["N0"], Es=f["Es"], T_max=3, reg=oracle.REG_MMSE)
    xg = x.cpu().numpy().astype(np.complex128)
    rel = np.linalg.norm(xg - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert rel.max() <= FP32_TOL

    dl = Case(dbp, "dl", "fp32", 40, 14, 256, 16, 16, 64, 5, seed=2201)
    xd, _ = _run_with(dbp, handle, dl, dbp.DBP_PREFACTOR_ON)
    Hd = dl.f["H"].astype(np.complex64).astype(np.complex128)
    sd = dl.f["s"].astype(np.complex64).astype(np.complex128)
    refd = oracle.admm_dl(Hd, sd, C=16, rho=1.0, T_max=5)
    xdg = xd.cpu().numpy().astype(np.complex128)
    assert (np.linalg.norm(xdg - refd, axis=-1) / np.linalg.norm(refd, axis=-1)).max() <= FP32_TOL


@pytest.mark.parametrize("kind", ["admm", "dl"])
def test_operator_kernel_fp64_retry(dbp, handle, kind):
    """A near-singular cluster block makes an FP32 pivot fall below 2^-12 of
    the largest diagonal entry: the operator kernel recomputes that cluster
    in FP64 (one retry) and the result matches the run without it."""
    # S = 32 > U = 16: the other clusters stay far from the threshold
    if kind == "admm":
        case = Case(dbp, "admm", "fp16", 12, 14, 256, 8, 16, 16, 3, seed=2300, rho=1e-6)
    else:
        case = Case(dbp, "dl", "fp32", 12, 14, 128, 4, 16, 64, 3, seed=2301, rho=1e6)
    S = case.d.B // case.C
    Hc = case.f["H"][5, S:2 * S]
    u_, s_, vh = np.linalg.svd(Hc, full_matrices=False)
    s_[-1] = 1e-4 * s_[0]
    case.f["H"][5, S:2 * S] = (u_ * s_) @ vh
    case.H = _dev(case.f["H"], case.prec)
    dbp.dbp_fp64_retries(handle)
    on = _run_with(dbp, handle, case, dbp.DBP_PREFACTOR_ON)
    assert dbp.dbp_fp64_retries(handle) == 1
    off = _run_with(dbp, handle, case, dbp.DBP_PREFACTOR_OFF)
    assert dbp.dbp_fp64_retries(handle) == 1
    assert torch.equal(on[0], off[0])


def test_two_streams_with_operator_buffers(dbp, handle):
    """Frames on two streams at once, each call with its own operator buffer
    from the handle's pool: the same bits as the frames one after the other."""
    cases = [Case(dbp, "admm", "fp16", 400, 14, 256, 8, 32, 64, 3, seed=2400 + i) for i in range(4)]
    ref = [_run_with(dbp, handle, c, dbp.DBP_PREFACTOR_ON)[0] for c in cases]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    dbp.dbp_set_tuning(handle, prefactor=dbp.DBP_PREFACTOR_ON)
    try:
        for s in streams:
            s.wait_stream(torch.cuda.current_stream())
        for rep in range(3):
            for i, c in enumerate(cases):
                s = streams[i % 2]
                with torch.cuda.stream(s):
                    outs.append((i, c.run(dbp, handle, s)[0]))
        torch.cuda.synchronize()
    finally:
        dbp.dbp_set_tuning(handle)
    for i, x in outs:
        assert torch.equal(x, ref[i])


def test_tuning_rejects_bad_prefactor(dbp, handle):
    with pytest.raises(dbp.DbpError) as ei:
        dbp.dbp_set_tuning(handle, prefactor=3)
    assert ei.value.status == dbp.DBP_ERR_INVALID_ARG
    dbp.dbp_set_tuning(handle)


def test_operator_kernel_with_power_normalisation(dbp, handle):
    """The downlink with the per-frame power normalisation: x and beta are
    the same bits with and without the operator kernel."""
    f = synth.downlink_frame(120, 14, 256, 16, 64, seed=2500)
    H, s = _dev(f["H"], "fp32"), _dev(f["s"], "fp32")
    d = dbp.frame_desc(256, 16, 16, 120, 14, T_max=4, rho=1.0, flags=dbp.DBP_FLAG_NORMALIZE)
    outs = []
    for pf in (dbp.DBP_PREFACTOR_OFF, dbp.DBP_PREFACTOR_ON):
        x = torch.zeros((120, 14, 256), dtype=torch.complex64, device="cuda")
        beta = torch.zeros(1, dtype=torch.float64, device="cuda")
        try:
            dbp.dbp_set_tuning(handle, prefactor=pf)
            dbp.dbp_downlink_admm(handle, d, H, s, x, beta)
            torch.cuda.synchronize()
        finally:
            dbp.dbp_set_tuning(handle)
        outs.append((x, beta))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    assert abs(float((outs[1][0].abs() ** 2).mean()) - 1.0) < 1e-4
