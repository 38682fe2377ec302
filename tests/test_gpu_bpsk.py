"""The BPSK prox of Alg. 1 (DBP_REG_BPSK): s_u = sign(Re v_u) min(|Re v_u|, r),
Im s_u = 0, in every uplink ADMM kernel against the FP64 oracle on the same
inputs, with BPSK labels (qam_order 2) from the kernel's own estimate."""
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


def _inputs(a, prec):
    """Device copy of a complex array and the values the kernel sees."""
    if prec in ("fp32", "fp64"):
        ct = np.complex64 if prec == "fp32" else np.complex128
        seen = a.astype(ct).astype(np.complex128)
        return torch.from_numpy(a.astype(ct)).cuda(), seen
    dt = torch.float16 if prec == "fp16" else torch.bfloat16
    t = torch.from_numpy(np.stack([a.real, a.imag], -1).astype(np.float32)).to(dt).contiguous()
    q = t.float().numpy().astype(np.float64)
    return t.cuda(), q[..., 0] + 1j * q[..., 1]


CASES = [
    # (kernel path, precision, W, N, B, C, U, T)
    ("mma", "fp32", 23, 14, 128, 8, 8, 4),      # tensor-core kernel
    ("bcast", "fp32", 21, 14, 128, 8, 16, 4),   # CUDA-core kernel, U = 16
    ("bcast", "fp32", 17, 9, 64, 4, 4, 3),      # U = 4, ragged N
    ("generic", "fp32", 19, 14, 128, 8, 8, 4),  # generic fused kernel
    ("auto", "fp32", 13, 14, 256, 8, 32, 3),    # bulk-copy kernel, FP32 inputs at U = 32
    ("auto", "fp16", 13, 14, 256, 8, 32, 3),    # bulk-copy kernel, 16-bit inputs
    ("auto", "bf16", 11, 14, 128, 8, 16, 4),
    ("generic", "fp64", 9, 5, 32, 2, 4, 5),     # FP64 kernel
]


@pytest.mark.parametrize("path,prec,W,N,B,C,U,T", CASES)
def test_bpsk_prox_matches_oracle(dbp, handle, path, prec, W, N, B, C, U, T):
    f = synth.uplink_frame(W, N, B, U, 2, 4.0, seed=3100 + U + W)
    Hd, H = _inputs(f["H"], prec)
    yd, y = _inputs(f["y"], prec)
    r = oracle.box_radius(2)
    code = {"fp32": dbp.DBP_FP32, "fp64": dbp.DBP_FP64, "fp16": dbp.DBP_FP16, "bf16": dbp.DBP_BF16}[prec]
    d = dbp.frame_desc(B, C, U, W, N, qam_order=2, T_max=T, regularizer=dbp.DBP_REG_BPSK, precision=code,
                       rho=1.0, N0=f["N0"], Es=1.0, box_r=r)
    xd = torch.zeros((W, N, U), dtype=torch.complex128 if prec == "fp64" else torch.complex64, device="cuda")
    ld = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
    kernel = {"mma": dbp.DBP_PATH_MMA, "bcast": dbp.DBP_PATH_BCAST, "generic": dbp.DBP_PATH_GENERIC,
              "auto": dbp.DBP_PATH_AUTO}[path]
    try:
        dbp.dbp_set_tuning(handle, kernel=kernel)
        dbp.dbp_uplink_admm(handle, d, Hd, yd, xd, ld)
        torch.cuda.synchronize()
    finally:
        dbp.dbp_set_tuning(handle)
    x = xd.cpu().numpy().astype(np.complex128)
    lab = ld.cpu().numpy()
    ref = oracle.admm_ul(H, y, C=C, rho=1.0, N0=f["N0"], Es=1.0, T_max=T, reg=oracle.REG_BPSK, box_r=r)
    rel = np.linalg.norm(x - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert rel.max() <= (FP64_TOL if prec == "fp64" else FP32_TOL), rel.max()
    # the prox leaves no imaginary part, and the segment bound is active at 4 dB
    assert np.all(x.imag == 0.0)
    assert np.all(np.abs(x.real) <= r) and np.any(np.abs(x.real) == r)
    # labels: the oracle's BPSK slicer on the kernel's own estimate, in its precision,
    # and the oracle's labels wherever its estimate is not within 1e-3 of the boundary
    dt = np.float64 if prec == "fp64" else np.float32
    assert np.array_equal(lab, oracle.slice_labels(x, 2, dtype=dt))
    clear = np.abs(ref.real) > 1e-3
    assert np.array_equal(lab[clear], oracle.slice_labels(ref, 2)[clear])


def test_bpsk_beats_zf_at_low_snr(dbp, handle):
    """Per Sec. III-A the constrained equaliser outperforms the linear one: on
    a BPSK frame at 0 dB the BPSK prox makes fewer bit errors than ZF."""
    W, N, B, C, U = 300, 14, 32, 4, 16
    f = synth.uplink_frame(W, N, B, U, 2, 0.0, seed=3200)
    Hd = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
    yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
    errs = {}
    for name, reg in (("zf", dbp.DBP_REG_ZF), ("bpsk", dbp.DBP_REG_BPSK)):
        d = dbp.frame_desc(B, C, U, W, N, qam_order=0, T_max=30, regularizer=reg, rho=1.0, N0=f["N0"], Es=1.0,
                           box_r=1.0)
        xd = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
        dbp.dbp_uplink_admm(handle, d, Hd, yd, xd, None)
        torch.cuda.synchronize()
        lab = oracle.slice_labels(xd.cpu().numpy(), 2, dtype=np.float32)
        errs[name] = oracle.bit_errors(lab, f["labels"])
    assert errs["bpsk"] < errs["zf"], errs


@pytest.mark.parametrize("kind,bad", [
    ("admm", dict(qam_order=2)),                                         # BPSK labels with the MMSE prox
    ("admm", dict(regularizer=3, qam_order=16, box_r=1.0)),              # the BPSK prox slices BPSK only
    ("admm", dict(regularizer=3, qam_order=2, box_r=0.0)),               # no radius
    ("admm", dict(regularizer=3, qam_order=2, box_r=float("inf"))),
    ("cg", dict(regularizer=3, qam_order=2, box_r=1.0)),                 # CG takes ZF / MMSE only
    ("cg", dict(qam_order=2)),
    ("dl", dict(qam_order=2)),
])
def test_bpsk_descriptor_checks(dbp, handle, kind, bad):
    kw = dict(B=32, C=4, U=4, W=3, N=2, qam_order=4, T_max=2, N0=0.1)
    kw.update(bad)
    d = dbp.frame_desc(**kw)
    buf = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    fn = {"admm": dbp.dbp_uplink_admm, "cg": dbp.dbp_uplink_cg, "dl": dbp.dbp_downlink_admm}[kind]
    with pytest.raises(dbp.DbpError) as ei:
        fn(handle, d, buf, buf, buf, None)
    assert ei.value.status == dbp.DBP_ERR_INVALID_ARG


def test_bpsk_full_size_sampled(dbp, handle):
    """B=128, C=8, U=8, BPSK, 1200 x 14 at -6 dB, ADMM T=3 with the BPSK prox
    (the bench's bpsk_prox line): the whole frame on the GPU, the oracle on
    48 sampled subcarriers; labels from the kernel's estimate."""
    W, N, B, C, U, T = 1200, 14, 128, 8, 8, 3
    f = synth.uplink_frame(W, N, B, U, 2, -6.0, seed=synth.frame_seed(2, 90))
    Hd = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
    yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
    d = dbp.frame_desc(B, C, U, W, N, qam_order=2, T_max=T, regularizer=dbp.DBP_REG_BPSK, rho=1.0, N0=f["N0"],
                       Es=1.0, box_r=1.0)
    xd = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
    ld = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
    dbp.dbp_uplink_admm(handle, d, Hd, yd, xd, ld)
    torch.cuda.synchronize()
    x, lab = xd.cpu().numpy().astype(np.complex128), ld.cpu().numpy()
    idx = np.sort(np.random.default_rng(10).choice(W, size=48, replace=False))
    H = f["H"][idx].astype(np.complex64).astype(np.complex128)
    y = f["y"][idx].astype(np.complex64).astype(np.complex128)
    ref = oracle.admm_ul(H, y, C=C, rho=1.0, N0=f["N0"], Es=1.0, T_max=T, reg=oracle.REG_BPSK, box_r=1.0)
    rel = np.linalg.norm(x[idx] - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert rel.max() <= FP32_TOL
    assert np.array_equal(lab, oracle.slice_labels(x, 2, dtype=np.float32))
    assert np.all(x.imag == 0.0)
