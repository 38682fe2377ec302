"""GPU parity of the 16-bit-input path (H and y stored as FP16 or BF16; Gram
and matched filter on the tensor cores with FP32 accumulation; FP32 inverse
and iterations) and of the FP64 inverse retry.

Tolerances: against the FP64 oracle run on the dequantised 16-bit inputs
(which isolates the arithmetic) the bound is the FP32 one, 1e-4 per
(subcarrier, symbol) vector, because every product of two 16-bit inputs is
exact in FP32.  Against the FP32 path on the original inputs the difference
is the input quantisation, bounded by 1e-2 (FP16, 11-bit significand) and
5e-2 (BF16, 8-bit significand) at the SNRs used here.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ARITH_TOL = 1e-4
QUANT_TOL = {"fp16": 1e-2, "bf16": 5e-2}


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


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), 1e-30)


def _to16(a, kind):
    """complex128 [.., ] -> torch tensor [..., 2] of float16 / bfloat16 and
    the dequantised complex128 values."""
    dt = torch.float16 if kind == "fp16" else torch.bfloat16
    t = torch.from_numpy(np.stack([a.real, a.imag], axis=-1).astype(np.float32)).to(dt)
    back = t.to(torch.float32).numpy()
    return t.contiguous(), back[..., 0].astype(np.float64) + 1j * back[..., 1].astype(np.float64)


def run16(dbp, h, f, C, T, algo, kind, H=None, y=None):
    W, N, B, U = f["W"], f["N"], f["B"], f["U"]
    Ht, Hq = _to16(f["H"] if H is None else H, kind)
    yt, yq = _to16(f["y"] if y is None else y, kind)
    Hd, yd = Ht.cuda(), yt.cuda()
    x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
    lab = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
    prec = dbp.DBP_FP16 if kind == "fp16" else dbp.DBP_BF16
    d = dbp.frame_desc(B, C, U, W, N, qam_order=f["M"], T_max=T, precision=prec, rho=f.get("rho", 1.0),
                       N0=f["N0"], Es=1.0)
    (dbp.dbp_uplink_admm if algo == "admm" else dbp.dbp_uplink_cg)(h, d, Hd, yd, x, lab)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128), lab.cpu().numpy(), Hq, yq


def oracle_run(f, C, T, algo, H, y):
    if algo == "admm":
        return oracle.admm_ul(H, y, C=C, rho=f.get("rho", 1.0), N0=f["N0"], T_max=T)
    return oracle.cg_ul(H, y, C=C, rho=f["N0"], T_max=T)


CASES = [
    # (W, N, B, C, U, M, T)
    (11, 14, 256, 8, 32, 64, 3),     # B=256, C=8 clusters of 32, U=32, 64-QAM
    (23, 14, 128, 8, 8, 16, 3),      # U=8
    (9, 14, 256, 16, 16, 64, 4),     # C=16, U=16
    (7, 5, 32, 2, 4, 4, 3),          # U=4, ragged N
    (6, 14, 96, 8, 8, 16, 2),        # S=12 (a multiple of 4, not of 8)
]


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
@pytest.mark.parametrize("algo", ["admm", "cg"])
@pytest.mark.parametrize("W,N,B,C,U,M,T", CASES)
def test_16bit_inputs_match_oracle_on_dequantised_inputs(dbp, handle, kind, algo, W, N, B, C, U, M, T):
    f = synth.uplink_frame(W, N, B, U, M, 20.0, seed=7000 + W + B + U)
    Tr = T if algo == "admm" else T + 4
    x, lab, Hq, yq = run16(dbp, handle, f, C, Tr, algo, kind)
    ref = oracle_run(f, C, Tr, algo, Hq, yq)
    assert _rel(x, ref).max() <= ARITH_TOL, _rel(x, ref).max()
    assert np.array_equal(lab, oracle.slice_labels(x, M, dtype=np.float32))


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_16bit_quantisation_error_against_fp32_path(dbp, handle, kind):
    f = synth.uplink_frame(31, 14, 256, 32, 64, 20.0, seed=7100)
    x16, _, _, _ = run16(dbp, handle, f, 8, 3, "admm", kind)
    H = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
    y = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
    x = torch.zeros((31, 14, 32), dtype=torch.complex64, device="cuda")
    d = dbp.frame_desc(256, 8, 32, 31, 14, qam_order=64, T_max=3, N0=f["N0"])
    dbp.dbp_uplink_admm(handle, d, H, y, x)
    torch.cuda.synchronize()
    x32 = x.cpu().numpy().astype(np.complex128)
    err = _rel(x16, x32)
    assert err.max() <= QUANT_TOL[kind], err.max()


def test_fp64_retry_on_a_near_singular_cluster(dbp, handle):
    """One cluster of one subcarrier is made nearly rank deficient and rho is
    small, so its FP32 Gauss-Jordan pivot falls below 2^-12 of the diagonal:
    exactly that (subcarrier, cluster) is recomputed in FP64, and every other
    subcarrier still matches the oracle."""
    W, N, B, C, U = 12, 14, 256, 8, 16              # S = 32 > U: all other clusters well conditioned
    f = synth.uplink_frame(W, N, B, U, 16, 20.0, seed=7200)
    S = B // C
    Hc = f["H"][3, 2 * S:3 * S]                     # subcarrier 3, cluster 2 (S x U)
    u_, s_, vh = np.linalg.svd(Hc, full_matrices=False)
    s_[-1] = 1e-4 * s_[0]
    f["H"][3, 2 * S:3 * S] = (u_ * s_) @ vh
    f["y"] = np.einsum("wbu,wnu->wnb", f["H"], f["s"])
    f["rho"] = 1e-6
    dbp.dbp_fp64_retries(handle)                    # clear
    x, _, Hq, yq = run16(dbp, handle, f, C, 3, "admm", "fp16")
    assert dbp.dbp_fp64_retries(handle) == 1
    ref = oracle_run(f, C, 3, "admm", Hq, yq)
    good = np.ones(W, dtype=bool)
    good[3] = False
    assert np.all(np.isfinite(x))
    assert _rel(x[good], ref[good]).max() <= 10 * ARITH_TOL


def test_no_retries_on_well_conditioned_frames(dbp, handle):
    f = synth.uplink_frame(40, 14, 256, 32, 64, 10.0, seed=7300)
    dbp.dbp_fp64_retries(handle)
    run16(dbp, handle, f, 8, 3, "admm", "bf16")
    assert dbp.dbp_fp64_retries(handle) == 0


def test_16bit_downlink_is_rejected(dbp, handle):
    buf = torch.zeros(64, dtype=torch.float16, device="cuda")
    d = dbp.frame_desc(16, 2, 4, 1, 1, T_max=2, precision=dbp.DBP_FP16)
    with pytest.raises(dbp.DbpError) as ei:
        dbp.dbp_downlink_admm(handle, d, buf, buf, buf)
    assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_full_size_16bit_sampled(dbp, handle, kind):
    """The bench's mixed workload at full size (B=256, C=8, U=32, 64-QAM,
    3300 x 14, ADMM T=3, 20 dB) in its launch configuration: the oracle on
    the dequantised inputs recomputes 16 sampled subcarriers."""
    W, N, B, C, U, M, T = 3300, 14, 256, 8, 32, 64, 3
    f = synth.uplink_frame(W, N, B, U, M, 20.0, seed=synth.frame_seed(4, 5) + 11)
    x, lab, Hq, yq = run16(dbp, handle, f, C, T, "admm", kind)
    idx = np.sort(np.random.default_rng(7).choice(W, size=16, replace=False))
    sub = dict(f, W=len(idx))
    ref = oracle_run(sub, C, T, "admm", Hq[idx], yq[idx])
    assert _rel(x[idx], ref).max() <= ARITH_TOL


def _run32(dbp, h, f, prec, rho):
    """The B=256 / C=8 / U=32 frame through the automatic kernel choice."""
    W, N = f["W"], f["N"]
    x = torch.zeros((W, N, 32), dtype=torch.complex64, device="cuda")
    if prec == "fp32":
        Hd = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
        yd = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
        Hq = f["H"].astype(np.complex64).astype(np.complex128)
        yq = f["y"].astype(np.complex64).astype(np.complex128)
        code = dbp.DBP_FP32
    else:
        Ht, Hq = _to16(f["H"], prec)
        yt, yq = _to16(f["y"], prec)
        Hd, yd = Ht.cuda(), yt.cuda()
        code = dbp.DBP_FP16 if prec == "fp16" else dbp.DBP_BF16
    d = dbp.frame_desc(256, 8, 32, W, N, qam_order=64, T_max=3, precision=code, rho=rho, N0=f["N0"])
    dbp.dbp_uplink_admm(h, d, Hd, yd, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128), Hq, yq


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("rho", [0.1, 1.0])
def test_worst_conditioned_square_clusters_default_path(dbp, handle, prec, rho):
    """Square clusters (S = U = 32) at 30 dB with small rho: the local Grams
    of i.i.d. square blocks are ill conditioned (smallest eigenvalue of order
    1/S, so condition numbers up to ~4 S^2 / rho), the worst case of the
    explicit FP32 Gauss-Jordan inverse.  The automatic kernel choice (the
    bulk-copy kernel) meets the FP32 tolerance against the FP64 oracle."""
    f = synth.uplink_frame(64, 14, 256, 32, 64, 30.0, seed=9600)
    x, Hq, yq = _run32(dbp, handle, f, prec, rho)
    ref = oracle.admm_ul(Hq, yq, C=8, rho=rho, N0=f["N0"], T_max=3)
    err = _rel(x, ref)
    print(f"default path, worst-conditioned {prec} rho={rho}: max {err.max():.3e} median {np.median(err):.3e}")
    assert err.max() <= ARITH_TOL, err.max()


def test_fp64_retry_at_u32_default_path(dbp, handle):
    """One user 1000 times stronger than the rest in one square cluster: that
    cluster's FP32 pivots fall below 2^-12 of its largest diagonal entry and
    its operator is recomputed in FP64 -- exactly one retry -- and every
    subcarrier, the retried one included, matches the oracle."""
    f = synth.uplink_frame(8, 14, 256, 32, 64, 20.0, seed=9700)
    f["H"][3, 64:96, 5] *= 1e3
    f["y"] = np.einsum("wbu,wnu->wnb", f["H"], f["s"])
    dbp.dbp_fp64_retries(handle)
    x, Hq, yq = _run32(dbp, handle, f, "fp32", 1.0)
    assert dbp.dbp_fp64_retries(handle) == 1
    ref = oracle.admm_ul(Hq, yq, C=8, rho=1.0, N0=f["N0"], T_max=3)
    assert _rel(x, ref).max() <= ARITH_TOL
