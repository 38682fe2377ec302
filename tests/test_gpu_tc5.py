"""The tcgen05 uplink ADMM kernel (DBP_PATH_TC5: U = S = 32, every dense
product on the fifth-generation tensor cores with FP16 hi / lo operand
pairs) against the FP64 oracle on the same seeded inputs.

Tolerances as for every FP32 kernel: 1e-4 relative per (subcarrier, symbol)
vector against the oracle on the FP32-rounded inputs (16-bit inputs: on the
dequantised inputs); labels bit for bit with the oracle slicer applied to
the kernel's own output in FP32.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def dbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_04458_b300 as p
    return p


@pytest.fixture(scope="module")
def handle(dbp):
    h = dbp.dbp_create(0)
    dbp.dbp_set_tuning(h, kernel=dbp.DBP_PATH_TC5)
    yield h
    torch.cuda.synchronize()
    dbp.dbp_destroy(h)


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), 1e-30)


def _c64(a):
    return a.astype(np.complex64).astype(np.complex128)


def _to16(a, kind):
    dt = torch.float16 if kind == "fp16" else torch.bfloat16
    t = torch.from_numpy(np.stack([a.real, a.imag], axis=-1).astype(np.float32)).to(dt)
    back = t.to(torch.float32).numpy()
    return t.contiguous(), back[..., 0].astype(np.float64) + 1j * back[..., 1].astype(np.float64)


def run(dbp, h, H, y, C, T, M, N0, prec="fp32", reg=None, rho=1.0, box_r=0.0):
    W, N, B = y.shape
    U = H.shape[2]
    if prec == "fp32":
        Hd = torch.from_numpy(H.astype(np.complex64)).cuda()
        yd = torch.from_numpy(y.astype(np.complex64)).cuda()
        Hq, yq = _c64(H), _c64(y)
        code = dbp.DBP_FP32
    else:
        Ht, Hq = _to16(H, prec)
        yt, yq = _to16(y, prec)
        Hd, yd = Ht.cuda(), yt.cuda()
        code = dbp.DBP_FP16 if prec == "fp16" else dbp.DBP_BF16
    x = torch.zeros((W, N, U), dtype=torch.complex64, device="cuda")
    lab = torch.zeros((W, N, U), dtype=torch.uint8, device="cuda")
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, precision=code,
                       regularizer=dbp.DBP_REG_MMSE if reg is None else reg, rho=rho, N0=N0, Es=1.0, box_r=box_r)
    dbp.dbp_uplink_admm(h, d, Hd, yd, x, lab)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128), lab.cpu().numpy(), Hq, yq


CASES = [
    # (W, N, C, T, M, snr)                 covers
    (7, 14, 8, 3, 64, 20.0),             # the B=256 / C=8 / U=32 frame, few subcarriers
    (301, 14, 8, 3, 64, 14.0),           # more subcarriers than CTA slots on a small part
    (13, 16, 4, 4, 16, 10.0),            # B=128, C=4, N=16 (the 16-slot instance)
    (9, 9, 2, 2, 4, 6.0),                # B=64, C=2 (one pair), ragged N
    (5, 1, 8, 1, 64, 25.0),              # N=1, T=1 (init and prox only)
    (4, 14, 8, 6, 256, 30.0),            # T=6, 256-QAM
    (11, 14, 6, 3, 64, 18.0),            # C=6: three pairs, the second Gram round holds one
]


@pytest.mark.parametrize("W,N,C,T,M,snr", CASES)
def test_tc5_fp32_matches_oracle(dbp, handle, W, N, C, T, M, snr):
    B, U = 32 * C, 32
    f = synth.uplink_frame(W, N, B, U, M, snr, seed=9100 + W + N + C)
    x, lab, Hq, yq = run(dbp, handle, f["H"], f["y"], C, T, M, f["N0"])
    ref = oracle.admm_ul(Hq, yq, C=C, rho=1.0, N0=f["N0"], T_max=T)
    err = _rel(x, ref)
    assert err.max() <= TOL, err.max()
    assert np.array_equal(lab, oracle.slice_labels(x, M, dtype=np.float32))


@pytest.mark.parametrize("reg", ["zf", "box", "bpsk"])
def test_tc5_regularisers(dbp, handle, reg):
    C, W, N, T = 8, 11, 14, 4
    M = 2 if reg == "bpsk" else 16
    f = synth.uplink_frame(W, N, 256, 32, M, 8.0, seed=9200)
    r = 1.0 if reg == "bpsk" else oracle.box_radius(M)
    code_d = {"zf": dbp.DBP_REG_ZF, "box": dbp.DBP_REG_BOX, "bpsk": dbp.DBP_REG_BPSK}[reg]
    code_o = {"zf": oracle.REG_ZF, "box": oracle.REG_BOX, "bpsk": oracle.REG_BPSK}[reg]
    x, lab, Hq, yq = run(dbp, handle, f["H"], f["y"], C, T, M, f["N0"], reg=code_d, box_r=r)
    ref = oracle.admm_ul(Hq, yq, C=C, rho=1.0, N0=f["N0"], T_max=T, reg=code_o, box_r=r)
    assert _rel(x, ref).max() <= TOL


@pytest.mark.parametrize("rho", [0.5, 4.0])
def test_tc5_penalty(dbp, handle, rho):
    f = synth.uplink_frame(6, 14, 256, 32, 64, 18.0, seed=9300)
    x, _, Hq, yq = run(dbp, handle, f["H"], f["y"], 8, 5, 64, f["N0"], rho=rho)
    ref = oracle.admm_ul(Hq, yq, C=8, rho=rho, N0=f["N0"], T_max=5)
    assert _rel(x, ref).max() <= TOL


@pytest.mark.parametrize("hs,ys", [(2.0 ** 20, 2.0 ** -30), (2.0 ** -18, 2.0 ** 25), (1e-3, 1e3)])
def test_tc5_input_scale(dbp, handle, hs, ys):
    """The FP16 operand pairs are scaled per operand: channels and receive
    vectors far outside the FP16 range give the same relative accuracy."""
    f = synth.uplink_frame(5, 14, 256, 32, 64, 20.0, seed=9400)
    H, y = f["H"] * hs, f["y"] * ys
    N0 = f["N0"] * hs * hs      # N0 / rho unchanged: every iterate scales by ys / hs
    x, _, Hq, yq = run(dbp, handle, H, y, 8, 3, 64, N0, rho=hs * hs)
    ref = oracle.admm_ul(Hq, yq, C=8, rho=hs * hs, N0=N0, T_max=3)
    assert _rel(x, ref).max() <= TOL


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
@pytest.mark.parametrize("C", [8, 2])
def test_tc5_16bit_inputs(dbp, handle, kind, C):
    f = synth.uplink_frame(9, 14, 32 * C, 32, 64, 20.0, seed=9500 + C)
    x, lab, Hq, yq = run(dbp, handle, f["H"], f["y"], C, 3, 64, f["N0"], prec=kind)
    ref = oracle.admm_ul(Hq, yq, C=C, rho=1.0, N0=f["N0"], T_max=3)
    assert _rel(x, ref).max() <= TOL
    assert np.array_equal(lab, oracle.slice_labels(x, 64, dtype=np.float32))


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("rho", [0.1, 1.0])
def test_tc5_worst_conditioned_square_clusters(dbp, handle, prec, rho):
    """Square clusters (S = U = 32) at 30 dB: every local Gram H_c^H H_c of
    an i.i.d. square block is ill conditioned (its smallest eigenvalue is of
    order 1/S), so B_c = G_c + rho I has condition numbers up to ~4 S^2 / rho
    ... 10^4 at rho = 0.1.  The explicit FP32 inverse still meets the FP32
    tolerance against the FP64 oracle."""
    f = synth.uplink_frame(64, 14, 256, 32, 64, 30.0, seed=9600)
    x, _, Hq, yq = run(dbp, handle, f["H"], f["y"], 8, 3, 64, f["N0"], prec=prec, rho=rho)
    ref = oracle.admm_ul(Hq, yq, C=8, rho=rho, N0=f["N0"], T_max=3)
    err = _rel(x, ref)
    print(f"worst-conditioned {prec} rho={rho}: max {err.max():.3e} median {np.median(err):.3e}")
    assert err.max() <= TOL, err.max()


def test_tc5_fp64_retry(dbp, handle):
    """One user's channel in one cluster of one subcarrier is 1000 times
    stronger than the rest: that cluster's Gram spans seven decades, its FP32
    pivots fall below 2^-12 of the largest diagonal entry, and exactly that
    cluster's operator is recomputed in FP64.  Every subcarrier, the retried
    one included, matches the oracle."""
    W, N, C = 8, 14, 8
    f = synth.uplink_frame(W, N, 256, 32, 64, 20.0, seed=9700)
    f["H"][3, 64:96, 5] *= 1e3                      # subcarrier 3, cluster 2, user 5
    f["y"] = np.einsum("wbu,wnu->wnb", f["H"], f["s"])
    dbp.dbp_fp64_retries(handle)
    x, _, Hq, yq = run(dbp, handle, f["H"], f["y"], C, 3, 64, f["N0"])
    assert dbp.dbp_fp64_retries(handle) == 1
    ref = oracle.admm_ul(Hq, yq, C=C, rho=1.0, N0=f["N0"], T_max=3)
    assert np.all(np.isfinite(x))
    assert _rel(x, ref).max() <= TOL


def test_tc5_full_size_sampled(dbp, handle):
    """The B=256 / C=8 / U=32 / 64-QAM / 3300 x 14 frame in its launch
    configuration; the oracle recomputes 16 sampled subcarriers."""
    W, N, C, T = 3300, 14, 8, 3
    f = synth.uplink_frame(W, N, 256, 32, 64, 20.0, seed=synth.frame_seed(4, 5))
    x, lab, Hq, yq = run(dbp, handle, f["H"], f["y"], C, T, 64, f["N0"])
    idx = np.sort(np.random.default_rng(11).choice(W, size=16, replace=False))
    ref = oracle.admm_ul(Hq[idx], yq[idx], C=C, rho=1.0, N0=f["N0"], T_max=T)
    assert _rel(x[idx], ref).max() <= TOL
    assert np.array_equal(lab, oracle.slice_labels(x, 64, dtype=np.float32))


def test_tc5_rejects_other_shapes(dbp, handle):
    buf = torch.zeros(1 << 16, dtype=torch.complex64, device="cuda")
    for (B, C, U, N) in ((256, 16, 16, 14), (256, 8, 16, 14), (256, 8, 32, 17), (96, 3, 32, 14)):
        d = dbp.frame_desc(B, C, U, 2, N, T_max=2)
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_uplink_admm(handle, d, buf, buf, buf)
        assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED


def test_tc5_is_the_default_for_eligible_shapes(dbp, handle):
    """AUTO runs uplink ADMM at U = S = 32 on the tcgen05 kernel (bit-identical
    to asking for it), and on the bulk-copy kernel when the separate operator
    kernel is asked for (bit-identical to asking for that path)."""
    W, N, C, T, M = 40, 14, 8, 3, 64
    f = synth.uplink_frame(W, N, 32 * C, 32, M, 20.0, seed=9800)
    outs = {}
    for name, kw in (("auto", {}), ("tc5", {"kernel": dbp.DBP_PATH_TC5}),
                     ("auto_pre", {"prefactor": dbp.DBP_PREFACTOR_ON}),
                     ("tma_pre", {"kernel": dbp.DBP_PATH_TMA, "prefactor": dbp.DBP_PREFACTOR_ON})):
        dbp.dbp_set_tuning(handle, **kw)
        try:
            outs[name] = run(dbp, handle, f["H"], f["y"], C, T, M, f["N0"])[:2]
        finally:
            dbp.dbp_set_tuning(handle, kernel=dbp.DBP_PATH_TC5)     # the module's setting
    assert np.array_equal(outs["auto"][0], outs["tc5"][0]) and np.array_equal(outs["auto"][1], outs["tc5"][1])
    assert np.array_equal(outs["auto_pre"][0], outs["tma_pre"][0])
    assert not np.array_equal(outs["auto"][0], outs["auto_pre"][0])     # two different kernels
