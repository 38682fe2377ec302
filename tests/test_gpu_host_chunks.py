"""Host-buffer entry points on frames large enough to run in chunks of
subcarriers (input copies, kernels and output copies overlapping on three
streams): the results equal those of the device-buffer call on the whole
frame, bit for bit, including a ragged last chunk, 16-bit inputs and the
tcgen05 kernel.  A downlink with power normalisation (a whole-frame pass)
runs unchunked and matches to rounding (its energy sum is in no fixed order)."""
import numpy as np
import pytest
import torch

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
    torch.cuda.synchronize()
    dbp.dbp_destroy(h)


def _host_inputs(a, prec):
    if prec == "fp32":
        return np.ascontiguousarray(a.astype(np.complex64))
    if prec == "fp64":
        return np.ascontiguousarray(a.astype(np.complex128))
    return np.ascontiguousarray(np.stack([a.real, a.imag], -1).astype(np.float16))


UL_CASES = [
    # (algo, W, B, C, U, M, prec): chunks of 16 k subcarriers, at least 256 each
    ("admm", 777, 128, 8, 8, 16, "fp32"),      # 3 chunks, the last one ragged (272, 272, 233)
    ("cg", 1200, 128, 8, 8, 16, "fp32"),       # 4 chunks
    ("admm", 600, 256, 8, 32, 64, "fp32"),     # the tcgen05 kernel, 2 chunks
    ("admm", 600, 256, 8, 32, 64, "fp16"),
    ("admm", 520, 32, 2, 4, 4, "fp64"),        # FP64 (generic kernel), 2 chunks of 272 and 248
]


@pytest.mark.parametrize("algo,W,B,C,U,M,prec", UL_CASES)
def test_chunked_uplink_equals_device_call(dbp, handle, algo, W, B, C, U, M, prec):
    f = synth.uplink_frame(W, 14, B, U, M, 15.0, seed=9950 + W + U)
    H, y = _host_inputs(f["H"], prec), _host_inputs(f["y"], prec)
    code = {"fp32": dbp.DBP_FP32, "fp16": dbp.DBP_FP16, "fp64": dbp.DBP_FP64}[prec]
    d = dbp.frame_desc(B, C, U, W, 14, qam_order=M, T_max=3 if algo == "admm" else 6,
                       precision=code, N0=f["N0"], Es=1.0)
    ct = np.complex128 if prec == "fp64" else np.complex64
    fd = dbp.dbp_uplink_admm if algo == "admm" else dbp.dbp_uplink_cg
    fh = dbp.dbp_uplink_admm_host if algo == "admm" else dbp.dbp_uplink_cg_host
    xd = torch.zeros((W, 14, U), dtype=torch.complex128 if prec == "fp64" else torch.complex64, device="cuda")
    ld = torch.zeros((W, 14, U), dtype=torch.uint8, device="cuda")
    fd(handle, d, torch.from_numpy(H).cuda(), torch.from_numpy(y).cuda(), xd, ld)
    torch.cuda.synchronize()
    xh = np.full((W, 14, U), np.nan, dtype=ct)
    lh = np.full((W, 14, U), 255, dtype=np.uint8)
    fh(handle, d, H, y, xh, lh)
    assert np.array_equal(xh, xd.cpu().numpy())
    assert np.array_equal(lh, ld.cpu().numpy())


@pytest.mark.parametrize("normalize", [False, True])
def test_chunked_downlink_equals_device_call(dbp, handle, normalize):
    W, N, B, C, U = 600, 14, 256, 16, 16
    f = synth.downlink_frame(W, N, B, U, 64, seed=9960)
    H, s = _host_inputs(f["H"], "fp32"), _host_inputs(f["s"], "fp32")
    d = dbp.frame_desc(B, C, U, W, N, T_max=5, flags=dbp.DBP_FLAG_NORMALIZE if normalize else 0)
    xd = torch.zeros((W, N, B), dtype=torch.complex64, device="cuda")
    bd = torch.zeros(1, dtype=torch.float64, device="cuda")
    dbp.dbp_downlink_admm(handle, d, torch.from_numpy(H).cuda(), torch.from_numpy(s).cuda(), xd,
                          bd if normalize else None)
    torch.cuda.synchronize()
    xh = np.full((W, N, B), np.nan, dtype=np.complex64)
    bh = np.zeros(1, dtype=np.float64)
    dbp.dbp_downlink_admm_host(handle, d, H, s, xh, bh if normalize else None)
    if not normalize:
        assert np.array_equal(xh, xd.cpu().numpy())
    else:
        # the frame energy is summed with atomics, in no fixed order: beta and
        # the scaled x agree to rounding
        b = float(bd.cpu()[0])
        assert bh[0] > 0.0 and abs(bh[0] - b) <= 1e-12 * b
        assert np.allclose(xh, xd.cpu().numpy(), rtol=1e-6, atol=0.0)
