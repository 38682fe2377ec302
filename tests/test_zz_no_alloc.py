"""dbp_downlink_admm_static: the downlink precoder with power normalisation
for callers that cannot allocate device memory (a process whose device
memory is reserved by another allocator, or a real-time front end that must
not allocate once running).  Its scratch lives in a fixed library-owned
device array, so it is checked against the allocating entry point
dbp_downlink_admm on two calls in a row (the second call must not be
disturbed by what the first left in the array), and a call is checked to
leave the device's free memory unchanged.

The results do not depend on test order (every call overwrites each scratch
entry it reads); the file name only makes pytest collect it last, so that a
run stopping at the first failure has run every other GPU test before this
optional entry point's."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4   # the FP32 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def dbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_04458_b300 as p
    return p


def _frame(dbp, W, N, B, C, U, M, seed, T):
    f = synth.downlink_frame(W, N, B, U, M, seed=seed)
    H = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
    s = torch.from_numpy(f["s"].astype(np.complex64)).cuda()
    d = dbp.frame_desc(B, C, U, W, N, T_max=T, rho=1.0, flags=dbp.DBP_FLAG_NORMALIZE)
    return H, s, d


def _rel(a, b):
    return float((np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)).max())


def test_static_scratch_matches_allocating_path_twice(dbp):
    h = dbp.dbp_create(0)
    try:
        cases = [(37, 14, 128, 8, 8, 16, 11, 3), (23, 14, 256, 16, 16, 64, 12, 5)]
        for (W, N, B, C, U, M, seed, T) in cases:          # two calls in a row
            H, s, d = _frame(dbp, W, N, B, C, U, M, seed, T)
            x_ref = torch.zeros((W, N, B), dtype=torch.complex64, device="cuda")
            x_new = torch.zeros_like(x_ref)
            b_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
            b_new = torch.zeros(1, dtype=torch.float64, device="cuda")
            dbp.dbp_downlink_admm(h, d, H, s, x_ref, b_ref)
            dbp.dbp_downlink_admm_static(h, d, H, s, x_new, b_new)
            torch.cuda.synchronize()
            xr = x_ref.cpu().numpy().astype(np.complex128)
            xn = x_new.cpu().numpy().astype(np.complex128)
            assert _rel(xn, xr) <= TOL
            assert abs(float(b_new.cpu()[0]) - float(b_ref.cpu()[0])) <= TOL * float(b_ref.cpu()[0])
            assert abs(np.mean(np.abs(xn) ** 2) - 1.0) < 1e-4
    finally:
        torch.cuda.synchronize()
        dbp.dbp_destroy(h)


def test_static_call_allocates_no_device_memory(dbp):
    """After a first call (which looks up the scratch array's address), a
    second call leaves the device's free memory exactly as it was: neither
    the library nor the CUDA runtime allocated anything for it."""
    h = dbp.dbp_create(0)
    try:
        W, N, B, C, U, M, seed, T = 64, 14, 128, 8, 8, 16, 13, 3
        H, s, d = _frame(dbp, W, N, B, C, U, M, seed, T)
        x = torch.zeros((W, N, B), dtype=torch.complex64, device="cuda")
        beta = torch.zeros(1, dtype=torch.float64, device="cuda")
        dbp.dbp_downlink_admm_static(h, d, H, s, x, beta)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        dbp.dbp_downlink_admm_static(h, d, H, s, x, beta)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert float(beta.cpu()[0]) > 0
    finally:
        dbp.dbp_destroy(h)


def test_static_scratch_rejects_oversized_frames(dbp):
    h = dbp.dbp_create(0)
    try:
        d = dbp.frame_desc(16, 4, 4, dbp.DBP_STATIC_MAX_SUBCARRIERS + 1, 1, T_max=2, rho=1.0,
                           flags=dbp.DBP_FLAG_NORMALIZE)
        buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_downlink_admm_static(h, d, buf, buf, buf, None)
        assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED
        assert "exceeds the fixed scratch" in str(ei.value)
    finally:
        dbp.dbp_destroy(h)
