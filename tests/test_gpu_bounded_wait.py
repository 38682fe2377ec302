"""Every wait of a kernel on its input copies is bounded: a wait that runs
out raises a device status bit, the kernel returns normally and the host
reports DBP_ERR_TIMEOUT.  The test hook dbp_set_test_faults(DBP_TEST_STARVE_COPY)
arms each input copy's mbarrier with more bytes than the copy delivers, so
the barrier never completes, and shortens the wait to about 1 ms: every
persistent bulk-copy kernel must then give up, return and report the
timeout -- without a fault, without a hang -- and the handle keeps working
(the next frame matches the oracle)."""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_04458_b300 as p
    return p


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), 1e-30)


# (name, kernel path, kind, B, C, U): one shape per persistent kernel
KERNELS = [
    ("tc8", "MMA", "ul_admm", 64, 4, 8),
    ("bcast", "BCAST", "ul_cg", 64, 4, 16),
    ("tma", "TMA", "ul_admm", 64, 4, 32),
    ("tcdl", "MMA", "dl_admm", 64, 4, 16),
    ("tc32", "TC5", "ul_admm", 256, 8, 32),
]


@pytest.mark.parametrize("name,path,kind,B,C,U", KERNELS)
def test_starved_copy_wait_runs_out_and_reports_timeout(dbp, name, path, kind, B, C, U):
    h = dbp.dbp_create(0)
    try:
        dbp.dbp_set_tuning(h, kernel=getattr(dbp, "DBP_PATH_" + path))
        W, N, T = 6, 14, 3
        dl = kind == "dl_admm"
        f = synth.downlink_frame(W, N, B, U, 16, seed=77) if dl else synth.uplink_frame(W, N, B, U, 16, 12.0, seed=77)
        H = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
        inp = torch.from_numpy((f["s"] if dl else f["y"]).astype(np.complex64)).cuda()
        x = torch.zeros((W, N, B if dl else U), dtype=torch.complex64, device="cuda")
        d = dbp.frame_desc(B, C, U, W, N, qam_order=0 if dl else 16, T_max=T, N0=f.get("N0", 0.1))

        def call():
            if dl:
                dbp.dbp_downlink_admm(h, d, H, inp, x)
            elif kind == "ul_admm":
                dbp.dbp_uplink_admm(h, d, H, inp, x)
            else:
                dbp.dbp_uplink_cg(h, d, H, inp, x)

        dbp.dbp_device_status(h)                       # nothing pending
        dbp.dbp_set_test_faults(h, dbp.DBP_TEST_STARVE_COPY)
        t0 = time.perf_counter()
        call()
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_device_status(h)                   # waits for the kernel: it returned
        assert ei.value.status == dbp.DBP_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0         # gave up after ~ms, not the default limit
        dbp.dbp_set_test_faults(h, 0)
        dbp.dbp_device_status(h)                       # cleared
        call()
        torch.cuda.synchronize()
        dbp.dbp_device_status(h)                       # a normal frame: no timeout
        Hq = f["H"].astype(np.complex64).astype(np.complex128)
        iq = (f["s"] if dl else f["y"]).astype(np.complex64).astype(np.complex128)
        if dl:
            ref = oracle.admm_dl(Hq, iq, C=C, rho=1.0, T_max=T)
        elif kind == "ul_admm":
            ref = oracle.admm_ul(Hq, iq, C=C, rho=1.0, N0=f["N0"], T_max=T)
        else:
            ref = oracle.cg_ul(Hq, iq, C=C, rho=f["N0"], T_max=T)
        assert _rel(x.cpu().numpy().astype(np.complex128), ref).max() <= 1e-4
    finally:
        dbp.dbp_set_test_faults(h, 0)
        torch.cuda.synchronize()
        dbp.dbp_destroy(h)


def test_host_variant_reports_the_timeout_itself(dbp):
    h = dbp.dbp_create(0)
    try:
        f = synth.uplink_frame(4, 14, 64, 8, 16, 12.0, seed=78)
        Hh, yh = f["H"].astype(np.complex64), f["y"].astype(np.complex64)
        x = np.zeros((4, 14, 8), np.complex64)
        d = dbp.frame_desc(64, 4, 8, 4, 14, qam_order=16, T_max=3, N0=f["N0"])
        dbp.dbp_set_test_faults(h, dbp.DBP_TEST_STARVE_COPY)
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_uplink_admm_host(h, d, Hh, yh, x)
        assert ei.value.status == dbp.DBP_ERR_TIMEOUT
        dbp.dbp_set_test_faults(h, 0)
        dbp.dbp_uplink_admm_host(h, d, Hh, yh, x)      # works again
        with pytest.raises(dbp.DbpError):
            dbp.dbp_set_test_faults(h, 0x80)           # unknown hook
    finally:
        dbp.dbp_set_test_faults(h, 0)
        dbp.dbp_destroy(h)
