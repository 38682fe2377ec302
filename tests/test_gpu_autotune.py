"""Autotuner: it picks a launch choice that accepts the frame, later fully
automatic calls of that shape use it (bit-identical to forcing it), and the
table survives a save / clear / load round trip."""
import os
import tempfile

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbp():
    import paper_1702_04458_b300 as m
    return m


@pytest.fixture()
def handle(dbp):
    h = dbp.dbp_create(0)
    yield h
    dbp.dbp_destroy(h)


def _ul(dbp, W, N, B, C, U, M, T, seed):
    f = synth.uplink_frame(W, N, B, U, M, 12.0, seed=seed)
    d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, N0=f["N0"])
    H = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
    y = torch.from_numpy(f["y"].astype(np.complex64)).cuda()
    return d, H, y


def _run(dbp, h, fn, d, H, y, U):
    x = torch.zeros((d.W, d.N, U), dtype=torch.complex64, device="cuda")
    lab = torch.zeros((d.W, d.N, U), dtype=torch.uint8, device="cuda")
    fn(h, d, H, y, x, lab)
    torch.cuda.synchronize()
    return x, lab


@pytest.mark.parametrize("kind,U,C", [("admm", 8, 8), ("cg", 16, 4), ("admm", 5, 2)])
def test_autotune_choice_is_used_by_auto_calls(dbp, handle, kind, U, C):
    d, H, y = _ul(dbp, 300, 14, 128, C, U, 16, 3 if kind == "admm" else 8, seed=1500 + U)
    k = dbp.DBP_KIND_UPLINK_ADMM if kind == "admm" else dbp.DBP_KIND_UPLINK_CG
    fn = dbp.dbp_uplink_admm if kind == "admm" else dbp.dbp_uplink_cg
    x = torch.zeros((d.W, d.N, U), dtype=torch.complex64, device="cuda")
    best = dbp.dbp_autotune(handle, k, d, H, y, x, None, reps=3)
    assert best.kernel in (dbp.DBP_PATH_MMA, dbp.DBP_PATH_BCAST, dbp.DBP_PATH_TMA, dbp.DBP_PATH_GENERIC)
    # a different W of the same shape uses the tuned choice
    d2, H2, y2 = _ul(dbp, 77, 14, 128, C, U, 16, d.T_max, seed=1600 + U)
    auto = _run(dbp, handle, fn, d2, H2, y2, U)
    dbp.dbp_set_tuning(handle, best.mapping, best.cluster_size, best.warps_per_cta, best.kernel, best.prefactor)
    forced = _run(dbp, handle, fn, d2, H2, y2, U)
    dbp.dbp_set_tuning(handle)
    assert torch.equal(auto[0], forced[0]) and torch.equal(auto[1], forced[1])


def test_autotune_table_round_trip(dbp, handle):
    d, H, y = _ul(dbp, 200, 14, 128, 8, 8, 16, 3, seed=1700)
    x = torch.zeros((d.W, d.N, 8), dtype=torch.complex64, device="cuda")
    best = dbp.dbp_autotune(handle, dbp.DBP_KIND_UPLINK_ADMM, d, H, y, x, None, reps=2)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "tuned.txt")
        dbp.dbp_autotune_save(handle, path)
        line = open(path).read().split()
        assert [int(v) for v in line] == [dbp.DBP_KIND_UPLINK_ADMM, 128, 8, 8, 14, dbp.DBP_FP32, best.mapping,
                                          best.cluster_size, best.warps_per_cta, best.kernel, best.prefactor]
        dbp.dbp_autotune_clear(handle)
        dbp.dbp_autotune_load(handle, path)
        dbp.dbp_autotune_save(handle, path + "2")
        assert open(path + "2").read() == open(path).read()
        bad = os.path.join(tmp, "bad.txt")
        open(bad, "w").write("0 128 8 8 14 0 0 0 0 0\n")        # ten fields
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_autotune_load(handle, bad)
        assert ei.value.status == dbp.DBP_ERR_INVALID_ARG
        with pytest.raises(dbp.DbpError):
            dbp.dbp_autotune_load(handle, os.path.join(tmp, "missing.txt"))


def test_autotune_rejects_bad_requests(dbp, handle):
    d, H, y = _ul(dbp, 10, 2, 32, 4, 4, 4, 2, seed=1800)
    x = torch.zeros((10, 2, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(dbp.DbpError) as ei:
        dbp.dbp_autotune(handle, 7, d, H, y, x)
    assert ei.value.status == dbp.DBP_ERR_INVALID_ARG
    d.C = 3
    with pytest.raises(dbp.DbpError) as ei:
        dbp.dbp_autotune(handle, dbp.DBP_KIND_UPLINK_ADMM, d, H, y, x)
    assert ei.value.status == dbp.DBP_ERR_INVALID_ARG


def test_plan_resolves_the_automatic_choice(dbp, handle):
    """dbp_plan names the kernel AUTO runs (tcgen05 at U = S = 32, the U = 8
    tensor-core kernel), and forcing the planned tuning reproduces the
    automatic call bit for bit."""
    K = dbp.DBP_KIND_UPLINK_ADMM
    d, H, y = _ul(dbp, 40, 14, 256, 8, 32, 64, 3, seed=1900)
    x = torch.zeros((d.W, d.N, 32), dtype=torch.complex64, device="cuda")
    p = dbp.dbp_plan(handle, K, d, H, y, x)
    assert p.kernel == dbp.DBP_PATH_TC5 and p.mapping == dbp.DBP_MAP_CTA and p.cluster_size == 1
    assert p.prefactor == dbp.DBP_PREFACTOR_OFF and p.warps_per_cta == 8
    auto = _run(dbp, handle, dbp.dbp_uplink_admm, d, H, y, 32)
    dbp.dbp_set_tuning(handle, p.mapping, 0, 0, p.kernel, p.prefactor)
    forced = _run(dbp, handle, dbp.dbp_uplink_admm, d, H, y, 32)
    dbp.dbp_set_tuning(handle)
    assert torch.equal(auto[0], forced[0]) and torch.equal(auto[1], forced[1])
    # the U = 8 frame
    d8, H8, y8 = _ul(dbp, 30, 14, 128, 8, 8, 16, 3, seed=1901)
    x8 = torch.zeros((d8.W, d8.N, 8), dtype=torch.complex64, device="cuda")
    assert dbp.dbp_plan(handle, K, d8, H8, y8, x8).kernel == dbp.DBP_PATH_MMA
    # a handle tuning is reported as resolved, never as AUTO
    dbp.dbp_set_tuning(handle, dbp.DBP_MAP_CTA, 0, 0, dbp.DBP_PATH_TMA, dbp.DBP_PREFACTOR_AUTO)
    p = dbp.dbp_plan(handle, K, d, H, y, x)
    dbp.dbp_set_tuning(handle)
    assert p.kernel == dbp.DBP_PATH_TMA and p.prefactor == dbp.DBP_PREFACTOR_OFF


def test_plan_follows_the_autotuned_table_and_rejects_what_calls_reject(dbp, handle):
    K = dbp.DBP_KIND_UPLINK_ADMM
    d, H, y = _ul(dbp, 200, 14, 128, 8, 8, 16, 3, seed=1902)
    x = torch.zeros((d.W, d.N, 8), dtype=torch.complex64, device="cuda")
    best = dbp.dbp_autotune(handle, K, d, H, y, x, None, reps=2)
    p = dbp.dbp_plan(handle, K, d, H, y, x)
    assert p.kernel == best.kernel
    dbp.dbp_autotune_clear(handle)
    with pytest.raises(dbp.DbpError) as ei:
        dbp.dbp_plan(handle, 7, d, H, y, x)
    assert ei.value.status == dbp.DBP_ERR_INVALID_ARG
    dbp.dbp_set_tuning(handle, dbp.DBP_MAP_AUTO, 0, 0, dbp.DBP_PATH_TC5, dbp.DBP_PREFACTOR_AUTO)
    with pytest.raises(dbp.DbpError) as ei:
        dbp.dbp_plan(handle, K, d, H, y, x)            # U = 8: no tcgen05 kernel
    dbp.dbp_set_tuning(handle)
    assert ei.value.status == dbp.DBP_ERR_UNSUPPORTED
