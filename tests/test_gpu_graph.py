"""A batch of frames of mixed kinds and shapes captured into one CUDA graph
(dbp_graph_create) gives, launch after launch, the results of the same
frames issued one by one."""
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
    dbp.dbp_destroy(h)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


# (kind, W, N, B, C, U, M, T, normalise)
MIX = [
    ("admm", 120, 14, 128, 8, 8, 16, 3, False),     # tensor-core uplink kernel
    ("cg", 60, 14, 64, 4, 16, 64, 6, False),        # broadcast CG kernel, U = 16
    ("dl", 50, 14, 256, 16, 16, 64, 5, True),       # tensor-core downlink kernel, normalised
    ("admm", 33, 5, 80, 2, 5, 16, 4, False),        # generic kernel (U = 5)
    ("dl", 40, 14, 64, 4, 8, 16, 3, False),         # bulk-copy downlink kernel, U = 8
    ("cg", 17, 20, 32, 2, 4, 4, 5, False),          # two symbol chunks
]


def _frames(dbp, seed0):
    out = []
    for i, (kind, W, N, B, C, U, M, T, norm) in enumerate(MIX):
        if kind == "dl":
            f = synth.downlink_frame(W, N, B, U, M, seed=seed0 + i)
            d = dbp.frame_desc(B, C, U, W, N, T_max=T, flags=dbp.DBP_FLAG_NORMALIZE if norm else 0)
            fr = dict(kind=dbp.DBP_KIND_DOWNLINK_ADMM, desc=d, H=_dev(f["H"]), inp=_dev(f["s"]),
                      out=torch.zeros((W, N, B), dtype=torch.complex64, device="cuda"), labels=None,
                      beta=torch.zeros(1, dtype=torch.float64, device="cuda") if norm else None)
        else:
            f = synth.uplink_frame(W, N, B, U, M, 12.0, seed=seed0 + i)
            d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, N0=f["N0"])
            fr = dict(kind=dbp.DBP_KIND_UPLINK_ADMM if kind == "admm" else dbp.DBP_KIND_UPLINK_CG, desc=d,
                      H=_dev(f["H"]), inp=_dev(f["y"]),
                      out=torch.zeros((W, N, U), dtype=torch.complex64, device="cuda"),
                      labels=torch.zeros((W, N, U), dtype=torch.uint8, device="cuda"), beta=None)
        out.append(fr)
    return out


def _one_by_one(dbp, h, frames):
    res = []
    for fr in frames:
        o = torch.zeros_like(fr["out"])
        lab = torch.zeros_like(fr["labels"]) if fr["labels"] is not None else None
        beta = torch.zeros_like(fr["beta"]) if fr["beta"] is not None else None
        if fr["kind"] == dbp.DBP_KIND_DOWNLINK_ADMM:
            dbp.dbp_downlink_admm(h, fr["desc"], fr["H"], fr["inp"], o, beta)
        elif fr["kind"] == dbp.DBP_KIND_UPLINK_ADMM:
            dbp.dbp_uplink_admm(h, fr["desc"], fr["H"], fr["inp"], o, lab)
        else:
            dbp.dbp_uplink_cg(h, fr["desc"], fr["H"], fr["inp"], o, lab)
        res.append((o, lab, beta))
    torch.cuda.synchronize()
    return res


def _items(dbp, frames):
    return [dbp.graph_item(fr["kind"], fr["desc"], fr["H"], fr["inp"], fr["out"], fr["labels"], fr["beta"])
            for fr in frames]


@pytest.mark.parametrize("branches", [1, 4])
def test_graph_of_mixed_frames_equals_single_calls(dbp, handle, branches):
    frames = _frames(dbp, 1100)
    ref = _one_by_one(dbp, handle, frames)
    g = dbp.dbp_graph_create(handle, _items(dbp, frames), branches)
    try:
        for _ in range(2):
            for fr in frames:
                fr["out"].zero_()
            g.launch()
            torch.cuda.synchronize()
            for fr, (o, lab, beta) in zip(frames, ref):
                assert torch.equal(fr["out"], o)
                if lab is not None:
                    assert torch.equal(fr["labels"], lab)
                if beta is not None:
                    assert torch.equal(fr["beta"], beta)
    finally:
        g.close()
    dbp.dbp_device_status(handle)              # no device-side timeout


def test_graph_recomputes_from_new_inputs(dbp, handle):
    frames = _frames(dbp, 1200)
    g = dbp.dbp_graph_create(handle, _items(dbp, frames))
    try:
        g.launch()
        newer = _frames(dbp, 1300)
        for fr, nf in zip(frames, newer):          # new data in the captured buffers
            fr["H"].copy_(nf["H"])
            fr["inp"].copy_(nf["inp"])
        g.launch()
        torch.cuda.synchronize()
        ref = _one_by_one(dbp, handle, newer)
        for fr, (o, lab, beta) in zip(frames, ref):
            assert torch.equal(fr["out"], o)
    finally:
        g.close()


def test_graph_rejects_a_bad_item(dbp, handle):
    frames = _frames(dbp, 1400)
    items = _items(dbp, frames)
    items[2].desc.C = 7                             # B = 256 is not a multiple of 7
    with pytest.raises(dbp.DbpError) as ei:
        dbp.dbp_graph_create(handle, items)
    assert ei.value.status == dbp.DBP_ERR_INVALID_ARG
    assert "item 2" in dbp.dbp_last_error(handle)
    with pytest.raises(dbp.DbpError):
        dbp.dbp_graph_create(handle, items[:1], branches=17)


def test_graph_with_operator_kernel_tuning(dbp, handle):
    """With DBP_PREFACTOR_ON on the handle, frames captured into a graph run
    without the separate operator kernel (no stream-ordered buffer inside a
    capture) and still equal the single calls, which do use it."""
    frames = _frames(dbp, 1500)
    f = synth.downlink_frame(64, 14, 256, 16, 64, seed=1510)          # tensor-core downlink
    frames.append(dict(kind=dbp.DBP_KIND_DOWNLINK_ADMM, desc=dbp.frame_desc(256, 16, 16, 64, 14, T_max=4),
                       H=_dev(f["H"]), inp=_dev(f["s"]),
                       out=torch.zeros((64, 14, 256), dtype=torch.complex64, device="cuda"),
                       labels=None, beta=None))
    dbp.dbp_set_tuning(handle, prefactor=dbp.DBP_PREFACTOR_ON)
    try:
        ref = _one_by_one(dbp, handle, frames)
        g = dbp.dbp_graph_create(handle, _items(dbp, frames), 2)
        try:
            g.launch()
            torch.cuda.synchronize()
            for fr, (o, lab, beta) in zip(frames, ref):
                assert torch.equal(fr["out"], o)
        finally:
            g.close()
    finally:
        dbp.dbp_set_tuning(handle)
