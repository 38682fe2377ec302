"""The request loop (dbp_server_start / dbp_submit / dbp_poll / dbp_wait /
dbp_cancel): every frame's result is the same alone and in a mix of uneven
frames whose work is in flight on the device at the same time; frames of one
coherence block reuse the resident channel and per-cluster operator; a pool
too small for all frames at once still completes every frame; frames that
could never fit the pool and bad requests are refused at submission; queued
frames can be cancelled; requests on caller-owned device buffers run in
place; the handle's HBM budget caps the library's own allocations."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_04458_b300 as p
    return p


def _pin(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def _c16(a, kind):
    dt = torch.float16 if kind == "fp16" else torch.bfloat16
    t = torch.from_numpy(np.stack([a.real, a.imag], -1).astype(np.float32)).to(dt)
    return t.contiguous().pin_memory()


class Frame:
    """One served frame: host inputs, host outputs and its descriptor."""

    def __init__(self, dbp, kind, B, C, U, W, N, M, T, seed, prec="fp32", key=0, epoch=0, H=None):
        self.kind, self.prec = kind, prec
        if kind == dbp.DBP_KIND_DOWNLINK_ADMM:
            f = synth.downlink_frame(W, N, B, U, M, seed=seed)
            inp = f["s"]
        else:
            f = synth.uplink_frame(W, N, B, U, M, 15.0, seed=seed)
            inp = f["y"]
        if H is not None:
            f["H"] = H
            if kind != dbp.DBP_KIND_DOWNLINK_ADMM:
                inp = np.einsum("wbu,wnu->wnb", H, f["s"])
        self.Hc = f["H"]
        if prec == "fp32":
            self.H, self.inp = _pin(f["H"].astype(np.complex64)), _pin(inp.astype(np.complex64))
            p = dbp.DBP_FP32
        else:
            self.H, self.inp = _c16(f["H"], prec), _c16(inp, prec)
            p = dbp.DBP_FP16 if prec == "fp16" else dbp.DBP_BF16
        shape = (W, N, B) if kind == dbp.DBP_KIND_DOWNLINK_ADMM else (W, N, U)
        self.out = _pin(np.zeros(shape, dtype=np.complex64))
        self.lab = _pin(np.zeros((W, N, U), dtype=np.uint8))
        self.desc = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, precision=p, rho=1.0,
                                   N0=f.get("N0", 0.1), Es=1.0)
        self.key, self.epoch = key, epoch

    def request(self, dbp, tag):
        lab = self.lab if self.kind != dbp.DBP_KIND_DOWNLINK_ADMM else None
        return dbp.request(self.kind, self.desc, self.H, self.inp, self.out, lab, None,
                           self.key, self.epoch, tag)

    def run_alone(self, dbp, h):
        """The same frame through the synchronous host-buffer entry points."""
        out = np.zeros_like(self.out)
        lab = np.zeros_like(self.lab)
        if self.kind == dbp.DBP_KIND_DOWNLINK_ADMM:
            dbp.dbp_downlink_admm_host(h, self.desc, self.H, self.inp, out)
        elif self.kind == dbp.DBP_KIND_UPLINK_ADMM:
            dbp.dbp_uplink_admm_host(h, self.desc, self.H, self.inp, out, lab)
        else:
            dbp.dbp_uplink_cg_host(h, self.desc, self.H, self.inp, out, lab)
        return out, lab


def _mix(dbp):
    K = dbp
    specs = [
        (K.DBP_KIND_UPLINK_ADMM, 128, 8, 8, 300, 14, 16, 3, "fp32"),
        (K.DBP_KIND_UPLINK_CG, 128, 8, 8, 600, 14, 16, 8, "fp32"),
        (K.DBP_KIND_DOWNLINK_ADMM, 256, 16, 16, 300, 14, 64, 5, "fp32"),
        (K.DBP_KIND_UPLINK_ADMM, 256, 8, 32, 300, 14, 64, 3, "fp16"),
        (K.DBP_KIND_UPLINK_CG, 64, 4, 4, 1200, 14, 16, 4, "fp32"),
        (K.DBP_KIND_UPLINK_ADMM, 64, 1, 16, 300, 14, 64, 6, "fp32"),      # C=1, S=64
        (K.DBP_KIND_DOWNLINK_ADMM, 128, 2, 32, 300, 14, 16, 3, "fp32"),   # S=64 > U
        (K.DBP_KIND_UPLINK_ADMM, 256, 16, 16, 600, 14, 64, 4, "bf16"),
        (K.DBP_KIND_UPLINK_CG, 256, 16, 32, 300, 14, 64, 5, "fp32"),      # cluster mapping
        (K.DBP_KIND_UPLINK_ADMM, 128, 4, 5, 300, 14, 16, 3, "fp32"),      # U=5: generic kernel
    ]
    return [Frame(dbp, *sp[:8], seed=900 + i, prec=sp[8]) for i, sp in enumerate(specs)]


def test_results_are_the_same_alone_and_in_the_mix(dbp):
    h = dbp.dbp_create(0)
    try:
        frames = _mix(dbp)
        alone = [f.run_alone(dbp, h) for f in frames]
        dbp.dbp_server_start(h, streams=4)
        tickets = [dbp.dbp_submit(h, f.request(dbp, i)) for i, f in enumerate(frames)]
        results = [dbp.dbp_wait(h, t, 120.0) for t in tickets]
        dbp.dbp_server_stop(h)
        for i, (f, r) in enumerate(zip(frames, results)):
            assert r is not None and r.status == dbp.DBP_OK and r.user_tag == i
            assert r.submit_us <= r.start_us <= r.finish_us
            # same kernels, same shape: bit-identical
            assert np.array_equal(f.out, alone[i][0]), i
            if f.kind != dbp.DBP_KIND_DOWNLINK_ADMM:
                assert np.array_equal(f.lab, alone[i][1]), i
        # the frames were in flight together: some admitted frame's
        # [start, finish] interval (work enqueued on its stream .. completion
        # seen) overlaps another's
        iv = sorted((r.start_us, r.finish_us) for r in results)
        overlaps = sum(1 for a in range(len(iv)) for b in range(a + 1, len(iv)) if iv[b][0] < iv[a][1])
        assert overlaps >= 1, iv
    finally:
        dbp.dbp_destroy(h)


def test_coherence_block_reuses_resident_channel(dbp):
    h = dbp.dbp_create(0)
    try:
        K = dbp.DBP_KIND_UPLINK_ADMM
        first = Frame(dbp, K, 128, 8, 8, 1200, 14, 16, 3, seed=1, key=77, epoch=3)
        block = [first] + [Frame(dbp, K, 128, 8, 8, 1200, 14, 16, 3, seed=2 + i, key=77, epoch=3, H=first.Hc)
                           for i in range(3)]
        dl = Frame(dbp, dbp.DBP_KIND_DOWNLINK_ADMM, 128, 8, 8, 1200, 14, 16, 4, seed=9, key=77, epoch=3,
                   H=first.Hc)
        alone = [f.run_alone(dbp, h) for f in block + [dl]]
        dbp.dbp_server_start(h, streams=2)
        hits = []
        for f in block + [dl]:                       # one after the other
            r = dbp.dbp_wait(h, dbp.dbp_submit(h, f.request(dbp, 0)), 60.0)
            assert r.status == dbp.DBP_OK
            hits.append(r.resident_hit)
        # a new epoch of the same key replaces the resident channel
        nxt = Frame(dbp, K, 128, 8, 8, 1200, 14, 16, 3, seed=20, key=77, epoch=4)
        r = dbp.dbp_wait(h, dbp.dbp_submit(h, nxt.request(dbp, 0)), 60.0)
        hits.append(r.resident_hit)
        ref_next = nxt.run_alone(dbp, h)
        dbp.dbp_server_stop(h)
        assert hits == [0, 1, 1, 1, 1, 0]
        for f, a in zip(block + [dl], alone):
            # the resident operator is the one the first frame computed:
            # identical arithmetic, identical results
            assert np.array_equal(f.out, a[0])
        assert np.array_equal(nxt.out, ref_next[0])
    finally:
        dbp.dbp_destroy(h)


def test_small_pool_admits_frames_as_memory_frees(dbp):
    h = dbp.dbp_create(0)
    try:
        K = dbp.DBP_KIND_UPLINK_CG
        frames = [Frame(dbp, K, 128, 8, 8, 1200, 14, 16, 6, seed=40 + i) for i in range(6)]
        alone = [f.run_alone(dbp, h) for f in frames]
        per = frames[0].H.nbytes + frames[0].inp.nbytes + frames[0].out.nbytes + frames[0].lab.nbytes
        dbp.dbp_server_start(h, streams=4, hbm_bytes=int(per * 1.6))   # room for one frame at a time
        tickets = [dbp.dbp_submit(h, f.request(dbp, i)) for i, f in enumerate(frames)]
        res = [dbp.dbp_wait(h, t, 120.0) for t in tickets]
        dbp.dbp_server_stop(h)
        for f, a, r in zip(frames, alone, res):
            assert r.status == dbp.DBP_OK
            assert np.array_equal(f.out, a[0])
        # one frame at a time: each starts after the previous one finished
        starts = sorted((r.start_us, r.finish_us) for r in res)
        for (s0, f0), (s1, f1) in zip(starts, starts[1:]):
            assert s1 >= f0 - 50.0
    finally:
        dbp.dbp_destroy(h)


def test_submission_errors_and_waits(dbp):
    h = dbp.dbp_create(0)
    try:
        dbp.dbp_server_start(h)
        f = Frame(dbp, dbp.DBP_KIND_UPLINK_ADMM, 128, 8, 8, 1200, 14, 16, 3, seed=60)
        bad = f.request(dbp, 0)
        bad.desc.C = 7                              # 128 % 7 != 0
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_submit(h, bad)
        assert ei.value.status == dbp.DBP_ERR_INVALID_ARG
        t = dbp.dbp_submit(h, f.request(dbp, 5))
        assert dbp.dbp_wait(h, t, 0.0) is None      # cannot be done yet
        r = dbp.dbp_wait(h, t, 60.0)
        assert r.status == dbp.DBP_OK and r.user_tag == 5
        with pytest.raises(dbp.DbpError):
            dbp.dbp_poll(h, t)                      # released
        dbp.dbp_server_stop(h)
    finally:
        dbp.dbp_destroy(h)


def test_box_and_bpsk_frames_through_the_request_loop(dbp):
    """Frames with the BOX and BPSK proxes (BPSK labels, qam_order 2) in a mix
    with an MMSE frame: each result is bit-identical to the same frame alone."""
    K = dbp
    bpsk = Frame(dbp, K.DBP_KIND_UPLINK_ADMM, 128, 8, 8, 300, 14, 2, 3, seed=950)
    bpsk.desc.regularizer, bpsk.desc.box_r = K.DBP_REG_BPSK, 1.0
    box = Frame(dbp, K.DBP_KIND_UPLINK_ADMM, 128, 8, 8, 600, 14, 16, 3, seed=951)
    box.desc.regularizer, box.desc.box_r = K.DBP_REG_BOX, float(3 * np.sqrt(3.0 / 30.0))
    mmse = Frame(dbp, K.DBP_KIND_UPLINK_ADMM, 256, 8, 32, 300, 14, 64, 3, seed=952)
    frames = [bpsk, box, mmse]
    h = dbp.dbp_create(0)
    try:
        alone = [f.run_alone(dbp, h) for f in frames]
        dbp.dbp_server_start(h, streams=3)
        tickets = [dbp.dbp_submit(h, f.request(dbp, i)) for i, f in enumerate(frames)]
        results = [dbp.dbp_wait(h, t, 120.0) for t in tickets]
        dbp.dbp_server_stop(h)
        for i, (f, r) in enumerate(zip(frames, results)):
            assert r is not None and r.status == dbp.DBP_OK and r.user_tag == i
            assert np.array_equal(f.out, alone[i][0]), i
            assert np.array_equal(f.lab, alone[i][1]), i
        assert np.all(bpsk.out.imag == 0.0) and set(np.unique(bpsk.lab)) <= {0, 1}
    finally:
        dbp.dbp_destroy(h)


def test_frame_larger_than_the_pool_is_refused(dbp):
    """A frame whose staged inputs and outputs alone exceed the pool is
    refused by dbp_submit with DBP_ERR_NOMEM instead of blocking the loop;
    frames submitted after it still run."""
    h = dbp.dbp_create(0)
    try:
        big = Frame(dbp, dbp.DBP_KIND_UPLINK_ADMM, 256, 8, 32, 300, 14, 64, 3, seed=70)    # ~27 MB staged
        small = Frame(dbp, dbp.DBP_KIND_UPLINK_ADMM, 64, 4, 8, 300, 14, 16, 3, seed=71)
        ref = small.run_alone(dbp, h)
        dbp.dbp_server_start(h, streams=2, hbm_bytes=16 << 20)
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_submit(h, big.request(dbp, 0))
        assert ei.value.status == dbp.DBP_ERR_NOMEM
        assert "pool" in str(ei.value)
        r = dbp.dbp_wait(h, dbp.dbp_submit(h, small.request(dbp, 1)), 60.0)
        dbp.dbp_server_stop(h)
        assert r is not None and r.status == dbp.DBP_OK
        assert np.array_equal(small.out, ref[0])
    finally:
        dbp.dbp_destroy(h)


def test_cancel_a_queued_frame(dbp):
    """One slot, several large frames submitted back to back: the last one is
    still queued when it is cancelled; its ticket finishes with
    DBP_ERR_CANCELLED and the others complete with their normal results."""
    h = dbp.dbp_create(0)
    try:
        K = dbp.DBP_KIND_UPLINK_ADMM
        frames = [Frame(dbp, K, 256, 8, 32, 1200, 14, 64, 3, seed=80 + i) for i in range(5)]
        ref = frames[0].run_alone(dbp, h)
        dbp.dbp_server_start(h, streams=1)
        tickets = [dbp.dbp_submit(h, f.request(dbp, i)) for i, f in enumerate(frames)]
        assert dbp.dbp_cancel(h, tickets[-1]) is True
        res = [dbp.dbp_wait(h, t, 120.0) for t in tickets]
        dbp.dbp_server_stop(h)
        assert [r.status for r in res[:-1]] == [dbp.DBP_OK] * 4
        assert res[-1].status == dbp.DBP_ERR_CANCELLED
        assert np.all(frames[-1].out == 0)               # nothing ran for it
        assert np.array_equal(frames[0].out, ref[0])
        with pytest.raises(dbp.DbpError):
            dbp.dbp_cancel(h, tickets[0])              # finished and released
    finally:
        dbp.dbp_destroy(h)


def test_device_buffer_requests_run_in_place(dbp):
    """Requests flagged DBP_REQ_DEVICE_BUFFERS run on the caller's CUDA
    buffers with no host copies: results bit-identical to the synchronous
    device-pointer entry points on the same kernel path, also when a
    coherence block reuses the resident operator.  (A resident operator
    needs the bulk-copy kernel, so the loop runs uplink ADMM at U = S = 32
    there, where a synchronous call defaults to the tcgen05 kernel; the
    reference pins that path.)"""
    h = dbp.dbp_create(0)
    try:
        K = dbp
        specs = [(K.DBP_KIND_UPLINK_ADMM, 256, 8, 32, 300, 64, 3), (K.DBP_KIND_UPLINK_CG, 128, 8, 8, 600, 16, 8),
                 (K.DBP_KIND_DOWNLINK_ADMM, 256, 16, 16, 300, 64, 5), (K.DBP_KIND_UPLINK_ADMM, 256, 16, 16, 300, 64, 4)]
        items, refs = [], []
        for i, (kind, B, C, U, W, M, T) in enumerate(specs):
            dl = kind == K.DBP_KIND_DOWNLINK_ADMM
            f = synth.downlink_frame(W, 14, B, U, M, seed=500 + i) if dl else \
                synth.uplink_frame(W, 14, B, U, M, 15.0, seed=500 + i)
            Hd = torch.from_numpy(f["H"].astype(np.complex64)).cuda()
            ind = torch.from_numpy((f["s"] if dl else f["y"]).astype(np.complex64)).cuda()
            shape = (W, 14, B) if dl else (W, 14, U)
            out = torch.zeros(shape, dtype=torch.complex64, device="cuda")
            lab = None if dl else torch.zeros((W, 14, U), dtype=torch.uint8, device="cuda")
            d = dbp.frame_desc(B, C, U, W, 14, qam_order=0 if dl else M, T_max=T, rho=1.0, N0=f.get("N0", 0.1))
            ro = torch.zeros_like(out)
            rl = None if dl else torch.zeros_like(lab)
            if dl:
                dbp.dbp_downlink_admm(h, d, Hd, ind, ro)
            elif kind == K.DBP_KIND_UPLINK_ADMM:
                if U == 32 and B == 32 * C:
                    dbp.dbp_set_tuning(h, kernel=dbp.DBP_PATH_TMA)
                dbp.dbp_uplink_admm(h, d, Hd, ind, ro, rl)
                dbp.dbp_set_tuning(h)
            else:
                dbp.dbp_uplink_cg(h, d, Hd, ind, ro, rl)
            items.append((kind, d, Hd, ind, out, lab))
            refs.append((ro, rl))
        torch.cuda.synchronize()
        dbp.dbp_server_start(h, streams=4, hbm_bytes=256 << 20)
        tickets = []
        for rep in range(2):        # the second round hits the resident operators
            for i, (kind, d, Hd, ind, out, lab) in enumerate(items):
                req = dbp.request(kind, d, Hd, ind, out, lab, None, 100 + i, 1, i,
                                  flags=dbp.DBP_REQ_DEVICE_BUFFERS)
                tickets.append(dbp.dbp_wait(h, dbp.dbp_submit(h, req), 60.0))
        dbp.dbp_server_stop(h)
        assert all(r.status == dbp.DBP_OK for r in tickets)
        for (kind, d, Hd, ind, out, lab), (ro, rl) in zip(items, refs):
            assert torch.equal(out, ro)
            if lab is not None:
                assert torch.equal(lab, rl)
    finally:
        dbp.dbp_destroy(h)


def test_hbm_budget_caps_the_library_allocations(dbp):
    """dbp_config.hbm_budget_bytes: a host-buffer call whose staging buffers
    exceed the budget and a request pool larger than it are refused with
    DBP_ERR_NOMEM; the default pool takes what the budget leaves."""
    h = dbp.dbp_create(0, hbm_budget_bytes=8 << 20)
    try:
        f = Frame(dbp, dbp.DBP_KIND_UPLINK_ADMM, 128, 8, 8, 1200, 14, 16, 3, seed=90)   # 27 MB staged
        with pytest.raises(dbp.DbpError) as ei:
            f.run_alone(dbp, h)
        assert ei.value.status == dbp.DBP_ERR_NOMEM
        with pytest.raises(dbp.DbpError) as ei:
            dbp.dbp_server_start(h, streams=2, hbm_bytes=64 << 20)
        assert ei.value.status == dbp.DBP_ERR_NOMEM
        small = Frame(dbp, dbp.DBP_KIND_UPLINK_ADMM, 64, 4, 8, 100, 14, 16, 3, seed=91)
        ref = small.run_alone(dbp, h)                   # fits the budget
        dbp.dbp_server_start(h, streams=2)              # pool = what the budget leaves
        r = dbp.dbp_wait(h, dbp.dbp_submit(h, small.request(dbp, 0)), 60.0)
        dbp.dbp_server_stop(h)
        assert r.status == dbp.DBP_OK and np.array_equal(small.out, ref[0])
    finally:
        dbp.dbp_destroy(h)
