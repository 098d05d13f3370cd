"""Serving loop and batched sweeps.

CPU: the scheduler's admission by footprint, arrival order, retirement and
statistics, driven by a fake backend (no GPU).  GPU: every result is the
same alone and in the mix, and batched sweeps equal one-at-a-time sweeps.
"""
import numpy as np
import pytest

from paper_2112_13184_gb300 import inputs as I
from paper_2112_13184_gb300.serve import Request, Server


class FakeBackend:
    """Handles that 'converge' after a set number of sweeps; a launched
    sweep of request rid completes after lag[rid] polls (0: at once);
    records order."""

    def __init__(self, bytes_of, sweeps_to_converge, lag=None, floor=None):
        self.bytes_of = bytes_of
        self.need = sweeps_to_converge
        self.lag = lag or {}
        self.floor = floor or {}
        self.opened, self.closed, self.live, self.peak, self.refined = [], [], 0, 0, []
        self.launches = []

    def footprint(self, r):
        return self.bytes_of[r.rid]

    def open(self, r, block=None):
        self.opened.append(r.rid)
        self.live += self.bytes_of[r.rid]
        self.peak = max(self.peak, self.live)
        return {"rid": r.rid, "n": 0, "wait": 0, "refined": False}

    def launch(self, h, n):
        h["n"] += n
        h["wait"] = self.lag.get(h["rid"], 0)
        self.launches.append(h["rid"])

    def ready(self, h):
        if h["wait"] > 0:
            h["wait"] -= 1
            return False
        return True

    def delta(self, h):
        if h["rid"] in self.floor and not h["refined"]:
            return self.floor[h["rid"]]  # stuck at a rounding floor until refined
        return 0.0 if h["n"] >= self.need[h["rid"]] else 1.0

    def measure(self, h, r):
        return np.full(12, float(r.rid))

    def close(self, h):
        self.closed.append(h["rid"])
        self.live -= self.bytes_of[h["rid"]]


class RefiningBackend(FakeBackend):
    def refine(self, h):
        if h["refined"]:
            return False
        h["refined"] = True
        self.refined.append(h["rid"])
        return True


def req(i, tol=0.5, max_sweeps=100):
    return Request(i, 2, 2, 4, None, None, None, None, tol=tol, max_sweeps=max_sweeps, arrival=float(i))


def test_first_fit_admission_respects_budget():
    sizes = {0: 60, 1: 50, 2: 30, 3: 10}
    fb = FakeBackend(sizes, {0: 3, 1: 1, 2: 2, 3: 1})
    t = iter(range(1000))
    srv = Server(100, fb, clock=lambda: float(next(t)))
    for i in range(4):
        srv.submit(req(i))
    srv.poll()
    # 0 (60) admitted; 1 (50) does not fit; 2 (30) and 3 (10) fit behind it
    assert fb.opened == [0, 2, 3] and [r.rid for r in srv.waiting] == [1]
    res = srv.drain()
    assert fb.peak <= 100
    assert fb.opened == [0, 2, 3, 1]
    assert sorted(r.rid for r in res) == [0, 1, 2, 3]
    assert all(r.converged for r in res)
    assert fb.live == 0 and srv.in_use == 0 and srv.pool.stats() == (0, 100, 1)  # pool merged back
    for r in res:
        assert np.all(r.observables == r.rid)


def test_head_of_queue_ages():
    """The head may be passed over max_skip times; then it goes next."""
    sizes = {0: 90, 1: 50, 2: 5, 3: 5, 4: 5}
    fb = FakeBackend(sizes, {0: 4, 1: 1, 2: 50, 3: 50, 4: 50})
    srv = Server(100, fb, max_skip=1)
    for i in range(5):
        srv.submit(req(i))
    srv.poll()
    # 0 admitted; 1 blocked; 2 passes it once; 3 and 4 must now wait behind 1
    assert fb.opened == [0, 2]
    srv.drain()
    assert fb.opened.index(1) < fb.opened.index(3) < fb.opened.index(4)


def test_requests_advance_at_their_own_pace():
    """A request whose sweeps take many polls does not hold back another."""
    fb = FakeBackend({0: 10, 1: 10}, {0: 3, 1: 6}, lag={0: 20, 1: 0})
    srv = Server(100, fb)
    srv.submit(req(0))
    srv.submit(req(1))
    for _ in range(15):
        srv.poll()
    done = {r.rid for r in srv.done}
    assert done == {1}  # 1 finished its 6 sweeps while 0's first sweep was still running
    srv.drain()
    assert {r.rid for r in srv.done} == {0, 1}


def test_pool_first_fit_and_merge():
    """The native pool: 256-byte granules, first fit, merging on free, and
    no double free."""
    from paper_2112_13184_gb300 import ctm
    from paper_2112_13184_gb300.serve import DevicePool
    p = DevicePool(1024, 256)
    a, b, c = p.alloc(100), p.alloc(300), p.alloc(200)
    assert (a, b, c) == (0, 256, 768) and p.alloc(10) is None  # 256-byte granules
    assert p.stats() == (1024, 0, 0)
    p.release(b, 300)
    assert p.alloc(256) == 256 and p.stats() == (768, 256, 1)
    p.release(a, 100)
    p.release(256, 256)
    assert p.stats() == (256, 768, 1)  # [0, 768) merged
    p.release(c, 200)
    assert p.stats() == (0, 1024, 1)
    with pytest.raises(ctm.CtmError):
        p.release(c, 200)  # second free
    with pytest.raises(ctm.CtmError):
        p.release(5, 256)  # not a block
    with pytest.raises(ctm.CtmError):
        DevicePool(1024, 100)  # grain not a power of two


def test_stall_triggers_refinement():
    fb = RefiningBackend({0: 1}, {0: 5}, floor={0: 1e-8})
    srv = Server(10, fb)
    srv.submit(req(0, tol=1e-10))
    res = srv.drain()
    assert fb.refined == [0] and res[0].converged


def test_max_sweeps_and_stats():
    fb = FakeBackend({0: 1, 1: 1}, {0: 10 ** 9, 1: 2})
    srv = Server(10, fb)
    srv.submit(req(0, max_sweeps=5))
    srv.submit(req(1))
    res = {r.rid: r for r in srv.drain()}
    assert res[0].sweeps == 5 and not res[0].converged
    assert res[1].sweeps == 2 and res[1].converged
    st = srv.stats()
    assert st["requests"] == 2 and st["converged"] == 1 and st["p99_s"] >= st["p50_s"]
    assert st["sweeps_total"] == 7


def test_cancel_waiting_and_active():
    fb = FakeBackend({0: 60, 1: 60, 2: 50}, {0: 10 ** 9, 1: 1, 2: 1})
    srv = Server(100, fb)
    for i in range(3):
        srv.submit(req(i))
    srv.poll()  # 0 active; 1 and 2 wait (no room for either)
    assert srv.cancel(2) and [r.rid for r in srv.waiting] == [1]
    assert srv.cancel(0)  # frees 60: 1 is admitted at once
    assert fb.closed[:1] == [0] and [a.req.rid for a in srv.active] == [1]
    res = srv.drain()
    assert [r.rid for r in res] == [1] and srv.in_use == 0 and fb.live == 0
    assert not srv.cancel(0) and not srv.cancel(7)


def test_oversized_request_rejected():
    srv = Server(10, FakeBackend({0: 11}, {0: 1}))
    with pytest.raises(ValueError):
        srv.submit(req(0))


@pytest.mark.gpu
def test_alone_equals_mix_and_batched_equals_sequential():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_13184_gb300 import ctm
    from paper_2112_13184_gb300.serve import CtmBackend

    def make(j):
        q = I.serving_request(j, ds=(2, 3), Ds=(2, 3), chis=(8, 12, 16))
        return Request(j, q["d"], q["D"], q["chi"], q["As"], q["envs"], q["op1"], q["op2"], tol=0.0,
                       max_sweeps=6 + j % 3, arrival=0.0)

    reqs = [make(j) for j in range(5)]
    alone = {}
    for r in reqs:
        srv = Server(8 << 30, CtmBackend("mixed"))
        srv.submit(r)
        alone[r.rid] = srv.drain()[0]
    srv = Server(8 << 30, CtmBackend("mixed"))
    for r in reqs:
        srv.submit(r)
    mix = {x.rid: x for x in srv.drain()}
    for rid, a in alone.items():
        assert a.sweeps == mix[rid].sweeps
        np.testing.assert_allclose(mix[rid].observables, a.observables, rtol=0, atol=1e-12)

    # ctm_batch_sweep over several handles == ctm_sweep on each in turn
    specs = [I.batch_instance(i) for i in range(3)]

    def build():
        hs = []
        for q in specs:
            c = ctm.CTMRG(q["d"], q["D"], q["chi"], precision=ctm.CTM_OZAKI_BF16)
            c.set_tensors(q["As"])
            c.set_envs(q["envs"])
            hs.append(c)
        return hs

    seq = build()
    for c in seq:
        c.sweep(4)
    bat = build()
    ctm.ctm_batch_sweep([c.h for c in bat], 4)
    for q, a, b in zip(specs, seq, bat):
        np.testing.assert_allclose(b.measure1(0, q["op1"]), a.measure1(0, q["op1"]), rtol=0, atol=1e-12)
        a.close()
        b.close()
