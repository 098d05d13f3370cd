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
    """Handles that 'converge' after a set number of sweeps; records order."""

    def __init__(self, bytes_of, sweeps_to_converge):
        self.bytes_of = bytes_of
        self.need = sweeps_to_converge
        self.opened, self.closed, self.live, self.peak = [], [], 0, 0

    def footprint(self, r):
        return self.bytes_of[r.rid]

    def open(self, r):
        self.opened.append(r.rid)
        self.live += self.bytes_of[r.rid]
        self.peak = max(self.peak, self.live)
        return {"rid": r.rid, "n": 0}

    def sweep_async(self, h):
        h["n"] += 1

    def delta(self, h):
        return 0.0 if h["n"] >= self.need[h["rid"]] else 1.0

    def measure(self, h, r):
        return np.full(12, float(r.rid))

    def close(self, h):
        self.closed.append(h["rid"])
        self.live -= self.bytes_of[h["rid"]]


def req(i, tol=0.5, max_sweeps=100):
    return Request(i, 2, 2, 4, None, None, None, None, tol=tol, max_sweeps=max_sweeps, arrival=float(i))


def test_admission_respects_budget_and_order():
    sizes = {0: 60, 1: 50, 2: 30, 3: 10}
    fb = FakeBackend(sizes, {0: 3, 1: 1, 2: 2, 3: 1})
    t = iter(range(1000))
    srv = Server(100, fb, clock=lambda: float(next(t)))
    for i in range(4):
        srv.submit(req(i))
    srv.step()
    # 0 (60) admitted; 1 (50) does not fit and blocks 2, 3 behind it
    assert fb.opened[:1] == [0] and 1 not in fb.opened[:1]
    res = srv.drain()
    assert fb.peak <= 100
    assert fb.opened == [0, 1, 2, 3]  # arrival order
    assert sorted(r.rid for r in res) == [0, 1, 2, 3]
    assert all(r.converged for r in res)
    assert fb.live == 0 and srv.in_use == 0
    for r in res:
        assert np.all(r.observables == r.rid)


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


def test_cancel_waiting_and_active():
    fb = FakeBackend({0: 60, 1: 60, 2: 30}, {0: 10 ** 9, 1: 1, 2: 1})
    srv = Server(100, fb)
    for i in range(3):
        srv.submit(req(i))
    srv.step()  # 0 active; 1 waits (no room), 2 waits behind it
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
        srv = Server(1 << 40, CtmBackend("mixed"))
        srv.submit(r)
        alone[r.rid] = srv.drain()[0]
    srv = Server(1 << 40, CtmBackend("mixed"))
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
