"""Continuous-batching serving loop and batched sweeps for CTMRG requests.

A request asks for the environment of one 2x2-cell iTPS (d, D, chi, site
tensors, initial C/T) converged until the gauge-invariant loop moments of
ctm_loop_delta change by less than `tol` per sweep (Sec. 2.2 iterates to
convergence), and for one- and two-site expectation values (Sec. 5.3).

Serving (continuous batching):
  * device memory: one region of `budget` bytes is reserved when the server
    starts; a first-fit pool (libctm's ctm_pool_*) hands each admitted request a block
    of its ctm_footprint_bytes, from which ctm_create_in carves the handle,
    so admission and retirement never call cudaMalloc / cudaFree (cudaFree
    waits for every stream on the device);
  * every admitted request keeps its C/T resident in its block and runs on
    its own CUDA stream;
  * admission: the waiting queue is scanned in arrival order and every
    request whose block fits is admitted (first fit), so small requests do
    not wait behind a large one; the head of the queue may be passed over
    at most `max_skip` times, after which nothing is admitted ahead of it;
  * cadence: each request advances independently -- `check_every` sweeps
    are enqueued (ctm_sweep_async), the server polls the request's stream
    without blocking, and only a request whose sweeps have finished has its
    convergence measure read (ctm_loop_delta) and is retired or given its
    next sweeps; a large request's sweep paces nobody else;
  * an emulated-FP64 request whose measure has stopped halving for
    `STALL_CHECKS` checks below `REFINE_BELOW` (the emulated products'
    rounding floor) continues in FP64;
  * latency = finish - arrival (queue wait + service); stats report p50 /
    p99 of each and the throughput.

Batching: ctm_batch_sweep advances many independent instances together
(round-robin graph launches over their streams) instead of one at a time.

The device work all runs in libctm's kernels; this module only orders calls.

    python -m paper_2112_13184_gb300.serve serve --rate 2 --requests 24
    python -m paper_2112_13184_gb300.serve batch --instances 64 --sweeps 20
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass
from typing import Any, Callable, Dict, List, Optional, Tuple

import numpy as np

from . import inputs as I


# an emulated-FP64 request whose measure has not halved for STALL_CHECKS
# checks while below REFINE_BELOW continues in FP64
STALL_CHECKS = 3
REFINE_BELOW = 1e-6


@dataclass
class Request:
    rid: int
    d: int
    D: int
    chi: int
    As: Any
    envs: Any
    op1: np.ndarray
    op2: np.ndarray
    tol: float = 1e-10
    max_sweeps: int = 100
    arrival: float = 0.0


@dataclass
class Result:
    rid: int
    observables: np.ndarray  # <op1> on the 4 sites, then <op2> on the 8 bonds
    sweeps: int
    delta: float
    converged: bool
    arrival: float
    start: float
    finish: float

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class CtmBackend:
    """Device side of the server: one libctm handle per request, on its own
    stream, carved from the server's reserved region."""

    def __init__(self, precision: str = "mixed", slices: int = 5):
        from . import ctm
        self.ctm = ctm
        self.precision = ctm.CTM_OZAKI_BF16 if precision == "mixed" else ctm.CTM_FP64
        self.slices = slices
        self._region = None

    def footprint(self, r: Request) -> int:
        o = self.ctm.ctm_default_options(chi=r.chi, precision=self.precision, ozaki_slices=self.slices)
        return self.ctm.ctm_footprint_bytes(r.d, r.D, o)

    def reserve(self, nbytes: int) -> int:
        """One device region for every handle the server opens; returns its address."""
        import torch
        self._region = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        return self._region.data_ptr()

    def open(self, r: Request, block: Optional[Tuple[int, int]] = None):
        import torch
        c = self.ctm.CTMRG(r.d, r.D, r.chi, stream=torch.cuda.Stream(), arena=block, precision=self.precision,
                           ozaki_slices=self.slices)
        c.set_tensors(r.As)
        c.set_envs(r.envs)
        c.loop_delta()  # reference loop moments of the initial environment
        return c

    def launch(self, c, n: int) -> None:
        c.sweep_async(n)

    def ready(self, c) -> bool:
        return c.stream.query()

    def delta(self, c) -> float:
        # the gauge-invariant measure: single-corner spectra keep moving with
        # the chi-bond gauge after the network has converged
        return c.loop_delta()

    def refine(self, c) -> bool:
        """Switches an emulated-FP64 handle to FP64 contractions; returns
        whether it switched."""
        if self.precision != self.ctm.CTM_OZAKI_BF16 or getattr(c, "_refined", False):
            return False
        self.ctm.ctm_set_precision(c.h, self.ctm.CTM_FP64)
        c._refined = True
        return True

    def measure(self, c, r: Request) -> np.ndarray:
        one = [c.measure1(i, r.op1) for i in range(4)]
        two = [c.measure2(i, dx, dy, r.op2) for (i, dx, dy) in I.SQUARE_2X2_BONDS]
        return np.array(one + two)

    def close(self, c):
        c.close()


class DevicePool:
    """First-fit offsets in one reserved region, kept by libctm's native pool
    (ctm_pool_*): blocks rounded up to `grain` bytes (256 for device memory),
    freed neighbours merge, a second free of a block is refused."""

    def __init__(self, size: int, grain: int = 1):
        from . import ctm
        self._ctm = ctm
        self.size = int(size)
        self.grain = int(grain)
        self._p = ctm.ctm_pool_create(self.size, self.grain)

    def alloc(self, n: int) -> Optional[int]:
        return self._ctm.ctm_pool_alloc(self._p, int(n))

    def release(self, off: int, n: int) -> None:
        self._ctm.ctm_pool_free(self._p, int(off), int(n))

    def largest(self) -> int:
        return self._ctm.ctm_pool_stats(self._p)[1]

    def stats(self) -> Tuple[int, int, int]:
        """(bytes allocated, largest free block, number of free blocks)."""
        return self._ctm.ctm_pool_stats(self._p)

    def __del__(self):
        try:
            if self._p:
                self._ctm.ctm_pool_destroy(self._p)
                self._p = None
        except Exception:
            pass


@dataclass
class _Active:
    req: Request
    handle: Any
    bytes: int
    offset: int
    start: float
    sweeps: int = 0
    inflight: int = 0
    delta: float = float("inf")
    best: float = float("inf")
    stall: int = 0


class Server:
    """Admits by device footprint (first fit with aging), advances each
    request at its own pace and retires converged ones (module docstring)."""

    def __init__(self, budget_bytes: int, backend=None, clock: Callable[[], float] = time.perf_counter,
                 check_every: int = 1, max_skip: int = 8):
        self.budget = int(budget_bytes)
        self.backend = backend if backend is not None else CtmBackend()
        self.clock = clock
        self.check_every = max(1, int(check_every))
        self.max_skip = int(max_skip)
        self.base = self.backend.reserve(self.budget) if hasattr(self.backend, "reserve") else None
        # device blocks start on 256-byte boundaries (ctm_create_in requires it)
        self.pool = DevicePool(self.budget, 256 if self.base is not None else 1)
        self.waiting: List[Request] = []
        self.active: List[_Active] = []
        self.done: List[Result] = []
        self.in_use = 0
        self.head_skips = 0
        self.progressed = False

    def submit(self, r: Request) -> None:
        if self.backend.footprint(r) > self.budget:
            raise ValueError(f"request {r.rid} needs more device memory than the whole budget")
        self.waiting.append(r)

    def _admit(self) -> None:
        i, head_blocked = 0, False
        while i < len(self.waiting):
            r = self.waiting[i]
            b = self.backend.footprint(r)
            if i > 0 and head_blocked and self.head_skips >= self.max_skip:
                break  # the head has been passed over often enough: it goes next
            off = self.pool.alloc(b)
            if off is None:
                head_blocked = head_blocked or i == 0
                i += 1
                continue
            block = (self.base + off, b) if self.base is not None else None
            self.active.append(_Active(r, self.backend.open(r, block), b, off, self.clock()))
            self.waiting.pop(i)
            self.in_use += b
            if i == 0:
                self.head_skips = 0
            elif head_blocked:
                self.head_skips += 1

    def _retire(self, a: _Active, conv: bool) -> Result:
        obs = self.backend.measure(a.handle, a.req)
        self.backend.close(a.handle)
        self.pool.release(a.offset, a.bytes)
        self.in_use -= a.bytes
        return Result(a.req.rid, obs, a.sweeps, a.delta, conv, a.req.arrival, a.start, self.clock())

    def poll(self) -> List[Result]:
        """One non-blocking pass over the active requests; returns the
        requests finished in it.  self.progressed tells whether anything
        was read or launched."""
        self._admit()
        finished: List[Result] = []
        self.progressed = False
        for a in list(self.active):
            if a.inflight:
                if not self.backend.ready(a.handle):
                    continue
                a.sweeps += a.inflight
                a.inflight = 0
                a.delta = self.backend.delta(a.handle)
                self.progressed = True
                conv = a.delta < a.req.tol
                if a.delta < 0.5 * a.best:
                    a.best, a.stall = a.delta, 0
                else:
                    a.stall += 1
                if (not conv and a.stall >= STALL_CHECKS and a.delta < REFINE_BELOW
                        and hasattr(self.backend, "refine")):
                    if self.backend.refine(a.handle):
                        a.stall = 0
                if conv or a.sweeps >= a.req.max_sweeps:
                    finished.append(self._retire(a, conv))
                    self.active.remove(a)
                    continue
            n = min(self.check_every, a.req.max_sweeps - a.sweeps)
            self.backend.launch(a.handle, n)
            a.inflight = n
            self.progressed = True
        if finished:
            self.done.extend(finished)
            self._admit()
        return finished

    def step(self) -> List[Result]:
        return self.poll()

    def cancel(self, rid: int) -> bool:
        """Withdraws a request: a waiting one is dropped, an active one has
        its handle freed once its enqueued sweeps have finished (closing the
        handle waits for its own stream only).  Returns False when the
        request is unknown or already finished."""
        for r in list(self.waiting):
            if r.rid == rid:
                self.waiting.remove(r)
                return True
        for a in self.active:
            if a.req.rid == rid:
                self.backend.close(a.handle)
                self.pool.release(a.offset, a.bytes)
                self.in_use -= a.bytes
                self.active.remove(a)
                self._admit()
                return True
        return False

    def idle(self) -> bool:
        return not self.waiting and not self.active

    def drain(self, nap: float = 2e-4) -> List[Result]:
        while not self.idle():
            self.poll()
            if not self.active and self.waiting:
                raise RuntimeError("waiting requests fit no free block of the pool")
            if not self.progressed:
                time.sleep(nap)
        return self.done

    def stats(self) -> Dict[str, float]:
        lat = np.array([r.latency for r in self.done]) if self.done else np.zeros(1)
        wait = np.array([r.start - r.arrival for r in self.done]) if self.done else np.zeros(1)
        span = (max(r.finish for r in self.done) - min(r.arrival for r in self.done)) if self.done else 0.0
        return {"requests": len(self.done), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)),
                "queue_p50_s": float(np.percentile(wait, 50)), "queue_p99_s": float(np.percentile(wait, 99)),
                "throughput_req_per_s": len(self.done) / span if span > 0 else None,
                "converged": int(sum(r.converged for r in self.done)),
                "sweeps_total": int(sum(r.sweeps for r in self.done))}


def make_request(j: int, arrival: float, tol: float, max_sweeps: int, **family) -> Request:
    q = I.serving_request(j, **family)
    return Request(j, q["d"], q["D"], q["chi"], q["As"], q["envs"], q["op1"], q["op2"], tol, max_sweeps, arrival)


def serve_poisson(rate: float, n: int, budget_bytes: int, precision: str, tol: float, max_sweeps: int,
                  seed: int = 0, **family) -> Dict[str, Any]:
    """Real-time Poisson stream of n requests at `rate` per second."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    srv = Server(budget_bytes, CtmBackend(precision))
    t0 = time.perf_counter()
    arrivals = t0 + np.cumsum(gaps)
    j = 0
    while j < n or not srv.idle():
        now = time.perf_counter()
        while j < n and arrivals[j] <= now:
            srv.submit(make_request(j, float(arrivals[j]), tol, max_sweeps, **family))
            j += 1
        if srv.idle():
            time.sleep(max(0.0, min(0.01, arrivals[j] - now)) if j < n else 0.0)
            continue
        srv.poll()
        if not srv.progressed:
            time.sleep(2e-4)
    out = srv.stats()
    out.update(rate=rate, precision=precision, budget_gb=budget_bytes / 1e9, tol=tol, max_sweeps=max_sweeps)
    return out


def rate_sweep(rates, n: int, budget_bytes: int, precision: str, tol: float, max_sweeps: int, seed: int = 0,
               **family) -> List[Dict[str, Any]]:
    """serve_poisson at each rate (requests 0 .. n-1 of the family at every
    rate, the same arrival-gap seed): latency percentiles against load."""
    return [serve_poisson(rate, n, budget_bytes, precision, tol, max_sweeps, seed=seed, **family) for rate in rates]


def batch_compare(instances: int, sweeps: int, precision: str) -> Dict[str, Any]:
    """Aggregate sweeps/s of `instances` uneven instances: one ctm_batch_sweep
    over all handles against ctm_sweep on each handle in turn (same inputs,
    results compared)."""
    from . import ctm
    import torch
    prec = ctm.CTM_OZAKI_BF16 if precision == "mixed" else ctm.CTM_FP64
    specs = [I.batch_instance(i) for i in range(instances)]

    def build():
        hs = []
        for q in specs:
            c = ctm.CTMRG(q["d"], q["D"], q["chi"], precision=prec)
            c.set_tensors(q["As"])
            c.set_envs(q["envs"])
            hs.append(c)
        return hs

    out: Dict[str, Any] = {"instances": instances, "sweeps": sweeps, "precision": precision}
    obs = {}
    for mode in ("one_at_a_time", "batched"):
        hs = build()
        # one untimed sweep each: the cold sweep and CUDA-graph capture
        ctm.ctm_batch_sweep([c.h for c in hs], 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if mode == "batched":
            ctm.ctm_batch_sweep([c.h for c in hs], sweeps)
        else:
            for c in hs:
                c.sweep(sweeps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[mode + "_sweeps_per_s"] = instances * sweeps / dt
        obs[mode] = np.array([c.measure1(0, specs[i]["op1"]) for i, c in enumerate(hs)])
        for c in hs:
            c.close()
    out["speedup"] = out["batched_sweeps_per_s"] / out["one_at_a_time_sweeps_per_s"]
    out["max_abs_diff_batched_vs_one"] = float(np.abs(obs["batched"] - obs["one_at_a_time"]).max())
    return out


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    s = sub.add_parser("serve")
    s.add_argument("--rate", type=float, default=2.0)
    s.add_argument("--requests", type=int, default=24)
    s.add_argument("--budget-gb", type=float, default=60.0)
    s.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    s.add_argument("--tol", type=float, default=1e-8)
    s.add_argument("--max-sweeps", type=int, default=60)
    s.add_argument("--Ds", default="4,6")
    s.add_argument("--chis", default="32,64")
    w = sub.add_parser("sweep", help="latency against load: one Poisson stream per rate")
    w.add_argument("--rates", default="1,2,5,10,20,50,100,200")
    w.add_argument("--requests", type=int, default=16)
    w.add_argument("--budget-gb", type=float, default=200.0)
    w.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    w.add_argument("--tol", type=float, default=1e-10)
    w.add_argument("--max-sweeps", type=int, default=300)
    w.add_argument("--Ds", default="4,6,8")
    w.add_argument("--chis", default="32,64,128")
    b = sub.add_parser("batch")
    b.add_argument("--instances", type=int, default=64)
    b.add_argument("--sweeps", type=int, default=20)
    b.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    a = ap.parse_args()
    if a.cmd == "serve":
        fam = dict(Ds=tuple(int(x) for x in a.Ds.split(",")), chis=tuple(int(x) for x in a.chis.split(",")))
        r = serve_poisson(a.rate, a.requests, int(a.budget_gb * 1e9), a.precision, a.tol, a.max_sweeps, **fam)
        r.update(Ds=fam["Ds"], chis=fam["chis"])
    elif a.cmd == "sweep":
        fam = dict(Ds=tuple(int(x) for x in a.Ds.split(",")), chis=tuple(int(x) for x in a.chis.split(",")))
        r = {"Ds": fam["Ds"], "chis": fam["chis"], "requests": a.requests,
             "runs": rate_sweep([float(x) for x in a.rates.split(",")], a.requests, int(a.budget_gb * 1e9),
                                a.precision, a.tol, a.max_sweeps, **fam)}
    else:
        r = batch_compare(a.instances, a.sweeps, a.precision)
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
