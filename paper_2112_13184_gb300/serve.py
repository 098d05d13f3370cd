"""Continuous-batching serving loop and batched sweeps for CTMRG requests.

A request asks for the environment of one 2x2-cell iTPS (d, D, chi, site
tensors, initial C/T) converged until the gauge-invariant loop moments of
ctm_loop_delta change by less than `tol` per sweep (Sec. 2.2 iterates to
convergence), and for one- and two-site expectation values (Sec. 5.3).

Serving (continuous batching):
  * every admitted request keeps its C/T resident on the device in its own
    CTMRG handle, on its own CUDA stream;
  * requests are admitted in arrival order while the summed device
    footprint (ctm_footprint_bytes) fits the budget; a request that does not
    fit waits until retirements free memory;
  * one server step enqueues one sweep for every active request
    (ctm_sweep_async, so the requests' kernels overlap on the GPU), then
    reads each request's convergence measure (ctm_loop_delta); an
    emulated-FP64 request whose measure is below 1e-8 (about where the
    emulated products' rounding holds it) continues in FP64; requests that
    converged or reached max_sweeps are measured, their handles freed, and
    waiting requests admitted in the same step.
  * latency = finish - arrival; the stats report p50 / p99 and throughput.

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
from collections import deque
from dataclasses import dataclass
from typing import Any, Callable, Deque, Dict, List

import numpy as np

from . import inputs as I


# below this change per sweep an emulated-FP64 request continues in FP64
REFINE_AT = 1e-8


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
    """Device side of the server: one libctm handle per request."""

    def __init__(self, precision: str = "mixed", slices: int = 5):
        from . import ctm
        self.ctm = ctm
        self.precision = ctm.CTM_OZAKI_BF16 if precision == "mixed" else ctm.CTM_FP64
        self.slices = slices

    def footprint(self, r: Request) -> int:
        o = self.ctm.ctm_default_options(chi=r.chi, precision=self.precision, ozaki_slices=self.slices)
        return self.ctm.ctm_footprint_bytes(r.d, r.D, o)

    def open(self, r: Request):
        c = self.ctm.CTMRG(r.d, r.D, r.chi, precision=self.precision, ozaki_slices=self.slices)
        c.set_tensors(r.As)
        c.set_envs(r.envs)
        c.loop_delta()  # reference loop moments of the initial environment
        return c

    def sweep_async(self, c):
        c.sweep_async(1)

    def delta(self, c) -> float:
        # the gauge-invariant measure: single-corner spectra keep moving with
        # the chi-bond gauge after the network has converged
        return c.loop_delta()

    def refine(self, c) -> bool:
        """Switches an emulated-FP64 handle to FP64 contractions (the
        emulated products' rounding holds the measure near 1e-8); returns
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


@dataclass
class _Active:
    req: Request
    handle: Any
    bytes: int
    start: float
    sweeps: int = 0
    delta: float = float("inf")


class Server:
    """Admits by device footprint, advances all active requests one sweep per
    step, retires converged requests (see the module docstring)."""

    def __init__(self, budget_bytes: int, backend=None, clock: Callable[[], float] = time.perf_counter):
        self.budget = int(budget_bytes)
        self.backend = backend if backend is not None else CtmBackend()
        self.clock = clock
        self.waiting: Deque[Request] = deque()
        self.active: List[_Active] = []
        self.done: List[Result] = []
        self.in_use = 0

    def submit(self, r: Request) -> None:
        if self.backend.footprint(r) > self.budget:
            raise ValueError(f"request {r.rid} needs more device memory than the whole budget")
        self.waiting.append(r)

    def _admit(self) -> None:
        while self.waiting:
            r = self.waiting[0]
            b = self.backend.footprint(r)
            if self.in_use + b > self.budget:
                break  # arrival order: later requests wait behind this one
            self.waiting.popleft()
            self.active.append(_Active(r, self.backend.open(r), b, self.clock()))
            self.in_use += b

    def step(self) -> List[Result]:
        """One scheduling round; returns the requests finished in it."""
        self._admit()
        for a in self.active:
            self.backend.sweep_async(a.handle)
        finished: List[Result] = []
        keep: List[_Active] = []
        for a in self.active:
            a.sweeps += 1
            a.delta = self.backend.delta(a.handle)
            conv = a.delta < a.req.tol
            if not conv and a.delta < REFINE_AT and hasattr(self.backend, "refine"):
                self.backend.refine(a.handle)
            if conv or a.sweeps >= a.req.max_sweeps:
                obs = self.backend.measure(a.handle, a.req)
                self.backend.close(a.handle)
                self.in_use -= a.bytes
                finished.append(Result(a.req.rid, obs, a.sweeps, a.delta, conv, a.req.arrival, a.start,
                                       self.clock()))
            else:
                keep.append(a)
        self.active = keep
        self.done.extend(finished)
        self._admit()
        return finished

    def cancel(self, rid: int) -> bool:
        """Withdraws a request: a waiting one is dropped, an active one has
        its handle freed between steps (none of its work is in flight then).
        Returns False when the request is unknown or already finished."""
        for r in list(self.waiting):
            if r.rid == rid:
                self.waiting.remove(r)
                return True
        for a in self.active:
            if a.req.rid == rid:
                self.backend.close(a.handle)
                self.in_use -= a.bytes
                self.active.remove(a)
                self._admit()
                return True
        return False

    def idle(self) -> bool:
        return not self.waiting and not self.active

    def drain(self) -> List[Result]:
        while not self.idle():
            self.step()
        return self.done

    def stats(self) -> Dict[str, float]:
        lat = np.array([r.latency for r in self.done]) if self.done else np.zeros(1)
        span = (max(r.finish for r in self.done) - min(r.arrival for r in self.done)) if self.done else 0.0
        return {"requests": len(self.done), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)),
                "throughput_req_per_s": len(self.done) / span if span > 0 else None,
                "converged": int(sum(r.converged for r in self.done))}


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
        srv.step()
    out = srv.stats()
    out.update(rate=rate, precision=precision, budget_gb=budget_bytes / 1e9, tol=tol, max_sweeps=max_sweeps)
    return out


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
    b = sub.add_parser("batch")
    b.add_argument("--instances", type=int, default=64)
    b.add_argument("--sweeps", type=int, default=20)
    b.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    a = ap.parse_args()
    if a.cmd == "serve":
        fam = dict(Ds=tuple(int(x) for x in a.Ds.split(",")), chis=tuple(int(x) for x in a.chis.split(",")))
        r = serve_poisson(a.rate, a.requests, int(a.budget_gb * 1e9), a.precision, a.tol, a.max_sweeps, **fam)
        r.update(Ds=fam["Ds"], chis=fam["chis"])
    else:
        r = batch_compare(a.instances, a.sweeps, a.precision)
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
