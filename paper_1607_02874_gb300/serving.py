"""Continuous-batching request loop over resident simulations.

Requests (box, porosity, correlation length, Da, seed) arrive over time. The
loop:

- admits them in arrival order while their device footprint fits the budget;
- builds each geometry on a worker thread, so the host-side generator
  overlaps the GPU work;
- keeps every admitted lattice resident on the device;
- advances all resident simulations together, one batched launch per time
  step (``lbm_step_batch``).

A simulation retires when its conversion efficiency eta is positive and
changes by less than ``tol`` (relative) over ``check_every`` steps, or at
``max_steps``. Retiring
frees its memory, which admits waiting requests. The loop reports the
time-to-steady-state of each request, its p50/p99, and the throughput.

Failures are per request and the loop carries on. Each ends with a status:
- "rejected": the footprint exceeds the whole budget;
- "failed": the build raised, for instance on an allocation failure. The
  reservation is released;
- "diverged": the observables reported NaN or a non-positive carrier mass.
  The simulation is freed.
A failing batched step is not per request. It raises, because the state of
every simulation in the launch is then unknown.

The device side sits behind a small backend interface: ``LbmBackend`` drives
the C library. The tests drive the same loop with a fake backend to check
admission and batching on the CPU.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import time
from typing import Any, Callable

import numpy as np


@dataclasses.dataclass
class Request:
    id: int
    arrival: float
    nx: int
    ny: int
    nz: int
    slab: tuple
    porosity: float
    corr_len: float
    Da: float
    seed: int


@dataclasses.dataclass
class Record:
    id: int
    arrival: float
    admitted: float = float("nan")
    finished: float = float("nan")
    steps: int = 0
    converged: bool = False
    eta: float = float("nan")
    cells: int = 0
    footprint: int = 0
    status: str = "waiting"  # converged | capped | rejected | failed | diverged
    error: str = ""


LBM_ERR_DIVERGED = -4


class Diverged(RuntimeError):
    """A resident simulation's observables show NaN or a non-positive mass."""


class LbmBackend:
    """Device operations through liblbm (all on one device)."""

    def __init__(self, storage, layout, n_species=2, tau=0.8, rho_in=1.001, rho_out=1.0, c_in=1.0, pS_R=0.95,
                 pS_P=0.0, deterministic=True):
        import torch

        from . import lbm

        self.lbm = lbm
        self.torch = torch
        # deterministic wall-hit sums: a request's result does not depend on
        # which other requests share its launches
        self.kw = dict(tau=tau, rho_in=rho_in, rho_out=rho_out, c_in=c_in, pS_R=pS_R, pS_P=pS_P,
                       n_species=n_species, storage=storage, layout=layout, deterministic=deterministic)
        self.step_stream = torch.cuda.Stream()

    def footprint(self, r: Request) -> int:
        return self.lbm.request_footprint(r.nx, r.ny, r.nz, n_species=self.kw["n_species"],
                                          storage=self.kw["storage"])

    def create(self, r: Request):
        """Runs on the worker thread: geometry + initial state, synchronised.
        Each request gets a stream of its own, so that polling its
        conversion (on that stream) never waits behind another request's
        build."""
        st = self.torch.cuda.Stream()
        g = self.lbm.Geometry(r.nx, r.ny, r.nz, slab=r.slab, porosity=r.porosity, corr_len=r.corr_len,
                              seed=r.seed, stream=st)
        s = self.lbm.Simulation(g, Da=r.Da, stream=st, **self.kw)
        return (g, s, st), g.info()["n_fluid"]

    def step(self, handles, nsteps):
        self.lbm.step_batch([h[1] for h in handles], nsteps, stream=self.step_stream)

    def eta(self, h) -> float:
        """eta of a resident simulation; raises Diverged on NaN."""
        try:
            return h[1].observables_noalloc()["eta"]
        except self.lbm.LbmError as e:
            if e.code == LBM_ERR_DIVERGED:
                raise Diverged(str(e)) from e
            raise

    def free(self, h):
        h[1].close()
        h[0].close()


class ServingLoop:
    def __init__(self, backend, budget_bytes: int, steps_per_tick=100, check_every=1000, max_steps=20000,
                 tol=1e-8, clock: Callable[[], float] = time.perf_counter, sleep=time.sleep, workers=1):
        assert check_every % steps_per_tick == 0, "checks fall on tick boundaries"
        self.be = backend
        self.budget = int(budget_bytes)
        self.k = int(steps_per_tick)
        self.check_every = int(check_every)
        self.max_steps = int(max_steps)
        self.tol = float(tol)
        self.clock = clock
        self.sleep = sleep
        self.workers = workers
        self.trace: list = []  # (time, event, request id) for tests and logs

    def run(self, requests):
        reqs = sorted(requests, key=lambda r: (r.arrival, r.id))
        recs = {r.id: Record(r.id, r.arrival) for r in reqs}
        waiting = collections.deque(reqs)
        building: dict = {}  # future -> request
        resident: list = []  # [request, handle, steps, eta_prev]
        used = 0
        cell_updates = 0
        t0 = self.clock()
        # workers = 0 builds inline (deterministic; used by the tests)
        ex = concurrent.futures.ThreadPoolExecutor(self.workers) if self.workers > 0 else _InlineExecutor()
        try:
            while waiting or building or resident:
                now = self.clock() - t0
                # admission: arrived, in order, while the footprint fits
                while waiting and waiting[0].arrival <= now:
                    r = waiting[0]
                    fp = self.be.footprint(r)
                    if fp > self.budget:
                        waiting.popleft()
                        self._end(recs[r.id], now, "rejected", f"needs {fp} bytes, budget {self.budget}")
                        self.trace.append((now, "reject", r.id))
                        continue
                    if used + fp > self.budget:
                        break
                    waiting.popleft()
                    used += fp
                    recs[r.id].footprint = fp
                    recs[r.id].admitted = now
                    self.trace.append((now, "admit", r.id))
                    building[ex.submit(self.be.create, r)] = r
                # geometries that finished building join the batch
                for fut in [f for f in building if f.done()]:
                    r = building.pop(fut)
                    try:
                        h, cells = fut.result()
                    except Exception as e:  # the build failed: release the reservation
                        used -= recs[r.id].footprint
                        self._end(recs[r.id], self.clock() - t0, "failed", repr(e))
                        self.trace.append((self.clock() - t0, "fail", r.id))
                        continue
                    recs[r.id].cells = cells
                    resident.append([r, h, 0, None])
                    self.trace.append((self.clock() - t0, "resident", r.id))
                if not resident:
                    nxt = waiting[0].arrival - now if waiting else 0.0
                    if building:
                        concurrent.futures.wait(list(building), timeout=max(nxt, 0.0) or None,
                                                return_when=concurrent.futures.FIRST_COMPLETED)
                    elif nxt > 0:
                        self.sleep(nxt)
                    continue
                # one tick: every resident simulation advances k steps, one
                # batched launch per step
                self.be.step([x[1] for x in resident], self.k)
                self.trace.append((self.clock() - t0, "tick", len(resident)))
                done = []
                for x in resident:
                    r = x[0]
                    x[2] += self.k
                    cell_updates += recs[r.id].cells * self.k
                    if x[2] % self.check_every == 0 or x[2] >= self.max_steps:
                        try:
                            eta = self.be.eta(x[1])
                        except Diverged as e:
                            recs[r.id].steps = x[2]
                            self._end(recs[r.id], self.clock() - t0, "diverged", str(e))
                            done.append(x)
                            continue
                        prev = x[3]
                        # eta = 0 means no product has reached the outlet yet:
                        # not a steady state however flat it looks
                        conv = prev is not None and eta > 0.0 and abs(eta - prev) <= self.tol * abs(eta)
                        x[3] = eta
                        if conv or x[2] >= self.max_steps:
                            rec = recs[r.id]
                            rec.steps = x[2]
                            rec.converged = bool(conv)
                            rec.eta = eta
                            self._end(rec, self.clock() - t0, "converged" if conv else "capped")
                            done.append(x)
                for x in done:
                    resident.remove(x)
                    self.be.free(x[1])
                    used -= recs[x[0].id].footprint
                    self.trace.append((self.clock() - t0, "retire", x[0].id))
        finally:
            ex.shutdown(wait=True)
        wall = self.clock() - t0
        return summarize(list(recs.values()), wall, cell_updates)

    @staticmethod
    def _end(rec, t, status, error=""):
        rec.finished = t
        rec.status = status
        rec.error = error


class _InlineExecutor:
    def submit(self, fn, *args):
        f = concurrent.futures.Future()
        try:
            f.set_result(fn(*args))
        except Exception as e:
            f.set_exception(e)
        return f

    def shutdown(self, wait=True):
        pass


def summarize(recs, wall, cell_updates):
    """Latency percentiles over the requests that ran to the end (converged or
    capped); failures are counted by status."""
    ok = [r for r in recs if r.status in ("converged", "capped")] or recs
    lat = np.array([r.finished - r.arrival for r in ok])
    svc = np.array([r.finished - r.admitted for r in ok])
    pct = lambda a, q: float(np.percentile(a, q)) if a.size else float("nan")
    out = {
        "requests": len(recs),
        "wall_s": wall,
        "p50_s": pct(lat, 50),
        "p99_s": pct(lat, 99),
        "service_p50_s": pct(svc, 50),
        "service_p99_s": pct(svc, 99),
        "throughput_req_s": len(ok) / wall if wall > 0 else float("nan"),
        "MLUPS": cell_updates / wall / 1e6 if wall > 0 else float("nan"),
        "converged": int(sum(r.converged for r in recs)),
        "status": {k: sum(r.status == k for r in recs)
                   for k in ("converged", "capped", "rejected", "failed", "diverged")},
    }
    out["records"] = [dataclasses.asdict(r) for r in recs]
    return out


def requests_from_workload(items) -> list:
    return [Request(id=d["id"], arrival=d["arrival"], nx=d["nx"], ny=d["ny"], nz=d["nz"], slab=tuple(d["slab"]),
                    porosity=d["porosity"], corr_len=d["corr_len"], Da=d["Da"], seed=d["seed"]) for d in items]
