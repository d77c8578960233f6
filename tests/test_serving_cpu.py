"""Serving loop logic on the CPU with a fake device backend and a fake clock:
admission by footprint in arrival order, continuous batching, retirement on
convergence or at the step cap, the latency statistics, and per-request
failures (rejected, failed build, diverged) that leave the other requests
running. The failures are made on the host by the fake backend."""
import pytest

from paper_1607_02874_gb300.serving import Diverged, Request, ServingLoop, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeBackend:
    """Each step of a batched tick costs `step_cost` seconds per resident
    simulation. Request i's eta stops changing after converge_after[i] steps."""

    def __init__(self, clock, footprints, converge_after, step_cost=1e-4, fail_build=(), diverge_at=None):
        self.fail_build = set(fail_build)
        self.diverge_at = diverge_at or {}
        self.clock = clock
        self.fp = footprints
        self.conv = converge_after
        self.cost = step_cost
        self.steps = {}
        self.batches = []
        self.freed = []

    def footprint(self, r):
        return self.fp[r.id]

    def create(self, r):
        if r.id in self.fail_build:
            raise MemoryError(f"allocation failed for request {r.id}")
        self.steps[r.id] = 0
        return r.id, 1000

    def step(self, handles, nsteps):
        self.batches.append(sorted(handles))
        for h in handles:
            self.steps[h] += nsteps
        self.clock.t += self.cost * nsteps * len(handles)

    def eta(self, h):
        if h in self.diverge_at and self.steps[h] >= self.diverge_at[h]:
            raise Diverged(f"request {h}: NaN in a plane sum")
        s = min(self.steps[h], self.conv[h])
        return 0.5 * (1.0 - 0.5 ** (s / 100.0))

    def free(self, h):
        self.freed.append(h)


def _req(i, t):
    return Request(id=i, arrival=t, nx=8, ny=8, nz=8, slab=(2, 6), porosity=0.6, corr_len=2.0, Da=1.0, seed=i)


def test_admission_respects_budget_and_order():
    clk = FakeClock()
    be = FakeBackend(clk, {0: 60, 1: 60, 2: 30}, {0: 1000, 1: 1000, 2: 1000})
    loop = ServingLoop(be, budget_bytes=100, steps_per_tick=100, check_every=500, max_steps=5000, tol=1e-12,
                       clock=clk, sleep=clk.sleep, workers=0)
    out = loop.run([_req(0, 0.0), _req(1, 0.0), _req(2, 0.01)])
    adm = [e for e in loop.trace if e[1] == "admit"]
    ret = [e for e in loop.trace if e[1] == "retire"]
    # request 1 (60) cannot join request 0 (60) under a budget of 100: it is
    # admitted only after 0 retires; request 2 queues behind 1 (arrival order)
    assert [a[2] for a in adm] == [0, 1, 2]
    t_ret0 = next(e[0] for e in ret if e[2] == 0)
    assert next(a[0] for a in adm if a[2] == 1) >= t_ret0
    assert next(a[0] for a in adm if a[2] == 2) >= next(a[0] for a in adm if a[2] == 1)
    # 1 and 2 (60 + 30 <= 100) were resident together: batched in one launch
    assert any(b == [1, 2] for b in be.batches)
    assert sorted(be.freed) == [0, 1, 2]
    assert out["requests"] == 3 and out["converged"] == 3


def test_continuous_batching_admits_arrivals_into_running_batch():
    clk = FakeClock()
    be = FakeBackend(clk, {i: 10 for i in range(4)}, {0: 3000, 1: 3000, 2: 1000, 3: 1000})
    loop = ServingLoop(be, budget_bytes=100, steps_per_tick=100, check_every=500, max_steps=10000, tol=1e-12,
                       clock=clk, sleep=clk.sleep, workers=0)
    loop.run([_req(0, 0.0), _req(1, 0.0), _req(2, 0.05), _req(3, 0.05)])
    # the late arrivals joined the batch while 0 and 1 were still running
    assert any(b == [0, 1, 2, 3] for b in be.batches)
    assert be.batches[0] == [0, 1]


def test_step_cap_and_convergence_flags():
    clk = FakeClock()
    be = FakeBackend(clk, {0: 1, 1: 1}, {0: 500, 1: 10 ** 9})
    loop = ServingLoop(be, budget_bytes=10, steps_per_tick=250, check_every=500, max_steps=2000, tol=1e-12,
                       clock=clk, sleep=clk.sleep, workers=0)
    out = loop.run([_req(0, 0.0), _req(1, 0.0)])
    recs = {r["id"]: r for r in out["records"]}
    assert recs[0]["converged"] and recs[0]["steps"] == 1000  # flat from 500 on: seen at the second check
    assert not recs[1]["converged"] and recs[1]["steps"] == 2000  # cap


def test_oversized_request_is_rejected_and_others_run():
    clk = FakeClock()
    be = FakeBackend(clk, {0: 500, 1: 50}, {0: 100, 1: 500})
    loop = ServingLoop(be, budget_bytes=100, steps_per_tick=100, check_every=500, max_steps=5000, tol=1e-12,
                       clock=clk, sleep=clk.sleep, workers=0)
    out = loop.run([_req(0, 0.0), _req(1, 0.0)])
    recs = {r["id"]: r for r in out["records"]}
    assert recs[0]["status"] == "rejected" and "budget" in recs[0]["error"]
    assert recs[1]["status"] == "converged"
    assert out["status"]["rejected"] == 1 and out["status"]["converged"] == 1
    assert 0 not in be.steps  # never built


def test_failed_build_releases_its_reservation():
    clk = FakeClock()
    # 0 and 1 cannot be resident together (60 + 60 > 100): 1 waits for 0's
    # reservation, which the failed build must give back
    be = FakeBackend(clk, {0: 60, 1: 60}, {0: 500, 1: 500}, fail_build={0})
    loop = ServingLoop(be, budget_bytes=100, steps_per_tick=100, check_every=500, max_steps=5000, tol=1e-12,
                       clock=clk, sleep=clk.sleep, workers=0)
    out = loop.run([_req(0, 0.0), _req(1, 0.0)])
    recs = {r["id"]: r for r in out["records"]}
    assert recs[0]["status"] == "failed" and "MemoryError" in recs[0]["error"]
    assert recs[1]["status"] == "converged"
    assert be.freed == [1]


def test_diverged_simulation_retires_and_the_batch_continues():
    clk = FakeClock()
    be = FakeBackend(clk, {0: 10, 1: 10, 2: 10}, {0: 1000, 1: 1000, 2: 1000}, diverge_at={1: 500})
    loop = ServingLoop(be, budget_bytes=100, steps_per_tick=100, check_every=500, max_steps=5000, tol=1e-12,
                       clock=clk, sleep=clk.sleep, workers=0)
    out = loop.run([_req(0, 0.0), _req(1, 0.0), _req(2, 0.0)])
    recs = {r["id"]: r for r in out["records"]}
    assert recs[1]["status"] == "diverged" and recs[1]["steps"] == 500
    assert recs[0]["status"] == recs[2]["status"] == "converged"
    assert sorted(be.freed) == [0, 1, 2]
    # after the divergence, 1 is no longer in any launch
    assert all(1 not in b for b in be.batches[5:])
    assert out["status"]["diverged"] == 1
    # latency percentiles cover only the requests that ran to the end
    assert out["p50_s"] == pytest.approx(recs[0]["finished"])


def test_summary_percentiles():
    from paper_1607_02874_gb300.serving import Record

    recs = [Record(id=i, arrival=0.0, admitted=0.0, finished=float(i + 1), status="converged") for i in range(100)]
    s = summarize(recs, wall=100.0, cell_updates=10 ** 9)
    assert s["p50_s"] == pytest.approx(50.5)
    assert s["p99_s"] == pytest.approx(99.01)
    assert s["MLUPS"] == pytest.approx(10.0)
