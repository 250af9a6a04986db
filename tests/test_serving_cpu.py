"""Host logic of the serving loop, on the CPU with fake executors and a fake
clock: admission by HBM budget, FIFO order, rejection of malformed and
oversized requests, failures injected on the host, quantum accounting,
latency percentiles, the cap on concurrent large lattices and shortest-job-first
order -- with the synchronous executor (every quantum waits for the whole
device) and the asynchronous one (each lattice's quantum completes on its own,
as CUDA events on separate streams report it)."""
import math
from dataclasses import dataclass

import pytest

from paper_2504_19941_gb300.serving import Scheduler, serial_run, summarize  # noqa: E402


@dataclass
class Req:
    rid: int
    arrival: float
    steps: int
    n: int
    nbytes: int = 100
    bad: bool = False


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeExecutor:
    """Each step of a lattice costs `cost` seconds of fake time; a quantum over
    several lattices costs the sum (one device)."""

    def __init__(self, clock, cost=1e-3, fail=(), nan=(), large_n=None):
        self.clock = clock
        self.cost = cost
        self.fail = set(fail)      # rids whose advance reports an error
        self.nan = set(nan)        # rids whose finish reports a non-finite state
        self.large_n = large_n     # requests with n above this count as large
        self.live = {}
        self.steps = {}
        self.peak = 0
        self.peak_large = 0

    def is_large(self, req):
        return self.large_n is not None and req.n > self.large_n

    def bytes_needed(self, req):
        if req.bad:
            raise ValueError("malformed request")
        return req.nbytes

    def admit(self, req):
        h = ("h", req.rid)
        self.live[h] = req
        self.steps[req.rid] = 0
        self.peak = max(self.peak, sum(r.nbytes for r in self.live.values()))
        self.peak_large = max(self.peak_large, sum(self.is_large(r) for r in self.live.values()))
        return h

    def advance(self, work):
        errs = {}
        for h, k in work:
            self.steps[h[1]] += k
            self.clock.t += self.cost * k
            if h[1] in self.fail:
                errs[h] = "injected device error"
        return errs

    def finish(self, h):
        req = self.live.pop(h)
        if req.rid in self.nan:
            return {"error": "non-finite population"}
        return {"steps": self.steps[req.rid]}

    def release(self, h):
        self.live.pop(h, None)


class FakeAsyncExecutor(FakeExecutor):
    """launch / poll: a queued quantum of k steps completes cost * k seconds of
    fake time after it was queued, and quanta of different lattices overlap
    (streams); poll moves the clock to the next completion."""

    def __init__(self, clock, **kw):
        super().__init__(clock, **kw)
        self.due = {}
        self.launches = 0

    def launch(self, work):
        self.launches += 1
        for h, k in work:
            self.steps[h[1]] += k
            self.due[h] = self.clock.t + self.cost * k
        return [h for h, _ in work]

    def poll(self, timeout):
        if not self.due:
            return []
        t_next = min(self.due.values())
        if timeout is not None and t_next > self.clock.t + timeout:
            self.clock.t += timeout
            return []
        self.clock.t = max(self.clock.t, t_next)
        done = [h for h, t in self.due.items() if t <= self.clock.t]
        for h in done:
            del self.due[h]
        return [(h, "injected device error" if h[1] in self.fail else None) for h in done]


MODES = ["sync", "async"]


def _run(reqs, budget=1000, quantum=10, max_large=None, order="fifo", mode="sync", **kw):
    clk = Clock()
    ex = (FakeAsyncExecutor if mode == "async" else FakeExecutor)(clk, **kw)
    sch = Scheduler(ex, budget, quantum, clock=clk, sleep=clk.sleep, max_large=max_large,
                    order=order)
    recs = sch.run(reqs)
    return recs, ex, clk


@pytest.mark.parametrize("mode", MODES)
def test_every_request_gets_exactly_its_steps(mode):
    reqs = [Req(i, 0.01 * i, steps=7 + 13 * i, n=10) for i in range(8)]
    recs, ex, _ = _run(reqs, quantum=10, mode=mode)
    assert all(r.status == "done" for r in recs)
    assert all(ex.steps[r.rid] == r.steps for r in reqs)
    assert all(r.finished >= r.admitted >= r.arrival - 1e-12 for r in recs)


@pytest.mark.parametrize("mode", MODES)
def test_budget_is_never_exceeded_and_admission_is_fifo(mode):
    reqs = [Req(i, 0.0, steps=50, n=10, nbytes=400) for i in range(6)]
    recs, ex, _ = _run(reqs, budget=1000, quantum=10, mode=mode)
    assert ex.peak <= 1000
    adm = [r.admitted for r in recs]
    assert adm == sorted(adm)               # FIFO
    assert adm[2] > adm[1] and adm[1] == adm[0]  # only two fit at a time


@pytest.mark.parametrize("mode", MODES)
def test_rejections_and_failures_do_not_stop_the_loop(mode):
    reqs = [Req(0, 0.0, 30, 10), Req(1, 0.0, 30, 10, bad=True),
            Req(2, 0.0, 30, 10, nbytes=5000), Req(3, 0.0, 30, 10), Req(4, 0.0, 30, 10),
            Req(5, 0.0, 30, 10)]
    recs, ex, _ = _run(reqs, budget=1000, fail={3}, nan={4}, mode=mode)
    st = {r.rid: r.status for r in recs}
    assert st == {0: "done", 1: "rejected", 2: "rejected", 3: "failed", 4: "failed", 5: "done"}
    assert not ex.live                      # everything released
    s = summarize(recs, 1.0)
    assert s["solves"] == 2 and s["rejected"] == 2 and s["failed"] == 2


@pytest.mark.parametrize("mode", MODES)
def test_continuous_batching_admits_arrivals_between_quanta(mode):
    # a long request is running when a short one arrives; the short one must
    # not wait for the long one to finish
    reqs = [Req(0, 0.0, steps=1000, n=10), Req(1, 0.05, steps=20, n=10)]
    recs, _, _ = _run(reqs, quantum=10, cost=1e-3, mode=mode)
    r0, r1 = recs
    assert r1.finished < r0.finished
    assert r1.admitted < 0.08


def test_serial_baseline_serves_in_order():
    reqs = [Req(i, 0.0, steps=100, n=10) for i in range(4)]
    clk = Clock()
    ex = FakeExecutor(clk)
    recs = serial_run(ex, reqs, clock=clk, sleep=clk.sleep)
    fin = [r.finished for r in recs]
    assert fin == sorted(fin)
    assert math.isclose(fin[-1], 4 * 100 * 1e-3)


def test_percentiles():
    from paper_2504_19941_gb300.serving import Record
    recs = [Record(i, 0.0, finished=float(i + 1), status="done", steps=1, nodes=1)
            for i in range(100)]
    s = summarize(recs, 10.0)
    assert s["p50_s"] == 50.0 and s["p99_s"] == 99.0 and s["solves_per_s"] == 10.0


@pytest.mark.parametrize("mode", MODES)
def test_large_cap_lets_small_requests_through(mode):
    # three large requests (n = 1000) and two small ones, all at once, cap 1:
    # never two large lattices at a time, and the small ones do not wait
    reqs = [Req(0, 0.0, 200, 1000), Req(1, 0.0, 200, 1000), Req(2, 0.0, 200, 1000),
            Req(3, 0.0, 30, 10), Req(4, 0.0, 30, 10)]
    recs, ex, _ = _run(reqs, budget=10 ** 6, quantum=10, max_large=1, large_n=100, mode=mode)
    assert all(r.status == "done" for r in recs)
    assert ex.peak_large == 1
    assert recs[3].admitted == 0.0 and recs[4].admitted == 0.0
    fin = [recs[i].finished for i in range(3)]
    assert fin == sorted(fin)              # FIFO among the large ones
    assert recs[3].finished < recs[0].finished


@pytest.mark.parametrize("mode", MODES)
def test_shortest_job_first_for_large_requests(mode):
    reqs = [Req(0, 0.0, 300, 1000), Req(1, 0.0, 100, 1000), Req(2, 0.0, 200, 1000)]
    recs, ex, _ = _run(reqs, budget=10 ** 6, quantum=10, max_large=1, order="sjf", large_n=100, mode=mode)
    order = sorted(range(3), key=lambda i: recs[i].finished)
    assert order == [1, 2, 0]
    # shortest first lowers the mean latency against arrival order
    fifo, _, _ = _run(reqs, budget=10 ** 6, quantum=10, max_large=1, large_n=100, mode=mode)
    assert sum(r.latency for r in recs) < sum(r.latency for r in fifo)
    with pytest.raises(ValueError):
        Scheduler(ex, 1, order="lifo")


def test_async_quanta_complete_on_their_own():
    """A long lattice's quanta (1000 steps, 1 s of device time each) do not
    hold back a short request arriving meanwhile: with the asynchronous
    executor it is admitted, advanced and finished while the long quantum is
    still running; with the synchronous one it waits for that quantum."""
    reqs = [Req(0, 0.0, steps=3000, n=10), Req(1, 0.2, steps=50, n=10)]
    rec_a, ex_a, _ = _run(reqs, quantum=1000, cost=1e-3, mode="async")
    rec_s, _, _ = _run(reqs, quantum=1000, cost=1e-3, mode="sync")
    assert all(r.status == "done" for r in rec_a + rec_s)
    assert ex_a.steps == {0: 3000, 1: 50}
    assert rec_a[1].finished < 0.3            # 0.2 arrival + 50 steps
    assert rec_s[1].finished > 1.0            # after the long lattice's first quantum
    assert rec_a[0].finished == pytest.approx(3.0)
