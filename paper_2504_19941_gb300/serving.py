"""Serving loop: continuous batching of wetting studies on one GPU.

Requests (lattices of different sizes, geometries and contact angles) arrive
over time.  The scheduler admits them FIFO as soon as their workspace fits in
the HBM budget, keeps every admitted lattice resident, and advances them in
quanta of steps: the small lattices in one persistent batched launch
(``dsm_batch_step``), each large one with ``dsm_step`` on its own CUDA stream so
their work overlaps on the device.  With an executor that launches without
waiting (``launch`` / ``poll``), each lattice's quantum completes on its own: a
CUDA event per stream tells the host which lattices are idle, those get their
next quantum at once, finished requests retire and free their memory, and new
arrivals are admitted, without waiting for the rest of the device.  A
request's latency is finish time minus arrival time; its result is the
lattice's observables and the apparent contact angle of its drop.

One large lattice nearly fills the GPU by itself, so advancing every admitted
large lattice at once only makes them all finish late.  ``max_large`` caps how
many large lattices are active together (small ones are still admitted
freely), and ``order="sjf"`` takes waiting large requests shortest work
(nodes x steps) first.

``Scheduler`` is host logic only; ``GpuExecutor`` does the device work through
libdsm.  Tests drive the scheduler with fake executors on the CPU.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field


@dataclass
class Record:
    rid: int
    arrival: float
    admitted: float = math.nan
    finished: float = math.nan
    status: str = "pending"      # done | rejected | failed
    steps: int = 0
    nodes: int = 0
    result: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Slot:
    req: object
    rec: Record
    handle: object
    nbytes: int
    remaining: int
    inflight: int = 0            # steps of the quantum on the device (asynchronous path)


class Scheduler:
    """Admission by HBM budget + continuous batching in quanta of steps.

    executor interface:
      bytes_needed(req) -> int            workspace bytes (host-side, no device work)
      is_large(req) -> bool               (optional) counts against max_large
      admit(req) -> handle                 create and initialise the lattice
      advance([(handle, steps)]) -> {handle: error-or-None}
                                           advance every active lattice, wait for it
      finish(handle) -> dict               result of a finished lattice, release it
      release(handle)                      release a failed lattice
    or, instead of advance, the asynchronous pair
      launch([(handle, steps)]) -> handles queue a quantum for each lattice, do not wait;
                                           returns the lattices it queued (None: all;
                                           the others stay idle and are offered again)
      poll(timeout) -> [(handle, error-or-None)]
                                           lattices whose quantum completed (waits at
                                           most timeout seconds for one; None: until one)
    and optionally drain(), called once at the end (results computed in the
    background are complete after it).
    """

    def __init__(self, executor, budget_bytes: int, quantum: int = 200, clock=time.perf_counter,
                 sleep=time.sleep, max_large=None, order: str = "fifo"):
        if order not in ("fifo", "sjf"):
            raise ValueError("order must be 'fifo' or 'sjf'")
        self.ex = executor
        self.budget = int(budget_bytes)
        self.quantum = int(quantum)
        self.clock = clock
        self.sleep = sleep
        self.max_large = max_large
        self.order = order

    def _large(self, req) -> bool:
        f = getattr(self.ex, "is_large", None)
        return bool(f(req)) if f is not None else False

    def run(self, requests):
        if hasattr(self.ex, "launch") and hasattr(self.ex, "poll"):
            recs = self._run_async(requests)
        else:
            recs = self._run_sync(requests)
        drain = getattr(self.ex, "drain", None)
        if drain is not None:
            drain()
        return recs

    def _admit(self, waiting, active, recs, used, t0):
        """Admission in arrival order (large requests shortest work first under
        "sjf") while the next request fits in the budget; a large request waits
        for a free large slot without holding up the rest.  Returns the bytes
        now in use."""
        if self.order == "sjf":
            queue = sorted(waiting, key=lambda r: (1, r.n * r.steps, r.arrival)
                           if self._large(r) else (0, r.arrival, 0))
        else:
            queue = list(waiting)
        n_large = sum(1 for sl in active if self._large(sl.req))
        for req in queue:
            rec = recs[req.rid]
            try:
                need = int(self.ex.bytes_needed(req))
            except Exception as e:  # malformed request: reject, keep serving
                waiting.remove(req)
                rec.status, rec.finished = "rejected", self.clock() - t0
                rec.result = {"error": str(e)}
                continue
            if need > self.budget:
                waiting.remove(req)
                rec.status, rec.finished = "rejected", self.clock() - t0
                rec.result = {"error": f"needs {need} bytes, budget {self.budget}"}
                continue
            if used + need > self.budget:
                break
            large = self._large(req)
            if large and self.max_large is not None and n_large >= self.max_large:
                continue
            waiting.remove(req)
            try:
                h = self.ex.admit(req)
            except Exception as e:
                rec.status, rec.finished = "failed", self.clock() - t0
                rec.result = {"error": str(e)}
                continue
            used += need
            n_large += large
            rec.admitted = self.clock() - t0
            active.append(_Slot(req, rec, h, need, int(req.steps)))
        return used

    def _retire(self, s, k, err, t0):
        """Account a completed quantum of k steps; True when the slot is done
        (finished or failed) and released."""
        if err is not None:
            self.ex.release(s.handle)
            s.rec.status, s.rec.finished = "failed", self.clock() - t0
            s.rec.result = {"error": str(err)}
            return True
        s.remaining -= k
        if s.remaining <= 0:
            s.rec.result = self.ex.finish(s.handle)
            s.rec.status = "failed" if "error" in s.rec.result else "done"
            s.rec.finished = self.clock() - t0
            return True
        return False

    def _run_async(self, requests):
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque = deque()
        active: list[_Slot] = []
        used = 0
        recs = {r.rid: Record(r.rid, r.arrival, steps=r.steps, nodes=int(r.n)) for r in requests}
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            used = self._admit(waiting, active, recs, used, t0)
            idle = [s for s in active if s.inflight == 0]
            if idle:
                work = [(s.handle, min(self.quantum, s.remaining)) for s in idle]
                queued = self.ex.launch(work)
                queued = None if queued is None else set(queued)
                for s, (_, k) in zip(idle, work):
                    if queued is None or s.handle in queued:
                        s.inflight = k
            if not active:
                if pending:
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(min(wait, 0.05))
                continue
            # wait for a quantum to complete, or until the next arrival is due
            timeout = None
            if pending:
                timeout = max(0.0, min(pending[0].arrival - (self.clock() - t0), 0.05))
            elif waiting:
                timeout = 0.05
            done = dict(self.ex.poll(timeout))
            if not done:
                continue
            still = []
            for s in active:
                if s.handle in done:
                    k, s.inflight = s.inflight, 0
                    if self._retire(s, k, done[s.handle], t0):
                        used -= s.nbytes
                        continue
                still.append(s)
            active = still
        return [recs[r.rid] for r in requests]

    def _run_sync(self, requests):
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque = deque()
        active: list[_Slot] = []
        used = 0
        recs = {r.rid: Record(r.rid, r.arrival, steps=r.steps, nodes=int(r.n)) for r in requests}
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            used = self._admit(waiting, active, recs, used, t0)
            if not active:
                if pending:
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(min(wait, 0.05))
                continue
            work = [(s.handle, min(self.quantum, s.remaining)) for s in active]
            errors = self.ex.advance(work) or {}
            still = []
            for s, (_, k) in zip(active, work):
                if self._retire(s, k, errors.get(s.handle), t0):
                    used -= s.nbytes
                else:
                    still.append(s)
            active = still
        return [recs[r.rid] for r in requests]


def serial_run(executor, requests, clock=time.perf_counter, sleep=time.sleep):
    """Baseline: the same stream served one request at a time, in arrival order."""
    recs = []
    t0 = clock()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if req.arrival > now:
            sleep(req.arrival - now)
        rec = Record(req.rid, req.arrival, steps=req.steps, nodes=int(req.n))
        try:
            h = executor.admit(req)
        except Exception as e:
            rec.status, rec.finished, rec.result = "failed", clock() - t0, {"error": str(e)}
            recs.append(rec)
            continue
        rec.admitted = clock() - t0
        err = (executor.advance([(h, int(req.steps))]) or {}).get(h)
        if err is not None:
            executor.release(h)
            rec.status, rec.result = "failed", {"error": str(err)}
        else:
            rec.result = executor.finish(h)
            rec.status = "failed" if "error" in rec.result else "done"
        rec.finished = clock() - t0
        recs.append(rec)
    drain = getattr(executor, "drain", None)
    if drain is not None:
        drain()
    return recs


def _angle(c2, c1):
    from .analysis import apparent_contact_angle
    return apparent_contact_angle(c2, c1)


def summarize(records, wall: float) -> dict:
    done = [r for r in records if r.status == "done"]
    lat = sorted(r.latency for r in done)

    def pct(p):
        if not lat:
            return math.nan
        k = min(len(lat) - 1, max(0, int(math.ceil(p / 100.0 * len(lat))) - 1))
        return lat[k]
    lu = sum(r.nodes * r.steps for r in done)
    return {"solves": len(done), "rejected": sum(r.status == "rejected" for r in records),
            "failed": sum(r.status == "failed" for r in records), "wall_s": wall,
            "solves_per_s": len(done) / wall if wall > 0 else math.nan,
            "p50_s": pct(50), "p99_s": pct(99), "mean_s": sum(lat) / len(lat) if lat else math.nan,
            "glups": lu / wall / 1e9 if wall > 0 else math.nan}


class GpuExecutor:
    """Device work of the scheduler through libdsm: one Lattice per request,
    small lattices advanced together by dsm_batch_step on the current stream
    (one launch per lattice kind), large ones by dsm_step, each on a stream of
    its own.

    ``advance`` waits for the whole quantum (the synchronous interface);
    ``launch`` / ``poll`` queue the quanta and report lattices whose quantum
    completed through CUDA events, each large lattice on its own stream; at most
    one batched launch of small lattices is in flight (dsm_batch_step waits for
    its stream while it stages the work list).  A finished lattice's result is
    its observables and, with angles=True, the apparent contact angle of its
    drop (analysis.apparent_contact_angle on the final C2 and C1), fitted in a
    worker thread so that the loop goes on; drain() waits for the fits."""

    def __init__(self, precision="f32", small_nodes=300_000, device="cuda", angles=True):
        import torch
        from concurrent.futures import ThreadPoolExecutor
        self.torch = torch
        self.precision = precision
        self.small_nodes = small_nodes
        self.device = torch.device(device)
        self.batch_scratch = None
        self.angles = angles
        self.inflight = {}        # lattice -> CUDA event of its queued quantum
        self.batch_event = None   # event of the batched launch in flight
        self.pool = ThreadPoolExecutor(max_workers=4) if angles else None
        self.pending_fits = []

    def _params(self, case):
        from . import make_params
        return make_params(case.lattice, case.shape, self.precision, theta_deg=case.theta_deg,
                           g12=case.g12, g23=case.g23, alpha=case.alpha, alpha_s=case.alpha_s,
                           rho2=case.rho2, rho3=case.rho3, tau2=case.tau2, tau3=case.tau3,
                           tau_g=case.tau_g, body=case.body, faces=case.faces)

    def is_large(self, req) -> bool:
        return req.n > self.small_nodes

    def bytes_needed(self, req):
        from . import _lib, make_params
        p = make_params(req.lattice, req.shape, self.precision, theta_deg=req.theta_deg)
        return _lib.dsm_workspace_bytes(p)

    def admit(self, req):
        from . import Lattice
        torch = self.torch
        case = getattr(req, "payload", None) or req.case()
        main = torch.cuda.current_stream(self.device)
        # large lattices, and lattices with mirror or wall faces (which the
        # batched step does not take), get a stream of their own (their steps
        # overlap on the device); small ones share the current stream, which
        # the batched launch requires
        solo = req.n > self.small_nodes or any(f not in (None, 0, "periodic")
                                                for f in (case.faces or ()))
        stream = torch.cuda.Stream(self.device) if solo else main
        lat = Lattice(self._params(case), device=self.device, stream=stream)
        lat.solo = solo
        sd = torch.as_tensor(case.solid_sd, dtype=lat.real, device=self.device)
        c2 = torch.as_tensor(case.c2, dtype=lat.real, device=self.device)
        stream.wait_stream(main)
        lat.set_solid_distance(sd)
        lat.set_fluid(c2)
        torch.cuda.synchronize(self.device)  # inputs may be freed after this
        lat.req = req
        return lat

    def _queue(self, work):
        """Queue the quanta: large lattices with dsm_step on their own streams,
        small ones in one batched launch per lattice kind on the current
        stream.  Returns {lattice: event recorded after its quantum}."""
        from . import _lib
        torch = self.torch
        small = [(h, k) for h, k in work if not h.solo and k > 0]
        large = [(h, k) for h, k in work if h.solo and k > 0]
        events = {}
        for h, k in large:  # queued on each lattice's own stream
            _lib.dsm_step(h.h, k)
            ev = torch.cuda.Event()
            ev.record(h.stream)
            events[h] = ev
        # one batched launch per lattice kind (a batch shares kind and precision)
        for kind in sorted({h.params.lattice for h, _ in small}):
            grp = [(h, k) for h, k in small if h.params.lattice == kind]
            hs = [h.h for h, _ in grp]
            nb = _lib.dsm_batch_scratch_bytes(hs)
            if self.batch_scratch is None or self.batch_scratch.numel() < nb:
                self.batch_scratch = torch.empty(max(nb, 1 << 20), dtype=torch.uint8,
                                                 device=self.device)
            _lib.dsm_batch_step(hs, [k for _, k in grp], self.batch_scratch,
                                self.batch_scratch.numel())
        if small:
            ev = torch.cuda.Event()
            ev.record(torch.cuda.current_stream(self.device))
            for h, _ in small:
                events[h] = ev
            self.batch_event = ev
        for h, k in work:           # a zero-step quantum completes at once
            if k <= 0:
                events[h] = None
        return events

    def advance(self, work):
        self._queue(work)
        self.torch.cuda.synchronize(self.device)
        self.batch_event = None
        return {}

    def launch(self, work):
        # at most one batched launch in flight: small lattices whose batch is
        # still running, or that would start a second batch, wait for the next
        # round (they stay idle and are offered again)
        if self.batch_event is not None and not self.batch_event.query():
            work = [(h, k) for h, k in work if h.solo]
        else:
            self.batch_event = None
        self.inflight.update(self._queue(work))
        return [h for h, _ in work]

    def poll(self, timeout=None):
        """Lattices whose queued quantum has completed, waiting up to timeout
        seconds (None: until one does)."""
        t_end = None if timeout is None else time.perf_counter() + timeout
        while True:
            done = [h for h, ev in self.inflight.items() if ev is None or ev.query()]
            if done:
                for h in done:
                    del self.inflight[h]
                return [(h, None) for h in done]
            if not self.inflight or (t_end is not None and time.perf_counter() >= t_end):
                return []
            time.sleep(1e-4)

    def finish(self, lat):
        """Result of a finished lattice (its observables, and the apparent
        contact angle fitted in the background), then release it.  A lattice
        whose state holds a NaN/Inf, or whose batched launch timed out, reports
        an error instead."""
        from . import _lib
        ob = lat.observables(check=False)   # synchronises the lattice's stream
        if ob["status"] != 0:
            self.release(lat)
            return {"error": _lib.status_string(ob["status"]), "step": ob["step"]}
        res = {"mass_c2": ob["mass_c2"], "max_u": ob["max_u"], "step": ob["step"]}
        if self.angles:
            nx, ny, nz = lat.shape
            shape = (ny, nx) if lat.params.lattice == 0 else (nz, ny, nx)
            c2 = lat.field("C2")            # written on the lattice's stream:
            c1 = lat.field("C1")
            lat.stream.synchronize()        # complete before torch reads them
            c2 = c2.double().cpu().numpy().reshape(shape)
            c1 = c1.double().cpu().numpy().reshape(shape)
            self.pending_fits.append((res, self.pool.submit(_angle, c2, c1)))
        self.release(lat)
        return res

    def drain(self):
        """Wait for the background contact-angle fits and store them."""
        for res, fut in self.pending_fits:
            res["theta_deg"] = fut.result()
        self.pending_fits = []

    def release(self, lat):
        lat.__del__()          # destroys the handle
        lat.workspace = None   # returns the workspace to torch's allocator
