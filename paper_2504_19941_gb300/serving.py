"""Serving loop: continuous batching of wetting studies on one GPU.

Requests (lattices of different sizes, geometries and contact angles) arrive
over time.  The scheduler admits them FIFO as soon as their workspace fits in
the HBM budget, keeps every admitted lattice resident, and advances all of them
together in quanta of steps: the small lattices in one persistent batched launch
(``dsm_batch_step``), each large one with ``dsm_step`` on its own CUDA stream so
their work overlaps on the device.  Between quanta finished requests retire and
free their memory, and new arrivals are admitted.  A request's latency is
finish time minus arrival time.

One large lattice nearly fills the GPU by itself, so advancing every admitted
large lattice at once only makes them all finish late.  ``max_large`` caps how
many large lattices are active together (small ones are still admitted
freely), and ``order="sjf"`` takes waiting large requests shortest work
(nodes x steps) first.

``Scheduler`` is host logic only; ``GpuExecutor`` does the device work through
libdsm.  Tests drive the scheduler with a fake executor on the CPU.
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
            # admission in arrival order (large requests shortest work first
            # under "sjf") while the next request fits in the budget; a large
            # request waits for a free large slot without holding up the rest
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
                err = errors.get(s.handle)
                if err is not None:
                    self.ex.release(s.handle)
                    used -= s.nbytes
                    s.rec.status, s.rec.finished = "failed", self.clock() - t0
                    s.rec.result = {"error": str(err)}
                    continue
                s.remaining -= k
                if s.remaining <= 0:
                    s.rec.result = self.ex.finish(s.handle)
                    used -= s.nbytes
                    s.rec.status = "failed" if "error" in s.rec.result else "done"
                    s.rec.finished = self.clock() - t0
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
    return recs


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
    its own."""

    def __init__(self, precision="f32", small_nodes=300_000, device="cuda"):
        import torch
        self.torch = torch
        self.precision = precision
        self.small_nodes = small_nodes
        self.device = torch.device(device)
        self.batch_scratch = None

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

    def advance(self, work):
        from . import _lib
        torch = self.torch
        small = [(h, k) for h, k in work if not h.solo and k > 0]
        large = [(h, k) for h, k in work if h.solo and k > 0]
        for h, k in large:  # queued on each lattice's own stream
            _lib.dsm_step(h.h, k)
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
        torch.cuda.synchronize(self.device)
        return {}

    def finish(self, lat):
        """Result of a finished lattice (its observables), then release it.  A
        lattice whose state holds a NaN/Inf, or whose batched launch timed out,
        reports an error instead."""
        from . import _lib
        ob = lat.observables(check=False)
        self.release(lat)
        if ob["status"] != 0:
            return {"error": _lib.status_string(ob["status"]), "step": ob["step"]}
        return {"mass_c2": ob["mass_c2"], "max_u": ob["max_u"], "step": ob["step"]}

    def release(self, lat):
        lat.__del__()          # destroys the handle
        lat.workspace = None   # returns the workspace to torch's allocator
