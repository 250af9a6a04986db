"""Critical pressure of the Cassie-Baxter to Wenzel transition on micropillars
by energy minimisation (Sec. III, "Critical Pressure on Micropillared
Surfaces"; Eq. [frozen:pressure_const], Eq. [frozen:critical-pressure-cyl-2d]).

A liquid layer rests on the tops of pillars with gas in the gap between them.
The free energy carries a pressure term -dP V (V = sum_x C2), so a larger dP
pushes the liquid down into the gap.  Below the critical pressure the meniscus
stays on the pillar tops; above it the minimum is the collapsed state with the
gap full of liquid.  The critical pressure is found by bisection on dP to a set
tolerance (the paper uses 1e-4), each probe being a full L-BFGS minimisation of
the discrete free energy from the suspended initial state; a probe counts as
collapsed when the mean liquid concentration over the lower half of the gap
exceeds one half.  For the 2D geometry the paper compares with
dP_c = -2 gamma_lg cos(theta) / s, s the gap width.

All device work goes through libdsm: the solid profile (dsm_set_solid), the
energy and gradient (dsm_fe_energy_grad), the L-BFGS kernels, and the gap mean
(dsm_vec_dot against an indicator vector).

A sweep over several cases (contact angles, gap widths) runs its searches
concurrently (critical_sweep): one host thread and one CUDA stream per case.
The native L-BFGS loop releases the interpreter lock and waits only on its own
stream, so one search's host work (bisection, line search) overlaps the other
searches' kernels.
"""
from __future__ import annotations

import math
import time
from concurrent.futures import ThreadPoolExecutor

import torch

from . import Lattice, _lib, make_params
from .energy import FreeEnergy, _Vec, lbfgs


def critical_theory(gamma_lg: float, theta_deg: float, s: float) -> float:
    """dP_c = -2 gamma_lg cos(theta) / s (Eq. [frozen:critical-pressure-cyl-2d])."""
    return -2.0 * gamma_lg * math.cos(math.radians(theta_deg)) / s


class PillarGap:
    """One pillar-gap problem on the GPU: C1 from the solid's signed distance, the
    suspended initial liquid field, and the indicator of the gap's lower half.
    All of its work is queued on `stream` (None: the current stream)."""

    def __init__(self, case, device="cuda", tol=1e-6, max_iter=20000, stream=None):
        dev = torch.device(device)
        self.case = case
        self.tol, self.max_iter = tol, max_iter
        self.stream = stream
        self.params = make_params(case.lattice, case.shape, "f32", theta_deg=case.theta_deg,
                                  g12=case.g12, g23=case.g23, alpha=case.alpha,
                                  alpha_s=case.alpha_s)
        # C1 = 1/2 + tanh(d / (2 alpha_s)) / 2 by the library's solid-profile kernel
        lat = Lattice(self.params, device=dev, stream=stream)
        lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=torch.float32, device=dev))
        self.c1 = lat.field("C1").clone()
        del lat
        self.c2_0 = torch.as_tensor(case.c2, dtype=torch.float32, device=dev)
        gap = torch.as_tensor(case.extra["gap"], dtype=torch.long, device=dev)
        self.ind = torch.zeros(self.c2_0.numel(), dtype=torch.float32, device=dev)
        self.ind[gap] = 1.0
        self.n_gap = int(gap.numel())
        self.fe = FreeEnergy(self.params, device=dev, stream=stream)
        self.vec = _Vec(self.c2_0.numel(), dev, stream)
        self.iterations = 0
        self.probes = 0

    def relax(self, dP: float):
        """Minimise at pressure dP from the suspended state: (C2, energy, info)."""
        x, E, info = lbfgs(self.fe, self.c2_0, self.c1, active=2, dP=dP, tol=self.tol,
                           max_iter=self.max_iter)
        self.iterations += info["iterations"]
        self.probes += 1
        return x, E, info

    def gap_liquid(self, c2) -> float:
        """Mean C2 over the lower half of the gap."""
        return float(self.vec.dot(c2, self.ind).item()) / self.n_gap

    def collapsed(self, dP: float) -> bool:
        x, _, _ = self.relax(dP)
        return self.gap_liquid(x) > 0.5


def bisect_critical(collapsed, lo: float, hi: float, tol: float = 1e-4, max_widen: int = 8):
    """Bisection for the pressure where collapsed(dP) switches from False (lo) to
    True (hi).  The bracket is widened outward (doubling its width) until it
    holds the switch.  Returns (dP_c, lo, hi)."""
    width = hi - lo
    for _ in range(max_widen):
        if collapsed(hi):
            break
        lo, hi = hi, hi + width
        width *= 2.0
    else:
        raise RuntimeError("no collapse within the widened bracket")
    for _ in range(max_widen):
        if not collapsed(lo):
            break
        hi, lo = lo, lo - width
        width *= 2.0
    else:
        raise RuntimeError("collapsed at every pressure of the widened bracket")
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if collapsed(mid):
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi), lo, hi


def critical_pressure(case, tol: float = 1e-4, device="cuda", rms_tol=1e-6, max_iter=20000,
                      stream=None):
    """Critical pressure of a pillar-gap case (synthetic.pillar_gap_2d) by
    bisection, bracketed around the closed form.  Returns a dict with dP_c, the
    closed form, and the work done."""
    dev = torch.device(device)
    with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream(dev)):
        pg = PillarGap(case, device=dev, tol=rms_tol, max_iter=max_iter, stream=stream)
        th = critical_theory(case.g23, case.theta_deg, case.extra["s"])
        t0 = time.perf_counter()
        dpc, lo, hi = bisect_critical(pg.collapsed, th - 0.5 * abs(th) - 5e-3,
                                      th + 0.5 * abs(th) + 5e-3, tol)
        torch.cuda.current_stream(dev).synchronize()
    return {"dP_c": dpc, "bracket": (lo, hi), "theory": th, "ratio": dpc / th if th else math.nan,
            "probes": pg.probes, "iterations": pg.iterations,
            "seconds": time.perf_counter() - t0}


def critical_sweep(cases, tol: float = 1e-4, device="cuda", rms_tol=1e-6, max_iter=20000,
                   workers=None):
    """Critical pressures of several cases at once, each search on its own host
    thread and CUDA stream (at most `workers` at a time; default: all).  Every
    search owns its workspace and runs the same kernels as critical_pressure
    alone, so each result equals its one-at-a-time result.  Returns (results in
    case order, wall seconds)."""
    dev = torch.device(device)
    cases = list(cases)
    if not cases:
        return [], 0.0
    workers = len(cases) if workers is None else max(1, min(int(workers), len(cases)))
    streams = [torch.cuda.Stream(device=dev) for _ in cases]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(critical_pressure, c, tol, dev, rms_tol, max_iter, s)
                for c, s in zip(cases, streams)]
        res = [f.result() for f in futs]
    torch.cuda.synchronize(dev)
    return res, time.perf_counter() - t0
