"""Oracle critical pressure on micropillars (Sec. III, "Critical Pressure on
Micropillared Surfaces") -- TEST INFRASTRUCTURE ONLY.

For a pressure difference dP the discrete free energy with the pressure term
-dP V (Eq. [frozen:pressure_const]) is minimised over C2 from the suspended
state by the FP64 oracle L-BFGS; the state counts as collapsed when the mean
C2 over the lower half of the gap exceeds 1/2.  The critical pressure is the
switch point, found by plain bisection to a tolerance (the paper: 1e-4) from a
bracket [lo, hi] with lo suspended and hi collapsed.  Pinned against the closed
form dP_c = -2 gamma cos(theta) / s of Eq. [frozen:critical-pressure-cyl-2d].
"""
from __future__ import annotations

import numpy as np

from . import energy_grad
from .lbfgs import minimize


def collapsed(p, c1, c2_0, gap, dP, tol=1e-6, max_iter=20000):
    """True when the minimum at pressure dP (from c2_0) has liquid in the gap."""
    x, _, _, _ = minimize(lambda v: energy_grad(p, c1, v, active=2, dP=dP)[:2], c2_0, tol=tol,
                          max_iter=max_iter)
    return float(np.mean(x[gap])) > 0.5


def critical_pressure(p, c1, c2_0, gap, lo, hi, tol=1e-4):
    """Bisection between a suspended lo and a collapsed hi."""
    if not collapsed(p, c1, c2_0, gap, hi) or collapsed(p, c1, c2_0, gap, lo):
        raise ValueError("the bracket does not hold the transition")
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if collapsed(p, c1, c2_0, gap, mid):
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)
