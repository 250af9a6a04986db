"""Oracle L-BFGS minimiser (FP64 numpy) -- TEST INFRASTRUCTURE ONLY.

The paper minimises the discrete free energy with L-BFGS (Sec. II.A, citing
Nocedal 1980 and Liu & Nocedal 1989) and stops on an rms-gradient criterion.
It fixes neither the history length nor the line search; reading: m = 10
pairs, initial inverse Hessian (s.y / y.y) I, pairs with s.y <= 1e-12 |s||y|
skipped, and a strong-Wolfe line search (c1 = 1e-4, c2 = 0.9) by bracketing
and zooming with cubic interpolation, at most 20 trials per iteration
(Nocedal & Wright, Numerical Optimization, Algorithms 3.5 and 3.6).

Parity unpinned: the iteration-by-iteration trajectory is not fixed by the
paper; only converged energies and fields are compared.  Its steps are pinned
against independent definitions: the two-loop direction against explicit BFGS
matrix updates, the line search against the strong Wolfe conditions, and the
minimiser against closed-form minima.
"""
from __future__ import annotations

import math

import numpy as np


def _cubic_min(a, fa, ga, b, fb, gb):
    """Minimiser of the cubic through (a, fa, ga), (b, fb, gb); None if degenerate."""
    d1 = ga + gb - 3.0 * (fa - fb) / (a - b)
    rad = d1 * d1 - ga * gb
    if rad < 0.0:
        return None
    d2 = math.copysign(math.sqrt(rad), b - a)
    den = gb - ga + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (gb + d2 - d1) / den


def _interp(lo, flo, glo, hi, fhi, ghi):
    t = _cubic_min(lo, flo, glo, hi, fhi, ghi)
    a, b = min(lo, hi), max(lo, hi)
    if t is None or not (a + 0.1 * (b - a) <= t <= b - 0.1 * (b - a)):
        t = 0.5 * (lo + hi)
    return t


def line_search(fg, x, fx, gx, d, alpha0=1.0, c1=1e-4, c2=0.9, max_trials=20):
    """Strong-Wolfe step along d.  Returns (alpha, x_new, f_new, g_new, trials)."""
    dg0 = float(np.dot(gx, d))
    if dg0 >= 0.0:
        return 0.0, x, fx, gx, 0
    trials = 0

    def phi(a):
        xn = x + a * d
        f, g = fg(xn)
        return xn, f, g, float(np.dot(g, d))

    a_prev, f_prev, dg_prev = 0.0, fx, dg0
    a = alpha0
    best = None
    while trials < max_trials:
        xn, f, g, dg = phi(a)
        trials += 1
        if f > fx + c1 * a * dg0 or (trials > 1 and f >= f_prev):
            return _zoom(phi, fx, dg0, a_prev, f_prev, dg_prev, a, f, dg, c1, c2,
                         max_trials - trials, trials, best, x, gx)
        if abs(dg) <= -c2 * dg0:
            return a, xn, f, g, trials
        best = (a, xn, f, g)
        if dg >= 0.0:
            return _zoom(phi, fx, dg0, a, f, dg, a_prev, f_prev, dg_prev, c1, c2,
                         max_trials - trials, trials, best, x, gx)
        a_prev, f_prev, dg_prev = a, f, dg
        a = 2.0 * a
    if best is not None:
        return best[0], best[1], best[2], best[3], trials
    return 0.0, x, fx, gx, trials


def _zoom(phi, f0, dg0, lo, flo, dglo, hi, fhi, dghi, c1, c2, budget, trials, best, x, gx):
    for _ in range(max(budget, 0)):
        a = _interp(lo, flo, dglo, hi, fhi, dghi)
        xn, f, g, dg = phi(a)
        trials += 1
        if f > f0 + c1 * a * dg0 or f >= flo:
            hi, fhi, dghi = a, f, dg
        else:
            best = (a, xn, f, g)
            if abs(dg) <= -c2 * dg0:
                return a, xn, f, g, trials
            if dg * (hi - lo) >= 0.0:
                hi, fhi, dghi = lo, flo, dglo
            lo, flo, dglo = a, f, dg
    if best is not None:
        return best[0], best[1], best[2], best[3], trials
    return 0.0, x, f0, gx, trials


def two_loop(g, S, Y, R, gamma):
    """H g for the L-BFGS inverse Hessian H of the pairs (S[k], Y[k]), oldest
    first, R[k] = 1 / (S[k].Y[k]), from H0 = gamma I: the two-loop recursion
    (Nocedal & Wright, Algorithm 7.4)."""
    q = np.array(g, dtype=np.float64, copy=True)
    al = []
    for s, y, r in zip(reversed(S), reversed(Y), reversed(R)):
        a = r * float(np.dot(s, q))
        al.append(a)
        q -= a * y
    r_ = gamma * q
    for (s, y, rr), a in zip(zip(S, Y, R), reversed(al)):
        b = rr * float(np.dot(y, r_))
        r_ += (a - b) * s
    return r_


def minimize(fg, x0, *, m=10, tol=1e-6, max_iter=10000, callback=None):
    """Minimise f with gradient fg(x) -> (f, g).  Stops when sqrt(mean(g^2)) < tol
    or after max_iter iterations.  Returns (x, f, g, info)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    f, g = fg(x)
    S, Y, R = [], [], []
    it = 0
    evals = 1
    n = x.size
    while it < max_iter:
        rms = math.sqrt(float(np.dot(g, g)) / n)
        if rms < tol:
            break
        if S:
            gamma = float(np.dot(S[-1], Y[-1])) / float(np.dot(Y[-1], Y[-1]))
        else:
            gamma = 1.0 / max(math.sqrt(float(np.dot(g, g))), 1e-300)
        d = -two_loop(g, S, Y, R, gamma)
        step, xn, fn, gn, tr = line_search(fg, x, f, g, d)
        evals += tr
        if step == 0.0:
            if S:  # restart from steepest descent once
                S, Y, R = [], [], []
                continue
            break
        s = xn - x
        y = gn - g
        sy = float(np.dot(s, y))
        if sy > 1e-12 * math.sqrt(float(np.dot(s, s)) * float(np.dot(y, y))):
            S.append(s)
            Y.append(y)
            R.append(1.0 / sy)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
                R.pop(0)
        x, f, g = xn, fn, gn
        it += 1
        if callback is not None:
            callback(it, x, f, g)
    info = dict(iterations=it, evaluations=evals,
                rms_grad=math.sqrt(float(np.dot(g, g)) / n))
    return x, f, g, info
