"""Phase-field energy minimisation on the GPU (Sec. II.A of the paper).

``FreeEnergy`` evaluates the discrete free energy and its gradient with
``dsm_fe_energy_grad`` (FP32 fields, FP64 energy).  ``Energy`` exposes it to
autograd: the forward pass returns E and keeps the hand-written adjoint dE/dC,
the backward pass scales it by the incoming gradient (``dsm_vec_axpy_dev``).
``lbfgs`` minimises E over one component with the L-BFGS kernels of libdsm
(FP64 dot products, two-loop recursion on the device); only the scalar
decisions of the line search run on the host.

The paper names L-BFGS (Nocedal 1980; Liu & Nocedal 1989) and an rms-gradient
stop; it fixes neither the history length nor the line search.  Here: m = 10
pairs, H0 = (s.y / y.y) I, pairs with s.y <= 1e-12 |s||y| dropped, a strong-Wolfe
search (c1 = 1e-4, c2 = 0.9) that brackets and then bisects/interpolates with a
safeguarded cubic, at most 20 trials per iteration.
"""
from __future__ import annotations

import math

import torch

from . import _lib
from ._lib import dsm_params


class FreeEnergy:
    """Energy + gradient of one grid (shape and material fixed by ``params``)."""

    def __init__(self, params: dsm_params, device="cuda", stream=None):
        self.params = params
        self.device = torch.device(device)
        self.stream = stream
        self.n = params.nx * params.ny * params.nz
        self.sb = _lib.dsm_fe_scratch_bytes(params.lattice, params.nx, params.ny, params.nz)
        self.scratch = torch.empty(self.sb, dtype=torch.uint8, device=self.device)
        self.terms = torch.zeros(6, dtype=torch.float64, device=self.device)

    def __call__(self, c1, c2, *, active=2, mask=None, dP=0.0, kcs=0.0, V0=0.0, fg=0.0,
                 energy=None, grad=None):
        """Returns (E as a 1-element float64 device tensor, gradient w.r.t. the
        active field as a float32 device tensor)."""
        if energy is None:
            energy = torch.empty(1, dtype=torch.float64, device=self.device)
        if grad is None:
            grad = torch.empty(self.n, dtype=torch.float32, device=self.device)
        _lib.dsm_fe_energy_grad(self.params, c1, c2, mask, active, dP, kcs, V0, fg, energy, grad,
                                self.terms, self.scratch, self.sb, self.stream)
        return energy, grad


class Energy(torch.autograd.Function):
    """E(C) with the hand-written adjoint.  Differentiable in the active field."""

    @staticmethod
    def forward(ctx, c_active, c_other, fe: FreeEnergy, active: int = 2, mask=None, dP=0.0,
                kcs=0.0, V0=0.0, fg=0.0):
        c1, c2 = (c_other, c_active) if active == 2 else (c_active, c_other)
        E, grad = fe(c1.detach().contiguous(), c2.detach().contiguous(), active=active,
                     mask=mask, dP=dP, kcs=kcs, V0=V0, fg=fg)
        ctx.save_for_backward(grad)
        ctx.fe = fe
        return E.reshape(())

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        out = torch.empty_like(grad)
        n = grad.numel()
        go = gout.detach().to(torch.float64).reshape(1).contiguous()
        _lib.dsm_vec_axpby(n, 0.0, grad, 0.0, out, ctx.fe.stream)          # out = 0
        _lib.dsm_vec_axpy_dev(n, 1.0, go, None, grad, out, ctx.fe.stream)  # out += gout grad
        return out, None, None, None, None, None, None, None, None


class _Vec:
    """Device vector helpers over libdsm (no torch arithmetic)."""

    def __init__(self, n, device, stream):
        self.n = n
        self.device = device
        self.stream = stream
        self.sb = _lib.dsm_vec_scratch_bytes(n)
        self.scratch = torch.empty(self.sb, dtype=torch.uint8, device=device)
        self.out = torch.zeros(4, dtype=torch.float64, device=device)

    def dot(self, x, y, slot=0):
        _lib.dsm_vec_dot(self.n, x, y, self.out[slot:slot + 1], self.scratch, self.sb, self.stream)
        return self.out[slot:slot + 1]

    def axpby(self, a, x, b, y):
        _lib.dsm_vec_axpby(self.n, a, x, b, y, self.stream)


def compact_direction(SY, YY, a, b, gamma):
    """Coefficients of d = -H g for the L-BFGS inverse Hessian in its compact
    form (Byrd, Nocedal & Schnabel 1994, Theorem 2.2), the same matrix the
    two-loop recursion applies:
      H = gamma I + [S  gamma Y] [[R^-T (D + gamma Y^T Y) R^-1, -R^-T], [-R^-1, 0]] [S^T; gamma Y^T]
    with R the upper triangle of S^T Y (pairs oldest first) and D its diagonal.
    SY[i, j] = s_i.y_j, YY[i, j] = y_i.y_j, a = S^T g, b = Y^T g (host float64).
    Solving R w = a and R^T u = (D + gamma Y^T Y) w - gamma b gives
    H g = gamma g + S u - gamma Y w, so d = cx g + sum cs_i s_i + sum cy_i y_i with
    (cx, cs, cy) = (-gamma, -u, gamma w)."""
    import numpy as np
    R = np.triu(SY)
    w = np.linalg.solve(R, a)
    z = (np.diag(np.diag(SY)) + gamma * YY) @ w - gamma * b
    u = np.linalg.solve(R.T, z)
    return -gamma, -u, gamma * w


def lbfgs(fe: FreeEnergy, x0, other, *, active=2, mask=None, dP=0.0, kcs=0.0, V0=0.0, fg=0.0,
          m=10, tol=1e-6, max_iter=10000, callback=None):
    """Minimise E over the active field from x0 (FP32 device vector, not
    modified).  Stops when sqrt(mean(grad^2)) < tol.  Returns (x, E, info).

    The direction uses the compact form of the L-BFGS matrix
    (compact_direction): per iteration one batched pass of dot products over the
    stored pairs and one linear combination, instead of the 2m dependent dot and
    axpy passes of the two-loop recursion.  The small m x m solves run on the
    host, which reads the dot products once per iteration."""
    import numpy as np
    n = x0.numel()
    dev = x0.device
    V = _Vec(n, dev, fe.stream)
    f32 = dict(dtype=torch.float32, device=dev)
    x = x0.detach().clone().contiguous()
    xt = torch.empty(n, **f32)
    g = torch.empty(n, **f32)
    gt = torch.empty(n, **f32)
    d = torch.empty(n, **f32)
    hist = torch.zeros(2 * m * n, **f32)        # slots: s_0..s_{m-1}, y_0..y_{m-1}
    dots = torch.zeros(4 * m, dtype=torch.float64, device=dev)
    dsb = _lib.dsm_vec_dots_scratch_bytes(n, 2 * m)
    dscratch = torch.empty(dsb, dtype=torch.uint8, device=dev)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    Et = torch.empty(1, dtype=torch.float64, device=dev)
    kw = dict(active=active, mask=mask, dP=dP, kcs=kcs, V0=V0, fg=fg)
    SY = np.zeros((m, m))   # SY[i, j] = s_i . y_j by slot (j's column set when y_j is stored)
    YY = np.zeros((m, m))
    Ag = np.zeros(m)        # s_i . g and y_i . g for the current g, by slot
    Bg = np.zeros(m)

    def evaluate(point, e_out, g_out):
        c1, c2 = (other, point) if active == 2 else (point, other)
        fe(c1, c2, energy=e_out, grad=g_out, **kw)

    def host(*ts):
        return [float(v) for v in torch.cat([t.reshape(-1) for t in ts]).cpu()]

    def slot_s(k):
        return hist[k * n:(k + 1) * n]

    def slot_y(k):
        return hist[(m + k) * n:(m + k + 1) * n]

    evaluate(x, E, g)
    f_val, gg = host(E, V.dot(g, g))
    order = []   # slots of the stored pairs, oldest first
    nxt = 0
    gamma = 1.0
    it = evals = 0
    coef = np.zeros(2 * m)
    while it < max_iter:
        rms = math.sqrt(gg / n)
        if rms < tol:
            break
        if order:
            ix = np.array(order)
            cx, cs, cy = compact_direction(SY[np.ix_(ix, ix)], YY[np.ix_(ix, ix)], Ag[ix], Bg[ix],
                                           gamma)
            coef[:] = 0.0
            coef[ix] = cs
            coef[m + ix] = cy
            dg0 = cx * gg + float(cs @ Ag[ix]) + float(cy @ Bg[ix])
        if not order or not dg0 < 0.0:  # no pairs, or not a descent direction
            order = []
            cx = -1.0 / max(math.sqrt(gg), 1e-300)
            coef[:] = 0.0
            dg0 = cx * gg
        _lib.dsm_vec_lincomb(n, 2 * m if order else 0, hist, n, coef, g, cx, d, fe.stream)
        step, trials, ft, dgt = _wolfe(lambda a: _trial(a, x, d, xt, Et, gt, evaluate, V, host),
                                       f_val, dg0)
        evals += trials
        if step == 0.0:
            if order:
                order = []
                continue
            break
        if ft is None:
            _trial(step, x, d, xt, Et, gt, evaluate, V, host)
            evals += 1
            (ft,) = host(Et)
        # the new pair s = step d, y = g_new - g into slot nxt
        if nxt in order:  # the ring is full: the oldest pair leaves
            order.remove(nxt)
        V.axpby(step, d, 0.0, slot_s(nxt))
        V.axpby(1.0, gt, 0.0, slot_y(nxt))
        V.axpby(-1.0, g, 1.0, slot_y(nxt))
        # one batched pass each: every stored s, y against y_new and against g_new
        _lib.dsm_vec_dots(n, 2 * m, hist, n, slot_y(nxt), dots[0:2 * m], dscratch, dsb, fe.stream)
        _lib.dsm_vec_dots(n, 2 * m, hist, n, gt, dots[2 * m:4 * m], dscratch, dsb, fe.stream)
        V.dot(slot_s(nxt), slot_s(nxt), 1)
        V.dot(gt, gt, 2)
        hv = host(dots, V.out[1:3])
        ss, gg = hv[4 * m], hv[4 * m + 1]
        sy, yy = hv[nxt], hv[m + nxt]
        Ag[:] = hv[2 * m:3 * m]
        Bg[:] = hv[3 * m:4 * m]
        if sy > 1e-12 * math.sqrt(ss * yy):
            SY[:, nxt] = hv[0:m]          # s_i . y_new
            YY[:, nxt] = hv[m:2 * m]      # y_i . y_new
            YY[nxt, :] = hv[m:2 * m]
            gamma = sy / yy
            order.append(nxt)
            nxt = (nxt + 1) % m
        x, xt = xt, x
        g, gt = gt, g
        E, Et = Et, E
        f_val = ft
        it += 1
        if callback is not None:
            callback(it, x, f_val, math.sqrt(gg / n))
    info = dict(iterations=it, evaluations=evals + 1, rms_grad=math.sqrt(gg / n), energy=f_val)
    return x, f_val, info


def _trial(a, x, d, xt, Et, gt, evaluate, V, host):
    V.axpby(1.0, x, 0.0, xt)
    V.axpby(a, d, 1.0, xt)
    evaluate(xt, Et, gt)
    return host(Et, V.dot(gt, d))


def _wolfe(phi, f0, dg0, c1=1e-4, c2=0.9, max_trials=20, eps=1e-6):
    """Strong-Wolfe step length along a descent direction (Nocedal & Wright,
    Numerical Optimization, Algorithms 3.5 and 3.6): expand until the minimum is
    bracketed, then shrink the bracket with a safeguarded cubic.  phi(a) ->
    (f, f') evaluates the trial point and leaves it in the trial buffers.
    Returns (a, trials, f(a), f'(a)); f(a) is None when the accepted point is
    not the last one evaluated.

    Near a minimum the energy change of a step falls below the rounding noise
    of an energy summed from FP32 node densities, so the sufficient-decrease
    test on f stops being informative.  There (|f - f0| <= eps |f0|) the test
    is replaced by its derivative form, f'(a) <= (2 c1 - 1) f'(0) (the
    approximate Wolfe condition of Hager & Zhang 2005), using the FP64
    directional derivatives."""
    noise = eps * abs(f0)

    def too_high(a, f, df):
        if abs(f - f0) <= noise:
            return df > (2.0 * c1 - 1.0) * dg0
        return f > f0 + c1 * a * dg0

    trials = 0
    a_prev, f_prev, d_prev = 0.0, f0, dg0
    a = 1.0
    lo = hi = None
    while trials < max_trials:
        f, df = phi(a)
        trials += 1
        if too_high(a, f, df) or (trials > 1 and f >= f_prev and abs(f - f0) > noise):
            lo, hi = (a_prev, f_prev, d_prev), (a, f, df)
            break
        if abs(df) <= -c2 * dg0:
            return a, trials, f, df
        if df >= 0.0:
            lo, hi = (a, f, df), (a_prev, f_prev, d_prev)
            break
        a_prev, f_prev, d_prev = a, f, df
        a *= 2.0
    if lo is None:  # never bracketed: the last point evaluated still descends
        return a_prev, trials, f_prev, d_prev
    last = a
    while trials < max_trials:
        a = _cubic_step(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2])
        f, df = phi(a)
        trials += 1
        last = a
        if too_high(a, f, df) or (f >= lo[1] and abs(f - f0) > noise):
            hi = (a, f, df)
        else:
            if abs(df) <= -c2 * dg0:
                return a, trials, f, df
            if df * (hi[0] - lo[0]) >= 0.0:
                hi = lo
            lo = (a, f, df)
    if lo[0] > 0.0:
        same = last == lo[0]
        return lo[0], trials, (lo[1] if same else None), (lo[2] if same else None)
    return 0.0, trials, None, None


def _cubic_step(a, fa, da, b, fb, db):
    """Minimiser of the cubic interpolating (a, fa, da) and (b, fb, db), kept
    inside the middle 80 % of the bracket (bisection otherwise)."""
    lo, hi = min(a, b), max(a, b)
    t = None
    den = b - a
    if den != 0.0:
        z = 3.0 * (fa - fb) / den + da + db
        w2 = z * z - da * db
        if w2 >= 0.0:
            w = math.copysign(math.sqrt(w2), den)
            q = db - da + 2.0 * w
            if q != 0.0:
                t = b - den * (db + w - z) / q
    if t is None or not (lo + 0.1 * (hi - lo) <= t <= hi - 0.1 * (hi - lo)):
        t = 0.5 * (lo + hi)
    return t
