"""Oracle free energy of N fluid components on a frozen solid -- TEST
INFRASTRUCTURE ONLY.

The N+1-component free energy of Sec. II.A (Eq. [frozen:total_energy] with
the bulk term of Eq. [frozen:bulk_energy] and the gradient term of
Eq. [frozen:interface_energy]), written for any number N of fluids: C_1 is the
solid, C_2 .. C_{N+1} the fluids, and C_{N+1} = 1 - C_1 - (C_2 + .. + C_N)
(Sec. II.A: the order parameters sum to one).  The paper states the model for
general N and demonstrates N = 2.  Readings for N > 2: every component carries
the same two terms with its own kappa_m, so the tension between any two
components is alpha (kappa_m + kappa_n) / 6 (Eq. [frozen:interface_tension]);
the gradient term is the lattice-weighted pair sum of the N = 2 oracle (its
exact derivative is -alpha^2 kappa_m L[C_m]); and the pressure term
-dP_m V_m (Eq. [frozen:pressure_const]) or the volume constraint
kcs_m (V_m - V0_m)^2 / 2 applies to each free fluid m = 2 .. N separately,
V_m = sum_x C_m.  No gravity term, and the solid stays fixed.

Plain numpy in FP64: one neighbour table per lattice direction (faces as in the
C oracle: beyond a mirror or wall face the stencil sees the edge node), sums
over directions in lattice order.
"""
from __future__ import annotations

import numpy as np

from . import Params, lattice


def _axis(v, dv, n, lo, hi):
    w = v + dv
    out = np.mod(w, n)
    if lo:
        out = np.where(w < 0, -w - 1, out)
    if hi:
        out = np.where(w >= n, 2 * n - w - 1, out)
    return out


def neighbours(p: Params) -> np.ndarray:
    """(q, N) node index of x + c_i for every node x (the stencil's view of the
    faces)."""
    c, _ = lattice(p.kind)
    nx, ny, nz = p.nx, p.ny, p.nz
    n = np.arange(nx * ny * nz)
    x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
    f = list(p.face)
    out = np.empty((len(c), n.size), dtype=np.int64)
    for i, (cx, cy, cz) in enumerate(c):
        xx = _axis(x, cx, nx, f[0], f[1])
        yy = _axis(y, cy, ny, f[2], f[3])
        zz = _axis(z, cz, nz, f[4], f[5])
        out[i] = xx + nx * (yy + ny * zz)
    return out


def energy_grad_multi(p: Params, kappa, c1, C, *, dP=None, kcs=None, V0=None):
    """E, dE/dC_m for the free fluids m = 2..N (shape (N-1, nodes)), and the
    terms (bulk, gradient, constraint, V_2, .., V_N).  kappa holds kappa_1 ..
    kappa_{N+1}; C the free fluid fields C_2 .. C_N (shape (N-1, nodes))."""
    C = np.atleast_2d(np.asarray(C, dtype=np.float64))
    nf = C.shape[0]
    kappa = np.asarray(kappa, dtype=np.float64)
    assert kappa.size == nf + 2
    dP = np.zeros(nf) if dP is None else np.asarray(dP, dtype=np.float64)
    kcs = np.zeros(nf) if kcs is None else np.asarray(kcs, dtype=np.float64)
    V0 = np.zeros(nf) if V0 is None else np.asarray(V0, dtype=np.float64)
    c1 = np.asarray(c1, dtype=np.float64).ravel()
    comps = [c1] + [C[m] for m in range(nf)] + [1.0 - c1 - C.sum(axis=0)]
    nb = neighbours(p)
    _, w = lattice(p.kind)
    a2 = p.alpha * p.alpha
    bulk = grad_e = 0.0
    d = []
    for m, cm in enumerate(comps):
        q = cm * (1.0 - cm)
        bulk += 0.5 * kappa[m] * np.sum(q * q)
        pair = np.zeros_like(cm)
        lap = np.zeros_like(cm)
        for i in range(1, len(w)):
            diff = cm[nb[i]] - cm
            pair += w[i] * diff * diff
            lap += w[i] * diff
        lap *= 6.0                                   # 2 / c_s^2
        grad_e += 1.5 * a2 * kappa[m] * np.sum(pair)  # alpha^2 kappa / (2 c_s^2)
        d.append(kappa[m] * cm * (1.0 - cm) * (1.0 - 2.0 * cm) - a2 * kappa[m] * lap)
    V = C.sum(axis=1)
    cons = 0.0
    g = np.empty_like(C)
    for m in range(nf):
        if kcs[m] == 0.0:
            cons += -dP[m] * V[m]
            extra = -dP[m]
        else:
            cons += 0.5 * kcs[m] * (V[m] - V0[m]) ** 2
            extra = kcs[m] * (V[m] - V0[m])
        g[m] = d[m + 1] - d[-1] + extra
    E = bulk + grad_e + cons
    return E, g, np.concatenate([[bulk, grad_e, cons], V])
