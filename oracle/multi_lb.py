"""Oracle lattice Boltzmann step for N fluid components on a frozen diffuse
solid -- TEST INFRASTRUCTURE ONLY.

Sec. II.B states the method for the N + 1-component model and demonstrates
N = 2.  This is the stage-2 step of the C oracle written for N fluids in
plain numpy (FP64), in the same order: pull (streaming, interpolated
bounce-back at the diffuse solid, the face rules), moments and forces,
collision.  Readings for N > 2 (with N = 2 each reduces to the C oracle's):
  * every free fluid f = 2 .. N carries its own Cahn-Hilliard populations g_f
    (same tau_g, same streaming rules); C_{N+1} = 1 - C_1 - sum_f C_f;
  * mu_f = d_f - d_{N+1}, d_k = kappa_k b(C_k) - alpha^2 kappa_k L[C_k]: the
    exact derivative of the N-fluid energy of oracle/multi.py;
  * F = sum_f mu_f G[C_f] + C_2 b: the potential form of the capillary force
    for every free fluid, the body force on fluid 2;
  * rho = rho_{N+1} + sum_f (rho_f - rho_{N+1}) phi_f, with the volume fractions
    phi_f = C_f / (1 - C_1) clamped to [0, 1] (0 where 1 - C_1 <= 1e-6);
  * tau = the relaxation time of the locally largest fluid concentration, ties
    to the later fluid (N = 2: H(C_2 - C_3) with H(0) = 0).
"""
from __future__ import annotations

import numpy as np

from . import D2Q9, Params, lattice, link_q
from .multi import neighbours

CS2 = 1.0 / 3.0


def _opp(c):
    return np.array([next(j for j in range(len(c)) if np.all(c[j] == -c[i]))
                     for i in range(len(c))])


def pull_tables(p: Params):
    """For every direction j and node n: the node and direction whose
    post-collision value moves into direction j at n, and which faces the link
    crosses (0 none, 1 mirrors only, 2 a wall) -- the C oracle's pull rule."""
    c, _ = lattice(p.kind)
    opp = _opp(c)
    nx, ny, nz = p.nx, p.ny, p.nz
    n = np.arange(nx * ny * nz)
    v = [n % nx, (n // nx) % ny, n // (nx * ny)]
    e = [nx, ny, nz]
    f = list(p.face)
    q = len(c)
    src = np.empty((q, n.size), dtype=np.int64)
    kdir = np.empty((q, n.size), dtype=np.int64)
    cross = np.zeros((q, n.size), dtype=np.int64)
    for j in range(q):
        crossed = np.zeros(n.size, dtype=bool)
        wall = np.zeros(n.size, dtype=bool)
        flip = []
        coord = []
        for a in range(3):
            w = v[a] - c[j][a]
            t = np.where(w < 0, f[2 * a], np.where(w >= e[a], f[2 * a + 1], 0))
            crossed |= t > 0
            wall |= t == 2
            flip.append(t > 0)
            # the image node beyond a mirror or wall: the edge node; else periodic
            img = np.where((w < 0) & (f[2 * a] > 0), -w - 1,
                           np.where((w >= e[a]) & (f[2 * a + 1] > 0), 2 * e[a] - w - 1,
                                    np.mod(w, e[a])))
            coord.append(img)
        node = coord[0] + nx * (coord[1] + ny * coord[2])
        # reflected direction for mirror crossings
        kk = np.full(n.size, j)
        for s in np.flatnonzero(crossed & ~wall):
            cc = [(-c[j][a] if flip[a][s] else c[j][a]) for a in range(3)]
            kk[s] = next(i for i in range(q) if list(c[i]) == cc)
        kk[wall] = opp[j]
        node = np.where(wall, n, node)
        src[j], kdir[j] = node, kk
        cross[j] = np.where(wall, 2, np.where(crossed, 1, 0))
    return src, kdir, cross, opp


class MultiLB:
    """Stage-2 LB of N = nf + 1 fluids.  kappa: kappa_1 .. kappa_{N+1}; rho,
    tau: per fluid C_2 .. C_{N+1}; tau_g, body, alpha, alpha_s, faces from p."""

    def __init__(self, p: Params, kappa, rho, tau, c1):
        self.p = p
        self.c, self.w = lattice(p.kind)
        self.q = len(self.w)
        self.kappa = np.asarray(kappa, dtype=np.float64)
        self.rho = np.asarray(rho, dtype=np.float64)
        self.tau = np.asarray(tau, dtype=np.float64)
        self.nf = self.kappa.size - 2
        assert self.rho.size == self.nf + 1 and self.tau.size == self.nf + 1
        self.c1 = np.asarray(c1, dtype=np.float64).ravel()
        self.nb = neighbours(p)
        self.src, self.kdir, self.cross, self.opp = pull_tables(p)
        self.gc1 = self.grad(self.c1)
        self.solid = self.c1 >= 0.5

    def grad(self, phi):
        g = np.zeros((3, phi.size))
        for i in range(1, self.q):
            v = phi[self.nb[i]]
            for a in range(3):
                if self.c[i][a]:
                    g[a] += self.w[i] * self.c[i][a] * v
        return g / CS2

    def lap(self, phi):
        s = np.zeros_like(phi)
        for i in range(1, self.q):
            s += self.w[i] * (phi[self.nb[i]] - phi)
        return 2.0 * s / CS2

    def mus(self, C):
        """mu_f of the free fluids (nf x N) for free concentrations C."""
        a2 = self.p.alpha ** 2
        comps = [self.c1] + [C[f] for f in range(self.nf)] + [1.0 - self.c1 - C.sum(axis=0)]
        d = [k * cm * (1 - cm) * (1 - 2 * cm) - a2 * k * self.lap(cm)
             for k, cm in zip(self.kappa, comps)]
        return np.stack([d[1 + f] - d[-1] for f in range(self.nf)])

    def init(self, C):
        """f = w, g_f = g_eq(C_f, mu_f(C), u = 0)."""
        C = np.atleast_2d(np.asarray(C, dtype=np.float64))
        n = C.shape[1]
        f = np.repeat(self.w[:, None], n, axis=1)
        mu = self.mus(C)
        g = np.empty((self.nf, self.q, n))
        for k in range(self.nf):
            g[k] = self.geq(C[k], mu[k], np.zeros((3, n)))
        return f, g

    def s_of(self, u):
        cu = self.c.astype(float) @ u               # q x N
        uu = (u * u).sum(axis=0)
        return cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2)

    def geq(self, Cf, mu, u):
        s = self.s_of(u)
        g = self.w[:, None] * (mu + Cf * s)
        g[0] = Cf - (1 - self.w[0]) * mu + self.w[0] * Cf * s[0]
        return g

    def stream(self, f, g):
        n = f.shape[1]
        cols = np.arange(n)
        fs = np.empty_like(f)
        gs = np.empty_like(g)
        for j in range(self.q):
            fs[j] = f[self.kdir[j], self.src[j]]
            for k in range(self.nf):
                gs[k, j] = g[k, self.kdir[j], self.src[j]]
        # interpolated bounce-back at the diffuse solid (links inside the
        # lattice, or across mirrors, whose upstream node is solid)
        for j in range(1, self.q):
            up = self.src[j]
            hit = np.flatnonzero(~self.solid & self.solid[up] & (self.cross[j] != 2))
            i = self.opp[j]
            for nn in hit:
                q = link_q(self.p.kind, self.p.alpha_s, self.c1[nn], self.gc1[:, nn], i)
                z, kz, cz = self.src[i, nn], self.kdir[i, nn], self.cross[i, nn]
                if q < 0.5 and cz != 2 and not self.solid[z]:
                    fs[j, nn] = 2 * q * f[i, nn] + (1 - 2 * q) * f[kz, z]
                elif q < 0.5:
                    fs[j, nn] = f[i, nn]
                else:
                    fs[j, nn] = f[i, nn] / (2 * q) + (1 - 1 / (2 * q)) * f[j, nn]
        fs[:, self.solid] = self.w[:, None]
        del cols
        return fs, gs

    def macroscopic(self, fs, gs):
        C = gs.sum(axis=1)                          # nf x N
        den = 1.0 - self.c1
        safe = den > 1e-6
        phis = np.where(safe, np.clip(C / np.where(safe, den, 1.0), 0.0, 1.0), 0.0)
        rho = self.rho[-1] + ((self.rho[:-1, None] - self.rho[-1]) * phis).sum(axis=0)
        allc = np.vstack([C, 1.0 - self.c1 - C.sum(axis=0)])
        # the largest fluid concentration, ties to the later fluid
        idx = allc.shape[0] - 1 - np.argmax(allc[::-1], axis=0)
        tau = self.tau[idx]
        mu = self.mus(C)
        F = np.zeros((3, C.shape[1]))
        for k in range(self.nf):
            F += mu[k] * self.grad(C[k])
        b = np.array([self.p.bx, self.p.by, self.p.bz])
        F += C[0] * b[:, None]
        grho = self.grad(rho)
        m0 = fs.sum(axis=0)
        m1 = self.c.T.astype(float) @ fs
        u = (m1 + 0.5 * F) / rho
        u[:, self.solid] = 0.0
        pt = m0 + 0.5 * (u * grho).sum(axis=0)
        pt[self.solid] = 1.0
        return dict(C=C, mu=mu, rho=rho, tau=tau, F=F, grho=grho, u=u, pt=pt)

    def collide(self, fs, gs, M):
        u, tau = M["u"], M["tau"]
        s = self.s_of(u)
        feq = self.w[:, None] * (M["pt"] + M["rho"] * s)
        cmg = (self.c.astype(float) @ M["grho"]) - (u * M["grho"]).sum(axis=0)
        cF = self.c.astype(float) @ M["F"]
        Fi = (1 - 1 / (2 * tau)) * self.w[:, None] * (cmg * s + cF / CS2)
        f = fs - (fs - feq) / tau + Fi
        f[:, self.solid] = self.w[:, None]
        g = np.empty_like(gs)
        for k in range(self.nf):
            ge = self.geq(M["C"][k], M["mu"][k], u)
            g[k] = gs[k] - (gs[k] - ge) / self.p.tau_g
        return f, g

    def run(self, f, g, nsteps):
        for _ in range(nsteps):
            fs, gs = self.stream(f, g)
            f, g = self.collide(fs, gs, self.macroscopic(fs, gs))
        return f, g

    def fields(self, f, g):
        """Moments at the current time level (after the pull, before the
        collision)."""
        return self.macroscopic(*self.stream(f, g))
