"""Pins of the oracle's free energy for N fluid components (oracle/multi.py)
against what the paper and the mathematics fix, independent of the oracle's
own arithmetic:

  * with the fourth component absent it is the N = 2 energy of the C oracle
    (itself pinned in test_oracle_pins), and the difference of its two
    gradients is the N = 2 gradient;
  * its gradient matches brute-force central differences (N = 3 and 4);
  * renaming fluids (with their kappa and constraints) leaves it unchanged;
  * the flat interface between two fluids of a four-component system has the
    tension alpha (kappa_m + kappa_n) / 6 of Eq. [frozen:interface_tension]
    whatever the other components' kappa, and the absent fluid stays absent.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import lbfgs
from oracle import multi as M


def _fd(fun, x, h=1e-6):
    g = np.zeros_like(x)
    flat = x.ravel()
    for j in range(flat.size):
        a, b = flat.copy(), flat.copy()
        a[j] += h
        b[j] -= h
        g.ravel()[j] = (fun(a.reshape(x.shape)) - fun(b.reshape(x.shape))) / (2 * h)
    return g


FACES = ("mirror", "mirror", "periodic", "periodic", "wall", "wall")


@pytest.mark.parametrize("kind,shape,faces", [(O.D2Q9, (9, 7), None),
                                              (O.D3Q19, (5, 4, 3), FACES)])
def test_reduces_to_two_fluids(kind, shape, faces):
    n = int(np.prod(shape))
    c1, c2 = S.random_fields(n, seed=2)
    c1, c2 = 0.4 * c1, 0.5 * c2
    p = O.make_params(kind, shape, (0.7, 1.3, 0.9), alpha=1.2, faces=faces)
    for kw2, kwm in ((dict(dP=0.01), dict(dP=(0.01, 0.0))),
                     (dict(kcs=0.3, V0=0.2 * n), dict(kcs=(0.3, 0.0), V0=(0.2 * n, 0.0)))):
        E2, g2, t2 = O.energy_grad(p, c1, c2, active=2, **kw2)
        Em, gm, tm = M.energy_grad_multi(p, (0.7, 1.3, 0.9, 0.55), c1,
                                         np.stack([c2, 1.0 - c1 - c2]), **kwm)
        assert abs(Em - E2) <= 1e-13 * abs(E2)
        np.testing.assert_allclose(gm[0] - gm[1], g2, rtol=0, atol=1e-13)
        np.testing.assert_allclose(tm[:3], t2[[0, 1, 3]], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind,shape,nf", [(O.D2Q9, (6, 5), 2), (O.D2Q9, (5, 4), 3),
                                           (O.D3Q19, (4, 3, 3), 2)])
def test_gradient_central_differences(kind, shape, nf):
    n = int(np.prod(shape))
    rng = np.random.default_rng(nf)
    c1 = 0.3 * rng.uniform(size=n)
    C = rng.uniform(0.05, 0.3, size=(nf, n))
    kappa = rng.uniform(0.5, 1.5, size=nf + 2)
    p = O.make_params(kind, shape, kappa[:3], alpha=1.1, faces=FACES if kind == O.D3Q19 else None)
    kw = dict(dP=rng.uniform(-0.02, 0.02, nf), kcs=np.r_[0.4, np.zeros(nf - 1)],
              V0=np.r_[0.15 * n, np.zeros(nf - 1)])
    E, g, _ = M.energy_grad_multi(p, kappa, c1, C, **kw)
    fd = _fd(lambda x: M.energy_grad_multi(p, kappa, c1, x, **kw)[0], C)
    assert np.max(np.abs(fd - g)) / np.max(np.abs(g)) < 1e-7


def test_renaming_fluids():
    shape, n = (7, 6), 42
    rng = np.random.default_rng(5)
    c1 = 0.2 * rng.uniform(size=n)
    A, B, Cc = rng.uniform(0.05, 0.3, size=(3, n))
    s = A + B + Cc
    A, B, Cc = A / s * (1 - c1), B / s * (1 - c1), Cc / s * (1 - c1)
    k = (0.8, 1.1, 0.6, 1.4)     # kappa_1, then fluids A, B and the dependent Cc
    p = O.make_params(O.D2Q9, shape, k[:3])
    E1, g1, _ = M.energy_grad_multi(p, k, c1, np.stack([A, B]), dP=(0.01, -0.02))
    E2, g2, _ = M.energy_grad_multi(p, (k[0], k[2], k[1], k[3]), c1, np.stack([B, A]),
                                    dP=(-0.02, 0.01))
    assert abs(E1 - E2) <= 1e-13 * abs(E1)
    np.testing.assert_allclose(g1[::-1], g2, atol=1e-14)
    # the dependent fluid exchanged with a free one
    E3, _, _ = M.energy_grad_multi(p, (k[0], k[3], k[2], k[1]), c1, np.stack([Cc, B]),
                                   dP=(0.0, -0.02))
    E4, _, _ = M.energy_grad_multi(p, k, c1, np.stack([A, B]), dP=(0.0, -0.02))
    assert abs(E3 - E4) <= 1e-13 * abs(E4)


def test_flat_interface_tension_between_two_of_four():
    nx = 96
    shape = (nx, 1)
    k3, k4 = 0.6, 0.9
    kappa = (0.3, 2.5, k3, k4)   # solid and fluid 2 absent
    p = O.make_params(O.D2Q9, shape, kappa[:3])
    x = np.arange(nx, dtype=float)
    c3 = ((x >= nx // 4) & (x < 3 * nx // 4)).astype(float)
    c1 = np.zeros(nx)
    V0 = c3.sum()
    kw = dict(kcs=(0.0, 1.0), V0=(0.0, V0))

    def fg(v):
        E, g, _ = M.energy_grad_multi(p, kappa, c1, v.reshape(2, nx), **kw)
        return E, g.ravel()
    v, E, g, info = lbfgs.minimize(fg, np.concatenate([np.zeros(nx), c3]), tol=1e-9,
                                   max_iter=20000)
    assert info["rms_grad"] < 1e-9
    C = v.reshape(2, nx)
    assert np.abs(C[0]).max() < 1e-6          # fluid 2 stays absent
    _, _, t = M.energy_grad_multi(p, kappa, c1, C, **kw)
    gamma = (t[0] + t[1]) / 2.0                 # two interfaces, unit area
    assert abs(gamma / ((k3 + k4) / 6.0) - 1.0) < 0.02
