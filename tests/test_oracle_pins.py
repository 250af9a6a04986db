"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle (``oracle/``) against something other than itself:
values printed in the paper (tests/golden), exact identities of the lattice and
the equilibria, closed forms (tanh profile, surface tension, Young, Laplace,
Jurin, Poiseuille), brute-force finite differences, invariants (mass,
quiescence, mirror symmetry).  A plausible mistake in the oracle -- a dropped
term, a wrong sign or index, a transposed operand -- fails at least one:

  lattice tables / weights ......... test_d2q9_matches_paper, test_lattice_isotropy
  kappa <-> tensions ............... test_kappa_golden, test_kappa_roundtrip
  solid tanh profile ............... test_solid_profile_width
  isotropic G and L ................ test_stencils_exact_on_quadratics
  equilibria and forcing ........... test_equilibrium_moments
  mu (stage 2) and energy .......... test_energy_gradient_fd, test_mu_equals_energy_gradient
  mirror faces of the energy ....... test_mirror_energy_is_half_the_symmetric_domain,
                                     test_mirror_energy_gradient_fd
  mu (stage 1) and confinement ..... test_stage1_mu_is_energy_gradient, test_solid_relaxation_keeps_shape
  streaming + collision ............ test_quiescent_fixed_point, test_mass_conservation,
                                     test_mirror_symmetry_2d, test_axis_swap_symmetry_3d
  interpolated bounce-back ......... test_link_q_planar, test_bouzidi_poiseuille
  interface thermodynamics ......... test_flat_interface_profile_and_tension, test_laplace_em
  wetting .......................... test_young_em, test_young_lb, test_laplace_lb
  gravity energy ................... test_jurin_em
  mirror and wall faces (LB) ....... test_lb_mirror_faces_match_reflected_periodic,
                                     test_wall_poiseuille_closed_form, test_faces_conserve_mass
  capillary filling analysis ....... test_lucas_washburn_fit_recovers_known_curve,
                                     test_meniscus_position_on_an_inclined_axis
  pressure term, wetting transition  test_critical_pressure_em
  density and relaxation maps ...... test_density_map_uniform_acceleration,
                                     test_viscosity_map_two_layer_channel,
                                     test_translating_interface_density_contrast,
                                     test_three_fluid_relaxation_map_three_layer_channel,
                                     test_density_viscosity_pins_catch_planted_mistakes
Parity unpinned: the L-BFGS iteration trajectory (only its converged results
are used, through the pins above).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import analysis as A
from oracle import lbfgs

HERE = os.path.dirname(os.path.abspath(__file__))
CS2 = 1.0 / 3.0


# ---------------------------------------------------------------- tables
def test_d2q9_matches_paper():
    rows = np.loadtxt(os.path.join(HERE, "golden", "d2q9_lattice.txt"))
    c, w = O.lattice(O.D2Q9)
    assert c.shape == (9, 3)
    np.testing.assert_array_equal(c[:, :2], rows[:, 1:3].astype(int))
    np.testing.assert_array_equal(c[:, 2], 0)
    np.testing.assert_allclose(w, rows[:, 3] / rows[:, 4], rtol=0, atol=1e-16)


@pytest.mark.parametrize("kind", [O.D2Q9, O.D3Q19])
def test_lattice_isotropy(kind):
    c, w = O.lattice(kind)
    d = 2 if kind == O.D2Q9 else 3
    c = c[:, :d].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * np.eye(d), atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    I = np.eye(d)
    iso4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                       + np.einsum("ad,bc->abcd", I, I))
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-16)
    # every velocity has its opposite in the set
    for ci in c:
        assert any(np.all(cj == -ci) for cj in c)


# ---------------------------------------------------------------- kappa
def test_kappa_golden():
    rows = np.loadtxt(os.path.join(HERE, "golden", "kappa_cases.txt"))
    for th, g23, g12, k1, k2, k3 in rows:
        k, rc = O.kappa_from_angle(th, g23, g12)
        assert rc == 0
        np.testing.assert_allclose(k, [k1, k2, k3], rtol=1e-12, atol=1e-15)


def test_kappa_roundtrip():
    # Eq. [frozen:interface_tension]: gamma_nm = alpha (kappa_n + kappa_m)/6 must
    # recover the tensions; Eq. [eqn:st_ca]: cos(theta) = (k3 - k2)/(k2 + k3).
    rng = np.random.default_rng(1)
    for _ in range(50):
        alpha = rng.uniform(0.5, 2.0)
        g12, g23 = rng.uniform(0.1, 1.0, 2)
        th = rng.uniform(10, 170)
        k, rc = O.kappa_from_angle(th, g23, g12, alpha)
        g13 = g12 + g23 * math.cos(math.radians(th))
        np.testing.assert_allclose(alpha * (k[0] + k[1]) / 6, g12, rtol=1e-12)
        np.testing.assert_allclose(alpha * (k[0] + k[2]) / 6, g13, rtol=1e-12)
        np.testing.assert_allclose(alpha * (k[1] + k[2]) / 6, g23, rtol=1e-12)
        assert abs(A.young_angle(k[1], k[2]) - th) < 1e-9
    # a contact angle of 180 degrees leaves no positive kappa_3
    assert O.kappa_from_angle(180.0, 1.0, 1.0)[1] != 0


def test_solid_profile_width():
    # Sec. II.A: planar profile 1/2 + tanh(x/(2 alpha))/2, C = 0.5 at the
    # boundary, 10-90 % transition over 4.4 alpha at alpha = 1.
    for a in (0.5, 1.0, 2.0):
        dx = 1e-3
        x = np.arange(-8000, 8001) * dx
        c = O.solid_profile(x, a)
        assert abs(c[8000] - 0.5) < 1e-16
        w = A.width_10_90(c) * dx
        assert abs(w - 2 * a * math.log(9)) < 2e-3 * a
        assert abs(w / a - 4.4) < 0.01 * 4.4


# ---------------------------------------------------------------- stencils
@pytest.mark.parametrize("kind,shape", [(O.D2Q9, (12, 11)), (O.D3Q19, (9, 10, 11))])
def test_stencils_exact_on_quadratics(kind, shape):
    d = len(shape)
    rng = np.random.default_rng(2)
    Q = rng.normal(size=(d, d))
    Q = Q + Q.T
    b = rng.normal(size=d)
    X = np.stack([x.ravel() for x in S._coords(shape)], axis=1)
    phi = 0.5 * np.einsum("na,ab,nb->n", X, Q, X) + X @ b + 0.3
    p = O.make_params(kind, shape, (1, 1, 1))
    G = O.gradient(p, phi)
    L = O.laplacian(p, phi)
    inner = np.all((X >= 1) & (X <= np.array(shape) - 2), axis=1)
    np.testing.assert_allclose(G[:d, inner].T, X[inner] @ Q + b, atol=1e-11)
    np.testing.assert_allclose(L[inner], np.trace(Q), atol=1e-11)
    if d == 2:
        assert np.all(G[2] == 0)


# ---------------------------------------------------------------- equilibria
@pytest.mark.parametrize("kind", [O.D2Q9, O.D3Q19])
def test_equilibrium_moments(kind):
    c, w = O.lattice(kind)
    c = c.astype(float)
    rng = np.random.default_rng(3)
    for _ in range(20):
        u = rng.normal(size=3) * 0.05
        if kind == O.D2Q9:
            u[2] = 0
        pt, rho, Cc, mu, tau = 1 + 0.1 * rng.normal(), rng.uniform(0.5, 2), rng.uniform(), \
            rng.normal() * 1e-2, rng.uniform(0.6, 2)
        grho, F = rng.normal(size=3) * 0.1, rng.normal(size=3) * 1e-3
        if kind == O.D2Q9:
            grho[2] = F[2] = 0
        feq, geq, Fi = O.equilibria(kind, pt, rho, u, Cc, mu, tau, grho, F)
        uu = np.outer(u, u)
        d = 2 if kind == O.D2Q9 else 3
        I = np.diag([1.0] * d + [0.0] * (3 - d))
        assert abs(feq.sum() - pt) < 1e-14
        np.testing.assert_allclose(c.T @ feq, rho * u, atol=1e-15)
        np.testing.assert_allclose(np.einsum("ia,ib,i->ab", c, c, feq), CS2 * pt * I + rho * uu,
                                   atol=1e-14)
        assert abs(geq.sum() - Cc) < 1e-14
        np.testing.assert_allclose(c.T @ geq, Cc * u, atol=1e-15)
        np.testing.assert_allclose(np.einsum("ia,ib,i->ab", c, c, geq), CS2 * mu * I + Cc * uu,
                                   atol=1e-14)
        k = 1.0 - 1.0 / (2.0 * tau)
        assert abs(Fi.sum() - k * u @ grho) < 1e-15
        np.testing.assert_allclose(c.T @ Fi, k * F, atol=1e-15)


# ---------------------------------------------------------------- energy, mu
def _fd_grad(fun, x, h=1e-6):
    g = np.zeros_like(x)
    for j in range(x.size):
        a, b = x.copy(), x.copy()
        a[j] += h
        b[j] -= h
        g[j] = (fun(a) - fun(b)) / (2 * h)
    return g


@pytest.mark.parametrize("kind,shape", [(O.D2Q9, (7, 6)), (O.D3Q19, (4, 4, 4))])
@pytest.mark.parametrize("active", [1, 2])
def test_energy_gradient_fd(kind, shape, active):
    n = int(np.prod(shape))
    c1, c2 = S.random_fields(n, seed=5)
    c1 = 0.6 * c1
    Smask = (np.arange(n) % 3 == 0).astype(np.uint8)
    p = O.make_params(kind, shape, (0.7, 1.3, 0.9), alpha=1.3, beta=10.0)
    kw = dict(active=active, S=Smask, kcs=0.3, V0=0.4 * n, fg=0.05)
    E, g, _ = O.energy_grad(p, c1, c2, **kw)
    if active == 1:
        fd = _fd_grad(lambda x: O.energy_grad(p, x, c2, want_grad=False, **kw)[0], c1)
    else:
        fd = _fd_grad(lambda x: O.energy_grad(p, c1, x, want_grad=False, **kw)[0], c2)
    assert np.max(np.abs(fd - g)) / np.max(np.abs(g)) < 1e-7
    # pressure form of the constraint
    kw2 = dict(active=2, dP=0.02, fg=0.0)
    E, g, t = O.energy_grad(p, c1, c2, **kw2)
    fd = _fd_grad(lambda x: O.energy_grad(p, c1, x, want_grad=False, **kw2)[0], c2)
    assert np.max(np.abs(fd - g)) / np.max(np.abs(g)) < 1e-7
    assert abs(t[3] + 0.02 * c2.sum()) < 1e-12


def _mirror_faces(mirror):
    """faces argument with both faces of each flagged axis a mirror."""
    return tuple(f for m in mirror for f in (("mirror",) * 2 if m else ("periodic",) * 2))


def _mirror_extend(a, shape, mirror):
    """The periodic field twice as long along each mirror axis: the lattice
    followed by its reflection (node x' >= n holds node 2n - 1 - x')."""
    v = np.asarray(a).reshape(tuple(reversed(shape)))
    for axis, m in enumerate(mirror[:len(shape)]):
        if m:
            ax = v.ndim - 1 - axis
            v = np.concatenate([v, np.flip(v, axis=ax)], axis=ax)
    return v


@pytest.mark.parametrize("kind,shape,mirror", [(O.D2Q9, (7, 6), (1, 1, 0)),
                                               (O.D2Q9, (5, 4), (0, 1, 0)),
                                               (O.D3Q19, (4, 5, 3), (1, 0, 1))])
@pytest.mark.parametrize("active", [1, 2])
def test_mirror_energy_is_half_the_symmetric_domain(kind, shape, mirror, active):
    """A lattice with mirror faces is half of the periodic lattice doubled by
    reflection across them: its energy is that lattice's energy over 2^k, and
    its gradient is the doubled lattice's gradient on the original nodes."""
    n = int(np.prod(shape))
    c1, c2 = S.random_fields(n, seed=11)
    c1 = 0.6 * c1
    Smask = (np.arange(n) % 3 == 0).astype(np.uint8)
    kw = dict(active=active, dP=0.013, fg=0.0)
    p = O.make_params(kind, shape, (0.7, 1.3, 0.9), alpha=1.2, beta=10.0,
                      faces=_mirror_faces(mirror))
    E, g, t = O.energy_grad(p, c1, c2, S=Smask, **kw)
    full = [_mirror_extend(v, shape, mirror) for v in (c1, c2, Smask)]
    fshape = tuple(reversed(full[0].shape))
    pf = O.make_params(kind, fshape, (0.7, 1.3, 0.9), alpha=1.2, beta=10.0)
    Ef, gf, tf = O.energy_grad(pf, full[0].ravel(), full[1].ravel(),
                               S=full[2].ravel().astype(np.uint8), **kw)
    k = sum(mirror[:len(shape)])
    assert E == pytest.approx(Ef / 2 ** k, rel=1e-13, abs=1e-13)
    np.testing.assert_allclose(t, tf / 2 ** k, rtol=1e-12, atol=1e-13)
    gfull = gf.reshape(full[0].shape)
    sl = tuple(slice(0, m) for m in reversed(shape))
    np.testing.assert_allclose(g, gfull[sl].ravel(), rtol=1e-12, atol=1e-13)
    # and the periodic lattice of the same size differs (the faces matter)
    p0 = O.make_params(kind, shape, (0.7, 1.3, 0.9), alpha=1.2, beta=10.0)
    assert abs(O.energy_grad(p0, c1, c2, S=Smask, **kw)[0] - E) > 1e-6


@pytest.mark.parametrize("kind,shape,mirror", [(O.D2Q9, (6, 5), (1, 0, 0)),
                                               (O.D3Q19, (4, 3, 4), (0, 1, 1))])
def test_mirror_energy_gradient_fd(kind, shape, mirror):
    n = int(np.prod(shape))
    c1, c2 = S.random_fields(n, seed=13)
    p = O.make_params(kind, shape, (0.8, 1.1, 0.9), alpha=1.0, faces=_mirror_faces(mirror))
    kw = dict(active=2, kcs=0.2, V0=0.5 * n, fg=0.03)
    E, g, _ = O.energy_grad(p, 0.5 * c1, c2, **kw)
    fd = _fd_grad(lambda x: O.energy_grad(p, 0.5 * c1, x, want_grad=False, **kw)[0], c2)
    assert np.max(np.abs(fd - g)) / np.max(np.abs(g)) < 1e-7


def test_wall_face_energy_is_the_mirror_energy():
    # a bounce-back wall is neutral: its stencil sees the edge node's image,
    # as a mirror face does, so the energy cannot tell them apart
    shape = (6, 5)
    c1, c2 = S.random_fields(30, seed=3)
    pm = O.make_params(O.D2Q9, shape, (0.8, 1.1, 0.9), faces=_mirror_faces((0, 1, 0)))
    pw = O.make_params(O.D2Q9, shape, (0.8, 1.1, 0.9),
                       faces=("periodic", "periodic", "wall", "wall", "periodic", "periodic"))
    Em, gm, _ = O.energy_grad(pm, 0.5 * c1, c2)
    Ew, gw, _ = O.energy_grad(pw, 0.5 * c1, c2)
    assert Em == Ew
    np.testing.assert_array_equal(gm, gw)
    with pytest.raises(ValueError):  # one face periodic, the other not
        O.make_params(O.D2Q9, shape, (0.8, 1.1, 0.9),
                      faces=("mirror", "periodic", "periodic", "periodic", "periodic", "periodic"))


@pytest.mark.parametrize("kind,shape", [(O.D2Q9, (16, 16)), (O.D3Q19, (16, 16, 16))])
def test_mu_equals_energy_gradient(kind, shape):
    n = int(np.prod(shape))
    c1, c2 = S.random_fields(n, seed=7)
    c1 = 0.5 * c1
    p = O.make_params(kind, shape, (0.011, 0.0037, 0.0112), alpha=1.0)
    E, g, _ = O.energy_grad(p, c1, c2, active=2)
    mu = O.mu_fluid(p, c1, c2)
    np.testing.assert_allclose(mu, g, rtol=0, atol=1e-15 * np.abs(g).max() * 10)
    # symbolic form at a few nodes
    L2 = O.laplacian(p, c2)
    Ls = O.laplacian(p, c1 + c2)
    b = lambda c: c * (1 - c) * (1 - 2 * c)
    s = c1 + c2
    ref = 0.0037 * b(c2) + 0.0112 * b(s) - 0.0037 * L2 - 0.0112 * Ls
    np.testing.assert_allclose(mu, ref, atol=1e-16)
    # central FD on a 16^d grid at a sample of nodes
    h = 1e-4
    for j in np.random.default_rng(0).choice(n, 8, replace=False):
        a, bb = c2.copy(), c2.copy()
        a[j] += h
        bb[j] -= h
        fd = (O.energy_grad(p, c1, a, active=2, want_grad=False)[0]
              - O.energy_grad(p, c1, bb, active=2, want_grad=False)[0]) / (2 * h)
        assert abs(fd - mu[j]) <= 1e-6 * max(abs(mu[j]), 1e-3)


def test_stage1_mu_is_energy_gradient():
    shape = (10, 9)
    n = 90
    rng = np.random.default_rng(9)
    c1 = rng.uniform(0.02, 0.98, n)
    Smask = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    p = O.make_params(O.D2Q9, shape, (0.02, 0.01, 0.03), beta=0.5, omega=0.7)
    mu1 = O.mu_solid(p, Smask, c1)
    E, g, _ = O.energy_grad(p, c1, np.zeros(n), active=1, S=Smask)
    np.testing.assert_allclose(mu1, g, atol=1e-15)
    # outside [0, 1] the range penalty pulls back inside: d/dC of Omega C^2 for C<0
    c1b = c1.copy()
    c1b[3], c1b[4] = -0.2, 1.3
    mu_b = O.mu_solid(p, Smask, c1b)
    Eb, gb, _ = O.energy_grad(p, c1b, np.zeros(n), active=1, S=Smask)
    assert abs(mu_b[3] - (gb[3] + 2 * 0.7 * -0.2)) < 1e-14
    assert abs(mu_b[4] - (gb[4] + 2 * 0.7 * 0.3)) < 1e-14


# ---------------------------------------------------------------- LB step
def _wall_drop(nx=40, ny=30, theta=60.0, g=0.01, body=(0.0, 0.0, 0.0), seed=0, centre_x=None):
    shape = (nx, ny)
    sd = S.slab_sd(shape, 1, 0, 6)
    a_s = S.width_to_alpha(4.0)
    c2 = S.cap_c2(shape, 5.5, 10.0, 80.0, 1.0, sd, a_s, centre_x=centre_x).ravel()
    if seed is not None:
        c2 = c2 + S.perturbation(seed, c2.size)
    k, _ = O.kappa_from_angle(theta, g, g)
    p = O.make_params(O.D2Q9, shape, k, alpha_s=a_s, body=body)
    c1 = O.solid_profile(sd.ravel(), a_s)
    return p, c1, c2


def test_quiescent_fixed_point():
    for kind, shape in [(O.D2Q9, (8, 7)), (O.D3Q19, (5, 4, 6))]:
        n = int(np.prod(shape))
        p = O.make_params(kind, shape, (0.01, 0.004, 0.007))
        c1 = np.zeros(n)
        c2 = np.full(n, 0.3)
        f, g = O.lb_init(p, 2, c1, c2)
        f1, g1 = O.lb_run(p, 2, c1, f, g, 1)
        np.testing.assert_allclose(f1, f, rtol=0, atol=1e-15)
        np.testing.assert_allclose(g1, g, rtol=0, atol=1e-15)


def test_mass_conservation():
    p, c1, c2 = _wall_drop(body=(1e-5, -2e-5, 0.0))
    f, g = O.lb_init(p, 2, c1, c2)
    m0 = O.observables(p, c1, f, g)["mass_c2"]
    f, g = O.lb_run(p, 2, c1, f, g, 300)
    ob = O.observables(p, c1, f, g)
    assert abs(ob["mass_c2"] - m0) / m0 < 1e-12
    assert ob["nonfinite"] == 0 and ob["kinetic"] > 0
    # stage 1 conserves C1
    n = c1.size
    Smask = (S.slab_sd((40, 30), 1, 0, 6).ravel() > 0).astype(np.uint8)
    p1 = O.make_params(O.D2Q9, (40, 30), (0.01, 0.004, 0.012), beta=1e-3, omega=2e-4)
    f, g = O.lb_init(p1, 1, None, Smask.astype(float), S=Smask)
    f, g = O.lb_run(p1, 1, None, f, g, 200, S=Smask)
    m1 = O.lb_fields(p1, 1, None, f, g, S=Smask)["C"].sum()
    assert abs(m1 - Smask.sum()) / Smask.sum() < 1e-12


def test_mirror_symmetry_2d():
    nx, ny = 41, 30
    p, c1, c2 = _wall_drop(nx=nx, ny=ny, seed=None, centre_x=(nx - 1) / 2.0)
    c2 = c2.reshape(ny, nx)
    c2 = 0.5 * (c2 + c2[:, ::-1])
    f, g = O.lb_init(p, 2, c1, c2.ravel())
    f, g, F = O.lb_run(p, 2, c1, f, g, 400, want_fields=True)
    C = F["C"].reshape(ny, nx)
    ux = F["ux"].reshape(ny, nx)
    uy = F["uy"].reshape(ny, nx)
    assert np.abs(ux).max() > 1e-6
    np.testing.assert_allclose(C, C[:, ::-1], atol=1e-13)
    np.testing.assert_allclose(ux, -ux[:, ::-1], atol=1e-13)
    np.testing.assert_allclose(uy, uy[:, ::-1], atol=1e-13)


def test_axis_swap_symmetry_3d():
    n = 14
    shape = (n, n, n)
    sd = S.slab_sd(shape, 2, 0, 3)
    a_s = S.width_to_alpha(3.0)
    c2 = S.drop_c2(shape, (6.0, 6.0, 5.0), 4.0, 1.0, sd, a_s)
    c2 = 0.5 * (c2 + np.swapaxes(c2, 1, 2))  # symmetric under x <-> y
    k, _ = O.kappa_from_angle(70.0, 0.01, 0.01)
    p = O.make_params(O.D3Q19, shape, k, alpha_s=a_s, body=(1e-5, 1e-5, -1e-5))
    c1 = O.solid_profile(sd.ravel(), a_s)
    f, g = O.lb_init(p, 2, c1, c2.ravel())
    f, g, F = O.lb_run(p, 2, c1, f, g, 40, want_fields=True)
    C = F["C"].reshape(n, n, n)
    ux = F["ux"].reshape(n, n, n)
    uy = F["uy"].reshape(n, n, n)
    np.testing.assert_allclose(C, np.swapaxes(C, 1, 2), atol=1e-13)
    np.testing.assert_allclose(ux, np.swapaxes(uy, 1, 2), atol=1e-13)


def _disc_sd(shape, centre, R):
    """Signed distance to a disc, sphere or cylinder (positive inside); a
    centre coordinate of None leaves that axis out."""
    axes = np.meshgrid(*[np.arange(m, dtype=float) for m in reversed(shape)], indexing="ij")
    r2 = sum((ax - c) ** 2 for ax, c in zip(reversed(axes), centre) if c is not None)
    return R - np.sqrt(r2)


@pytest.mark.parametrize("kind,half,mirror,steps", [(O.D2Q9, (14, 12), (1, 1, 0), 150),
                                                    (O.D3Q19, (7, 6, 5), (1, 1, 0), 25)])
def test_lb_mirror_faces_match_reflected_periodic(kind, half, mirror, steps):
    """Specular reflection at mirror faces: a lattice with mirror faces evolves
    exactly as its reflected periodic double does on the original nodes
    (corner links that cross two faces included)."""
    dim = len(half)
    full = tuple(2 * m if mirror[a] else m for a, m in enumerate(half))
    a_s = S.width_to_alpha(3.0)
    # a solid disc / sphere about the corner (-1/2, -1/2) and a drop about the
    # opposite corner: both symmetric under the reflections of the double
    import itertools
    hi = tuple(h - 0.5 if mirror[a] else None for a, h in enumerate(half))
    R = min(half[a] for a in range(dim) if mirror[a]) / 2.0
    # the corner (-1/2, -1/2) of the periodic double, with its periodic images
    corners = itertools.product(*[(-0.5, f - 0.5) if mirror[a] else (None,)
                                  for a, f in enumerate(full)])
    sd = np.max([_disc_sd(full, c, R) for c in corners], axis=0)
    c1f = O.solid_profile(sd.ravel(), a_s).reshape(sd.shape)
    dsd = _disc_sd(full, hi, R - 0.5)
    c2f = (0.5 + 0.5 * np.tanh(dsd / 2.0)) * (1.0 - c1f)
    # the double is symmetric under each reflection x -> 2n - 1 - x
    for a in range(dim):
        if mirror[a]:
            ax = dim - 1 - a
            np.testing.assert_allclose(c1f, np.flip(c1f, axis=ax), atol=1e-15)
            np.testing.assert_allclose(c2f, np.flip(c2f, axis=ax), atol=1e-15)
    k, _ = O.kappa_from_angle(70.0, 0.01, 0.01)
    body = (0.0, 0.0, 1e-5)[:3] if dim == 3 else (0.0, 0.0, 0.0)
    pf = O.make_params(kind, full, k, alpha_s=a_s, body=body)
    ph = O.make_params(kind, half, k, alpha_s=a_s, body=body, faces=_mirror_faces(mirror))
    sl = tuple(slice(0, m) for m in reversed(half))
    f, g = O.lb_init(pf, 2, c1f.ravel(), c2f.ravel())
    _, _, Ff = O.lb_run(pf, 2, c1f.ravel(), f, g, steps, want_fields=True)
    f, g = O.lb_init(ph, 2, c1f[sl].ravel(), c2f[sl].ravel())
    _, _, Fh = O.lb_run(ph, 2, c1f[sl].ravel(), f, g, steps, want_fields=True)
    assert np.abs(Fh["ux"]).max() > 1e-6
    for name in ("C", "mu", "ux", "uy", "uz", "pt"):
        np.testing.assert_allclose(Fh[name], Ff[name].reshape(sd.shape)[sl].ravel(),
                                   rtol=0, atol=1e-13, err_msg=name)


@pytest.mark.parametrize("kind,shape,faces,body", [
    (O.D2Q9, (3, 12), ("periodic", "periodic", "wall", "wall", "periodic", "periodic"),
     (1e-6, 0.0, 0.0)),
    (O.D3Q19, (2, 3, 10), ("mirror", "mirror", "periodic", "periodic", "wall", "wall"),
     (0.0, 1e-6, 0.0))])
@pytest.mark.parametrize("tau", [0.8, 0.5 + math.sqrt(3.0 / 16.0), 1.5])
def test_wall_poiseuille_closed_form(kind, shape, faces, body, tau):
    """Halfway bounce-back walls: body-force Poiseuille flow of the BGK scheme.
    The steady discrete solution is the parabola with walls half a node beyond
    the edge nodes plus a constant slip b/(2 nu) (16 tau^2 - 16 tau + 1)/12,
    which vanishes at tau = 1/2 + sqrt(3/16) (the known viscosity-dependent
    slip of bounce-back with BGK, He, Zou, Luo & Dembo, J. Stat. Phys. 87,
    1997)."""
    n = int(np.prod(shape))
    p = O.make_params(kind, shape, (0.01, 0.004, 0.007), tau2=tau, tau3=tau, body=body,
                      faces=faces)
    c1, c2 = np.zeros(n), np.ones(n)  # all liquid, no solid: mu = 0, F = b
    f, g = O.lb_init(p, 2, c1, c2)
    f, g, F = O.lb_run(p, 2, c1, f, g, int(8000 / math.sqrt(tau - 0.5)), want_fields=True)
    H = shape[-1]
    b = body[0] if kind == O.D2Q9 else body[1]
    u = (F["ux"] if kind == O.D2Q9 else F["uy"]).reshape(tuple(reversed(shape)))
    s = np.arange(H)
    nu = (tau - 0.5) / 3.0
    exact = b / (2 * nu) * ((s + 0.5) * (H - 0.5 - s) + (16 * tau * tau - 16 * tau + 1) / 12.0)
    exact = exact.reshape((H,) + (1,) * (u.ndim - 1))
    assert np.max(np.abs(u - exact)) < 1e-9 * np.max(exact)
    other = F["uy"] if kind == O.D2Q9 else F["ux"]
    assert np.abs(other).max() < 1e-14


def test_faces_conserve_mass():
    """Mirror and wall faces pass no mass: sum f and sum g are kept exactly
    while a drop is driven into a wall and along a mirror plane (equal
    densities: with a density contrast the pressure moment's u.G[rho]/2 term
    moves sum f by itself)."""
    nx, ny = 20, 16
    n = nx * ny
    dsd = _disc_sd((nx, ny), (4.0, 9.0), 5.0)
    c2 = (0.5 + 0.5 * np.tanh(dsd / 2.0)).ravel()
    k, _ = O.kappa_from_angle(90.0, 0.01, 0.01)
    for faces in [("mirror", "wall", "wall", "mirror", "periodic", "periodic"),
                  ("wall", "wall", "wall", "wall", "periodic", "periodic")]:
        p = O.make_params(O.D2Q9, (nx, ny), k, body=(-2e-5, 1e-5, 0.0), faces=faces,
                          tau2=0.8, tau3=1.0)
        c1 = np.zeros(n)
        f, g = O.lb_init(p, 2, c1, c2)
        f1, g1 = O.lb_run(p, 2, c1, f, g, 300)
        assert abs(f1.sum() - f.sum()) < 1e-12 * f.sum()
        assert abs(g1.sum() - g.sum()) < 1e-12 * g.sum()
        ob = O.observables(p, c1, f1, g1)
        assert ob["nonfinite"] == 0 and ob["kinetic"] > 0


def test_lucas_washburn_fit_recovers_known_curve():
    # the fit of Eq. [eqn:cfilling] on samples of L0 + k sqrt(t - t0), exact and
    # with noise; and the angle that gives a prefactor back
    t = np.linspace(2000.0, 300000.0, 60)
    k, L0, t0, rms = A.lucas_washburn_fit(t, 3.0 + 0.3 * np.sqrt(t - 50.0))
    assert abs(k - 0.3) < 1e-6 and abs(L0 - 3.0) < 1e-3 and rms < 1e-4
    noisy = 3.0 + 0.3 * np.sqrt(t - 50.0) + np.random.default_rng(0).normal(0.0, 0.05, t.size)
    assert abs(A.lucas_washburn_fit(t, noisy)[0] - 0.3) < 2e-3
    kk = math.sqrt(2.5e-3 * 40.0 * math.cos(math.radians(60.0)) / (3.0 / 6.0))
    assert abs(A.washburn_angle(kk, 2.5e-3, 40.0, 1.0 / 6.0) - 60.0) < 1e-9


def test_meniscus_position_on_an_inclined_axis():
    ny, nx = 120, 300
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    a = math.radians(20.0)
    d, e = (math.cos(a), math.sin(a)), (40.0, 20.0)
    s = (x - e[0]) * d[0] + (y - e[1]) * d[1]
    for s0 in (12.3, 57.71, 100.0):
        c2 = 0.5 * (1.0 - np.tanh((s - s0) / 2.0))
        assert abs(A.meniscus_position(c2, e, d, 200.0) - s0) < 0.02
    assert A.meniscus_position(np.ones((ny, nx)), e, d, 200.0) == 200.0


def _square(n=40, half=8):
    y, x = np.mgrid[0:n, 0:n]
    c = (n - 1) / 2.0
    return ((abs(x - c) < half) & (abs(y - c) < half)).astype(np.uint8).ravel()


def test_two_step_solid_rounds_the_corners():
    """Two-step solid initialisation (Sec. II.B): a diffuse profile cannot
    follow a square's corners, so a one-step relaxation leaves nodes where the
    confinement still pulls; after the redefinition S := {C1 > 1/2} the final
    C1 agrees with its region everywhere.  The redefined region has rounded
    corners; the stage-1 dynamics conserve sum C1, so the mass taken from the
    corners moves the middles of the edges out by a node; and it keeps the
    square's symmetry."""
    n = 40
    S0 = _square(n)
    k, _ = O.kappa_from_angle(90.0, 0.01, 0.01)
    p = O.make_params(O.D2Q9, (n, n), k)

    def wrong_side(c1, S):
        return int((((S == 1) & (c1 < 0.5)) | ((S == 0) & (c1 > 0.5))).sum())
    c1_one = O.relax_solid(p, S0, S0.astype(float), 3000, 1e-3, 2e-4)
    c1_two, S2 = O.solid_two_step(p, S0, S0.astype(float), 500, 1e-2, 2e-3, 2500, 1e-3, 2e-4)
    assert wrong_side(c1_one, S0) > 20
    assert wrong_side(c1_two, S2) == 0
    c1a = O.relax_solid(p, S0, S0.astype(float), 500, 1e-2, 2e-3)
    np.testing.assert_array_equal(S2, (c1a > 0.5).astype(np.uint8))
    assert abs(c1a.sum() - S0.sum()) < 1e-10 * S0.sum()
    c = (n - 1) / 2.0
    d = S2.astype(int) - S0.astype(int)
    for idx, corner in ((np.flatnonzero(d < 0), True), (np.flatnonzero(d > 0), False)):
        assert idx.size > 0
        y, x = np.divmod(idx, n)
        ax, ay = abs(x - c), abs(y - c)
        if corner:   # lost: near the corners (both offsets large)
            assert np.all(np.minimum(ax, ay) >= 5.5)
        else:        # gained: one row out, near the middle of an edge
            assert np.all((np.maximum(ax, ay) == 8.5) & (np.minimum(ax, ay) <= 2.5))
    sq = S2.reshape(n, n)
    np.testing.assert_array_equal(sq, sq.T)
    np.testing.assert_array_equal(sq, sq[::-1, :])


def test_link_q_planar():
    # a planar tanh profile with its C1 = 1/2 surface a distance delta from the
    # node: the link fraction is delta / (n.d) / |c|
    for kind in (O.D2Q9, O.D3Q19):
        c, w = O.lattice(kind)
        for a_s in (0.7, 1.0):
            for delta in (0.2, 0.5, 0.8):
                c1x = O.solid_profile(np.array([-delta]), a_s)[0]
                nrm = np.array([0.0, -1.0, 0.0])  # solid lies toward -y
                for i in range(len(c)):
                    ci = c[i].astype(float)
                    nd = nrm @ ci / np.linalg.norm(ci) if ci.any() else 0
                    q = O.link_q(kind, a_s, c1x, nrm * 0.3, i)
                    if nd > 1e-6 and delta / nd / np.linalg.norm(ci) <= 1:
                        assert abs(q - delta / nd / np.linalg.norm(ci)) < 1e-12
                    else:
                        assert q == 0.5
        assert O.link_q(kind, 1.0, 0.3, np.zeros(3), 1) == 0.5


def test_bouzidi_poiseuille():
    # Body-force channel flow between two diffuse plates, one fluid (C2 = 1,
    # kappa = 0 so no capillary force): the wall planes are the C1 = 1/2
    # surfaces at y = 7.8 and y = ny - 0.8, deliberately off the half-link.
    nx, ny, g = 3, 34, 1e-6
    shape = (nx, ny)
    sd = S.slab_sd(shape, 1, 0, 8) + 0.3
    c1 = O.solid_profile(sd.ravel(), 0.9)
    p = O.make_params(O.D2Q9, shape, (0.0, 0.0, 0.0), alpha_s=0.9, body=(g, 0, 0))
    c2 = np.ones(nx * ny)
    f, gg = O.lb_init(p, 2, c1, c2)
    f, gg, F = O.lb_run(p, 2, c1, f, gg, 12000, want_fields=True)
    y = np.arange(ny, dtype=float)
    ya, yb = 7.8, ny - 0.8
    nu = (1.0 - 0.5) / 3.0
    ux = F["ux"].reshape(ny, nx)[:, 1]
    fluid = c1.reshape(ny, nx)[:, 1] < 0.5
    exact = g / (2 * nu) * (y - ya) * (yb - y)
    err = np.sqrt(np.sum((ux[fluid] - exact[fluid]) ** 2) / np.sum(exact[fluid] ** 2))
    assert err < 0.01
    # with the wall on the half link the interpolation reduces to the halfway rule,
    # which is exact for this flow at tau = 1
    sd2 = S.slab_sd(shape, 1, 0, 8)
    c1b = O.solid_profile(sd2.ravel(), 0.9)
    f, gg = O.lb_init(p, 2, c1b, c2)
    f, gg, F = O.lb_run(p, 2, c1b, f, gg, 12000, want_fields=True)
    ux = F["ux"].reshape(ny, nx)[:, 1]
    exact = g / (2 * nu) * (y - 7.5) * (ny - 0.5 - y)
    fl = c1b.reshape(ny, nx)[:, 1] < 0.5
    assert np.max(np.abs(ux[fl] - exact[fl])) / exact.max() < 1e-3


# ---------------------------------------------------------------- thermodynamics
def _minimize_c2(p, c1, c2, **kw):
    def fg(x):
        E, g, _ = O.energy_grad(p, c1, x, active=2, **kw)
        return E, g
    x, E, g, info = lbfgs.minimize(fg, c2, tol=kw.pop("tol", 1e-8) if "tol" in kw else 1e-8,
                                   max_iter=20000)
    return x, E, info


@pytest.mark.parametrize("alpha,tol", [(1.0, 0.02), (2.0, 0.005)])
def test_flat_interface_profile_and_tension(alpha, tol):
    nx = 96 if alpha == 1.0 else 160
    shape = (nx, 1)
    k23 = 0.6
    p = O.make_params(O.D2Q9, shape, (0.0, k23, k23), alpha=alpha)
    x = np.arange(nx, dtype=float)
    c2 = ((x >= nx // 4) & (x < 3 * nx // 4)).astype(float)
    c1 = np.zeros(nx)
    V0 = c2.sum()
    x2, E, info = _minimize_c2(p, c1, c2, kcs=1.0, V0=V0)
    assert info["rms_grad"] < 1e-8
    _, _, terms = O.energy_grad(p, c1, x2, active=2, kcs=1.0, V0=V0, want_grad=False)
    gamma = (terms[0] + terms[1]) / 2.0  # two interfaces, unit area
    assert abs(gamma / (alpha * 2 * k23 / 6) - 1) < tol
    # profile across the left interface
    left = x2[: nx // 2]
    w = A.width_10_90(left)
    assert abs(w / (2 * alpha * math.log(9)) - 1) < tol
    # shape: 1/2 + tanh((x - x0)/(2 alpha))/2 with x0 at the 1/2 crossing
    k0 = np.nonzero(left >= 0.5)[0][0]
    x0 = k0 - 1 + (0.5 - left[k0 - 1]) / (left[k0] - left[k0 - 1])
    ref = 0.5 + 0.5 * np.tanh((x[: nx // 2] - x0) / (2 * alpha))
    assert np.max(np.abs(left - ref)) < 2 * tol


def test_lb_flat_interface_relaxes_to_em_profile():
    # the stationary LB state of a flat interface is the energy minimum
    # (uniform mu, no flow)
    nx = 32
    shape = (nx, 1)
    k23 = 0.3
    p = O.make_params(O.D2Q9, shape, (0.0, k23, k23))
    x = np.arange(nx, dtype=float)
    c2 = ((x >= 8) & (x < 24)).astype(float)
    c1 = np.zeros(nx)
    f, g = O.lb_init(p, 2, c1, c2)
    f, g, F = O.lb_run(p, 2, c1, f, g, 6000, want_fields=True)
    xm, E, info = _minimize_c2(p, c1, c2, kcs=1.0, V0=c2.sum(), tol=1e-11)
    assert np.max(np.abs(F["C"] - xm)) < 1e-7
    assert np.ptp(F["mu"]) < 1e-9
    assert np.abs(F["ux"]).max() < 1e-12


@pytest.mark.parametrize("R", [10.0, 15.0, 20.0])
def test_laplace_em(R):
    # 2D Young-Laplace (textbook): mu0 (C_in - C_out) = gamma_23 / R
    n = 72
    shape = (n, n)
    k23 = 0.6
    gamma = 2 * k23 / 6
    p = O.make_params(O.D2Q9, shape, (0.0, k23, k23))
    c2 = S.drop_c2(shape, (n / 2, n / 2), R).ravel()
    c1 = np.zeros(n * n)
    V0 = c2.sum()
    x, E, info = _minimize_c2(p, c1, c2, kcs=0.05, V0=V0)
    mu = O.mu_fluid(p, c1, x)
    mu0 = mu[n // 2 * n + n // 2]
    assert np.ptp(mu) < 1e-6
    cin, cout = x[n // 2 * n + n // 2], x[0]
    # equimolar radius: the drop's excess over the outer bulk value
    Req = math.sqrt((x.sum() - x.size * cout) / math.pi / (cin - cout))
    assert abs(mu0 * (cin - cout) * Req / gamma - 1) < 0.03


# ---------------------------------------------------------------- wetting
def _em_wall_case(nx, ny, wall, theta, R, beta=10.0, n_iter=10):
    """Two-stage energy minimisation of Sec. II.A: relax a sharp wall for
    n_iter L-BFGS iterations with the confinement, then minimise C2."""
    shape = (nx, ny)
    g23, g12 = math.sqrt(8.0 / 9.0), 1.0
    k, _ = O.kappa_from_angle(theta, g23, g12)
    p = O.make_params(O.D2Q9, shape, k, beta=beta)
    Smask = (S.slab_sd(shape, 1, 0, wall).ravel() > 0).astype(np.uint8)
    n = nx * ny
    c2z = np.zeros(n)

    def fg1(x):
        E, g, _ = O.energy_grad(p, x, c2z, active=1, S=Smask)
        return E, g
    c1, _, _, _ = lbfgs.minimize(fg1, Smask.astype(float), tol=0.0, max_iter=n_iter)
    sd = S.slab_sd(shape, 1, 0, wall)
    c2 = S.cap_c2(shape, wall - 0.5, R, 90.0, 1.0, sd, 1.0).ravel()
    return p, k, c1, c2


@pytest.mark.slow
@pytest.mark.parametrize("theta", [60.0, 90.0, 120.0])
def test_young_em(theta):
    nx, ny, wall, R = 100, 56, 8, 18.0
    p, k, c1, c2 = _em_wall_case(nx, ny, wall, theta, R)
    # keep C1 within the solid's own profile; constrain the drop volume
    x, E, info = _minimize_c2(p, c1, c2, kcs=0.05, V0=c2.sum(), tol=1e-6)
    th = A.contact_angle_flat(x.reshape(ny, nx), c1.reshape(ny, nx))
    assert abs(th - theta) < 2.0, (th, theta)


@pytest.mark.slow
@pytest.mark.parametrize("theta,shape,R,steps,tol", [
    (30.0, (160, 48), 24.0, 8000, 1.5), (60.0, (64, 36), 12.0, 6000, 1.5),
    (90.0, (64, 36), 12.0, 6000, 1.5), (120.0, (64, 36), 12.0, 6000, 1.5),
    (135.0, (64, 36), 12.0, 6000, 1.5), (150.0, (64, 36), 12.0, 18000, 3.0)])
def test_young_lb(theta, shape, R, steps, tol):
    """A drop started 5 degrees off relaxes on the flat diffuse wall to Young's
    angle arccos((k3 - k2)/(k2 + k3)) (Supp. D: within 1.5 degrees for
    15-165 degrees with drops of radius 40).  These drops are small (radius 12,
    24 at 30 degrees, so that the flat cap rises above the fit's margin): at 150
    degrees the diffuse interface (4.4 nodes) shifts the angle to 147.5 from
    either side, so that case allows 3 degrees; the paper's own setup runs on
    the GPU (tests/test_gpu_lb.py::test_young_lb_paper_setup)."""
    nx, ny = shape
    g = 0.03
    sd = S.slab_sd(shape, 1, 0, 6)
    a_s = S.width_to_alpha(4.0)
    c2 = S.cap_c2(shape, 5.5, R, theta + 5.0, 1.0, sd, a_s).ravel()
    k, _ = O.kappa_from_angle(theta, g, g)
    p = O.make_params(O.D2Q9, shape, k, alpha_s=a_s)
    c1 = O.solid_profile(sd.ravel(), a_s)
    f, gg = O.lb_init(p, 2, c1, c2)
    f, gg, F = O.lb_run(p, 2, c1, f, gg, steps, want_fields=True)
    th = A.contact_angle_flat(F["C"].reshape(ny, nx), c1.reshape(ny, nx))
    assert abs(th - theta) < tol, th


@pytest.mark.slow
def test_laplace_lb():
    """Laplace's law from the lattice Boltzmann equilibrium of a free drop (no
    solid, 2D): the chemical potential relaxes to one value mu0 inside and
    outside (here the drop's bulk plateau, the outside within 20 % of it after
    20k steps), and mu0 (C_in - C_out) = gamma_23 / R with R the radius of the
    C = 1/2 circle (the drop's Laplace pressure in the potential form of the
    force, reading R1), within 3 %."""
    n, g, R0 = 64, 0.03, 15.0
    shape = (n, n)
    k, _ = O.kappa_from_angle(90.0, g, g)
    p = O.make_params(O.D2Q9, shape, k)
    c2 = S.drop_c2(shape, (n / 2 - 0.5, n / 2 - 0.5), R0, 1.0).ravel()
    c1 = np.zeros(n * n)
    f, gg = O.lb_init(p, 2, c1, c2)
    f, gg, F = O.lb_run(p, 2, c1, f, gg, 20000, want_fields=True)
    C, mu = F["C"].reshape(n, n), F["mu"].reshape(n, n)
    mu_in, mu_out = mu[n // 2, n // 2], mu[0, 0]
    assert abs(mu_in - mu_out) < 0.2 * abs(mu_in)       # one value, inside and out
    _, R = A.kasa_fit(A.iso_points(C, 0.5))
    dC = C[n // 2, n // 2] - C[0, 0]
    # the drop's bulk plateau (the outside's mu approaches it by diffusion)
    assert abs(mu_in * dC * R / g - 1.0) < 0.03


@pytest.mark.slow
def test_solid_relaxation_keeps_shape():
    # LB stage 1 (Sec. II.B, Eq. [Free Energy1]): a sharp wall relaxes to the
    # tanh profile while the confinement keeps its C1 = 1/2 surface on the
    # boundary of S.
    nx, ny = 4, 48
    shape = (nx, ny)
    Smask = (S.slab_sd(shape, 1, 0, 20).ravel() > 0).astype(np.uint8)
    g12 = g23 = 2.5e-3
    k, _ = O.kappa_from_angle(60.0, g23, g12)
    p = O.make_params(O.D2Q9, shape, k, beta=1e-3, omega=2e-4)
    f, g = O.lb_init(p, 1, None, Smask.astype(float), S=Smask)
    f, g = O.lb_run(p, 1, None, f, g, 5000, S=Smask)
    c1 = O.lb_fields(p, 1, None, f, g, S=Smask)["C"].reshape(ny, nx)[:, 0]
    top = c1[10:40]  # the upper face of the slab, boundary between nodes 19 and 20
    k0 = np.nonzero(top < 0.5)[0][0]
    yh = 10 + k0 - 1 + (top[k0 - 1] - 0.5) / (top[k0 - 1] - top[k0])
    assert abs(yh - 19.5) < 0.25
    w = A.width_10_90(top)
    assert abs(w / (2 * math.log(9)) - 1) < 0.1
    assert c1.min() > -0.02 and c1.max() < 1.02


@pytest.mark.slow
def test_jurin_em():
    # Capillary rise between two plates (the 2D analogue of Sec. III.B): the mean
    # rise above the far-field level obeys h = 2 gamma cos(theta) / (f_g w)
    # (Eq. [frozen:capillary_rise_height] with the plate geometry), exact for the
    # mean height by the force balance on the raised column.
    nx, ny = 240, 80
    shape = (nx, ny)
    theta, gap, thick, base, bottom = 45.0, 20, 10, 8, 14
    g23, g12 = math.sqrt(8.0 / 9.0), 1.0
    h_target = 20.0
    fg = 2 * g23 * math.cos(math.radians(theta)) / (h_target * gap)
    k, _ = O.kappa_from_angle(theta, g23, g12)
    p = O.make_params(O.D2Q9, shape, k)
    x0 = nx // 2 - gap // 2 - thick
    # one solid block across the periodic seam carries both plates
    blk = S.slab_sd(shape, 1, ny - base, ny + base)
    p1 = S.box_sd(shape, (x0, bottom), (x0 + thick, ny - base))
    p2 = S.box_sd(shape, (x0 + thick + gap, bottom), (x0 + 2 * thick + gap, ny - base))
    sd = S.union_sd(blk, p1, p2)
    c1 = O.solid_profile(sd.ravel(), 1.0)
    c2 = S.layer_c2(shape, 1, base, 24, 1.0, sd, 1.0).ravel()
    x, E, info = _minimize_c2(p, c1, c2, kcs=0.05, V0=c2.sum(), fg=fg, tol=1e-7)
    # liquid fraction of the fluid, C2 / (1 - C1), so the diffuse walls do not count
    phi = x.reshape(ny, nx) / np.maximum(1.0 - c1.reshape(ny, nx), 1e-9)

    def half_crossing(col, lo):
        kk = np.nonzero(col[lo:ny - base] < 0.5)[0][0] + lo
        return kk - 1 + (col[kk - 1] - 0.5) / (col[kk - 1] - col[kk])
    y_r = half_crossing(phi[:, 5], base + 2)          # far-field reservoir level
    ys = [half_crossing(phi[:, xx], bottom) for xx in range(x0 + thick, x0 + thick + gap)]
    h = float(np.mean(ys)) - y_r                       # mean height of the C2 = 1/2 line
    assert abs(h / h_target - 1) < 0.05, (h, h_target)


@pytest.mark.parametrize("theta", [60.0, 112.0, 135.0])
def test_critical_pressure_em(theta):
    # Cassie-Baxter to Wenzel transition on 2D pillars (Sec. III): the pressure
    # at which the minimum of the pressure-constrained energy switches from the
    # suspended meniscus to the filled gap is dP_c = -2 gamma cos(theta) / s
    # (Eq. [frozen:critical-pressure-cyl-2d]); bisection to the paper's 1e-4.
    from oracle import critical as OC
    c = S.pillar_gap_2d(period=40, height=64, width=16, pillar=24, base=4, theta=theta)
    k, _ = O.kappa_from_angle(theta, c.g23, c.g12)
    p = O.make_params(O.D2Q9, c.shape, k, alpha_s=c.alpha_s)
    c1 = O.solid_profile(c.solid_sd, c.alpha_s)
    th = -2 * c.g23 * math.cos(math.radians(theta)) / c.extra["s"]
    dpc = OC.critical_pressure(p, c1, c.c2, c.extra["gap"], th - 0.5 * abs(th) - 5e-3,
                               th + 0.5 * abs(th) + 5e-3)
    # diffuse walls make the effective gap a little wider than s: within 4 %
    assert abs(dpc / th - 1) < 0.04, (dpc, th)


# ------------------------------------------------------ density and viscosity
# The density map rho = rho3 + (rho2 - rho3) C2/(C2 + C3) and the relaxation
# map tau = tau3 + (tau2 - tau3) H(C2 - C3) (Sec. II.B, the hydrodynamic
# equations for unequal densities and viscosities), pinned by closed forms of
# the flow they produce; test_density_viscosity_pins_catch_planted_mistakes
# shows that each pin fails for the plausible mistakes in these maps.
def _accel_dev(c1v, c2v, rho2, rho3, b=1e-5, steps=(1, 5, 20)):
    """Uniform composition under a uniform body force: every node is alike, so
    each step adds exactly the force F = C2 b to sum_i c_i f_i (the forcing
    term's first moment with u = (sum c f + F/2)/rho in the equilibrium), and
    the velocity at step n is (n + 1/2) F / rho with rho from the volume
    fraction phi = C2/(1 - C1), clamped to [0, 1].  Returns the largest
    relative deviation over the given steps."""
    shape, n = (4, 3), 12
    k, _ = O.kappa_from_angle(90.0, 0.01, 0.01)
    p = O.make_params(O.D2Q9, shape, k, rho2=rho2, rho3=rho3, tau2=0.8, tau3=1.3,
                      body=(b, 0.0, 0.0))
    c1, c2 = np.full(n, c1v), np.full(n, c2v)
    f, g = O.lb_init(p, 2, c1, c2)
    phi = min(1.0, max(0.0, c2v / (1.0 - c1v)))
    rho = rho3 + (rho2 - rho3) * phi
    dev, done = 0.0, 0
    for s in steps:
        f, g = O.lb_run(p, 2, c1, f, g, s - done)
        done = s
        ux = O.lb_fields(p, 2, c1, f, g)["ux"]
        exact = (s + 0.5) * c2v * b / rho
        dev = max(dev, float(np.max(np.abs(ux - exact))) / exact)
    return dev


ACCEL_CASES = [(0.0, 1.0, 1.0, 0.4), (0.2, 0.4, 1.0, 0.4), (0.3, 0.8, 1.0, 0.4),
               (0.1, 0.3, 0.25, 1.0)]


@pytest.mark.parametrize("c1v,c2v,rho2,rho3", ACCEL_CASES)
def test_density_map_uniform_acceleration(c1v, c2v, rho2, rho3):
    # (0.3, 0.8): C2 + C3 = 0.7 < C2, the clamp phi = 1 applies
    assert _accel_dev(c1v, c2v, rho2, rho3) < 1e-10


def _channel_ode(nu_node, force):
    """Steady unidirectional flow between no-slip walls half a node beyond the
    edge nodes: d/dy(nu du/dy) = -force on the nodes, finite volumes with the
    harmonic mean of the two nodes' viscosities on each link (continuous
    shear stress at a viscosity jump)."""
    H = nu_node.size
    A = np.zeros((H, H))
    for k in range(H):
        for m in (k - 1, k + 1):
            if 0 <= m < H:
                nl = 2 * nu_node[k] * nu_node[m] / (nu_node[k] + nu_node[m])
                A[k, k] -= nl
                A[k, m] += nl
            else:
                A[k, k] -= 2 * nu_node[k]  # wall at distance 1/2
    return np.linalg.solve(A, -force)


def _two_layer_dev(tau2, tau3, H=32, b=2e-6):
    """Liquid (y < H/2) under gas between two walls, the body force on the
    liquid along the walls: returns (max deviation of u from the channel
    solution with nu = (tau - 1/2)/3 of the locally larger fluid, over max u;
    relative deviation of the liquid bulk's curvature from -b/nu_2)."""
    faces = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")
    k, _ = O.kappa_from_angle(90.0, 0.01, 0.01)
    p = O.make_params(O.D2Q9, (2, H), k, tau2=tau2, tau3=tau3, body=(b, 0.0, 0.0), faces=faces)
    y = np.arange(H)
    c2 = np.repeat(0.5 * (1 - np.tanh((y - (H / 2 - 0.5)) / 2.0)), 2)
    c1 = np.zeros(2 * H)
    f, g = O.lb_init(p, 2, c1, c2)
    steps = int(6 * H * H / ((min(tau2, tau3) - 0.5) / 3))
    f, g, F = O.lb_run(p, 2, c1, f, g, steps, want_fields=True)
    u = F["ux"].reshape(H, 2)[:, 0]
    C = F["C"].reshape(H, 2)[:, 0]
    nu = np.where(C - (1 - C) > 0, (tau2 - 0.5) / 3, (tau3 - 0.5) / 3)
    ue = _channel_ode(nu, b * C)
    kk = np.arange(3, H // 2 - 5)
    curv = np.mean(u[kk + 1] - 2 * u[kk] + u[kk - 1])
    return (float(np.max(np.abs(u - ue)) / np.max(np.abs(ue))),
            abs(curv / (-b / ((tau2 - 0.5) / 3)) - 1.0))


@pytest.mark.parametrize("tau2,tau3", [(1.7, 0.8), (0.8, 1.7)])
def test_viscosity_map_two_layer_channel(tau2, tau3):
    prof, curv = _two_layer_dev(tau2, tau3)
    # discretisation and convergence error: profile 0.4-0.7 %, curvature
    # 0.03-0.1 %; a liquid layer relaxing with the gas's tau misses the
    # curvature by nu_3 / nu_2 - 1 (here -53 % or +112 %)
    assert prof < 0.02 and curv < 0.01, (prof, curv)


def _translate_dev(U=0.01, steps=300, rho3=0.3, nx=64):
    """A liquid slab in gas (density ratio rho3) moving at uniform velocity U
    normal to its interfaces: the continuum solution is a rigid translation
    (density advected, u = U, uniform pressure), which the pressure moment's
    u.G[rho]/2 term keeps in the discrete scheme.  Returns (max |u - U| / U,
    max |pt - mean pt|) after `steps` steps."""
    n = 2 * nx
    k, _ = O.kappa_from_angle(90.0, 0.01, 0.01)
    p = O.make_params(O.D2Q9, (nx, 2), k, rho2=1.0, rho3=rho3, tau2=0.9, tau3=0.7)
    x = np.arange(nx)
    c2 = np.tile(0.25 * (1 + np.tanh((x - 15.5) / 2.0)) * (1 + np.tanh((47.5 - x) / 2.0)), 2)
    c1 = np.zeros(n)
    mu = O.lb_fields(p, 2, c1, *O.lb_init(p, 2, c1, c2))["mu"]
    rho = rho3 + (1.0 - rho3) * c2
    f, g = np.zeros((9, n)), np.zeros((9, n))
    for m in range(n):
        f[:, m], g[:, m], _ = O.equilibria(O.D2Q9, 1.0, rho[m], [U, 0.0, 0.0], c2[m], mu[m],
                                           1.0, [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    f, g = O.lb_run(p, 2, c1, f, g, steps)
    F = O.lb_fields(p, 2, c1, f, g)
    return (float(np.max(np.abs(F["ux"] - U)) / U),
            float(np.max(np.abs(F["pt"] - F["pt"].mean()))))


def test_translating_interface_density_contrast():
    du, dp = _translate_dev()
    # the scheme's own error on the diffuse interface: 8 % of U, 6e-4 in pt
    # (without the u.G[rho]/2 term: 62 %, 3.2e-3)
    assert du < 0.2 and dp < 1.5e-3, (du, dp)


# mistakes a reader could make in the density and relaxation maps and in the
# moments that use them, as edits of the C oracle
PLANTED = [
    ("densities swapped", "w->rho[n] = p->rho3 + (p->rho2 - p->rho3) * phi;",
     "w->rho[n] = p->rho2 + (p->rho3 - p->rho2) * phi;"),
    ("volume fraction without 1 - C1", "phi = C / den;", "phi = C;"),
    ("no clamp of the volume fraction", "phi = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);",
     "phi = phi;"),
    ("relaxation map inverted", "w->tau[n] = (C - C3 > 0.0) ? p->tau2 : p->tau3;",
     "w->tau[n] = (C - C3 > 0.0) ? p->tau3 : p->tau2;"),
    ("u.G[rho]/2 dropped", "w->pt[n] = solid_n ? 1.0 : m0 + 0.5 * ug;",
     "w->pt[n] = solid_n ? 1.0 : m0;"),
    ("u.G[rho]/2 with the wrong sign", "w->pt[n] = solid_n ? 1.0 : m0 + 0.5 * ug;",
     "w->pt[n] = solid_n ? 1.0 : m0 - 0.5 * ug;"),
    ("no half-force in the velocity", "u[a] = (m1[a] + 0.5 * w->F[a * N + n]) / w->rho[n];",
     "u[a] = m1[a] / w->rho[n];"),
]


def _oracle_variant(tmp_path, old, new):
    src = open(os.path.join(os.path.dirname(O.__file__), "dsm_oracle.c")).read()
    assert src.count(old) == 1, old
    c = tmp_path / "variant.c"
    so = tmp_path / "variant.so"
    c.write_text(src.replace(old, new))
    import subprocess
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", str(c), "-o", str(so), "-lm"])
    return str(so)


@pytest.mark.parametrize("name,old,new", PLANTED, ids=[p[0] for p in PLANTED])
def test_density_viscosity_pins_catch_planted_mistakes(name, old, new, tmp_path, monkeypatch):
    """Each planted mistake, compiled into a copy of the oracle, fails at
    least one of the three pins above."""
    so = _oracle_variant(tmp_path, old, new)
    monkeypatch.setattr(O, "_lib", None)
    monkeypatch.setattr(O, "_LIB", so)
    monkeypatch.setattr(O, "build", lambda force=False: so)
    fails = []
    if max(_accel_dev(*c) for c in ACCEL_CASES) > 1e-10:
        fails.append("acceleration")
    du, dp = _translate_dev()
    if du > 0.2 or dp > 1.5e-3:
        fails.append("translation")
    if not fails:
        prof, curv = _two_layer_dev(1.7, 0.8)
        if prof > 0.02 or curv > 0.01:
            fails.append("two-layer channel")
    assert fails, name
    monkeypatch.setattr(O, "_lib", None)  # the real oracle again after the test


def test_three_fluid_relaxation_map_three_layer_channel():
    """N = 3 fluids (Sec. II.B for N + 1 components): three layers between two
    walls, the body force on fluid 2, tau of the locally largest fluid.  The
    N-fluid oracle's profile matches the channel solution with each node's
    viscosity from that rule, and each layer's bulk curvature is -b C2 / nu."""
    from oracle.multi_lb import MultiLB
    H = 36
    taus = (1.4, 0.8, 1.1)       # fluids 2, 3 (free) and 4 (dependent)
    b = 2e-6
    faces = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")
    kappa = (0.03, 0.02, 0.025, 0.03)
    p = O.make_params(O.D2Q9, (2, H), kappa[:3], body=(b, 0.0, 0.0), faces=faces)
    y = np.arange(H)
    s = lambda a: 0.5 * (1 + np.tanh(a / 2.0))  # noqa: E731
    c2 = s(11.5 - y)                   # fluid 2: y < 12
    c3 = s(y - 11.5) * s(23.5 - y)     # fluid 3: 12 <= y < 24; fluid 4 above
    Cm = np.stack([np.repeat(c2, 2), np.repeat(c3, 2)])
    m = MultiLB(p, kappa, (1.0, 1.0, 1.0), taus, np.zeros(2 * H))
    f, g = m.init(Cm)
    steps = int(5 * H * H / ((min(taus) - 0.5) / 3))
    f, g = m.run(f, g, steps)
    M = m.fields(f, g)
    u = M["u"][0].reshape(H, 2)[:, 0]
    C = M["C"].reshape(2, H, 2)[:, :, 0]
    allc = np.stack([C[0], C[1], 1.0 - C[0] - C[1]])
    idx = 2 - np.argmax(allc[::-1], axis=0)  # the largest, ties to the later fluid
    nu = (np.asarray(taus)[idx] - 0.5) / 3
    ue = _channel_ode(nu, b * C[0])
    assert np.max(np.abs(u - ue)) / np.max(np.abs(ue)) < 0.02
    kk = np.arange(3, 8)
    curv = np.mean(u[kk + 1] - 2 * u[kk] + u[kk - 1])
    assert abs(curv / (-b / ((taus[0] - 0.5) / 3)) - 1.0) < 0.01
