"""GPU parity of the N-fluid free energy (dsm_fe_energy_grad_multi) and of its
L-BFGS (dsm_lbfgs_minimize_multi) against the FP64 oracle (oracle/multi.py).

Tolerances as for the two-fluid energy: energy 1e-6 relative (FP32 per-node
densities, FP64 accumulation), gradients 1e-5 of their max; the converged
L-BFGS energy 1e-5 relative and fields 2e-3 absolute against the oracle's own
converged minimum (the iteration trajectory is not pinned)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import lbfgs as olbfgs
from oracle import multi as M

from dsm_helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2504_19941_gb300 as P  # noqa: E402
from paper_2504_19941_gb300 import _lib  # noqa: E402
from paper_2504_19941_gb300.energy import (FreeEnergy, FreeEnergyMulti,  # noqa: E402
                                           lbfgs_multi)

DEV = "cuda"
FACES = ("mirror", "mirror", "periodic", "periodic", "wall", "mirror")


def _t(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


@pytest.mark.parametrize("lat,shape,faces", [("D2Q9", (23, 17), None),
                                             ("D3Q19", (13, 9, 7), FACES),
                                             ("D3Q19", (32, 8, 5), None)])
@pytest.mark.parametrize("nfluid", [2, 3, 4])
def test_energy_grad_multi_parity(lat, shape, faces, nfluid):
    n = int(np.prod(shape))
    nf = nfluid - 1
    rng = np.random.default_rng(10 * nfluid + len(shape))
    c1 = 0.4 * rng.uniform(size=n)
    C = rng.uniform(0.02, 0.3, size=(nf, n)) * (1.0 - c1) / max(nf, 1)
    kappa = rng.uniform(0.5, 1.5, size=nfluid + 1)
    kappa[0] = -0.2                      # the solid's kappa may be negative
    dP = rng.uniform(-0.02, 0.02, nf)
    kcs = np.r_[0.3, np.zeros(nf - 1)]
    V0 = np.r_[0.1 * n, np.zeros(nf - 1)]
    p = P.make_params(lat, shape, "f32", theta_deg=90.0, alpha=1.2, faces=faces)
    kind = O.D2Q9 if lat == "D2Q9" else O.D3Q19
    po = O.make_params(kind, shape, (1.0, 1.0, 1.0), alpha=1.2, faces=faces)
    c1f, Cf = _t(c1), _t(C)
    fe = FreeEnergyMulti(p, nfluid, kappa)
    E, g = fe(c1f, Cf, dP=dP, kcs=kcs, V0=V0)
    Eo, go, to = M.energy_grad_multi(po, kappa, c1f.double().cpu().numpy(),
                                     Cf.double().cpu().numpy(), dP=dP, kcs=kcs, V0=V0)
    assert abs(E.item() - Eo) / abs(Eo) < 1e-6
    assert rel_err(g.double().cpu().numpy(), go) < 1e-5
    np.testing.assert_allclose(fe.terms.cpu().numpy(), to, rtol=1e-5, atol=1e-6)


def test_two_fluids_equal_the_two_fluid_entry_point():
    shape = (40, 30)
    n = 1200
    c1, c2 = S.random_fields(n, seed=4)
    c1, c2 = 0.5 * c1, 0.4 * c2
    p = P.make_params("D2Q9", shape, "f32", theta_deg=75.0, g23=0.9, g12=1.0, alpha=1.1)
    k = _lib.dsm_kappa(p)
    E2, g2 = FreeEnergy(p)(_t(c1), _t(c2), active=2, dP=0.01)
    Em, gm = FreeEnergyMulti(p, 2, k)(_t(c1), _t(c2[None, :]), dP=[0.01])
    assert abs(E2.item() - Em.item()) <= 1e-6 * abs(E2.item())
    assert rel_err(gm[0].double().cpu().numpy(), g2.double().cpu().numpy()) < 1e-6


def test_lbfgs_multi_lens_matches_oracle():
    # half a lens of fluid 2 at the flat interface between fluid 3 (below) and
    # the dependent fluid 4 (above), centred on the mirror face x = -1/2 (mirror
    # faces all round: a lens in a periodic box could slide freely, and the
    # minimum would not be unique); no solid; fluids 2 and 3
    # volume-constrained.  Tensions (kappa_m + kappa_n)/6: 0.30, 0.317, 0.283,
    # so the lens stays a lens (the spreading coefficient is negative).  Two
    # different oracle starts reach the same minimum (checked to 1e-6).
    nx, ny = 32, 40
    n = nx * ny
    faces = ("mirror", "mirror", "mirror", "mirror", "periodic", "periodic")
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    lens = 0.5 * (1.0 + np.tanh((8.0 - np.hypot(x + 0.5, y - 20.0)) / 2.0))
    below = 0.5 * (1.0 - np.tanh((y - 20.0) / 2.0)) * (1.0 - lens)
    C0 = np.stack([lens.ravel(), below.ravel()])
    kappa = (0.5, 1.0, 0.8, 0.9)
    V0 = C0.sum(axis=1)
    kcs = (0.05, 0.05)
    p = P.make_params("D2Q9", (nx, ny), "f32", theta_deg=90.0, faces=faces)
    po = O.make_params(O.D2Q9, (nx, ny), (1.0, 1.0, 1.0), faces=faces)
    c1 = np.zeros(n)
    fe = FreeEnergyMulti(p, 3, kappa)
    X, E, info = lbfgs_multi(fe, _t(C0), _t(c1), kcs=kcs, V0=V0, tol=1e-5, max_iter=6000)
    assert info["rms_grad"] < 1e-5

    def fg(v):
        e, g, _ = M.energy_grad_multi(po, kappa, c1, v.reshape(2, n), kcs=kcs, V0=V0)
        return e, g.ravel()
    xo, Eo, _, info_o = olbfgs.minimize(fg, _t(C0).double().cpu().numpy().ravel(), tol=1e-8,
                                        max_iter=20000)
    assert info_o["rms_grad"] < 1e-8
    assert abs(E - Eo) / abs(Eo) < 1e-5, (E, Eo)
    assert np.max(np.abs(X.double().cpu().numpy().ravel() - xo)) < 2e-3


# ---------------------------------------------------------------- LB, N fluids

from dsm_helpers import ml_compare, ml_run  # noqa: E402


def _ml_case_2d(nf):
    # a drop of fluid 2 on a diffuse wall, a layer of fluid 3 (and fluid 4 in
    # a second drop for N = 4) under the dependent fluid; mirror x faces
    nx, ny = 24, 20
    sd = S.slab_sd((nx, ny), 1, 0, 4)
    c1 = O.solid_profile(sd.ravel(), 1.0)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    free = 1.0 - c1.reshape(ny, nx)
    drop = 0.5 * (1 + np.tanh((5.0 - np.hypot(x - 6.0, y - 9.0)) / 2.0)) * free
    layer = np.clip(0.5 * (1 - np.tanh((y - 13.0) / 2.0)) * free - drop, 0, 1)
    C = [drop, layer]
    if nf == 3:
        d2 = 0.5 * (1 + np.tanh((3.0 - np.hypot(x - 17.0, y - 16.0)) / 2.0)) * free
        C.append(d2)
        C[1] = np.clip(C[1] - d2, 0, 1)
    C = np.stack([c.ravel() for c in C])
    kappa = (0.02, 0.03, 0.025, 0.035, 0.028)[:nf + 2]
    rho = (1.0, 0.7, 0.5, 0.8)[:nf + 1]
    tau = (0.8, 1.0, 0.7, 0.9)[:nf + 1]
    faces = ("mirror", "mirror", "periodic", "periodic", "periodic", "periodic")
    return (nx, ny), c1, C, kappa, rho, tau, faces, (1e-5, -1e-5, 0.0)


def _ml_case_3d(nf):
    shape = (14, 12, 10)
    nx, ny, nz = shape
    sd = S.pillars_sd(shape, 3, 4, 7, 5, offset=2)
    c1 = O.solid_profile(sd.ravel(), 1.0)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(float)
    free = 1.0 - c1.reshape(nz, ny, nx)
    drop = 0.5 * (1 + np.tanh((3.5 - np.hypot(np.hypot(x - 7, y - 6), z - 6.0)) / 2.0)) * free
    layer = np.clip(0.5 * (1 - np.tanh((z - 4.5) / 2.0)) * free - drop, 0, 1)
    C = [drop, layer]
    if nf == 3:
        C.append(0.5 * (1 + np.tanh((z - 8.0) / 2.0)) * free * 0.8)
    C = np.stack([c.ravel() for c in C])
    kappa = (0.02, 0.03, 0.025, 0.035, 0.028)[:nf + 2]
    rho = (1.0, 0.7, 0.5, 0.8)[:nf + 1]
    tau = (0.8, 1.0, 0.7, 0.9)[:nf + 1]
    faces = ("mirror", "mirror", "wall", "wall", "mirror", "wall")
    return shape, c1, C, kappa, rho, tau, faces, (0.0, 1e-5, -1e-5)


def _ml_run(case, prec, steps, tau_g=0.9):
    return ml_run(case, prec, steps, tau_g)


def _ml_compare(ml, m, f, g, kind):
    return ml_compare(ml, m, f, g, kind)


@pytest.mark.parametrize("make", [_ml_case_2d, _ml_case_3d])
@pytest.mark.parametrize("nf", [2, 3])
def test_ml_fp64_parity(make, nf):
    ml, m, f, g, kind = _ml_run(make(nf), "f64", 20)
    errs = _ml_compare(ml, m, f, g, kind)
    assert max(errs.values()) < 1e-12, errs


@pytest.mark.parametrize("make", [_ml_case_2d, _ml_case_3d])
def test_ml_fp32_parity(make):
    ml, m, f, g, kind = _ml_run(make(2), "f32", 40)
    e = _ml_compare(ml, m, f, g, kind)
    assert e["f"] < 1e-5 and e["g"] < 1e-5 and e["C0"] < 1e-5 and e["C1"] < 1e-5, e
    assert e["pt"] < 1e-5 and e["rho"] < 1e-5 and e["mu0"] < 1e-4 and e["mu1"] < 1e-4, e
    # the velocity is a cancelling sum of O(0.1) populations: its FP32 rounding
    # relative to max |u| is larger here, where three fluids' forces partly
    # cancel, than in the two-fluid case (2e-4)
    assert max(v for k_, v in e.items() if k_ in ("ux", "uy", "uz")) < 5e-4, e
    # the same fluid rules every node; tau comes back as 1 / (1 / tau) in FP32
    assert e["tau"] < 1e-7, e


def test_ml_two_fluids_equal_the_lattice():
    # N = 2 through the N-fluid path equals the two-fluid step (population form)
    case = _ml_case_2d(2)
    shape, c1, C, kappa, rho, tau, faces, body = case
    p = P.make_params("D2Q9", shape, "f64", theta_deg=90.0, tau_g=0.9, body=body, faces=faces,
                      alpha_s=1.0, rho2=rho[0], rho3=rho[2], tau2=tau[0], tau3=tau[2])
    k3 = (kappa[0], kappa[1], kappa[3])
    # the two-fluid lattice takes its kappa from the tensions: find them
    g12 = (k3[0] + k3[1]) / 6.0
    g13 = (k3[0] + k3[2]) / 6.0
    g23 = (k3[1] + k3[2]) / 6.0
    p.tension_mode, p.g12, p.g13, p.g23 = 0, g12, g13, g23
    np.testing.assert_allclose(_lib.dsm_kappa(p), k3, rtol=1e-12)
    lat = P.Lattice(p)
    lat.set_g_storage("populations")
    lat.set_solid_c1(_t(c1, torch.float64))
    lat.set_fluid(_t(C[0], torch.float64))
    lat.step(30)
    ml = P.MultiLattice(p, 2, k3, (rho[0], rho[2]), (tau[0], tau[2]))
    ml.set_solid_c1(_t(c1, torch.float64))
    ml.set_fluids(_t(C[:1], torch.float64))
    ml.step(30)
    f1, g1 = lat.populations()
    f2, g2 = ml.populations()
    assert rel_err(f2.cpu().numpy(), f1.cpu().numpy()) < 1e-12
    assert rel_err(g2.cpu().numpy(), g1.cpu().numpy()) < 1e-12


def test_ml_three_layers_relax_to_the_energy_minimum():
    # fluid 2 | fluid 3 | fluid 4 between walls: the stationary LB state is the
    # N-fluid energy minimum at the same volumes (the CPU pin stops at 6000
    # steps and 1e-4)
    nx = 48
    x = np.arange(nx, dtype=float)
    C = np.stack([0.5 * (1.0 - np.tanh((x - 16.0) / 2.0)),
                  0.5 * (np.tanh((x - 16.0) / 2.0) - np.tanh((x - 32.0) / 2.0))])
    kappa = (0.0, 0.1, 0.12, 0.11)
    faces = ("wall", "wall", "periodic", "periodic", "periodic", "periodic")
    p = P.make_params("D2Q9", (nx, 1), "f64", theta_deg=90.0, faces=faces)
    ml = P.MultiLattice(p, 3, kappa, (1.0, 1.0, 1.0), (1.0, 1.0, 1.0))
    ml.set_solid_c1(torch.zeros(nx, dtype=torch.float64, device=DEV))
    ml.set_fluids(_t(C, torch.float64))
    ml.step(200000)
    got = np.stack([ml.field("C", k).cpu().numpy() for k in range(2)])
    po = O.make_params(O.D2Q9, (nx, 1), kappa[:3], faces=faces)
    V0 = C.sum(axis=1)

    def fg(v):
        e, gr, _ = M.energy_grad_multi(po, kappa, np.zeros(nx), v.reshape(2, nx), kcs=(1.0, 1.0),
                                       V0=V0)
        return e, gr.ravel()
    v, E, gr, info = olbfgs.minimize(fg, C.ravel(), tol=1e-11, max_iter=20000)
    assert np.max(np.abs(got - v.reshape(2, nx))) < 1e-6
    assert np.abs(ml.field("ux").cpu().numpy()).max() < 1e-9


@pytest.mark.parametrize("shape,faces", [((13, 9, 7), ("mirror", "mirror", "periodic", "periodic",
                                                      "wall", "wall")),
                                         ((3, 1), ("wall", "wall", "mirror", "mirror", "periodic",
                                                   "periodic"))])
def test_ml_ragged_and_tiny_fp64(shape, faces):
    n = int(np.prod(shape))
    rng = np.random.default_rng(n)
    c1 = np.where(np.arange(n) % 5 == 0, 0.7, 0.02)
    C = rng.uniform(0.1, 0.3, size=(2, n)) * (1 - c1)
    case = (shape, c1, C, (0.02, 0.03, 0.025, 0.035), (1.0, 0.7, 0.5), (0.8, 1.0, 0.7), faces,
            (1e-5, 0.0, -1e-5) if len(shape) == 3 else (1e-5, 0.0, 0.0))
    ml, m, f, g, kind = _ml_run(case, "f64", 9)
    errs = _ml_compare(ml, m, f, g, kind)
    assert max(errs.values()) < 1e-12, errs


def _periodic(case):
    shape, c1, C, kappa, rho, tau, faces, body = case
    return shape, c1, C, kappa, rho, tau, None, body


@pytest.mark.parametrize("make", [_ml_case_2d, _ml_case_3d])
@pytest.mark.parametrize("nf", [2, 3])
def test_ml_geq_form_fp64_parity(make, nf):
    # tau_g = 1 and periodic faces: g held as g_eq (A_f, u); the same step as
    # the population-form oracle up to rounding
    ml, m, f, g, kind = _ml_run(_periodic(make(nf)), "f64", 20, tau_g=1.0)
    errs = _ml_compare(ml, m, f, g, kind)
    assert max(errs.values()) < 1e-12, errs


def test_ml_geq_form_fp32_parity():
    ml, m, f, g, kind = _ml_run(_periodic(_ml_case_3d(2)), "f32", 40, tau_g=1.0)
    e = _ml_compare(ml, m, f, g, kind)
    assert e["f"] < 1e-5 and e["g"] < 1e-5 and e["C0"] < 1e-5 and e["C1"] < 1e-5, e
    assert e["pt"] < 1e-5 and e["rho"] < 1e-5 and e["mu0"] < 1e-4 and e["mu1"] < 1e-4, e
    assert max(v for k_, v in e.items() if k_ in ("ux", "uy", "uz")) < 5e-4, e


def test_ml_geq_two_fluids_equal_the_lattice():
    # N = 2 in the g_eq form equals the two-fluid lattice in its g_eq form
    shape, c1, C, kappa, rho, tau, faces, body = _ml_case_2d(2)
    p = P.make_params("D2Q9", shape, "f64", theta_deg=90.0, tau_g=1.0, body=body,
                      alpha_s=1.0, rho2=rho[0], rho3=rho[2], tau2=tau[0], tau3=tau[2])
    k3 = (kappa[0], kappa[1], kappa[3])
    p.tension_mode = 0
    p.g12, p.g13, p.g23 = (k3[0] + k3[1]) / 6.0, (k3[0] + k3[2]) / 6.0, (k3[1] + k3[2]) / 6.0
    lat = P.Lattice(p)
    lat.set_solid_c1(_t(c1, torch.float64))
    lat.set_fluid(_t(C[0], torch.float64))
    lat.step(30)
    assert lat.g_implicit
    ml = P.MultiLattice(p, 2, k3, (rho[0], rho[2]), (tau[0], tau[2]))
    ml.set_solid_c1(_t(c1, torch.float64))
    ml.set_fluids(_t(C[:1], torch.float64))
    ml.step(30)
    f1, g1 = lat.populations()
    f2, g2 = ml.populations()
    assert rel_err(f2.cpu().numpy(), f1.cpu().numpy()) < 1e-12
    assert rel_err(g2.cpu().numpy(), g1.cpu().numpy()) < 1e-12
    for name in ("mu", "ux", "pt"):
        assert rel_err(ml.field(name).cpu().numpy(), lat.field(name).cpu().numpy()) < 1e-12


@pytest.mark.parametrize("tau_g", [0.9, 1.0])
def test_ml_nonfinite_is_latched(tau_g):
    # a NaN in the input fluids reaches the fused pass, which latches it;
    # dsm_ml_set_fluids clears the word again
    shape, c1, C, kappa, rho, tau, faces, body = _periodic(_ml_case_2d(2))
    p = P.make_params("D2Q9", shape, "f64", theta_deg=90.0, tau_g=tau_g, alpha_s=1.0)
    ml = P.MultiLattice(p, 3, kappa, rho, tau)
    ml.set_solid_c1(_t(c1, torch.float64))
    bad = C.copy()
    bad[0, 17] = np.nan
    ml.set_fluids(_t(bad, torch.float64))
    ml.step(3)
    assert ml.status() == _lib.DSM_E_NONFINITE
    ml.set_fluids(_t(C, torch.float64))
    assert ml.status() == 0
    ml.step(3)
    assert ml.status() == 0

