"""GPU parity of the energy-minimisation twin: the free energy and its
hand-written adjoint (dsm_fe_energy_grad), the autograd function, the L-BFGS
vector kernels and the minimiser, against the FP64 oracle.

Tolerances: energy 1e-6 relative (FP32 per-node densities, FP64 accumulation);
gradient 1e-5 of its max (FP32 arithmetic of O(1) fields); dot products 1e-12
relative (FP64 accumulation of FP32 products); converged L-BFGS energy 1e-5
relative and fields 2e-3 absolute against the oracle's converged minimum (the
iteration trajectory itself is not pinned by the paper)."""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import lbfgs as olbfgs

from dsm_helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2504_19941_gb300 as P  # noqa: E402
from paper_2504_19941_gb300 import _lib  # noqa: E402
from paper_2504_19941_gb300.energy import Energy, FreeEnergy, lbfgs  # noqa: E402

DEV = "cuda"


def _t(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


CASES = [("D2Q9", (23, 17)), ("D3Q19", (16, 16, 16)), ("D3Q19", (13, 9, 7))]


@pytest.mark.parametrize("lat,shape", CASES)
@pytest.mark.parametrize("active", [1, 2])
@pytest.mark.parametrize("constraint", ["volume", "pressure"])
def test_energy_grad_parity(lat, shape, active, constraint):
    n = int(np.prod(shape))
    c1, c2 = S.random_fields(n, seed=11)
    c1 = 0.6 * c1
    mask = (np.arange(n) % 3 == 0).astype(np.uint8)
    kw = dict(kcs=0.3, V0=0.4 * n, dP=0.0) if constraint == "volume" else dict(kcs=0.0, V0=0.0,
                                                                                dP=0.02)
    p = P.make_params(lat, shape, "f32", theta_deg=75.0, g23=0.9, g12=1.0, alpha=1.2, beta=10.0)
    k = _lib.dsm_kappa(p)
    kind = O.D2Q9 if lat == "D2Q9" else O.D3Q19
    po = O.make_params(kind, shape, k, alpha=1.2, beta=10.0)
    c1f, c2f = _t(c1), _t(c2)
    fe = FreeEnergy(p)
    E, g = fe(c1f, c2f, active=active, mask=_t(mask, torch.uint8), fg=0.01, **kw)
    # oracle on the FP32-rounded inputs
    c1r, c2r = c1f.double().cpu().numpy(), c2f.double().cpu().numpy()
    Eo, go, to = O.energy_grad(po, c1r, c2r, active=active, S=mask, fg=0.01, **kw)
    assert abs(E.item() - Eo) / abs(Eo) < 1e-6
    assert rel_err(g.double().cpu().numpy(), go) < 1e-5
    terms = fe.terms.cpu().numpy()
    np.testing.assert_allclose(terms, to, rtol=1e-5, atol=1e-6)
    d = fe.decomposition()
    assert abs(d["surface"] - (to[0] + to[1])) <= 1e-5 * abs(to[0] + to[1])
    assert abs(d["surface"] + d["confinement"] + d["constraint"] + d["gravity"] - Eo) \
        <= 1e-6 * abs(Eo)


MIRROR_CASES = [("D2Q9", (23, 17), ("mirror", "mirror", "wall", "wall", "periodic", "periodic")),
                ("D3Q19", (13, 9, 7), ("mirror", "mirror", "periodic", "periodic", "wall", "mirror")),
                ("D3Q19", (16, 16, 16), ("periodic", "periodic", "mirror", "mirror", "periodic",
                                         "periodic"))]


@pytest.mark.parametrize("lat,shape,faces", MIRROR_CASES)
@pytest.mark.parametrize("active", [1, 2])
def test_energy_grad_mirror_parity(lat, shape, faces, active):
    # symmetry planes and walls on some axes: dsm_fe_energy_grad and the
    # allocation-free entry point against the oracle with the same faces
    n = int(np.prod(shape))
    c1, c2 = S.random_fields(n, seed=17)
    c1 = 0.6 * c1
    mask = (np.arange(n) % 4 == 1).astype(np.uint8)
    kw = dict(kcs=0.0, V0=0.0, dP=0.015)
    p = P.make_params(lat, shape, "f32", theta_deg=65.0, g23=0.9, g12=1.0, alpha=1.1, beta=8.0,
                      faces=faces)
    k = _lib.dsm_kappa(p)
    kind = O.D2Q9 if lat == "D2Q9" else O.D3Q19
    po = O.make_params(kind, shape, k, alpha=1.1, beta=8.0, faces=faces)
    c1f, c2f, mf = _t(c1), _t(c2), _t(mask, torch.uint8)
    fe = FreeEnergy(p)
    E, g = fe(c1f, c2f, active=active, mask=mf, fg=0.01, **kw)
    c1r, c2r = c1f.double().cpu().numpy(), c2f.double().cpu().numpy()
    Eo, go, to = O.energy_grad(po, c1r, c2r, active=active, S=mask, fg=0.01, **kw)
    assert abs(E.item() - Eo) / abs(Eo) < 1e-6
    assert rel_err(g.double().cpu().numpy(), go) < 1e-5
    np.testing.assert_allclose(fe.terms.cpu().numpy(), to, rtol=1e-5, atol=1e-6)
    E2 = torch.empty(1, dtype=torch.float64, device=DEV)
    g2 = torch.empty(n, dtype=torch.float32, device=DEV)
    t2 = torch.empty(6, dtype=torch.float64, device=DEV)
    _lib.dsm_fe_energy_grad_noalloc(p, c1f, c2f, mf, active, kw["dP"], 0.0, 0.0, 0.01, E2, g2, t2)
    torch.cuda.synchronize()
    assert abs(E2.item() - Eo) / abs(Eo) < 1e-6
    assert rel_err(g2.double().cpu().numpy(), go) < 1e-5


def test_lbfgs_mirror_half_domain_matches_symmetric_full_domain():
    # a drop on a flat wall, symmetric about x = -1/2: the half lattice with a
    # mirror face at x = 0 reaches the full periodic lattice's minimum on its
    # nodes, with half its energy (volume constraint halved too)
    nx, ny, wall = 48, 40, 8
    full = (2 * nx, ny)
    pf = P.make_params("D2Q9", full, "f32", theta_deg=70.0, g23=math.sqrt(8 / 9), g12=1.0)
    ph = P.make_params("D2Q9", (nx, ny), "f32", theta_deg=70.0, g23=math.sqrt(8 / 9), g12=1.0,
                       faces=("mirror", "mirror", "periodic", "periodic", "periodic", "periodic"))
    sd = S.slab_sd(full, 1, 0, wall)
    c1 = O.solid_profile(sd.ravel(), 1.0).reshape(ny, 2 * nx)
    c2 = S.cap_c2(full, wall - 0.5, 14.0, 90.0, 1.0, sd, 1.0).reshape(ny, 2 * nx)
    # centre the drop on the plane between node 2nx-1 and node 0
    c2 = np.roll(c2, nx, axis=1)
    np.testing.assert_allclose(c2, c2[:, ::-1], atol=1e-12)
    V0 = float(_t(c2).double().sum())
    xf, Ef, inf_f = lbfgs(FreeEnergy(pf), _t(c2.ravel()), _t(c1.ravel()), active=2, kcs=0.05,
                          V0=V0, tol=1e-5, max_iter=5000)
    xh, Eh, inf_h = lbfgs(FreeEnergy(ph), _t(c2[:, :nx].ravel()), _t(c1[:, :nx].ravel()),
                          active=2, kcs=0.05 * 2, V0=V0 / 2, tol=1e-5, max_iter=5000)
    assert inf_f["rms_grad"] < 1e-5 and inf_h["rms_grad"] < 1e-5
    # kcs doubles with V0 halved: 0.5 (2 kcs) (V/2 - V0/2)^2 is half the full term
    assert abs(Eh - Ef / 2) / abs(Ef) < 1e-5, (Eh, Ef)
    xf2 = xf.double().cpu().numpy().reshape(ny, 2 * nx)
    assert np.max(np.abs(xh.double().cpu().numpy().reshape(ny, nx) - xf2[:, :nx])) < 2e-3


def _sinusoid_problem(case):
    p = P.make_params("D3Q19", case.shape, "f32", theta_deg=case.theta_deg, g23=case.g23,
                      g12=case.g12)
    c1 = O.solid_profile(case.solid_sd, case.alpha_s)
    return p, _t(c1), _t(case.c2)


def test_lbfgs_sinusoid_drop_full_size():
    # the 128^3 energy-minimisation case of a drop on the sinusoidal wall
    # z < 16 + 6 sin(2 pi x / 32), volume-constrained (k_cs = 1e-2): the native
    # L-BFGS converges, lowers the energy and keeps the volume
    case = S.em_sinusoid_drop()
    p, c1f, c2f = _sinusoid_problem(case)
    V0 = float(c2f.double().sum())
    fe = FreeEnergy(p)
    E0, _ = fe(c1f, c2f, active=2, kcs=case.extra["kcs"], V0=V0)
    x, E, info = lbfgs(fe, c2f, c1f, active=2, kcs=case.extra["kcs"], V0=V0, tol=1e-6,
                       max_iter=20000)
    assert info["converged"] and info["rms_grad"] < 1e-6, info
    assert E < E0.item()
    assert abs(float(x.double().sum()) / V0 - 1.0) < 5e-3
    assert float(x.min()) > -0.05 and float(x.max()) < 1.05


def test_lbfgs_sphere_at_interface_full_size():
    # the other 128^3 case: a solid sphere of radius 20 at a flat liquid/gas
    # interface (Sec. III, Liquid Contact Angle: particles at interfaces),
    # volume-constrained; the native L-BFGS reaches rms gradient 1e-6 (about
    # 3100 iterations), lowers the energy and keeps the liquid volume
    case = S.em_sphere_interface()
    p, c1f, c2f = _sinusoid_problem(case)
    V0 = float(c2f.double().sum())
    fe = FreeEnergy(p)
    E0, _ = fe(c1f, c2f, active=2, kcs=1e-2, V0=V0)
    x, E, info = lbfgs(fe, c2f, c1f, active=2, kcs=1e-2, V0=V0, tol=1e-6, max_iter=20000)
    assert info["converged"] and info["rms_grad"] < 1e-6, info
    assert E < E0.item()
    assert abs(float(x.double().sum()) / V0 - 1.0) < 1e-4
    assert float(x.min()) > -0.05 and float(x.max()) < 1.05


def test_lbfgs_sinusoid_drop_matches_oracle():
    # the same geometry scaled to 32^3: the GPU minimiser and the oracle's
    # reach the same minimum
    case = S.em_sinusoid_drop(n=32, amplitude=1.5, wavelength=8.0, base=4.0, radius=7.5)
    p, c1f, c2f = _sinusoid_problem(case)
    V0 = float(c2f.double().sum())
    kcs = case.extra["kcs"]
    x, E, info = lbfgs(FreeEnergy(p), c2f, c1f, active=2, kcs=kcs, V0=V0, tol=1e-5,
                       max_iter=20000)
    assert info["rms_grad"] < 1e-5
    po = O.make_params(O.D3Q19, case.shape, _lib.dsm_kappa(p))
    c1 = c1f.double().cpu().numpy()

    def fg(v):
        e, gr, _ = O.energy_grad(po, c1, v, active=2, kcs=kcs, V0=V0)
        return e, gr
    xo, Eo, _, info_o = olbfgs.minimize(fg, c2f.double().cpu().numpy(), tol=1e-7,
                                        max_iter=20000)
    assert info_o["rms_grad"] < 2e-7
    assert abs(E - Eo) / abs(Eo) < 1e-5, (E, Eo)
    assert np.max(np.abs(x.double().cpu().numpy() - xo)) < 2e-3


def test_energy_grad_large_grid():
    shape = (128, 128, 128)
    case = S.em_sphere_interface()
    p = P.make_params("D3Q19", shape, "f32", theta_deg=90.0, g23=math.sqrt(8 / 9), g12=1.0)
    k = _lib.dsm_kappa(p)
    po = O.make_params(O.D3Q19, shape, k)
    c1 = O.solid_profile(case.solid_sd, 1.0)
    c1f, c2f = _t(c1), _t(case.c2)
    fe = FreeEnergy(p)
    E, g = fe(c1f, c2f, active=2)
    Eo, go, _ = O.energy_grad(po, c1f.double().cpu().numpy(), c2f.double().cpu().numpy(), active=2)
    assert abs(E.item() - Eo) / abs(Eo) < 1e-6
    assert rel_err(g.double().cpu().numpy(), go) < 1e-5


def test_autograd_backward_is_the_adjoint():
    shape = (12, 10, 8)
    n = 960
    c1, c2 = S.random_fields(n, seed=3)
    c1 *= 0.5
    p = P.make_params("D3Q19", shape, "f32", theta_deg=120.0, g23=1.0, g12=1.0)
    fe = FreeEnergy(p)
    x = _t(c2).requires_grad_(True)
    E = Energy.apply(x, _t(c1), fe, 2)
    (3.0 * E).backward()
    _, g = fe(_t(c1), _t(c2), active=2)
    torch.testing.assert_close(x.grad, 3.0 * g, rtol=1e-6, atol=1e-7)
    # first-order check of the adjoint on the GPU itself (FP32 energies)
    rng = np.random.default_rng(0)
    v = _t(rng.normal(size=n))
    h = 1e-2
    Ep = Energy.apply(_t(c2) + h * v, _t(c1), fe, 2).item()
    Em = Energy.apply(_t(c2) - h * v, _t(c1), fe, 2).item()
    fd = (Ep - Em) / (2 * h)
    an = float(torch.dot(g.double(), v.double()))
    assert abs(fd - an) / abs(an) < 1e-3


def test_vector_kernels():
    n = 1_000_003
    rng = np.random.default_rng(5)
    x, y = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    xd, yd = _t(x), _t(y)
    sb = _lib.dsm_vec_scratch_bytes(n)
    sc = torch.empty(sb, dtype=torch.uint8, device=DEV)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    _lib.dsm_vec_dot(n, xd, yd, out, sc, sb)
    ref = float(np.dot(x.astype(np.float64), y.astype(np.float64)))
    assert abs(out.item() - ref) / abs(ref) < 1e-12
    out2 = torch.zeros(1, dtype=torch.float64, device=DEV)
    _lib.dsm_vec_dot(n, xd, yd, out2, sc, sb)
    assert out2.item() == out.item()  # deterministic
    z = yd.clone()
    _lib.dsm_vec_axpby(n, 0.5, xd, -2.0, z)
    np.testing.assert_allclose(z.cpu().numpy(), 0.5 * x - 2.0 * y, rtol=1e-6, atol=1e-6)
    a = torch.tensor([1.5], dtype=torch.float64, device=DEV)
    b = torch.tensor([0.25], dtype=torch.float64, device=DEV)
    z = yd.clone()
    _lib.dsm_vec_axpy_dev(n, -1.0, a, b, xd, z)
    np.testing.assert_allclose(z.cpu().numpy(), y - 1.25 * x, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("n,nv", [(1_000_003, 20), (4097, 7), (33, 1)])
def test_batched_dots_and_lincomb(n, nv):
    rng = np.random.default_rng(nv)
    V = rng.normal(size=(nv, n)).astype(np.float32)
    x = rng.normal(size=n).astype(np.float32)
    Vd, xd = _t(V.ravel()), _t(x)
    sb = _lib.dsm_vec_dots_scratch_bytes(n, nv)
    sc = torch.empty(sb, dtype=torch.uint8, device=DEV)
    out = torch.zeros(nv, dtype=torch.float64, device=DEV)
    _lib.dsm_vec_dots(n, nv, Vd, n, xd, out, sc, sb)
    ref = V.astype(np.float64) @ x.astype(np.float64)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # each equals the single dot of the same vectors bitwise
    sb1 = _lib.dsm_vec_scratch_bytes(n)
    sc1 = torch.empty(sb1, dtype=torch.uint8, device=DEV)
    one = torch.zeros(1, dtype=torch.float64, device=DEV)
    for k in (0, nv - 1):
        _lib.dsm_vec_dot(n, Vd[k * n:(k + 1) * n], xd, one, sc1, sb1)
        assert one.item() == out[k].item()
    coef = rng.normal(size=nv)
    y = torch.empty(n, dtype=torch.float32, device=DEV)
    _lib.dsm_vec_lincomb(n, nv, Vd, n, coef, xd, -0.75, y)
    ref = -0.75 * x.astype(np.float64) + coef @ V.astype(np.float64)
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    with pytest.raises(P.DSMError):
        _lib.dsm_vec_lincomb(n, 65, Vd, n, np.zeros(65), xd, 1.0, y)


def test_two_loop_recursion_matches_dense_inverse_hessian():
    # with m pairs from a quadratic, the two-loop product equals the textbook
    # recursion H_{k+1} = (I - rho s y^T) H_k (I - rho y s^T) + rho s s^T
    n, m = 50, 4
    rng = np.random.default_rng(2)
    A = rng.normal(size=(n, n))
    A = A @ A.T + n * np.eye(n)
    Ss = rng.normal(size=(m, n))
    Ys = Ss @ A.T
    g = rng.normal(size=n)
    rho = 1.0 / np.einsum("ij,ij->i", Ss, Ys)
    gamma = float(Ss[-1] @ Ys[-1] / (Ys[-1] @ Ys[-1]))
    H = gamma * np.eye(n)
    for s, y, r in zip(Ss, Ys, rho):
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    ref = -H @ g
    Sd = _t(Ss.astype(np.float32).ravel())
    Yd = _t(Ys.astype(np.float32).ravel())
    Sf, Yf = Sd.double().cpu().numpy().reshape(m, n), Yd.double().cpu().numpy().reshape(m, n)
    rho_f = 1.0 / np.einsum("ij,ij->i", Sf, Yf)
    rhod = torch.as_tensor(rho_f, dtype=torch.float64, device=DEV)
    gam = torch.tensor([gamma], dtype=torch.float64, device=DEV)
    gd = _t(g.astype(np.float32))
    r = torch.empty(n, dtype=torch.float32, device=DEV)
    alpha = torch.zeros(m, dtype=torch.float64, device=DEV)
    sb = _lib.dsm_vec_scratch_bytes(n)
    sc = torch.empty(sb, dtype=torch.uint8, device=DEV)
    _lib.dsm_lbfgs_direction(n, list(range(m)), Sd, Yd, rhod, gam, gd, r, alpha, sc, sb)
    assert rel_err(r.double().cpu().numpy(), ref) < 1e-4


def test_lbfgs_minimum_matches_oracle():
    # 2D drop on a flat diffuse wall, volume-constrained (Sec. III.A setup,
    # small): the GPU minimiser and the oracle's reach the same minimum
    nx, ny, wall = 64, 40, 8
    shape = (nx, ny)
    p = P.make_params("D2Q9", shape, "f32", theta_deg=70.0, g23=math.sqrt(8 / 9), g12=1.0)
    k = _lib.dsm_kappa(p)
    po = O.make_params(O.D2Q9, shape, k)
    sd = S.slab_sd(shape, 1, 0, wall)
    c1 = O.solid_profile(sd.ravel(), 1.0)
    c2 = S.cap_c2(shape, wall - 0.5, 14.0, 90.0, 1.0, sd, 1.0).ravel()
    c1f, c2f = _t(c1), _t(c2)
    V0 = float(c2f.double().sum())
    fe = FreeEnergy(p)
    x, E, info = lbfgs(fe, c2f, c1f, active=2, kcs=0.05, V0=V0, tol=1e-5, max_iter=5000)
    assert info["rms_grad"] < 1e-5

    def fg(v):
        e, gr, _ = O.energy_grad(po, c1f.double().cpu().numpy(), v, active=2, kcs=0.05, V0=V0)
        return e, gr
    xo, Eo, _, info_o = olbfgs.minimize(fg, c2f.double().cpu().numpy(), tol=1e-8, max_iter=20000)
    assert abs(E - Eo) / abs(Eo) < 1e-5, (E, Eo)
    assert np.max(np.abs(x.double().cpu().numpy() - xo)) < 2e-3
