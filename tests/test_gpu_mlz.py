"""The one-pass N-fluid step (dsm_ml_set_step_form, DSM_STEP_AUTO): D3Q19
lattices whose planes tile into 32 x 8 blocks, every g_f held as g_eq
(tau_g = 1), periodic faces; N = 2, 3, 4 fluids (1, 2, 3 free fluids).

Each step rebuilds every C_f = sum_i g_eq_i(x - c_i) on chip from the staged
(A_f, C_f, u) of the previous collision and runs the N-fluid fused pass in the
same launch, so it is the same step as the moments passes + fused pass
(Sec. II.B for N + 1 components).  Checked here:
  * against the FP64 N-fluid oracle (1e-12 per field and population in FP64,
    velocities against the speed scale; the FP32 tolerances of the two-pass
    N-fluid parity tests in FP32), with density and viscosity contrasts, on the
    smallest tiles (32 x 8, nz = 1 and 3) and on lattices of several tiles
    with a ragged z run;
  * against the two-pass step on the same lattice in FP32, to a few FP32 ulp
    of each field's scale;
  * that the result does not depend on the z planes per block (bitwise);
  * that reading fields and populations and switching forms mid-run leave the
    trajectory unchanged;
  * that lattices the single pass does not cover run the two passes.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

from dsm_helpers import ml_compare, ml_run, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2504_19941_gb300 as P  # noqa: E402

DEV = "cuda"


def _case(nf, shape=(64, 16, 11), contrast=True, body=(1e-5, -1e-5, 2e-6)):
    """Pillars on a base plate; a drop of fluid 2 over the pillars, a layer of
    fluid 3 on the plate (N >= 3), a top layer of fluid 4 (N = 4), the
    dependent fluid elsewhere; seeded perturbation."""
    nx, ny, nz = shape
    sd = S.pillars_sd(shape, min(3, nz - 1), 5, 16, 4, offset=2)
    c1 = O.solid_profile(sd.ravel(), 1.0)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(float)
    free = 1.0 - c1.reshape(nz, ny, nx)
    zc = min(7.0, nz / 2)
    drop = 0.5 * (1 + np.tanh((4.0 - np.hypot(np.hypot(x - nx / 2, y - ny / 2), z - zc)) / 2.0))
    drop = drop * free
    layer = np.clip(0.5 * (1 - np.tanh((z - min(5.0, nz / 2)) / 2.0)) * free - drop, 0, 1)
    top = np.clip(0.5 * (1 + np.tanh((z - (nz - 3.0)) / 2.0)) * free * 0.8 - drop - layer, 0, 1)
    C = [drop, layer, top][:nf] if nf > 1 else [drop + layer]
    n = nx * ny * nz
    C = np.stack([np.clip(c.ravel() + S.perturbation(11 + k, n), 0.0, None)
                  for k, c in enumerate(C)])
    kappa = (0.02, 0.03, 0.025, 0.035, 0.028)[:nf + 2]
    rho = (1.0, 0.7, 0.5, 0.8)[:nf + 1] if contrast else (1.0,) * (nf + 1)
    tau = (0.8, 1.0, 0.7, 0.9)[:nf + 1] if contrast else (1.0,) * (nf + 1)
    return shape, c1, C, kappa, rho, tau, None, body


@pytest.mark.parametrize("nf,shape,contrast", [(1, (64, 16, 11), True), (2, (64, 16, 11), True),
                                               (3, (64, 16, 11), True), (2, (32, 8, 1), False),
                                               (3, (32, 8, 3), True), (2, (32, 16, 2), False)])
def test_single_pass_fp64_parity(nf, shape, contrast):
    ml, m, f, g, kind = ml_run(_case(nf, shape, contrast), "f64", 12, tau_g=1.0)
    assert ml.single_pass
    errs = ml_compare(ml, m, f, g, kind, speed_scale=True)
    u = {k: errs.pop(k) for k in ("ux", "uy", "uz")}
    assert max(errs.values()) < 1e-12, errs
    # u is a cancelling sum of O(0.05) populations: its FP64 floor against the
    # speed scale (the two-fluid single-pass parity test's 5e-12)
    assert max(u.values()) < 5e-12, u


@pytest.mark.parametrize("nf", [2, 3])
def test_single_pass_fp32_parity(nf):
    ml, m, f, g, kind = ml_run(_case(nf), "f32", 40, tau_g=1.0)
    assert ml.single_pass
    e = ml_compare(ml, m, f, g, kind, speed_scale=True)
    assert e["f"] < 1e-5 and e["g"] < 1e-5, e
    assert max(e[f"C{k}"] for k in range(nf)) < 1e-5, e
    assert e["pt"] < 1e-5 and e["rho"] < 1e-5, e
    assert max(e[f"mu{k}"] for k in range(nf)) < 1e-4, e
    # the tolerance of the two-pass N-fluid FP32 parity test
    assert max(e["ux"], e["uy"], e["uz"]) < 5e-4, e
    assert e["tau"] < 1e-7, e


def _lattice(case, prec="f32", form="auto", zrun=0):
    shape, c1, C, kappa, rho, tau, faces, body = case
    real = torch.float64 if prec == "f64" else torch.float32
    p = P.make_params("D3Q19", shape, prec, theta_deg=90.0, tau_g=1.0, body=body, faces=faces,
                      alpha_s=1.0)
    ml = P.MultiLattice(p, C.shape[0] + 1, kappa, rho, tau)
    ml.set_step_form(form, zrun)
    ml.set_solid_c1(torch.as_tensor(c1, dtype=real, device=DEV))
    ml.set_fluids(torch.as_tensor(C, dtype=real, device=DEV))
    return ml


def _pops(ml):
    f, g = ml.populations()
    return f.double().cpu().numpy(), g.double().cpu().numpy()


@pytest.mark.parametrize("nf", [2, 3])
def test_single_pass_equals_two_pass(nf):
    case = _case(nf, (96, 16, 21))
    one = _lattice(case)
    two = _lattice(case, form="two_pass")
    assert one.single_pass and not two.single_pass
    one.step(30)
    two.step(30)
    f1, g1 = _pops(one)
    f2, g2 = _pops(two)
    # the same per-node arithmetic; a few FP32 ulp of the scale (the kernels
    # may contract different products into FMAs)
    assert rel_err(f1, f2) < 1e-6 and rel_err(g1, g2) < 1e-6, (rel_err(f1, f2), rel_err(g1, g2))
    for name, idx in (("C", 0), ("C", nf - 1), ("mu", 0), ("pt", 0)):
        a = one.field(name, idx).double().cpu().numpy()
        b = two.field(name, idx).double().cpu().numpy()
        assert rel_err(a, b) < 1e-5, (name, idx, rel_err(a, b))
    # u is a cancelling sum of O(0.1) populations: against the speed scale, at
    # the FP32 level the two-fluid single-pass parity test allows (2e-4)
    u1 = np.stack([one.field(k).double().cpu().numpy() for k in ("ux", "uy", "uz")])
    u2 = np.stack([two.field(k).double().cpu().numpy() for k in ("ux", "uy", "uz")])
    assert np.abs(u1 - u2).max() / np.abs(u2).max() < 2e-4


def test_zrun_does_not_change_the_result():
    case = _case(2, (64, 16, 23))
    ref = None
    for zrun in (0, 1, 4, 7, 23):
        ml = _lattice(case, zrun=zrun)
        ml.step(9)
        f, g = _pops(ml)
        if ref is None:
            ref = (f, g)
        else:
            assert np.array_equal(f, ref[0]) and np.array_equal(g, ref[1]), zrun


def test_reads_and_form_switches_keep_the_trajectory():
    case = _case(3, (32, 16, 10))
    plain = _lattice(case)
    plain.step(20)
    f_ref, g_ref = _pops(plain)

    runs = []
    for _ in range(2):
        ml = _lattice(case)
        ml.step(4)
        ml.field("mu", 1)                # canonical reads between one-pass steps
        ml.step(4)
        ml.populations()
        ml.step(4)
        ml.set_step_form("two_pass")
        ml.step(1)
        ml.set_step_form("auto")
        ml.step(7)
        runs.append(_pops(ml))
        assert ml.status() == 0
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    # one two-pass step in the mix: equal to the uninterrupted run up to FP32
    # contraction order
    assert rel_err(runs[0][0], f_ref) < 1e-6 and rel_err(runs[0][1], g_ref) < 1e-6


def test_a_new_solid_or_new_fluids_restart_from_the_canonical_state():
    case = _case(2, (32, 8, 6))
    a = _lattice(case)
    a.step(5)
    # new fluids after single-pass steps: the run restarts from them
    shape, c1, C, *_ = case
    a.set_fluids(torch.as_tensor(C, dtype=torch.float32, device=DEV))
    a.step(5)
    b = _lattice(case)
    b.step(5)
    fa, ga = _pops(a)
    fb, gb = _pops(b)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


@pytest.mark.parametrize("nf,shape", [(2, (45, 13, 7)), (3, (37, 11, 5)), (2, (33, 8, 1))])
def test_ragged_tiles_fp64_parity(nf, shape):
    # the last tiles ragged in x and y: same step as the oracle's
    ml, m, f, g, kind = ml_run(_case(nf, shape), "f64", 10, tau_g=1.0)
    assert ml.single_pass
    errs = ml_compare(ml, m, f, g, kind, speed_scale=True)
    u = {k: errs.pop(k) for k in ("ux", "uy", "uz")}
    assert max(errs.values()) < 1e-12, errs
    assert max(u.values()) < 5e-12, u


def test_ineligible_lattices_use_two_passes():
    for shape, kw in [((24, 16, 8), {}), ((32, 6, 8), {}), ((32, 16, 8), {"tau_g": 0.8}),
                      ((32, 16, 8), {"faces": ("mirror", "mirror", "periodic", "periodic",
                                               "periodic", "periodic")})]:
        shape_, c1, C, kappa, rho, tau, faces, body = _case(2, shape)
        p = P.make_params("D3Q19", shape, "f32", theta_deg=90.0, tau_g=kw.get("tau_g", 1.0),
                          faces=kw.get("faces"), alpha_s=1.0)
        ml = P.MultiLattice(p, 3, kappa, rho, tau)
        assert not ml.single_pass, (shape, kw)
    p = P.make_params("D2Q9", (64, 32), "f32", theta_deg=90.0, alpha_s=1.0)
    assert not P.MultiLattice(p, 3, (0.02, 0.03, 0.025, 0.035), (1, 1, 1), (1, 1, 1)).single_pass
