"""The one-pass stage-2 step (dsm_set_step_form, DSM_STEP_AUTO): D3Q19 lattices
whose planes tile into 32 x 8 blocks, g held as g_eq (tau_g = 1), periodic.

Each step rebuilds C = sum_i g_eq_i(x - c_i) on chip from the TMA-staged
(A, u, C) of the previous collision and collides in the same pass, so it is the
same step as the moments pass + fused pass (Sec. II.B, C = sum_i g_i feeding mu
of the same step).  Checked here:
  * against the FP64 oracle (1e-12 per field and population, FP64; the FP32
    tolerances of the two-pass parity tests in FP32), with and without a
    density contrast, on the smallest tiles (32 x 8, nz = 1 .. 3) and on
    lattices of several tiles with a ragged z run;
  * against the two-pass step on the same lattice: FP32 and both 16-bit
    storage forms to a few FP32 ulp of the field's scale (the per-node
    arithmetic is shared);
  * that the result does not depend on the z planes per block;
  * that every call reading the state in its canonical layout (fields,
    observables, populations, checkpoint) and switching forms mid-run leave the
    trajectory unchanged.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

from dsm_helpers import (compare, direction_map, gpu_fields, gpu_lattice, gpu_pops,
                         oracle_params, rel_err)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2504_19941_gb300 as P  # noqa: E402


def _case(shape=(64, 24, 19), theta=115.0, g=0.01, body=(2e-6, -1e-6, -5e-6)):
    nx, ny, nz = shape
    sd = S.pillars_sd(shape, min(4, nz - 1), 6, 16, 8, offset=3)
    a_s = S.width_to_alpha(3.0)
    zl = max(1, nz // 3)
    c2 = S.layer_c2(shape, 2, zl, min(zl + 6, nz), 1.0, sd, a_s) + \
        S.drop_c2(shape, (nx / 2, ny / 2, min(8.0, nz / 2)), min(5.0, nz / 3), 1.0, sd, a_s) * 0.5
    c2 = c2.ravel() + S.perturbation(7, nx * ny * nz)
    return S.Case("zstep", "D3Q19", shape, sd.ravel(), c2, theta_deg=theta, g23=g, g12=g,
                  alpha_s=a_s, body=body)


def _oracle_run(case, steps):
    p = oracle_params(case, O.D3Q19)
    c1 = O.solid_profile(case.solid_sd, case.alpha_s)
    f, g = O.lb_init(p, 2, c1, case.c2)
    f, g = O.lb_run(p, 2, c1, f, g, steps)
    return p, c1, f, g


@pytest.mark.parametrize("shape,contrast", [((64, 24, 19), False), ((64, 24, 19), True),
                                            ((32, 8, 3), False), ((32, 8, 1), False),
                                            ((32, 16, 2), True)])
def test_single_pass_fp64_parity(shape, contrast):
    case = _case(shape)
    if contrast:
        case.rho2, case.rho3, case.tau2, case.tau3 = 1.0, 0.5, 1.0, 0.7
    lat = gpu_lattice(case, "f64")
    assert lat.single_pass
    steps = 12
    lat.step(steps)
    p, c1, f, g = _oracle_run(case, steps)
    gfl, ofl = gpu_fields(lat), O.lb_fields(p, 2, c1, f, g)
    errs = compare(gfl, ofl, ("C", "mu", "pt", "rho"))
    gf, gg = gpu_pops(lat, direction_map(O.D3Q19))
    errs["f"], errs["g"] = rel_err(gf, f), rel_err(gg, g)
    # velocity components against the speed scale: on the thin lattices one
    # component's own maximum is many orders below the others' (nz = 1: u_z
    # only answers the body force), which a per-component ratio would amplify
    speed = max(np.max(np.abs(ofl[k])) for k in ("ux", "uy", "uz"))
    uerr = max(float(np.max(np.abs(gfl[k] - ofl[k]))) / speed for k in ("ux", "uy", "uz"))
    assert max(errs.values()) < 1e-12, errs
    # u is a cancelling sum of O(0.05) populations: its FP64 floor (the same
    # 5e-12 the two-pass parity tests allow the velocity)
    assert uerr < 5e-12, uerr


def test_single_pass_fp32_parity():
    case = _case()
    lat = gpu_lattice(case, "f32")
    assert lat.single_pass
    lat.step(50)
    p, c1, f, g = _oracle_run(case, 50)
    e = compare(gpu_fields(lat), O.lb_fields(p, 2, c1, f, g))
    gf, gg = gpu_pops(lat, direction_map(O.D3Q19))
    assert e["C"] < 1e-5 and e["pt"] < 1e-5 and e["mu"] < 1e-4, e
    assert max(e["ux"], e["uy"], e["uz"]) < 2e-4, e
    assert rel_err(gf, f) < 1e-5 and rel_err(gg, g) < 1e-5


def _pops(lat):
    f, g = lat.populations()
    return f.double().cpu().numpy(), g.double().cpu().numpy()


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
def test_single_pass_equals_two_pass(prec):
    case = _case((96, 16, 21))
    one = gpu_lattice(case, prec)
    two = gpu_lattice(case, prec)
    two.set_step_form("two_pass")
    assert one.single_pass and not two.single_pass
    one.step(30)
    two.step(30)
    f1, g1 = _pops(one)
    f2, g2 = _pops(two)
    # the same per-node arithmetic; allow a few FP32 ulp of the scale (the two
    # kernels may contract different products into FMAs)
    assert rel_err(f1, f2) < 1e-6 and rel_err(g1, g2) < 1e-6, (rel_err(f1, f2), rel_err(g1, g2))
    for name in ("C2", "ux", "pt"):
        a = one.field(name).double().cpu().numpy()
        b = two.field(name).double().cpu().numpy()
        assert rel_err(a, b) < 1e-5, name


def test_zrun_does_not_change_the_result():
    case = _case((64, 16, 23))
    ref = None
    for zrun in (0, 1, 4, 7, 23):
        lat = gpu_lattice(case, "f32")
        lat.set_step_form("auto", zrun)
        lat.step(9)
        f, g = _pops(lat)
        if ref is None:
            ref = (f, g)
        else:
            assert np.array_equal(f, ref[0]) and np.array_equal(g, ref[1]), zrun


def test_reads_and_form_switches_keep_the_trajectory():
    case = _case((32, 16, 10))
    plain = gpu_lattice(case, "f32")
    plain.step(24)
    f_ref, g_ref = _pops(plain)

    lat = gpu_lattice(case, "f32")
    lat.step(4)
    lat.observables()                    # canonical read between one-pass steps
    lat.step(4)
    lat.field("mu")
    lat.step(4)
    lat.populations()
    lat.step(4)
    state = lat.state()              # checkpoint, restored into a fresh lattice
    other = gpu_lattice(case, "f32")
    other.set_state(state)
    for x in (lat, other):
        x.step(4)
        x.set_step_form("two_pass")
        x.step(1)
        x.set_step_form("auto")
        x.step(3)
    f1, g1 = _pops(lat)
    f2, g2 = _pops(other)
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    # one two-pass step in the mix: equal to the uninterrupted run up to FP32
    # contraction order
    assert rel_err(f1, f_ref) < 1e-6 and rel_err(g1, g_ref) < 1e-6
    assert lat.observables()["step"] == 24


@pytest.mark.parametrize("shape", [(45, 13, 7), (40, 16, 8), (70, 9, 4), (33, 8, 1)])
def test_ragged_tiles_fp64_parity(shape):
    # nx not a multiple of 32 or ny not of 8: the last tiles are ragged (their
    # threads beyond the lattice rebuild C and keep the barriers but run no pass)
    case = _case(shape)
    case.rho2, case.rho3, case.tau2, case.tau3 = 1.0, 0.5, 1.0, 0.7
    lat = gpu_lattice(case, "f64")
    assert lat.single_pass
    lat.step(10)
    p, c1, f, g = _oracle_run(case, 10)
    gfl, ofl = gpu_fields(lat), O.lb_fields(p, 2, c1, f, g)
    errs = compare(gfl, ofl, ("C", "mu", "pt", "rho"))
    gf, gg = gpu_pops(lat, direction_map(O.D3Q19))
    errs["f"], errs["g"] = rel_err(gf, f), rel_err(gg, g)
    speed = max(np.max(np.abs(ofl[k])) for k in ("ux", "uy", "uz"))
    uerr = max(float(np.max(np.abs(gfl[k] - ofl[k]))) / speed for k in ("ux", "uy", "uz"))
    assert max(errs.values()) < 1e-12, errs
    assert uerr < 5e-12, uerr


def test_ragged_tiles_equal_two_passes_and_any_zrun():
    case = _case((75, 21, 13))
    two = gpu_lattice(case, "f32")
    two.set_step_form("two_pass")
    two.step(20)
    f2, g2 = _pops(two)
    ref = None
    for zrun in (0, 1, 5, 13):
        one = gpu_lattice(case, "f32")
        one.set_step_form("auto", zrun)
        assert one.single_pass
        one.step(20)
        f1, g1 = _pops(one)
        assert rel_err(f1, f2) < 1e-6 and rel_err(g1, g2) < 1e-6, zrun
        if ref is None:
            ref = (f1, g1)
        else:
            assert np.array_equal(f1, ref[0]) and np.array_equal(g1, ref[1]), zrun


def test_ineligible_lattices_use_two_passes():
    for shape, kw in [((24, 16, 8), {}), ((32, 6, 8), {}), ((32, 16, 8), {"tau_g": 0.8})]:
        case = _case(shape)
        for k, v in kw.items():
            setattr(case, k, v)
        lat = gpu_lattice(case, "f32")
        assert not lat.single_pass, shape
    case = _case((32, 16, 8))
    lat = gpu_lattice(case, "f32", g_storage="populations")
    assert not lat.single_pass
