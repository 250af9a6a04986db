"""The body-force ramp on the GPU: dsm_set_body_force between steps, and a
reduced pressure ramp on a vented 32 x 32 x 64 pillar unit cell, against the
FP64 oracle taking the same force at every step (the body force on the liquid
of Sec. IV; the critical-pressure geometry of Sec. III)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

from dsm_helpers import compare, direction_map, gpu_fields, gpu_pops, oracle_params, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2504_19941_gb300 as P  # noqa: E402
from paper_2504_19941_gb300 import _lib  # noqa: E402
from paper_2504_19941_gb300.ramp import pillar_ring, pressure_ramp  # noqa: E402


def _cell(prec):
    case = S.pillar_slab_3d(32, 32, 64, seed=1, liquid=(38, 58), vent=10)
    p = P.make_params("D3Q19", case.shape, prec, theta_deg=case.theta_deg, g12=case.g12,
                      g23=case.g23, alpha_s=case.alpha_s)
    lat = P.Lattice(p)
    real = lat.real
    lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=real, device="cuda"))
    lat.set_fluid(torch.as_tensor(case.c2, dtype=real, device="cuda"))
    return case, lat


def test_ramp_matches_oracle_fp64():
    """A force changed before every step: the reduced ramp's state equals the
    oracle's, field by field and population by population, to 1e-12."""
    case, lat = _cell("f64")
    assert lat.single_pass
    nz, ny, nx = 64, 32, 32
    c1g = lat.field("C1").double().cpu().numpy().reshape(nz, ny, nx)
    steps, f_max = 240, 40 * case.extra["f_max"]   # a steep ramp, so that the state moves
    r = pressure_ramp(lat, f_max, steps, c1g, pillar_ring(c1g[20]), 38, 20.0,
                      check_every=80, stop_at_depinning=False)
    assert [h[0] for h in r["history"]] == [80, 160, 240]
    # the oracle with the same force at each step
    c1 = O.solid_profile(case.solid_sd, case.alpha_s)
    p0 = oracle_params(case, O.D3Q19)
    f, g = O.lb_init(p0, 2, c1, case.c2)
    for s in range(1, steps + 1):
        case.body = (0.0, 0.0, -f_max * s / steps)
        f, g = O.lb_run(oracle_params(case, O.D3Q19), 2, c1, f, g, 1)
    of = O.lb_fields(oracle_params(case, O.D3Q19), 2, c1, f, g)
    gfl = gpu_fields(lat)
    e = compare(gfl, of, ("C", "mu", "pt"))
    speed = max(np.max(np.abs(of[k])) for k in ("ux", "uy", "uz"))
    assert speed > 1e-6                            # the ramp drives a flow
    du = max(float(np.max(np.abs(gfl[k] - of[k]))) for k in ("ux", "uy", "uz"))
    assert max(e.values()) < 1e-12 and du < 5e-12 * speed, (e, du, speed)
    gf, gg = gpu_pops(lat, direction_map(O.D3Q19))
    assert rel_err(gf, f) < 1e-12 and rel_err(gg, g) < 1e-12


def test_body_force_changes_only_the_following_steps():
    case, a = _cell("f32")
    _, b = _cell("f32")
    a.step(5)
    b.step(5)
    a.set_body_force((0.0, 0.0, -1e-5))
    a.step(3)
    b.set_body_force((0.0, 0.0, -1e-5))
    b.step(3)
    fa, _ = a.populations()
    fb, _ = b.populations()
    assert torch.equal(fa, fb)
    with pytest.raises(P.DSMError) as e:
        a.set_body_force((0.0, float("nan"), 0.0))
    assert e.value.status == _lib.DSM_E_INVAL


def test_reduced_ramp_runs_and_reports():
    case, lat = _cell("f32")
    nz, ny, nx = 64, 32, 32
    c1 = lat.field("C1").double().cpu().numpy().reshape(nz, ny, nx)
    ring = pillar_ring(c1[20])
    r = pressure_ramp(lat, case.extra["f_max"] * 3.0, 2000, c1, ring, 38, 20.0, check_every=250)
    forces = [h[1] for h in r["history"]]
    assert forces == sorted(forces) and forces[-1] <= case.extra["f_max"] * 3.0 * (1 + 1e-12)
    heights = [h[2] for h in r["history"]]
    assert all(30.0 < h < 38.5 for h in heights), heights
    if r["f_crit"] is not None:
        assert heights[-1] < 36.0 and r["dp_crit"] == pytest.approx(r["f_crit"] * 20.0)
    assert lat.observables()["nonfinite"] == 0
