"""The observables ring (dsm_set_observables_ring) on the GPU.

dsm_step appends a record after each step that is a multiple of `every`,
on the device and without a host synchronisation.  Checked here, for the
one-pass step, the two-pass step and D2Q9:
  * the ring keeps the last `capacity` records, oldest first, with the step of
    each, across several dsm_step calls;
  * each record equals, bitwise, what dsm_get_observables returns at that step
    on a twin lattice read at the same steps (the same kernels);
  * recording leaves the trajectory as it is: the populations equal the twin's
    bitwise, and a lattice never read to FP32 rounding;
  * every=0 turns recording off.
"""
import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2504_19941_gb300 as P  # noqa: E402


def _lattice(lat, shape, prec):
    sd = S.pillars_sd(shape, 3, 4, 9, 5, offset=2)
    a_s = S.width_to_alpha(3.0)
    centre = [s / 2 for s in shape]
    centre[-1] = 6.0
    c2 = S.drop_c2(shape, centre, min(shape) / 3, 1.0, sd, a_s).ravel()
    c2 = c2 + S.perturbation(5, c2.size)
    p = P.make_params(lat, shape, prec, theta_deg=70.0, g12=0.01, g23=0.01, alpha_s=a_s,
                      body=(1e-6, -2e-6, -3e-6))
    L = P.Lattice(p)
    L.set_solid_distance(torch.as_tensor(sd.ravel(), dtype=L.real, device="cuda"))
    L.set_fluid(torch.as_tensor(c2, dtype=L.real, device="cuda"))
    return L


def _pops(L):
    f, g = L.populations()
    return f.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("lat,shape,prec,single", [("D3Q19", (64, 24, 19), "f32", True),
                                                    ("D3Q19", (20, 17, 13), "f32", False),
                                                    ("D2Q9", (33, 17), "f64", False)])
def test_ring_records_equal_observables(lat, shape, prec, single):
    rec = _lattice(lat, shape, prec)
    twin = _lattice(lat, shape, prec)
    plain = _lattice(lat, shape, prec)
    assert rec.single_pass == single
    rec.set_observables_ring(4, 10)
    rec.step(30)
    rec.step(25)
    ring = rec.observables_ring()
    assert [r["step"] for r in ring] == [20, 30, 40, 50]
    got = {r["step"]: r for r in ring}
    for k in range(1, 6):
        twin.step(10)
        o = twin.observables()
        if 10 * k in got:
            r = got[10 * k]
            for name in ("mass_c2", "mass_c1", "kinetic", "max_u"):
                assert r[name] == o[name], (10 * k, name, r[name], o[name])
            assert r["nonfinite"] == 0
    twin.step(5)
    plain.step(55)
    f_r, g_r = _pops(rec)
    f_t, g_t = _pops(twin)
    assert np.array_equal(f_r, f_t) and np.array_equal(g_r, g_t)
    f_p, g_p = _pops(plain)
    tol = 1e-6 if prec == "f32" else 1e-13
    assert np.abs(f_r - f_p).max() <= tol * np.abs(f_p).max()
    assert np.abs(g_r - g_p).max() <= tol * np.abs(g_p).max()
    assert rec.observables()["step"] == 55
    # off: no further records
    rec.set_observables_ring(4, 0)
    rec.step(20)
    assert rec.observables_ring() == []
