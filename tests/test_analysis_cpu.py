"""Contact-angle measurement on fields with a known answer.

The oracle's circle fit (oracle/analysis.py: Kasa's algebraic least squares
and the angle against the wall plane, the measurement of Sec. III.A) and the
library's own apparent-angle fit (paper_2504_19941_gb300/analysis.py, used for
served results) are checked on exact circular / spherical caps, whose
C2 = 1/2 level is the circle itself, and on caps damped into a diffuse wall
as the initial conditions of the method are."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import analysis as A
from paper_2504_19941_gb300 import analysis as B


def _wall(shape, top=8):
    sd = S.slab_sd(shape, len(shape) - 1, 0, top)
    a_s = S.width_to_alpha(3.0)
    return sd, a_s, 0.5 * (1 + np.tanh(sd / (2 * a_s)))


@pytest.mark.parametrize("d", [2, 3])
def test_kasa_fit_recovers_an_exact_circle(d):
    rng = np.random.default_rng(4)
    centre = rng.uniform(-5, 5, d)
    R = 7.3
    v = rng.normal(size=(200, d))
    pts = centre + R * v / np.linalg.norm(v, axis=1)[:, None]
    c, r = A.kasa_fit(pts)
    assert np.allclose(c, centre, atol=1e-10) and abs(r - R) < 1e-10
    c, r = B.sphere_fit(pts)
    assert np.allclose(c, centre, atol=1e-10) and abs(r - R) < 1e-10


@pytest.mark.parametrize("d,R", [(2, 40.0), (3, 24.0)])
@pytest.mark.parametrize("theta", [60.0, 90.0, 120.0, 150.0])
def test_contact_angle_of_an_exact_cap(d, R, theta):
    """A cap whose C2 = 1/2 level is exactly a circle (sphere) meeting the wall
    plane (C1 = 1/2) at theta: the oracle's fit returns theta to 0.01 degrees,
    the library's to 0.1 (it fits the liquid fraction C2/(1 - C1))."""
    shape = (160, 100) if d == 2 else (96, 96, 70)
    _, _, c1 = _wall(shape)
    c2 = S.cap_c2(shape, 7.5, R, theta, 1.0)
    assert abs(A.contact_angle_flat(c2, c1) - theta) < 0.01
    assert abs(B.apparent_contact_angle(c2, c1) - theta) < 0.1


def test_contact_angle_of_a_flat_cap():
    # a thin cap (30 degrees) needs a large drop: enough of it lies above the
    # 3-node margin
    shape = (400, 80)
    _, _, c1 = _wall(shape)
    c2 = S.cap_c2(shape, 7.5, 120.0, 30.0, 1.0)
    assert abs(A.contact_angle_flat(c2, c1) - 30.0) < 0.02
    assert abs(B.apparent_contact_angle(c2, c1) - 30.0) < 0.1


@pytest.mark.parametrize("theta", [60.0, 120.0, 150.0])
def test_damped_caps_and_the_two_fits_agree(theta):
    # the initial condition of a sessile drop: the cap damped into the diffuse
    # wall; both fits stay within 0.1 degrees of theta and of each other
    shape = (96, 96, 70)
    sd, a_s, c1 = _wall(shape)
    c2 = S.cap_c2(shape, 7.5, 24.0, theta, 1.0, sd, a_s)
    a, b = A.contact_angle_flat(c2, c1), B.apparent_contact_angle(c2, c1)
    assert abs(a - theta) < 0.1 and abs(b - theta) < 0.1 and abs(a - b) < 0.1


def test_apparent_angle_is_read_against_the_top_of_the_roughness():
    # a cap resting on pillar tops: the reference plane is the pillars' top
    shape = (128, 128, 80)
    sd = S.pillars_sd(shape, 6, 8, 16, 20, offset=4)
    a_s = S.width_to_alpha(3.0)
    c1 = 0.5 * (1 + np.tanh(sd / (2 * a_s)))
    top = B.roughness_top(c1)
    assert abs(top - 25.5) < 0.01          # pillars fill z < 26
    c2 = S.cap_c2(shape, top, 30.0, 120.0, 1.0)
    assert abs(B.apparent_contact_angle(c2, c1) - 120.0) < 0.1
    # no solid, or no interface above the margin: not a number
    assert math.isnan(B.apparent_contact_angle(c2, np.zeros_like(c1)))
    assert math.isnan(B.apparent_contact_angle(np.zeros_like(c2), c1))
