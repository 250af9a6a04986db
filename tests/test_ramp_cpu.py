"""Host-side parts of the pressure ramp (paper_2504_19941_gb300/ramp.py): the
contact-line detector on fields with a known answer, the ring of gap columns
next to the pillars, and the vented base plate of the ramp geometry."""
import numpy as np

import synthetic as S
from paper_2504_19941_gb300.ramp import interface_height, pillar_ring


def _slab(nz, ny, nx, lo, hi, alpha=1.0):
    z = np.arange(nz)[:, None, None]
    c = 0.25 * (1 + np.tanh((z - lo + 0.5) / (2 * alpha))) * (1 + np.tanh((hi - 0.5 - z) / (2 * alpha)))
    return np.broadcast_to(c, (nz, ny, nx)).copy()


def test_interface_height_of_a_flat_slab():
    # the C2 = 1/2 level of the slab's lower interface lies half a node below
    # its first liquid node (the tanh is centred there)
    c2 = _slab(48, 6, 7, 20, 40)
    cols = np.ones((6, 7), bool)
    h = interface_height(c2, np.zeros_like(c2), cols, z_start=30)
    assert abs(h - 19.5) < 0.02, h


def test_interface_height_uses_the_liquid_fraction_and_the_floor():
    c2 = _slab(40, 4, 4, 12, 30)
    c1 = np.zeros_like(c2)
    c1[:, 0, 0] = 0.4            # a diffuse solid column: C2 = 0.6 x fraction
    c2[:, 0, 0] *= 0.6
    cols = np.zeros((4, 4), bool)
    cols[0, 0] = True
    assert abs(interface_height(c2, c1, cols, z_start=20) - 11.5) < 0.02
    # a column liquid all the way down counts the floor
    c2b = np.ones_like(c2)
    assert interface_height(c2b, np.zeros_like(c2b), cols, z_start=20, z_floor=3) == 3


def test_a_sagging_column_lowers_the_mean():
    c2 = _slab(48, 2, 2, 20, 40)
    c2[:, 0, 0] = _slab(48, 1, 1, 16, 40)[:, 0, 0]
    h = interface_height(c2, np.zeros_like(c2), np.ones((2, 2), bool), z_start=30)
    assert abs(h - (3 * 19.5 + 15.5) / 4) < 0.02


def test_pillar_ring_surrounds_each_pillar():
    c1 = np.zeros((32, 32))
    c1[11:21, 11:21] = 1.0
    ring = pillar_ring(c1)
    assert ring.sum() == 12 * 12 - 10 * 10
    assert not ring[11:21, 11:21].any() and ring[10, 10] and ring[21, 21] and not ring[9, 15]


def test_vented_plate_has_one_hole_per_gap_cell():
    case = S.pillar_slab_3d(64, 64, 96, seed=0, liquid=(38, 90), vent=10)
    solid = case.solid_sd.reshape(96, 64, 64) > 0
    plate = solid[3]
    assert (~plate).sum() == 4 * 100        # four cells, a 10 x 10 hole each
    # the holes sit in the gaps: never under a pillar
    assert not (~plate & solid[20]).any()
    closed = S.pillar_slab_3d(64, 64, 96, seed=0, liquid=(38, 90))
    assert (closed.solid_sd.reshape(96, 64, 64)[3] > 0).all()
