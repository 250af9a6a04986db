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
