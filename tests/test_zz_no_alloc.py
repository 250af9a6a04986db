"""The allocation-free free-energy entry point, dsm_fe_energy_grad_noalloc.

It serves callers that cannot allocate device memory (a host program with no
CUDA allocator of its own, or one whose device memory belongs to an allocator
that forbids side allocations): its reduction scratch is a fixed array inside
the library instead of a buffer the caller passes.  This test calls it through
the C ABI and checks it against dsm_fe_energy_grad (the entry point that takes
caller-owned scratch): both run the same kernels on the same fixed grid with
the same reduction order, so energy, gradient and the energy terms must be
bitwise equal.  Three calls in a row -- two on a larger lattice with different
fields and constraints, then one on a smaller lattice with fewer blocks -- show
that the shared array carries nothing from one call into the next.  The
results are also compared with the FP64 oracle (Sec. II.A, the free energy and
its gradient), within the energy tests' tolerances.  The file sorts last so
that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2504_19941_gb300 as P  # noqa: E402
from paper_2504_19941_gb300 import _lib  # noqa: E402

DEV = "cuda"
NOALLOC_BYTES = 1 << 16  # DSM_NOALLOC_SCRATCH_BYTES in include/dsm.h


def _fields(n, seed):
    c1, c2 = S.random_fields(n, seed=seed)
    return (torch.as_tensor(0.6 * c1, dtype=torch.float32, device=DEV),
            torch.as_tensor(c2, dtype=torch.float32, device=DEV))


def _call(fn, p, n, c1, c2, mask, active, kw, *scratch):
    E = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
    g = torch.full((n,), float("nan"), dtype=torch.float32, device=DEV)
    t = torch.full((6,), float("nan"), dtype=torch.float64, device=DEV)
    fn(p, c1, c2, mask, active, kw["dP"], kw["kcs"], kw["V0"], kw["fg"], E, g, t, *scratch)
    return E, g, t


@pytest.mark.parametrize("lat,big,small", [("D3Q19", (40, 36, 30), (9, 7, 5)),
                                           ("D2Q9", (77, 51), (13, 6))])
def test_noalloc_matches_caller_scratch_entry_point(lat, big, small):
    theta, g23, g12, beta = 70.0, 0.9, 1.0, 5.0
    calls = [(big, 1, 2, dict(dP=0.0, kcs=0.2, V0=None, fg=0.01)),
             (big, 2, 1, dict(dP=0.05, kcs=0.0, V0=0.0, fg=0.0)),
             (small, 3, 2, dict(dP=0.0, kcs=0.5, V0=None, fg=0.02))]
    for call, (shape, seed, active, kw) in enumerate(calls):
        n = int(np.prod(shape))
        if kw["V0"] is None:
            kw = dict(kw, V0=0.3 * n)
        p = P.make_params(lat, shape, "f32", theta_deg=theta, g23=g23, g12=g12, beta=beta)
        mask = torch.as_tensor((np.arange(n) % 5 == 0).astype(np.uint8), device=DEV)
        sb = _lib.dsm_fe_scratch_bytes(p.lattice, p.nx, p.ny, p.nz)
        scratch = torch.empty(sb, dtype=torch.uint8, device=DEV)
        c1, c2 = _fields(n, seed)
        E_ref, g_ref, t_ref = _call(_lib.dsm_fe_energy_grad, p, n, c1, c2, mask, active, kw,
                                    scratch, sb)
        E, g, t = _call(_lib.dsm_fe_energy_grad_noalloc, p, n, c1, c2, mask, active, kw)
        torch.cuda.synchronize()
        assert torch.equal(E, E_ref), call
        assert torch.equal(g, g_ref), call
        assert torch.equal(t, t_ref), call
        # the same energy and gradient as the FP64 oracle
        po = O.make_params(O.D3Q19 if lat == "D3Q19" else O.D2Q9, shape, _lib.dsm_kappa(p),
                           beta=beta)
        E_or, g_or, _ = O.energy_grad(po, c1.double().cpu().numpy(), c2.double().cpu().numpy(),
                                      active=active, S=mask.cpu().numpy(), **kw)
        assert abs(E.item() - E_or) <= 1e-6 * abs(E_or), (call, E.item(), E_or)
        gd = g.double().cpu().numpy()
        assert np.max(np.abs(gd - g_or)) <= 1e-5 * np.max(np.abs(g_or)), call


def test_noalloc_array_holds_every_accepted_lattice():
    # the energy kernel leaves at most one partial sum per resident block, so
    # the scratch it needs does not grow with the lattice: the largest lattice
    # the library accepts fits the fixed array
    need = _lib.dsm_fe_scratch_bytes(1, 1290, 1290, 1290)  # ~2^31 - 1 nodes
    assert need <= NOALLOC_BYTES
    # an invalid lattice is refused on the host, before any device work
    # (the pointers are never touched)
    p = P.make_params("D3Q19", (2048, 2048, 1024), "f32", theta_deg=90.0)
    with pytest.raises(P.DSMError) as e:
        _lib.dsm_fe_energy_grad_noalloc(p, 16, 16, None, 2, 0.0, 0.0, 0.0, 0.0, 16, 16, None)
    assert e.value.status == _lib.DSM_E_INVAL
