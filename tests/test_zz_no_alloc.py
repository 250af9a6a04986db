"""The allocation-free free-energy entry point, dsm_fe_energy_grad_noalloc.

It serves callers that cannot allocate device memory (a host program with no
CUDA allocator of its own, or one whose device memory belongs to an allocator
that forbids side allocations): its reduction scratch is a fixed array inside
the library instead of a buffer the caller passes.  This test calls it through
the C ABI and checks it against dsm_fe_energy_grad (the entry point that takes
caller-owned scratch) within the energy tests' tolerance, on two calls in a
row with different fields, so the shared array cannot carry a stale result
from one call into the next.  The file sorts last so that a run stopping at
the first failure has run every other test first."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("lat,shape", [("D3Q19", (40, 36, 30)), ("D2Q9", (77, 51))])
def test_noalloc_matches_caller_scratch_entry_point(lat, shape):
    n = int(np.prod(shape))
    p = P.make_params(lat, shape, "f32", theta_deg=70.0, g23=0.9, g12=1.0, beta=5.0)
    mask = torch.as_tensor((np.arange(n) % 5 == 0).astype(np.uint8), device=DEV)
    sb = _lib.dsm_fe_scratch_bytes(p.lattice, p.nx, p.ny, p.nz)
    scratch = torch.empty(sb, dtype=torch.uint8, device=DEV)
    for call, (seed, active, kw) in enumerate([
            (1, 2, dict(dP=0.0, kcs=0.2, V0=0.3 * n, fg=0.01)),
            (2, 1, dict(dP=0.05, kcs=0.0, V0=0.0, fg=0.0))]):
        c1, c2 = _fields(n, seed)
        E_ref = torch.zeros(1, dtype=torch.float64, device=DEV)
        g_ref = torch.empty(n, dtype=torch.float32, device=DEV)
        t_ref = torch.zeros(6, dtype=torch.float64, device=DEV)
        _lib.dsm_fe_energy_grad(p, c1, c2, mask, active, kw["dP"], kw["kcs"], kw["V0"], kw["fg"],
                                E_ref, g_ref, t_ref, scratch, sb)
        E = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
        g = torch.full((n,), float("nan"), dtype=torch.float32, device=DEV)
        t = torch.full((6,), float("nan"), dtype=torch.float64, device=DEV)
        _lib.dsm_fe_energy_grad_noalloc(p, c1, c2, mask, active, kw["dP"], kw["kcs"], kw["V0"],
                                        kw["fg"], E, g, t)
        torch.cuda.synchronize()
        assert abs(E.item() - E_ref.item()) <= 1e-6 * abs(E_ref.item()), call
        gmax = g_ref.abs().max().item()
        assert (g - g_ref).abs().max().item() <= 1e-5 * gmax, call
        torch.testing.assert_close(t, t_ref, rtol=1e-6, atol=1e-9)


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
