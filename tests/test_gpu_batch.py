"""The batched persistent step (dsm_batch_step) and the serving loop on the GPU.

Mix invariance: every lattice advanced inside a batch -- whatever the other
lattices, their sizes and step counts -- ends in exactly the state its solo
dsm_step run reaches (bitwise: the same per-node arithmetic)."""
import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2504_19941_gb300 as P  # noqa: E402
from paper_2504_19941_gb300 import _lib  # noqa: E402
from paper_2504_19941_gb300.serving import GpuExecutor, Scheduler, serial_run, summarize  # noqa

DEV = "cuda"


def _lattice(shape, seed, prec="f32", form="auto"):
    rng = np.random.default_rng(seed)
    d = len(shape)
    sd = S.pillars_sd(shape, 3, int(rng.integers(3, 6)), int(rng.integers(8, 14)), 5, offset=2)
    a_s = S.width_to_alpha(3.0)
    centre = [s / 2 for s in shape]
    centre[-1] = 6.0
    c2 = S.drop_c2(shape, centre, min(shape) / 4, 1.0, sd, a_s).ravel()
    p = P.make_params("D2Q9" if d == 2 else "D3Q19", shape, prec,
                      theta_deg=float(rng.uniform(40, 140)), g12=0.01, g23=0.01, alpha_s=a_s,
                      body=(1e-6, -2e-6, 0.0))
    lat = P.Lattice(p)
    lat.set_g_storage(form)
    lat.set_solid_distance(torch.as_tensor(sd.ravel(), dtype=lat.real, device=DEV))
    lat.set_fluid(torch.as_tensor(c2, dtype=lat.real, device=DEV))
    return lat


SETS = {
    "2d": [(64, 64), (80, 48), (33, 17), (128, 96), (7, 5)],
    "3d": [(32, 32, 24), (20, 17, 13), (40, 24, 16)],
}


@pytest.mark.parametrize("kind,prec,form", [("2d", "f32", "auto"), ("3d", "f32", "auto"),
                                            ("2d", "bf16", "auto"), ("3d", "bf16", "auto"),
                                            ("3d", "f32", "populations"),
                                            ("2d", "bf16", "populations")])
def test_batch_equals_solo_bitwise(kind, prec, form):
    shapes = SETS[kind]
    nsteps = [30, 17, 0, 45, 8][:len(shapes)]
    batch = [_lattice(s, i, prec, form) for i, s in enumerate(shapes)]
    solo = [_lattice(s, i, prec, form) for i, s in enumerate(shapes)]
    hs = [lat.h for lat in batch]
    nb = _lib.dsm_batch_scratch_bytes(hs)
    scratch = torch.empty(nb, dtype=torch.uint8, device=DEV)
    # two calls (quanta) per lattice budget: first the first half, then the rest
    first = [k // 2 for k in nsteps]
    _lib.dsm_batch_step(hs, first, scratch, nb)
    _lib.dsm_batch_step(hs, [k - f for k, f in zip(nsteps, first)], scratch, nb)
    for lat, k in zip(solo, nsteps):
        lat.step(k)
    for a, b, k in zip(batch, solo, nsteps):
        fa, ga = a.populations()
        fb, gb = b.populations()
        assert torch.equal(fa, fb) and torch.equal(ga, gb), (a.shape, k)
        oa, ob = a.observables(), b.observables()
        assert oa["step"] == ob["step"] == k
        assert oa["mass_c2"] == ob["mass_c2"]


def test_batch_argument_checks():
    a = _lattice((16, 16), 0, "f32")
    b = _lattice((16, 16), 1, "bf16")
    with pytest.raises(P.DSMError) as e:
        _lib.dsm_batch_scratch_bytes([a.h, b.h])
    assert e.value.status == _lib.DSM_E_INVAL
    s = torch.cuda.Stream()
    p = P.make_params("D2Q9", (16, 16), "f32", theta_deg=90)
    c = P.Lattice(p, stream=s)
    c.set_solid_distance(torch.full((256,), -5.0, device=DEV))
    c.set_fluid(torch.zeros(256, device=DEV))
    torch.cuda.synchronize()
    with pytest.raises(P.DSMError) as e:
        _lib.dsm_batch_scratch_bytes([a.h, c.h])  # different streams
    assert e.value.status == _lib.DSM_E_INVAL
    d = _lattice((16, 16), 2, "f32", form="populations")
    with pytest.raises(P.DSMError) as e:
        _lib.dsm_batch_scratch_bytes([a.h, d.h])  # g held as g_eq in one only
    assert e.value.status == _lib.DSM_E_INVAL
    nb = _lib.dsm_batch_scratch_bytes([a.h])
    scratch = torch.empty(nb, dtype=torch.uint8, device=DEV)
    with pytest.raises(P.DSMError) as e:
        _lib.dsm_batch_step([a.h], [1], scratch, nb - 1)
    assert e.value.status == _lib.DSM_E_WORKSPACE


def test_serving_results_equal_solo_runs():
    reqs = S.serving_stream(n_req=10, rate=200.0, seed=3, min_side=24, max_side_2d=160, max_side_3d=48,
                            steps=(40, 200))
    ex = GpuExecutor("f32", small_nodes=20_000)
    recs = Scheduler(ex, budget_bytes=8 << 30, quantum=32).run(reqs)
    assert all(r.status == "done" for r in recs), [r.result for r in recs]
    solo = serial_run(GpuExecutor("f32", small_nodes=20_000), reqs)
    for a, b in zip(recs, solo):
        assert a.result == b.result, (a.rid, a.result, b.result)
    s = summarize(recs, max(r.finished for r in recs))
    assert s["solves"] == 10 and s["p99_s"] >= s["p50_s"] > 0
