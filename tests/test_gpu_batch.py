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
    import math
    thetas = []
    for a, b in zip(recs, solo):
        # each served lattice ends in its solo state bitwise: the observables
        # and the apparent contact angle fitted to its final fields are equal
        ta, tb = a.result.pop("theta_deg"), b.result.pop("theta_deg")
        assert a.result == b.result, (a.rid, a.result, b.result)
        assert ta == tb or (math.isnan(ta) and math.isnan(tb)), (a.rid, ta, tb)
        thetas.append(ta)
    assert sum(math.isfinite(t) and 0.0 < t < 180.0 for t in thetas) >= 5, thetas
    s = summarize(recs, max(r.finished for r in recs))
    assert s["solves"] == 10 and s["p99_s"] >= s["p50_s"] > 0


# ------------------------------------------------- batched lattices vs oracle
def _case(shape, seed):
    """A small wetting case (pillars, a drop, a body force) as the oracle and
    the library both take it."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    sd = S.pillars_sd(shape, 3, int(rng.integers(3, 6)), int(rng.integers(8, 14)), 5, offset=2)
    a_s = S.width_to_alpha(3.0)
    centre = [s / 2 for s in shape]
    centre[-1] = 6.0
    c2 = S.drop_c2(shape, centre, min(shape) / 4, 1.0, sd, a_s).ravel() + \
        S.perturbation(seed, int(np.prod(shape)))
    return S.Case("batch", "D2Q9" if d == 2 else "D3Q19", shape, sd.ravel(), c2,
                  theta_deg=float(rng.uniform(40, 140)), g23=0.01, g12=0.01, alpha_s=a_s,
                  body=(1e-6, -2e-6, 0.0) if d == 2 else (1e-6, -2e-6, 3e-6))


BATCH_ORACLE_SETS = {"2d": ([(64, 48), (33, 17), (7, 5)], [25, 12, 30]),
                     "3d": ([(20, 17, 13), (32, 16, 8)], [15, 9])}


@pytest.mark.parametrize("kind", ["2d", "3d"])
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16", "f16"])
def test_batch_matches_oracle(kind, prec):
    """Lattices advanced together by dsm_batch_step (one persistent launch,
    its own brick shapes and phase order) against the FP64 oracle, element by
    element: FP64 to 1e-12 on every field and population (velocities 5e-12 of
    the speed scale, their FP64 floor); FP32 to the tolerances of the
    single-lattice parity tests; 16-bit storage: one batched step from a
    stored state stays within the encoding's rounding of the oracle's step."""
    from dsm_helpers import compare, direction_map, gpu_fields, gpu_lattice, gpu_pops, \
        oracle_params, rel_err
    import oracle as O
    shapes, steps = BATCH_ORACLE_SETS[kind]
    cases = [_case(s, i) for i, s in enumerate(shapes)]
    lats = [gpu_lattice(c, prec) for c in cases]
    hs = [lat.h for lat in lats]
    nb = _lib.dsm_batch_scratch_bytes(hs)
    scratch = torch.empty(nb, dtype=torch.uint8, device=DEV)
    ok = O.D2Q9 if kind == "2d" else O.D3Q19
    perm = direction_map(ok)
    inv = np.empty(len(perm), dtype=int)
    inv[perm] = np.arange(len(perm))
    if prec in ("f64", "f32"):
        _lib.dsm_batch_step(hs, steps, scratch, nb)
        for lat, case, k in zip(lats, cases, steps):
            p = oracle_params(case, ok)
            c1 = O.solid_profile(case.solid_sd, case.alpha_s)
            f, g = O.lb_init(p, 2, c1, case.c2)
            f, g = O.lb_run(p, 2, c1, f, g, k)
            of = O.lb_fields(p, 2, c1, f, g)
            gfl = gpu_fields(lat)
            e = compare(gfl, of, ("C", "mu", "pt"))
            gf, gg = gpu_pops(lat, perm)
            speed = max(np.max(np.abs(of[n])) for n in ("ux", "uy", "uz"))
            du = max(float(np.max(np.abs(gfl[n] - of[n]))) for n in ("ux", "uy", "uz"))
            if prec == "f64":
                assert max(e.values()) < 1e-12 and du < 5e-12 * speed, (case.shape, e, du)
                assert rel_err(gf, f) < 1e-12 and rel_err(gg, g) < 1e-12, case.shape
            else:
                assert e["C"] < 1e-5 and e["pt"] < 1e-5 and e["mu"] < 1e-4, (case.shape, e)
                # u is a cancelling sum of O(0.1) populations: besides 2e-4 of
                # the speed, an absolute FP32 rounding floor of a few 2^-24 per
                # term (the 7 x 5 lattice moves at a few 1e-4)
                assert du < 2e-4 * speed + 5e-7, (case.shape, du, speed)
                assert rel_err(gf, f) < 1e-5 and rel_err(gg, g) < 1e-5, case.shape
        return
    # 16-bit storage: from the stored state after some batched steps, one
    # batched step against the oracle's step of the same (decoded) state
    _lib.dsm_batch_step(hs, steps, scratch, nb)
    before = []
    for lat in lats:
        f, g = lat.populations()
        q = lat.q
        before.append((f.double().cpu().numpy().reshape(q, -1)[inv],
                       g.double().cpu().numpy().reshape(q, -1)[inv]))
    _lib.dsm_batch_step(hs, [1] * len(lats), scratch, nb)
    bits = 8 if prec == "bf16" else 11
    _, w = O.lattice(ok)
    for lat, case, (f0, g0) in zip(lats, cases, before):
        p = oracle_params(case, ok)
        c1 = lat.field("C1").double().cpu().numpy()
        f1, g1 = O.lb_run(p, 2, c1, f0, g0, 1)
        gf, gg = gpu_pops(lat, perm)
        u = 2.0 ** -bits
        bound_f = u * np.abs(f1 - w[:, None]) + 1e-6
        assert np.all(np.abs(gf - f1) <= bound_f), (case.shape, np.max(np.abs(gf - f1) - bound_f))
        bound_g = u * np.abs(g1[1:]) + 1e-7
        assert np.all(np.abs(gg[1:] - g1[1:]) <= bound_g), case.shape
        np.testing.assert_allclose(gg.sum(axis=0), g1.sum(axis=0), rtol=0, atol=5e-7)


def test_bounded_barrier_wait_times_out_and_the_handle_recovers():
    """A grid barrier of the persistent batched launch that gives up after a
    few polls (dsm_set_wait_limit): early blocks stop waiting, latch
    DSM_E_TIMEOUT and return, so the launch ends; the next synchronising call
    reports DSM_E_TIMEOUT, the handles refuse to step until a state is set
    again, and a restored checkpoint steps on as before."""
    lats = [_lattice(s, i) for i, s in enumerate([(64, 64), (80, 48), (128, 96)])]
    ref = _lattice((64, 64), 0)
    saved = lats[0].state()
    hs = [lat.h for lat in lats]
    nb = _lib.dsm_batch_scratch_bytes(hs)
    scratch = torch.empty(nb, dtype=torch.uint8, device=DEV)
    try:
        _lib.dsm_set_wait_limit(2)
        _lib.dsm_batch_step(hs, [40, 40, 40], scratch, nb)
        torch.cuda.synchronize()  # the launch ended: every wait is bounded
    finally:
        _lib.dsm_set_wait_limit(0)
    o = _lib.dsm_get_observables(lats[0].h, check=False)
    assert o["status"] == _lib.DSM_E_TIMEOUT
    with pytest.raises(P.DSMError) as e:
        lats[0].step(1)
    assert e.value.status == _lib.DSM_E_STATE
    # recovery: the checkpoint taken before the failed launch
    lats[0].set_state(saved)
    lats[0].step(10)
    ref.step(10)
    fa, ga = lats[0].populations()
    fb, gb = ref.populations()
    assert torch.equal(fa, fb) and torch.equal(ga, gb)
    assert lats[0].observables()["step"] == 10
    # the default limit again: a batched launch completes
    others = [_lattice(s, 5 + i) for i, s in enumerate([(64, 64), (80, 48)])]
    hs = [lat.h for lat in others]
    nb = _lib.dsm_batch_scratch_bytes(hs)
    _lib.dsm_batch_step(hs, [5, 5], torch.empty(nb, dtype=torch.uint8, device=DEV), nb)
    for lat in others:
        assert lat.observables()["step"] == 5
