"""The checked build (libdsm_checked.so, -DDSM_CHECKED) on the GPU.

In the checked build every neighbour, pull, store and padded-plane index that
the lattice Boltzmann kernels form is tested against its buffer.  An index
outside the buffer latches DSM_E_BOUNDS and is clamped to 0, so the kernel
reports the fault instead of making it.  ``test_parity_under_the_checked_build``
builds that library and reruns, in a child process that loads it
(DSM_LIB=checked), parity cases of every step form against the oracle:
  * the one-pass step, full and ragged tiles;
  * the two-pass step, face kinds and tiny lattices;
  * D2Q9;
  * N fluids, one and two passes;
  * the batched step.
The child also runs ``test_status_clean``, which drives each form and checks
that the error word stays clean: no index left its buffer.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = os.environ.get("DSM_LIB") == "checked"

CASES = [
    "tests/test_gpu_zstep.py::test_ragged_tiles_fp64_parity",
    "tests/test_gpu_zstep.py::test_single_pass_fp32_parity",
    "tests/test_gpu_mlz.py::test_ragged_tiles_fp64_parity",
    "tests/test_gpu_multi.py::test_ml_ragged_and_tiny_fp64",
    "tests/test_gpu_multi.py::test_ml_fp64_parity",
    "tests/test_gpu_lb.py::test_d3q19_fp64_parity",
    "tests/test_gpu_lb.py::test_faces_fp64_parity",
    "tests/test_gpu_lb.py::test_tiny_lattices_with_faces_fp64",
    "tests/test_gpu_lb.py::test_d2q9_tiled_moments_parity",
    "tests/test_gpu_lb.py::test_solid_relaxation_fp64_parity",
    "tests/test_gpu_batch.py::test_batch_matches_oracle",
]


@pytest.mark.skipif(CHILD, reason="the parent of the checked-build run")
def test_parity_under_the_checked_build():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "dsm_build", os.path.join(ROOT, "paper_2504_19941_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(checked=True)
    env = dict(os.environ, DSM_LIB="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *CASES, "tests/test_gpu_checked.py::test_status_clean"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = r.stdout[-4000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "skipped" not in r.stdout.splitlines()[-1], tail


def _lattice(P, lat, shape, prec, faces=None, form="auto", seed=0):
    rng = np.random.default_rng(seed)
    base = 1 if min(shape) < 8 else 3
    sd = S.pillars_sd(shape, base, 4, 9, 5 if min(shape) >= 8 else 1, offset=2)
    a_s = S.width_to_alpha(3.0)
    centre = [s / 2 for s in shape]
    centre[-1] = min(6.0, shape[-1] / 2)
    c2 = S.drop_c2(shape, centre, max(2.0, min(shape) / 3), 1.0, sd, a_s).ravel()
    c2 = c2 + S.perturbation(seed + 3, c2.size)
    p = P.make_params(lat, shape, prec, theta_deg=float(rng.uniform(50, 130)), g12=0.01,
                      g23=0.01, alpha_s=a_s, body=(1e-6, -2e-6, -3e-6), faces=faces,
                      rho2=1.0, rho3=0.5, tau2=0.8, tau3=0.6)
    L = P.Lattice(p)
    L.set_g_storage(form)
    L.set_solid_distance(torch.as_tensor(sd.ravel(), dtype=L.real, device="cuda"))
    L.c2_init = torch.as_tensor(c2, dtype=L.real, device="cuda")
    L.set_fluid(L.c2_init)
    return L


@pytest.mark.skipif(not CHILD, reason="runs in the child that loads the checked library")
def test_status_clean():
    import paper_2504_19941_gb300 as P
    from paper_2504_19941_gb300 import _lib
    assert _lib.checked_build()
    mw = ("mirror", "mirror", "wall", "wall", "periodic", "periodic")
    runs = [("D3Q19", (64, 24, 19), "f32", None, "auto", True),
            ("D3Q19", (45, 13, 7), "f64", None, "auto", True),
            ("D3Q19", (40, 16, 8), "bf16", None, "auto", True),
            ("D3Q19", (20, 17, 13), "f32", None, "populations", False),
            ("D3Q19", (13, 9, 7), "f64", mw, "auto", False),
            ("D2Q9", (64, 48), "f32", mw, "auto", False),
            ("D2Q9", (5, 4), "f64", None, "auto", False)]
    for k, (lat, shape, prec, faces, form, single) in enumerate(runs):
        L = _lattice(P, lat, shape, prec, faces, form, seed=k)
        assert L.single_pass == single, (lat, shape)
        L.step(25)
        if single:
            L.set_step_form("auto", 3)
            L.step(5)
        obs = L.observables()  # raises DSMError on DSM_E_BOUNDS
        assert obs["step"] == (30 if single else 25)
    # solid relaxation (the Allen-Cahn pass of the solid component)
    L = _lattice(P, "D3Q19", (14, 12, 10), "f64")
    mask = torch.zeros(14 * 12 * 10, dtype=torch.uint8, device="cuda")
    mask[: 14 * 12 * 3] = 1
    L.relax_solid(mask, 20, 1e-3, 2e-4)
    L.set_fluid(L.c2_init)  # relax_solid works in the population buffers: the fluid comes after
    L.step(3)
    L.observables()
    # the batched step over lattices of several sizes (one lattice kind per launch)
    for lat, shapes in (("D2Q9", [(33, 17), (7, 5), (64, 9)]),
                        ("D3Q19", [(20, 17, 13), (32, 24, 16)])):
        batch = [_lattice(P, lat, s, "f32", seed=10 + i) for i, s in enumerate(shapes)]
        hs = [b.h for b in batch]
        nb = _lib.dsm_batch_scratch_bytes(hs)
        scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
        _lib.dsm_batch_step(hs, [12, 5, 9][:len(hs)], scratch, nb)
        for b in batch:
            b.observables()
    # N fluids: one pass (D3Q19 g_eq form), two passes, D2Q9 with faces
    for nf, lat, shape, tau_g, faces, form in [(3, "D3Q19", (45, 13, 7), 1.0, None, "auto"),
                                               (4, "D3Q19", (37, 11, 5), 1.0, None, "auto"),
                                               (3, "D3Q19", (45, 13, 7), 1.0, None, "two_pass"),
                                               (3, "D3Q19", (13, 9, 7), 0.9, mw, "auto"),
                                               (4, "D2Q9", (23, 17), 0.9, mw, "auto")]:
        n = int(np.prod(shape))
        sd = S.pillars_sd(shape, 3 if len(shape) == 2 else 2, 4, 8, 5, offset=2)
        p = P.make_params(lat, shape, "f64", theta_deg=90.0, tau_g=tau_g, faces=faces,
                          body=(1e-6, 0.0, -2e-6), alpha_s=1.0)
        kappa = (0.02, 0.03, 0.025, 0.035, 0.028)[:nf + 1]
        ml = P.MultiLattice(p, nf, kappa, (1.0, 0.7, 0.5, 0.8)[:nf], (0.8, 0.6, 0.9, 0.7)[:nf])
        ml.set_step_form(form)
        ml.set_solid_distance(torch.as_tensor(sd.ravel(), dtype=ml.real, device="cuda"))
        C = np.stack([1.0 / nf + S.perturbation(nf + f, n, 0.02) for f in range(nf - 1)])
        ml.set_fluids(torch.as_tensor(C, dtype=ml.real, device="cuda"))
        assert ml.single_pass == (form == "auto" and tau_g == 1.0), (nf, lat, shape, form)
        ml.step(20)
        assert ml.status() == 0, (nf, lat, shape, form, _lib.status_string(ml.status()))
