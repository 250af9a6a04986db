"""The C-ABI library without a GPU: it loads, exports every entry point that
include/dsm.h declares, and its host-side logic (argument checks, kappa mapping,
lattice tables, workspace sizing) is right.  No compute call is made."""
import math
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "dsm_build", os.path.join(ROOT, "paper_2504_19941_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    from paper_2504_19941_gb300 import _lib
    return _lib


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dsm_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    L = lib.load()
    declared = _declared()
    assert len(declared) >= 20
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared <= set(lib.EXPORTED), declared - set(lib.EXPORTED)


def test_status_strings(lib):
    for s in range(8):
        assert lib.status_string(s) not in ("", "unknown status")


@pytest.mark.parametrize("kind", [0, 1])
def test_lattice_table_matches_oracle(lib, kind):
    c, w = lib.dsm_lattice_table(kind)
    co, wo = O.lattice(kind)
    got = sorted(zip(map(tuple, c), w))
    ref = sorted(zip(map(tuple, co), wo))
    assert len(got) == len(ref)
    for (ca, wa), (cb, wb) in zip(got, ref):
        assert ca == tuple(cb) and abs(wa - wb) < 1e-17
    if kind == 0:  # the paper's D2Q9 order is kept
        assert [tuple(x) for x in c] == [tuple(x) for x in co]


def test_kappa_matches_oracle(lib):
    import paper_2504_19941_gb300 as P
    rng = np.random.default_rng(0)
    for _ in range(40):
        th, g23, g12, a = rng.uniform(5, 175), rng.uniform(1e-3, 1), rng.uniform(1e-3, 1), \
            rng.uniform(0.5, 2)
        p = P.make_params("D3Q19", (4, 4, 4), theta_deg=th, g23=g23, g12=g12, alpha=a)
        k_ref, rc = O.kappa_from_angle(th, g23, g12, a)
        if rc != 0:
            with pytest.raises(P.DSMError):
                lib.dsm_kappa(p)
            continue
        np.testing.assert_allclose(lib.dsm_kappa(p), k_ref, rtol=1e-13, atol=1e-16)
    p = P.make_params("D2Q9", (4, 4), g12=0.3, g13=0.5, g23=0.4)
    np.testing.assert_allclose(lib.dsm_kappa(p), O.kappa_from_tensions(0.3, 0.5, 0.4)[0])


@pytest.mark.parametrize("bad", [
    dict(shape=(0, 4, 4)), dict(shape=(4, -1, 4)), dict(lattice="D2Q9", shape=(4, 4, 2)),
    dict(tau2=0.5), dict(tau_g=0.4), dict(rho3=0.0), dict(theta_deg=180.0),
    dict(precision=7), dict(alpha=0.0), dict(shape=(2048, 2048, 1024)), dict(alpha_s=-1.0)])
def test_invalid_parameters_rejected(lib, bad):
    import paper_2504_19941_gb300 as P
    kw = dict(lattice="D3Q19", shape=(8, 8, 8), theta_deg=90.0)
    kw.update(bad)
    lat, shape = kw.pop("lattice"), kw.pop("shape")
    prec = kw.pop("precision", "f32")
    p = P.make_params(lat, shape, prec, **kw)
    with pytest.raises(P.DSMError) as e:
        lib.dsm_workspace_bytes(p)
    assert e.value.status == lib.DSM_E_INVAL


@pytest.mark.parametrize("faces,ok", [
    (("mirror", "mirror", "wall", "wall", "periodic", "periodic"), True),
    (("wall", "mirror", "periodic", "periodic", "mirror", "wall"), True),
    (("mirror", "periodic", "periodic", "periodic", "periodic", "periodic"), False),
    ((3, 3, 0, 0, 0, 0), False), ((-1, 1, 0, 0, 0, 0), False)])
def test_face_validation(lib, faces, ok):
    import paper_2504_19941_gb300 as P
    p = P.make_params("D3Q19", (8, 8, 8), "f32", theta_deg=90.0, faces=faces)
    if ok:
        assert lib.dsm_workspace_bytes(p) > 0
    else:
        with pytest.raises(P.DSMError) as e:
            lib.dsm_workspace_bytes(p)
        assert e.value.status == lib.DSM_E_INVAL
    # the z faces of a D2Q9 lattice are periodic
    p2 = P.make_params("D2Q9", (8, 8), "f32", theta_deg=90.0,
                       faces=("periodic", "periodic", "wall", "wall", "mirror", "mirror"))
    with pytest.raises(P.DSMError):
        lib.dsm_workspace_bytes(p2)


def test_invalid_faces_refused_by_energy_functions(lib):
    # each call refuses before any device work, so the fake addresses are
    # never touched
    import ctypes as C
    import paper_2504_19941_gb300 as P
    L = lib.load()
    fake = 1 << 20
    sb = lib.dsm_fe_scratch_bytes(1, 8, 8, 8)
    bad = P.make_params("D3Q19", (8, 8, 8), "f32", theta_deg=90.0, faces=(0, 0, 1, 0, 0, 0))
    assert L.dsm_fe_energy_grad(C.byref(bad), fake, fake, None, 2, 0.0, 0.0, 0.0, 0.0, fake,
                                fake, fake, fake * 256, sb, None) == lib.DSM_E_INVAL
    assert L.dsm_fe_energy_grad_noalloc(C.byref(bad), fake, fake, None, 2, 0.0, 0.0, 0.0, 0.0,
                                        fake, fake, fake, None) == lib.DSM_E_INVAL
    nb = lib.dsm_lbfgs_workspace_bytes(bad, 5)
    info = lib.dsm_lbfgs_info()
    assert L.dsm_lbfgs_minimize(C.byref(bad), fake, None, 2, 0.0, 0.0, 0.0, 0.0, fake, 5, 1e-6,
                                10, fake * 256, nb, C.byref(info), None) == lib.DSM_E_INVAL


@pytest.mark.parametrize("prec,sb,extra", [("f64", 8, 0), ("f32", 4, 0), ("bf16", 2, 1),
                                           ("f16", 2, 1)])
@pytest.mark.parametrize("shape", [(37, 29, 23), (21, 29, 23)])
def test_workspace_size(lib, prec, sb, extra, shape):
    import paper_2504_19941_gb300 as P
    nx, ny, nz = shape
    n = nx * ny * nz
    p = P.make_params("D3Q19", shape, prec, theta_deg=100.0)
    nbytes = lib.dsm_workspace_bytes(p)
    pops = 4 * 19 * n * sb + extra * 2 * 4 * n
    # plus seven real fields (C1, C in two buffers, the four g_eq planes A, u),
    # the mask bytes and small reduction scratch
    rb = 8 if prec == "f64" else 4
    reals = 7 * n * rb
    # nx >= 32, ny >= 8: the one-pass step's padded buffers, 11 reals per node
    # of (nx + 8 rounded up to a multiple of 4) (ny + 4) nz
    if nx >= 32 and ny >= 8:
        reals += 11 * ((nx + 8 + 3) // 4 * 4) * (ny + 4) * nz * rb
    assert pops + reals + n <= nbytes <= pops + reals + n + 10 * 2 ** 16


def test_create_rejects_bad_workspace_without_touching_the_gpu(lib):
    import paper_2504_19941_gb300 as P
    p = P.make_params("D3Q19", (8, 8, 8), "f32", theta_deg=90)
    nb = lib.dsm_workspace_bytes(p)
    for ptr, size in [(None, nb), (4096, nb - 1), (4096 + 16, nb)]:
        with pytest.raises(P.DSMError) as e:
            lib.dsm_create(p, ptr, size, stream=0)
        assert e.value.status == lib.DSM_E_WORKSPACE


def test_scratch_sizes(lib):
    # one FP64 partial per term per reduction block, at most 4 blocks per SM
    assert 8 * 5 * 608 <= lib.dsm_fe_scratch_bytes(1, 128, 128, 128) <= 32768
    assert lib.dsm_fe_scratch_bytes(0, 7, 5, 1) >= 8 * 5
    assert lib.dsm_vec_scratch_bytes(10 ** 7) >= 8 * 152 * 4
    import paper_2504_19941_gb300 as P
    with pytest.raises(P.DSMError):
        lib.dsm_fe_scratch_bytes(0, 4, 4, 2)


def test_null_arguments_rejected(lib):
    L = lib.load()
    assert L.dsm_step(None, 1) == lib.DSM_E_INVAL
    assert L.dsm_destroy(None) == lib.DSM_E_INVAL
    assert L.dsm_get_observables(None, None) == lib.DSM_E_INVAL
    assert L.dsm_batch_step(None, 1, None, None, 0) == lib.DSM_E_INVAL
    assert L.dsm_batch_scratch_bytes(None, 1, None) == lib.DSM_E_INVAL
    assert L.dsm_set_observables_ring(None, None, 0, 0) == lib.DSM_E_INVAL
    assert L.dsm_observables_ring_count(None, None) == lib.DSM_E_INVAL
    assert L.dsm_checked_build() == (1 if lib.LIB_PATH.endswith("_checked.so") else 0)


def test_vector_and_minimiser_arguments_rejected(lib):
    # argument checks of the batched vector kernels and the native L-BFGS loop:
    # each refuses before any device work, so fake addresses are never touched
    import ctypes as C
    import paper_2504_19941_gb300 as P
    L = lib.load()
    fake = 1 << 20
    assert L.dsm_vec_dots(-1, 2, fake, 10, fake, fake, fake, 1 << 20, None) == lib.DSM_E_INVAL
    assert L.dsm_vec_dots(10, 2, fake, 5, fake, fake, fake, 1 << 20, None) == lib.DSM_E_INVAL  # stride < n
    sb = lib.dsm_vec_dots_scratch_bytes(1000, 4)
    assert sb >= 4 * 8
    assert L.dsm_vec_dots(1000, 4, fake, 1000, fake, fake, fake, sb - 1, None) == lib.DSM_E_WORKSPACE
    coef = (C.c_double * 65)()
    assert L.dsm_vec_lincomb(10, 65, fake, 10, coef, fake, 1.0, fake, None) == lib.DSM_E_INVAL
    assert L.dsm_vec_lincomb(10, 2, None, 10, coef, fake, 1.0, fake, None) == lib.DSM_E_INVAL
    p = P.make_params("D3Q19", (16, 16, 16), "f32", theta_deg=90)
    nb = lib.dsm_lbfgs_workspace_bytes(p, 10)
    # the history holds 2m vectors: the workspace grows with m
    assert nb > 20 * 16 ** 3 * 4 and lib.dsm_lbfgs_workspace_bytes(p, 5) < nb
    with pytest.raises(P.DSMError):
        lib.dsm_lbfgs_workspace_bytes(p, 33)  # 2m above the combination limit
    info = lib.dsm_lbfgs_info()
    args = dict(fixed=fake, mask=None, active=2, dP=0.0, kcs=0.0, V0=0.0, fg=0.0, x=fake, m=10,
                tol=1e-6, max_iter=10, work=fake * 256, work_bytes=nb)

    def call(**kw):
        a = dict(args, **kw)
        return L.dsm_lbfgs_minimize(C.byref(p), a["fixed"], a["mask"], a["active"], a["dP"],
                                    a["kcs"], a["V0"], a["fg"], a["x"], a["m"], a["tol"],
                                    a["max_iter"], a["work"], a["work_bytes"], C.byref(info), None)
    assert call(active=3) == lib.DSM_E_INVAL
    assert call(active=1) == lib.DSM_E_INVAL          # stage 1 needs the solid mask
    assert call(kcs=-1.0) == lib.DSM_E_INVAL
    assert call(m=0) == lib.DSM_E_INVAL
    assert call(x=None) == lib.DSM_E_INVAL
    assert call(work_bytes=nb - 1) == lib.DSM_E_WORKSPACE
    assert call(work=fake * 256 + 16) == lib.DSM_E_WORKSPACE   # misaligned
    cx = C.c_double()
    one = (C.c_double * 1)(0.0)
    assert L.dsm_lbfgs_compact(1, one, one, one, one, 1.0, C.byref(cx), one, one) == lib.DSM_E_INVAL


def test_multi_fluid_arguments_rejected(lib):
    # the N-fluid energy, its L-BFGS and the N-fluid lattice refuse bad
    # arguments before any device work, so the fake addresses are never touched
    import ctypes as C
    import paper_2504_19941_gb300 as P
    L = lib.load()
    fake = 1 << 20
    p = P.make_params("D3Q19", (8, 8, 8), "f32", theta_deg=90.0)
    d = lambda *v: (C.c_double * len(v))(*v)  # noqa: E731
    sb = lib.dsm_fe_multi_scratch_bytes(1, 8, 8, 8, 3)
    assert sb > 0

    def fe(nfluid, kappa, kcs=None, scratch_bytes=sb, c=fake):
        return L.dsm_fe_energy_grad_multi(C.byref(p), nfluid, kappa, fake, c, None, kcs, None,
                                          fake, fake, None, fake * 256, scratch_bytes, None)
    assert fe(5, d(1, 1, 1, 1, 1, 1)) == lib.DSM_E_INVAL            # N above 4
    assert fe(1, d(1, 1)) == lib.DSM_E_INVAL                        # N below 2
    assert fe(3, d(1, 1, 0.0, 1)) == lib.DSM_E_INVAL                # a fluid kappa <= 0
    assert fe(3, None) == lib.DSM_E_INVAL
    assert fe(3, d(1, 1, 1, 1), kcs=d(-1.0, 0.0)) == lib.DSM_E_INVAL
    assert fe(3, d(1, 1, 1, 1), c=None) == lib.DSM_E_INVAL
    assert fe(3, d(-0.5, 1, 1, 1), scratch_bytes=16) == lib.DSM_E_WORKSPACE  # kappa_1 < 0 is valid
    with pytest.raises(P.DSMError):
        lib.dsm_lbfgs_multi_workspace_bytes(p, 5, 10)
    nb = lib.dsm_lbfgs_multi_workspace_bytes(p, 3, 10)
    assert nb > lib.dsm_lbfgs_workspace_bytes(p, 10)                # two planes per vector
    info = lib.dsm_lbfgs_info()
    assert L.dsm_lbfgs_minimize_multi(C.byref(p), 3, d(1, 1, 1, 1), fake, None, None, None,
                                      fake, 10, 1e-6, 10, fake * 256, nb - 1, C.byref(info),
                                      None) == lib.DSM_E_WORKSPACE
    # the N-fluid lattice
    assert lib.dsm_ml_workspace_bytes(p, 3) > lib.dsm_ml_workspace_bytes(p, 2)
    with pytest.raises(P.DSMError) as e:
        lib.dsm_ml_workspace_bytes(P.make_params("D3Q19", (8, 8, 8), "bf16", theta_deg=90.0), 3)
    assert e.value.status == lib.DSM_E_UNSUPPORTED
    h = C.c_void_p()
    nbm = lib.dsm_ml_workspace_bytes(p, 3)

    def create(nfluid, kappa, rho, tau, ws=fake * 256, nbytes=nbm):
        return L.dsm_ml_create(C.byref(p), nfluid, kappa, rho, tau, ws, nbytes, None,
                               C.byref(h))
    assert create(5, d(1, 1, 1, 1, 1, 1), d(1, 1, 1, 1, 1), d(1, 1, 1, 1, 1)) == lib.DSM_E_INVAL
    assert create(3, d(1, 1, 1, 1), d(1, 0.0, 1), d(1, 1, 1)) == lib.DSM_E_INVAL   # rho <= 0
    assert create(3, d(1, 1, 1, 1), d(1, 1, 1), d(1, 0.5, 1)) == lib.DSM_E_INVAL   # tau <= 1/2
    assert create(3, d(1, 1, 1, 1), d(1, 1, 1), d(1, 1, 1), ws=None) == lib.DSM_E_WORKSPACE
    assert create(3, d(1, 1, 1, 1), d(1, 1, 1), d(1, 1, 1), nbytes=nbm - 1) == lib.DSM_E_WORKSPACE
    assert L.dsm_ml_step(None, 1) == lib.DSM_E_INVAL
    assert L.dsm_ml_get_field(None, 1, 0, fake) == lib.DSM_E_INVAL


def test_tensor_arguments_are_checked_before_any_launch():
    # the Python layer hands raw pointers to libdsm, so it checks every tensor's
    # device, type, size and layout first (here on CPU tensors and a CPU device)
    torch = pytest.importorskip("torch")
    from paper_2504_19941_gb300 import _lib as L
    cpu = torch.device("cpu")
    t = torch.zeros(12, dtype=torch.float32)
    assert L.tensor_arg(t, 12, torch.float32, cpu, "x") is t
    with pytest.raises(ValueError, match="elements"):
        L.tensor_arg(t, 13, torch.float32, cpu, "x")
    with pytest.raises(ValueError, match="dtype"):
        L.tensor_arg(t, 12, torch.float64, cpu, "x")
    with pytest.raises(ValueError, match="expected cuda"):
        L.tensor_arg(t, 12, torch.float32, torch.device("cuda", 0), "x")
    with pytest.raises(TypeError):
        L.tensor_arg([0.0] * 12, 12, torch.float32, cpu, "x")
    m = torch.zeros(12, dtype=torch.uint8)
    assert L.tensor_arg(m, 12, None, cpu, "mask", itemsize=1) is m
    with pytest.raises(ValueError, match="byte elements"):
        L.tensor_arg(t, 12, None, cpu, "mask", itemsize=1)
    nc = torch.zeros(4, 6, dtype=torch.float32)[:, ::2]       # 12 elements, strided
    with pytest.raises(ValueError, match="contiguous"):
        L.tensor_arg(nc, 12, torch.float32, cpu, "out")
    c = L.tensor_arg(nc, 12, torch.float32, cpu, "x", copy=True)
    assert c.is_contiguous() and torch.equal(c, nc)
    with pytest.raises(ValueError, match="CUDA device"):
        L.cuda_device("cpu")
    assert L.cuda_device("cuda:1") == torch.device("cuda", 1)


def test_ring_records_order():
    # host side of the observables ring: record k sits in slot k % capacity
    import numpy as np
    from paper_2504_19941_gb300 import ring_records
    fields = ("step", "mass_c2", "mass_c1", "kinetic", "max_u", "nonfinite")
    cap = 4
    rows = np.zeros((cap, 6))
    for k in range(7):  # steps 10 .. 70, the last four kept
        rows[k % cap] = (10 * (k + 1), k + 0.5, 0, 0, 0, 0)
    got = ring_records(rows, 7, fields)
    assert [r["step"] for r in got] == [40, 50, 60, 70]
    assert [r["mass_c2"] for r in got] == [3.5, 4.5, 5.5, 6.5]
    fresh = np.zeros((cap, 6))
    fresh[0, 0], fresh[1, 0] = 10, 20  # two appends: not yet wrapped
    assert [r["step"] for r in ring_records(fresh, 2, fields)] == [10, 20]
    assert ring_records(rows, 0, fields) == []


def test_status_codes_match_the_header(lib):
    # the binding's status constants are the header's enum values
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "dsm.h")).read()
    body = hdr[hdr.index("DSM_OK = 0"):]
    body = body[:body.index("} dsm_status;")]
    codes = dict((m.group(1), int(m.group(2))) for m in re.finditer(r"(DSM_\w+)\s*=\s*(\d+)", body))
    assert codes["DSM_OK"] == 0 and len(codes) == 9
    for name, value in codes.items():
        assert getattr(lib, name) == value, name
        if name != "DSM_OK":
            assert lib.status_string(value) not in ("unknown status", "libdsm not loaded"), name
