"""ctypes binding of libdsm.so: the C ABI of include/dsm.h under the same names.

Argument marshalling only.  Device buffers are torch tensors (their data_ptr),
streams are torch CUDA streams (their cuda_stream handle).  Every status other
than DSM_OK raises DSMError.  The library must have been built
(``paper_2504_19941_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# DSM_LIB=checked loads the bounds-checked build (build.build(checked=True))
LIB_PATH = os.path.join(HERE, "libdsm_checked.so" if os.environ.get("DSM_LIB") == "checked"
                        else "libdsm.so")

DSM_OK, DSM_E_INVAL, DSM_E_WORKSPACE, DSM_E_CUDA, DSM_E_NONFINITE, DSM_E_TIMEOUT, \
    DSM_E_STATE, DSM_E_UNSUPPORTED, DSM_E_BOUNDS = range(9)
DSM_D2Q9, DSM_D3Q19 = 0, 1
DSM_FACE_PERIODIC, DSM_FACE_MIRROR, DSM_FACE_WALL = 0, 1, 2
DSM_F64, DSM_F32, DSM_BF16_STORE, DSM_F16_STORE = 0, 1, 2, 3
DSM_G_AUTO, DSM_G_POPULATIONS = 0, 1
DSM_STEP_AUTO, DSM_STEP_TWO_PASS = 0, 1
(DSM_FIELD_C1, DSM_FIELD_C2, DSM_FIELD_C3, DSM_FIELD_MU, DSM_FIELD_UX, DSM_FIELD_UY,
 DSM_FIELD_UZ, DSM_FIELD_PT, DSM_FIELD_RHO, DSM_FIELD_TAU) = range(10)

EXPORTED = (
    "dsm_status_string", "dsm_checked_build", "dsm_lattice_table", "dsm_kappa", "dsm_workspace_bytes", "dsm_create",
    "dsm_set_solid", "dsm_relax_solid", "dsm_solid_region", "dsm_set_fluid", "dsm_step", "dsm_step_moments",
    "dsm_step_collide", "dsm_set_body_force", "dsm_set_step_form", "dsm_step_info", "dsm_get_observables",
    "dsm_set_observables_ring", "dsm_observables_ring_count",
    "dsm_get_field", "dsm_get_populations", "dsm_set_populations", "dsm_set_g_storage",
    "dsm_get_g_storage", "dsm_state_bytes", "dsm_get_state", "dsm_set_state", "dsm_fe_scratch_bytes",
    "dsm_fe_energy_grad", "dsm_fe_energy_grad_noalloc", "dsm_vec_scratch_bytes", "dsm_vec_dot", "dsm_vec_axpy_dev",
    "dsm_vec_axpby", "dsm_lbfgs_direction", "dsm_vec_dots_scratch_bytes", "dsm_vec_dots",
    "dsm_vec_lincomb", "dsm_lbfgs_workspace_bytes", "dsm_lbfgs_minimize", "dsm_lbfgs_compact",
    "dsm_fe_multi_scratch_bytes", "dsm_fe_energy_grad_multi", "dsm_lbfgs_multi_workspace_bytes",
    "dsm_lbfgs_minimize_multi",
    "dsm_batch_scratch_bytes", "dsm_batch_step", "dsm_set_wait_limit",
    "dsm_destroy", "dsm_ml_workspace_bytes", "dsm_ml_create", "dsm_ml_set_solid",
    "dsm_ml_set_fluids", "dsm_ml_step", "dsm_ml_get_field", "dsm_ml_get_populations",
    "dsm_ml_check", "dsm_ml_destroy", "dsm_ml_set_step_form", "dsm_ml_step_info",
)


class DSMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class dsm_params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("precision", C.c_int), ("alpha", C.c_double), ("alpha_s", C.c_double),
                ("tension_mode", C.c_int), ("g12", C.c_double), ("g13", C.c_double),
                ("g23", C.c_double), ("theta_deg", C.c_double), ("rho2", C.c_double),
                ("rho3", C.c_double), ("tau2", C.c_double), ("tau3", C.c_double),
                ("tau_g", C.c_double), ("body_force", C.c_double * 3), ("beta", C.c_double),
                ("omega", C.c_double), ("face", C.c_int * 6)]


class dsm_lbfgs_info(C.Structure):
    _fields_ = [("iterations", C.c_longlong), ("evaluations", C.c_longlong),
                ("energy", C.c_double), ("rms_grad", C.c_double), ("converged", C.c_int)]


class dsm_observables(C.Structure):
    _fields_ = [("mass_c2", C.c_double), ("mass_c1", C.c_double), ("kinetic", C.c_double),
                ("max_u", C.c_double), ("step", C.c_longlong), ("nonfinite", C.c_int)]


_lib = None


def load():
    """Load libdsm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "paper_2504_19941_gb300.build.build() (nvcc, sm_103a; "
                          "checked=True for the checked library)")
    lib = C.CDLL(LIB_PATH)
    vp, dp, fp = C.c_void_p, C.POINTER(C.c_double), C.c_void_p
    P = C.POINTER(dsm_params)
    st = C.c_int
    sig = {
        "dsm_status_string": (C.c_char_p, [st]),
        "dsm_checked_build": (C.c_int, []),
        "dsm_lattice_table": (st, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), dp]),
        "dsm_kappa": (st, [P, dp]),
        "dsm_workspace_bytes": (st, [P, C.POINTER(C.c_size_t)]),
        "dsm_create": (st, [P, vp, C.c_size_t, vp, C.POINTER(vp)]),
        "dsm_set_solid": (st, [vp, vp, C.c_int]),
        "dsm_relax_solid": (st, [vp, vp, C.c_int, C.c_double, C.c_double]),
        "dsm_solid_region": (st, [vp, vp]),
        "dsm_set_fluid": (st, [vp, vp]),
        "dsm_step": (st, [vp, C.c_longlong]),
        "dsm_step_moments": (st, [vp]),
        "dsm_step_collide": (st, [vp]),
        "dsm_set_body_force": (st, [vp, C.POINTER(C.c_double)]),
        "dsm_set_step_form": (st, [vp, C.c_int, C.c_int]),
        "dsm_step_info": (st, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "dsm_get_observables": (st, [vp, C.POINTER(dsm_observables)]),
        "dsm_set_observables_ring": (st, [vp, vp, C.c_int, C.c_longlong]),
        "dsm_observables_ring_count": (st, [vp, C.POINTER(C.c_longlong)]),
        "dsm_get_field": (st, [vp, C.c_int, vp]),
        "dsm_get_populations": (st, [vp, vp, vp]),
        "dsm_set_populations": (st, [vp, vp, vp]),
        "dsm_set_g_storage": (st, [vp, C.c_int]),
        "dsm_get_g_storage": (st, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "dsm_state_bytes": (st, [vp, C.POINTER(C.c_size_t)]),
        "dsm_get_state": (st, [vp, vp, C.c_size_t]),
        "dsm_set_state": (st, [vp, vp, C.c_size_t]),
        "dsm_fe_scratch_bytes": (st, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
        "dsm_fe_energy_grad": (st, [P, fp, fp, vp, C.c_int, C.c_double, C.c_double, C.c_double,
                                    C.c_double, vp, fp, vp, vp, C.c_size_t, vp]),
        "dsm_fe_energy_grad_noalloc": (st, [P, fp, fp, vp, C.c_int, C.c_double, C.c_double,
                                            C.c_double, C.c_double, vp, fp, vp, vp]),
        "dsm_vec_scratch_bytes": (st, [C.c_longlong, C.POINTER(C.c_size_t)]),
        "dsm_vec_dot": (st, [C.c_longlong, fp, fp, vp, vp, C.c_size_t, vp]),
        "dsm_vec_axpy_dev": (st, [C.c_longlong, C.c_double, vp, vp, fp, fp, vp]),
        "dsm_vec_axpby": (st, [C.c_longlong, C.c_double, fp, C.c_double, fp, vp]),
        "dsm_lbfgs_direction": (st, [C.c_longlong, C.c_int, C.POINTER(C.c_int), fp, fp, vp, vp, fp,
                                     fp, vp, vp, C.c_size_t, vp]),
        "dsm_vec_dots_scratch_bytes": (st, [C.c_longlong, C.c_int, C.POINTER(C.c_size_t)]),
        "dsm_vec_dots": (st, [C.c_longlong, C.c_int, fp, C.c_longlong, fp, vp, vp, C.c_size_t,
                              vp]),
        "dsm_vec_lincomb": (st, [C.c_longlong, C.c_int, fp, C.c_longlong, dp, fp, C.c_double, fp,
                                 vp]),
        "dsm_lbfgs_workspace_bytes": (st, [P, C.c_int, C.POINTER(C.c_size_t)]),
        "dsm_lbfgs_minimize": (st, [P, fp, vp, C.c_int, C.c_double, C.c_double, C.c_double,
                                    C.c_double, fp, C.c_int, C.c_double, C.c_longlong, vp,
                                    C.c_size_t, C.POINTER(dsm_lbfgs_info), vp]),
        "dsm_lbfgs_compact": (st, [C.c_int, dp, dp, dp, dp, C.c_double, dp, dp, dp]),
        "dsm_fe_multi_scratch_bytes": (st, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                            C.POINTER(C.c_size_t)]),
        "dsm_fe_energy_grad_multi": (st, [P, C.c_int, dp, fp, fp, dp, dp, dp, vp, fp, vp, vp,
                                          C.c_size_t, vp]),
        "dsm_lbfgs_multi_workspace_bytes": (st, [P, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
        "dsm_lbfgs_minimize_multi": (st, [P, C.c_int, dp, fp, dp, dp, dp, fp, C.c_int,
                                          C.c_double, C.c_longlong, vp, C.c_size_t,
                                          C.POINTER(dsm_lbfgs_info), vp]),
        "dsm_batch_scratch_bytes": (st, [C.POINTER(vp), C.c_int, C.POINTER(C.c_size_t)]),
        "dsm_batch_step": (st, [C.POINTER(vp), C.c_int, C.POINTER(C.c_longlong), vp, C.c_size_t]),
        "dsm_set_wait_limit": (st, [C.c_ulonglong]),
        "dsm_destroy": (st, [vp]),
        "dsm_ml_workspace_bytes": (st, [P, C.c_int, C.POINTER(C.c_size_t)]),
        "dsm_ml_create": (st, [P, C.c_int, dp, dp, dp, vp, C.c_size_t, vp, C.POINTER(vp)]),
        "dsm_ml_set_solid": (st, [vp, vp, C.c_int]),
        "dsm_ml_set_fluids": (st, [vp, vp]),
        "dsm_ml_step": (st, [vp, C.c_longlong]),
        "dsm_ml_get_field": (st, [vp, C.c_int, C.c_int, vp]),
        "dsm_ml_get_populations": (st, [vp, vp, vp]),
        "dsm_ml_check": (st, [vp]),
        "dsm_ml_destroy": (st, [vp]),
        "dsm_ml_set_step_form": (st, [vp, C.c_int, C.c_int]),
        "dsm_ml_step_info": (st, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def checked_build() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(load().dsm_checked_build())


def status_string(s: int) -> str:
    try:
        return load().dsm_status_string(int(s)).decode()
    except ImportError:
        return "libdsm not loaded"


def _check(s: int, where: str):
    if s != DSM_OK:
        raise DSMError(s, where)


def _ptr(t):
    """Device address of a torch tensor (or None / int passthrough)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def cuda_device(device):
    """torch.device of a CUDA device with its index filled in."""
    import torch
    d = torch.device(device)
    if d.type != "cuda":
        raise ValueError(f"a CUDA device is required, not {d}")
    return d if d.index is not None else torch.device("cuda", torch.cuda.current_device())


def tensor_arg(t, numel: int, dtype, device, what: str, copy: bool = False, itemsize=None):
    """A device tensor handed to libdsm as a raw pointer: a torch tensor on
    `device` with `numel` elements of `dtype` (or, with dtype None, of any type
    of `itemsize` bytes), contiguous (with copy=True an input that is not is
    copied instead).  Raises TypeError / ValueError otherwise, so that no launch
    reads or writes past a buffer."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch tensor, got {type(t).__name__}")
    if t.device != device:
        raise ValueError(f"{what}: tensor on {t.device}, expected {device}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{what}: dtype {t.dtype}, expected {dtype}")
    if itemsize is not None and t.element_size() != itemsize:
        raise ValueError(f"{what}: {t.element_size()}-byte elements, expected {itemsize}")
    if t.numel() != numel:
        raise ValueError(f"{what}: {t.numel()} elements, expected {numel}")
    if not t.is_contiguous():
        if not copy:
            raise ValueError(f"{what}: the tensor must be contiguous")
        t = t.contiguous()
    return t


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# --------------------------------------------------------------------------
# same-name wrappers
# --------------------------------------------------------------------------
def dsm_lattice_table(lattice: int):
    q = C.c_int()
    c = (C.c_int * 57)()
    w = (C.c_double * 19)()
    _check(load().dsm_lattice_table(lattice, C.byref(q), c, w), "dsm_lattice_table")
    return [tuple(c[3 * i:3 * i + 3]) for i in range(q.value)], list(w[:q.value])


def dsm_kappa(params: dsm_params):
    k = (C.c_double * 3)()
    _check(load().dsm_kappa(C.byref(params), k), "dsm_kappa")
    return list(k)


def dsm_workspace_bytes(params: dsm_params) -> int:
    n = C.c_size_t()
    _check(load().dsm_workspace_bytes(C.byref(params), C.byref(n)), "dsm_workspace_bytes")
    return n.value


def dsm_create(params: dsm_params, workspace, nbytes: int, stream=None) -> int:
    h = C.c_void_p()
    _check(load().dsm_create(C.byref(params), _ptr(workspace), nbytes, _stream(stream),
                             C.byref(h)), "dsm_create")
    return h.value


def dsm_set_solid(h: int, field, kind: int):
    _check(load().dsm_set_solid(h, _ptr(field), kind), "dsm_set_solid")


def dsm_relax_solid(h: int, mask, steps: int, beta: float, omega: float):
    _check(load().dsm_relax_solid(h, _ptr(mask), steps, beta, omega), "dsm_relax_solid")


def dsm_solid_region(h: int, mask):
    _check(load().dsm_solid_region(h, _ptr(mask)), "dsm_solid_region")


def dsm_set_fluid(h: int, c2):
    _check(load().dsm_set_fluid(h, _ptr(c2)), "dsm_set_fluid")


def dsm_step(h: int, nsteps: int):
    _check(load().dsm_step(h, nsteps), "dsm_step")


def dsm_step_moments(h: int):
    _check(load().dsm_step_moments(h), "dsm_step_moments")


def dsm_step_collide(h: int):
    _check(load().dsm_step_collide(h), "dsm_step_collide")


def dsm_set_body_force(h: int, body):
    b = (C.c_double * 3)(*[float(v) for v in body])
    _check(load().dsm_set_body_force(h, b), "dsm_set_body_force")


def dsm_set_step_form(h: int, form: int, zrun: int = 0):
    _check(load().dsm_set_step_form(h, form, zrun), "dsm_set_step_form")


def dsm_step_info(h: int):
    """(single_pass, zrun) of dsm_step_info."""
    sp, zr = C.c_int(0), C.c_int(0)
    _check(load().dsm_step_info(h, C.byref(sp), C.byref(zr)), "dsm_step_info")
    return bool(sp.value), zr.value


def dsm_get_observables(h: int, check: bool = True) -> dict:
    o = dsm_observables()
    s = load().dsm_get_observables(h, C.byref(o))
    if check:
        _check(s, "dsm_get_observables")
    return dict(mass_c2=o.mass_c2, mass_c1=o.mass_c1, kinetic=o.kinetic, max_u=o.max_u,
                step=o.step, nonfinite=o.nonfinite, status=s)


def dsm_set_observables_ring(h: int, ring, capacity: int, every: int):
    _check(load().dsm_set_observables_ring(h, _ptr(ring), int(capacity), int(every)),
           "dsm_set_observables_ring")


def dsm_observables_ring_count(h: int) -> int:
    n = C.c_longlong(0)
    _check(load().dsm_observables_ring_count(h, C.byref(n)), "dsm_observables_ring_count")
    return n.value


def dsm_get_field(h: int, field: int, dst):
    _check(load().dsm_get_field(h, field, _ptr(dst)), "dsm_get_field")


def dsm_get_populations(h: int, f, g):
    _check(load().dsm_get_populations(h, _ptr(f), _ptr(g)), "dsm_get_populations")


def dsm_set_populations(h: int, f, g):
    _check(load().dsm_set_populations(h, _ptr(f), _ptr(g)), "dsm_set_populations")


def dsm_set_g_storage(h: int, form: int):
    _check(load().dsm_set_g_storage(h, form), "dsm_set_g_storage")


def dsm_get_g_storage(h: int):
    """(form, 1 if the current state holds g as g_eq else 0)."""
    form, imp = C.c_int(), C.c_int()
    _check(load().dsm_get_g_storage(h, C.byref(form), C.byref(imp)), "dsm_get_g_storage")
    return form.value, imp.value


def dsm_state_bytes(h: int) -> int:
    n = C.c_size_t()
    _check(load().dsm_state_bytes(h, C.byref(n)), "dsm_state_bytes")
    return n.value


def dsm_get_state(h: int, dst, nbytes: int):
    _check(load().dsm_get_state(h, _ptr(dst), nbytes), "dsm_get_state")


def dsm_set_state(h: int, src, nbytes: int):
    _check(load().dsm_set_state(h, _ptr(src), nbytes), "dsm_set_state")


def dsm_fe_scratch_bytes(lattice: int, nx: int, ny: int, nz: int) -> int:
    n = C.c_size_t()
    _check(load().dsm_fe_scratch_bytes(lattice, nx, ny, nz, C.byref(n)), "dsm_fe_scratch_bytes")
    return n.value


def dsm_fe_energy_grad(params: dsm_params, c1, c2, mask, active: int, dP: float, kcs: float,
                       V0: float, fg: float, energy, grad, terms, scratch, scratch_bytes: int,
                       stream=None):
    _check(load().dsm_fe_energy_grad(C.byref(params), _ptr(c1), _ptr(c2), _ptr(mask), active,
                                     dP, kcs, V0, fg, _ptr(energy), _ptr(grad), _ptr(terms),
                                     _ptr(scratch), scratch_bytes, _stream(stream)),
           "dsm_fe_energy_grad")


def dsm_fe_energy_grad_noalloc(params: dsm_params, c1, c2, mask, active: int, dP: float,
                               kcs: float, V0: float, fg: float, energy, grad, terms,
                               stream=None):
    _check(load().dsm_fe_energy_grad_noalloc(C.byref(params), _ptr(c1), _ptr(c2), _ptr(mask),
                                             active, dP, kcs, V0, fg, _ptr(energy), _ptr(grad),
                                             _ptr(terms), _stream(stream)),
           "dsm_fe_energy_grad_noalloc")


def dsm_vec_scratch_bytes(n: int) -> int:
    b = C.c_size_t()
    _check(load().dsm_vec_scratch_bytes(n, C.byref(b)), "dsm_vec_scratch_bytes")
    return b.value


def dsm_vec_dot(n: int, x, y, out, scratch, scratch_bytes: int, stream=None):
    _check(load().dsm_vec_dot(n, _ptr(x), _ptr(y), _ptr(out), _ptr(scratch), scratch_bytes,
                              _stream(stream)), "dsm_vec_dot")


def dsm_vec_axpy_dev(n: int, sign: float, a, b, x, y, stream=None):
    _check(load().dsm_vec_axpy_dev(n, sign, _ptr(a), _ptr(b), _ptr(x), _ptr(y), _stream(stream)),
           "dsm_vec_axpy_dev")


def dsm_vec_axpby(n: int, a: float, x, b: float, y, stream=None):
    _check(load().dsm_vec_axpby(n, a, _ptr(x), b, _ptr(y), _stream(stream)), "dsm_vec_axpby")


def dsm_lbfgs_direction(n: int, order, S, Y, rho, gamma, g, r, alpha, scratch, scratch_bytes: int,
                        stream=None):
    m = len(order)
    arr = (C.c_int * max(m, 1))(*order)
    _check(load().dsm_lbfgs_direction(n, m, arr, _ptr(S), _ptr(Y), _ptr(rho), _ptr(gamma),
                                      _ptr(g), _ptr(r), _ptr(alpha), _ptr(scratch), scratch_bytes,
                                      _stream(stream)), "dsm_lbfgs_direction")


def dsm_vec_dots_scratch_bytes(n: int, nv: int) -> int:
    b = C.c_size_t()
    _check(load().dsm_vec_dots_scratch_bytes(n, nv, C.byref(b)), "dsm_vec_dots_scratch_bytes")
    return b.value


def dsm_vec_dots(n: int, nv: int, V, stride: int, x, out, scratch, scratch_bytes: int,
                 stream=None):
    _check(load().dsm_vec_dots(n, nv, _ptr(V), stride, _ptr(x), _ptr(out), _ptr(scratch),
                               scratch_bytes, _stream(stream)), "dsm_vec_dots")


def dsm_vec_lincomb(n: int, nv: int, V, stride: int, coef, x, cx: float, y, stream=None):
    arr = (C.c_double * max(nv, 1))(*[float(v) for v in coef[:nv]])
    _check(load().dsm_vec_lincomb(n, nv, _ptr(V), stride, arr, _ptr(x), float(cx), _ptr(y),
                                  _stream(stream)), "dsm_vec_lincomb")


def _doubles(v, n):
    """Host double array of n values (None -> None)."""
    if v is None:
        return None
    vals = [float(x) for x in v]
    if len(vals) != n:
        raise ValueError(f"expected {n} values, got {len(vals)}")
    return (C.c_double * n)(*vals)


def dsm_fe_multi_scratch_bytes(lattice: int, nx: int, ny: int, nz: int, nfluid: int) -> int:
    n = C.c_size_t()
    _check(load().dsm_fe_multi_scratch_bytes(lattice, nx, ny, nz, nfluid, C.byref(n)),
           "dsm_fe_multi_scratch_bytes")
    return n.value


def dsm_fe_energy_grad_multi(params: dsm_params, nfluid: int, kappa, c1, c, dP, kcs, V0, energy,
                             grad, terms, scratch, scratch_bytes: int, stream=None):
    nf = nfluid - 1
    _check(load().dsm_fe_energy_grad_multi(C.byref(params), nfluid, _doubles(kappa, nfluid + 1),
                                           _ptr(c1), _ptr(c), _doubles(dP, nf), _doubles(kcs, nf),
                                           _doubles(V0, nf), _ptr(energy), _ptr(grad),
                                           _ptr(terms), _ptr(scratch), scratch_bytes,
                                           _stream(stream)),
           "dsm_fe_energy_grad_multi")


def dsm_lbfgs_multi_workspace_bytes(params: dsm_params, nfluid: int, m: int) -> int:
    b = C.c_size_t()
    _check(load().dsm_lbfgs_multi_workspace_bytes(C.byref(params), nfluid, m, C.byref(b)),
           "dsm_lbfgs_multi_workspace_bytes")
    return b.value


def dsm_lbfgs_minimize_multi(params: dsm_params, nfluid: int, kappa, c1, dP, kcs, V0, x, m: int,
                             tol: float, max_iter: int, work, work_bytes: int, stream=None,
                             check=True) -> dict:
    info = dsm_lbfgs_info()
    nf = nfluid - 1
    s = load().dsm_lbfgs_minimize_multi(C.byref(params), nfluid, _doubles(kappa, nfluid + 1),
                                        _ptr(c1), _doubles(dP, nf), _doubles(kcs, nf),
                                        _doubles(V0, nf), _ptr(x), m, tol, max_iter, _ptr(work),
                                        work_bytes, C.byref(info), _stream(stream))
    if check:
        _check(s, "dsm_lbfgs_minimize_multi")
    return dict(iterations=info.iterations, evaluations=info.evaluations, energy=info.energy,
                rms_grad=info.rms_grad, converged=bool(info.converged), status=s)


def dsm_lbfgs_workspace_bytes(params: dsm_params, m: int) -> int:
    b = C.c_size_t()
    _check(load().dsm_lbfgs_workspace_bytes(C.byref(params), m, C.byref(b)),
           "dsm_lbfgs_workspace_bytes")
    return b.value


def dsm_lbfgs_minimize(params: dsm_params, fixed, mask, active: int, dP: float, kcs: float,
                       V0: float, fg: float, x, m: int, tol: float, max_iter: int, work,
                       work_bytes: int, stream=None, check=True) -> dict:
    info = dsm_lbfgs_info()
    s = load().dsm_lbfgs_minimize(C.byref(params), _ptr(fixed), _ptr(mask), active, dP, kcs, V0,
                                  fg, _ptr(x), m, tol, max_iter, _ptr(work), work_bytes,
                                  C.byref(info), _stream(stream))
    if check:
        _check(s, "dsm_lbfgs_minimize")
    return dict(iterations=info.iterations, evaluations=info.evaluations, energy=info.energy,
                rms_grad=info.rms_grad, converged=bool(info.converged), status=s)


def dsm_lbfgs_compact(SY, YY, a, b, gamma: float):
    """Host-only compact-form solve: (cx, cs, cy) of -H g (see the header)."""
    import numpy as np
    k = len(a)
    arr = lambda v: (C.c_double * max(len(v), 1))(*[float(t) for t in v])  # noqa: E731
    cx = C.c_double()
    cs, cy = (C.c_double * k)(), (C.c_double * k)()
    _check(load().dsm_lbfgs_compact(k, arr(np.ravel(SY)), arr(np.ravel(YY)), arr(a), arr(b),
                                    float(gamma), C.byref(cx), cs, cy), "dsm_lbfgs_compact")
    return cx.value, np.array(cs[:]), np.array(cy[:])


def dsm_batch_scratch_bytes(handles) -> int:
    n = len(handles)
    hs = (C.c_void_p * max(n, 1))(*handles)
    b = C.c_size_t()
    _check(load().dsm_batch_scratch_bytes(hs, n, C.byref(b)), "dsm_batch_scratch_bytes")
    return b.value


def dsm_batch_step(handles, nsteps, scratch, scratch_bytes: int):
    n = len(handles)
    hs = (C.c_void_p * max(n, 1))(*handles)
    ns = (C.c_longlong * max(n, 1))(*nsteps)
    _check(load().dsm_batch_step(hs, n, ns, _ptr(scratch), scratch_bytes), "dsm_batch_step")


def dsm_set_wait_limit(polls: int):
    _check(load().dsm_set_wait_limit(int(polls)), "dsm_set_wait_limit")


def dsm_destroy(h: int):
    _check(load().dsm_destroy(h), "dsm_destroy")


def dsm_ml_workspace_bytes(params: dsm_params, nfluid: int) -> int:
    n = C.c_size_t()
    _check(load().dsm_ml_workspace_bytes(C.byref(params), nfluid, C.byref(n)),
           "dsm_ml_workspace_bytes")
    return n.value


def dsm_ml_create(params: dsm_params, nfluid: int, kappa, rho, tau, workspace, nbytes: int,
                  stream=None) -> int:
    h = C.c_void_p()
    _check(load().dsm_ml_create(C.byref(params), nfluid, _doubles(kappa, nfluid + 1),
                                _doubles(rho, nfluid), _doubles(tau, nfluid), _ptr(workspace),
                                nbytes, _stream(stream), C.byref(h)), "dsm_ml_create")
    return h.value


def dsm_ml_set_solid(h: int, field, kind: int):
    _check(load().dsm_ml_set_solid(h, _ptr(field), kind), "dsm_ml_set_solid")


def dsm_ml_set_fluids(h: int, c):
    _check(load().dsm_ml_set_fluids(h, _ptr(c)), "dsm_ml_set_fluids")


def dsm_ml_step(h: int, nsteps: int):
    _check(load().dsm_ml_step(h, nsteps), "dsm_ml_step")


def dsm_ml_get_field(h: int, field: int, index: int, out):
    _check(load().dsm_ml_get_field(h, field, index, _ptr(out)), "dsm_ml_get_field")


def dsm_ml_get_populations(h: int, f, g):
    _check(load().dsm_ml_get_populations(h, _ptr(f), _ptr(g)), "dsm_ml_get_populations")


def dsm_ml_check(h: int, check=True) -> int:
    s = load().dsm_ml_check(h)
    if check:
        _check(s, "dsm_ml_check")
    return s


def dsm_ml_set_step_form(h: int, form: int, zrun: int = 0):
    _check(load().dsm_ml_set_step_form(h, form, zrun), "dsm_ml_set_step_form")


def dsm_ml_step_info(h: int):
    """(single_pass, zrun) of dsm_ml_step_info."""
    sp, zr = C.c_int(0), C.c_int(0)
    _check(load().dsm_ml_step_info(h, C.byref(sp), C.byref(zr)), "dsm_ml_step_info")
    return bool(sp.value), zr.value


def dsm_ml_destroy(h: int):
    _check(load().dsm_ml_destroy(h), "dsm_ml_destroy")
