"""FP64 CPU oracle of the Diffuse Solid Method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library under
``paper_2504_19941_gb300`` and its binding) never imports it and shares no
code with it.

The arithmetic lives in ``dsm_oracle.c`` (plain C, FP64, one loop per stage
of the method in the paper's order); this module compiles it with gcc on
first use and wraps it with numpy arrays.  ``lbfgs.py`` holds the oracle's
L-BFGS minimiser and ``analysis.py`` the contact-angle and profile analysis.

Parity status of each function (what pins it) is listed in the header of
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19 = 0, 1


def build(force: bool = False) -> str:
    """Compile dsm_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    """Mirror of ``or_params`` in dsm_oracle.c."""
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("alpha", C.c_double), ("alpha_s", C.c_double),
                ("kappa1", C.c_double), ("kappa2", C.c_double), ("kappa3", C.c_double),
                ("rho2", C.c_double), ("rho3", C.c_double), ("tau2", C.c_double),
                ("tau3", C.c_double), ("tau_g", C.c_double),
                ("bx", C.c_double), ("by", C.c_double), ("bz", C.c_double),
                ("beta", C.c_double), ("omega", C.c_double), ("face", C.c_int * 6)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            bp = C.POINTER(C.c_ubyte)
            pp = C.POINTER(Params)
            lib.or_lattice.argtypes = [C.c_int, ip, dp]
            lib.or_kappa_from_tensions.argtypes = [C.c_double] * 4 + [dp]
            lib.or_kappa_from_angle.argtypes = [C.c_double] * 4 + [dp]
            lib.or_solid_profile.argtypes = [C.c_long, dp, C.c_double, dp]
            lib.or_gradient.argtypes = [pp, dp, dp]
            lib.or_laplacian.argtypes = [pp, dp, dp]
            lib.or_mu_fluid.argtypes = [pp, dp, dp, dp]
            lib.or_mu_solid.argtypes = [pp, bp, dp, dp]
            lib.or_equilibria.argtypes = [C.c_int, C.c_double, C.c_double, dp, C.c_double,
                                          C.c_double, C.c_double, dp, dp, dp, dp, dp]
            lib.or_link_q.argtypes = [C.c_int, C.c_double, C.c_double, dp, C.c_int]
            lib.or_link_q.restype = C.c_double
            lib.or_lb_run.argtypes = [pp, C.c_int, bp, dp, dp, dp, C.c_long, dp]
            lib.or_lb_fields.argtypes = [pp, C.c_int, bp, dp, dp, dp, dp]
            lib.or_lb_init.argtypes = [pp, C.c_int, bp, dp, dp, dp, dp]
            lib.or_energy_grad.argtypes = [pp, dp, dp, bp, C.c_int, C.c_double, C.c_double,
                                           C.c_double, C.c_double, dp, dp]
            lib.or_energy_grad.restype = C.c_double
            lib.or_observables.argtypes = [pp, dp, dp, dp, dp]
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _b(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_ubyte))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------
def lattice(kind: int):
    """Velocity set c (q x 3, int) and weights w (q,) of D2Q9 / D3Q19."""
    lib = _load()
    c = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    q = lib.or_lattice(kind, c.ctypes.data_as(C.POINTER(C.c_int)), _d(w))
    return c[:3 * q].reshape(q, 3).copy(), w[:q].copy()


def kappa_from_tensions(g12, g13, g23, alpha=1.0):
    k = np.zeros(3)
    rc = _load().or_kappa_from_tensions(g12, g13, g23, alpha, _d(k))
    return k, rc


def kappa_from_angle(theta_deg, g23, g12, alpha=1.0):
    k = np.zeros(3)
    rc = _load().or_kappa_from_angle(theta_deg, g23, g12, alpha, _d(k))
    return k, rc


def make_params(kind, shape, kappa, *, alpha=1.0, alpha_s=None, rho2=1.0, rho3=1.0,
                tau2=1.0, tau3=1.0, tau_g=1.0, body=(0.0, 0.0, 0.0), beta=0.0,
                omega=0.0, faces=None) -> Params:
    """faces: the boundary of the faces x-, x+, y-, y+, z-, z+, each "periodic",
    "mirror" (symmetry plane) or "wall" (halfway bounce-back), or 0, 1, 2;
    None: all periodic."""
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    return Params(kind, nx, ny, nz, alpha, alpha if alpha_s is None else alpha_s,
                  kappa[0], kappa[1], kappa[2], rho2, rho3, tau2, tau3, tau_g,
                  body[0], body[1], body[2], beta, omega, (C.c_int * 6)(*face_codes(faces)))


FACE_CODES = {"periodic": 0, "mirror": 1, "wall": 2}


def face_codes(faces):
    if faces is None:
        return (0,) * 6
    if len(faces) != 6:
        raise ValueError("faces: six entries, x-, x+, y-, y+, z-, z+")
    codes = tuple(FACE_CODES[f] if isinstance(f, str) else int(f) for f in faces)
    for a in range(3):
        if (codes[2 * a] == 0) != (codes[2 * a + 1] == 0) or not 0 <= codes[2 * a] <= 2 \
                or not 0 <= codes[2 * a + 1] <= 2:
            raise ValueError("faces: an axis is periodic on both faces or on neither")
    return codes


def _n(p: Params) -> int:
    return p.nx * p.ny * p.nz


def _q(p: Params) -> int:
    return 9 if p.kind == D2Q9 else 19


def solid_profile(sd, alpha_s):
    sd = _f64(sd).ravel()
    out = np.empty_like(sd)
    _load().or_solid_profile(sd.size, _d(sd), alpha_s, _d(out))
    return out


def gradient(p: Params, phi):
    phi = _f64(phi).ravel()
    out = np.empty(3 * _n(p))
    _load().or_gradient(C.byref(p), _d(phi), _d(out))
    return out.reshape(3, -1)


def laplacian(p: Params, phi):
    phi = _f64(phi).ravel()
    out = np.empty(_n(p))
    _load().or_laplacian(C.byref(p), _d(phi), _d(out))
    return out


def mu_fluid(p: Params, c1, c):
    c1, c = _f64(c1).ravel(), _f64(c).ravel()
    out = np.empty(_n(p))
    _load().or_mu_fluid(C.byref(p), _d(c1), _d(c), _d(out))
    return out


def mu_solid(p: Params, S, c1):
    S = np.ascontiguousarray(S, dtype=np.uint8).ravel()
    c1 = _f64(c1).ravel()
    out = np.empty(_n(p))
    _load().or_mu_solid(C.byref(p), _b(S), _d(c1), _d(out))
    return out


def equilibria(kind, pt, rho, u, Cc, mu, tau, grho, F):
    q = 9 if kind == D2Q9 else 19
    feq, geq, Fi = np.zeros(q), np.zeros(q), np.zeros(q)
    u, grho, F = _f64(u), _f64(grho), _f64(F)
    _load().or_equilibria(kind, pt, rho, _d(u), Cc, mu, tau, _d(grho), _d(F),
                          _d(feq), _d(geq), _d(Fi))
    return feq, geq, Fi


def link_q(kind, alpha_s, c1x, gc1, i):
    gc1 = _f64(gc1)
    return _load().or_link_q(kind, alpha_s, c1x, _d(gc1), i)


def lb_init(p: Params, stage: int, c1, cfield, S=None):
    """Quiescent initial post-collision state (f, g), each q x N."""
    n, q = _n(p), _q(p)
    f = np.empty(q * n)
    g = np.empty(q * n)
    c1a = _f64(c1 if c1 is not None else np.zeros(n)).ravel()
    cf = _f64(cfield).ravel()
    Sa = None if S is None else np.ascontiguousarray(S, dtype=np.uint8).ravel()
    _load().or_lb_init(C.byref(p), stage, _b(Sa), _d(c1a), _d(cf), _d(f), _d(g))
    return f.reshape(q, n), g.reshape(q, n)


FIELD_NAMES = ("C", "mu", "ux", "uy", "uz", "pt", "rho", "tau")


def lb_run(p: Params, stage: int, c1, f, g, nsteps: int, S=None, want_fields=False):
    """Advance the post-collision state (f, g) by nsteps (copies, returns new)."""
    n = _n(p)
    f = _f64(f).copy()
    g = _f64(g).copy()
    c1a = _f64(c1 if c1 is not None else np.zeros(n)).ravel()
    Sa = None if S is None else np.ascontiguousarray(S, dtype=np.uint8).ravel()
    fields = np.zeros(8 * n) if want_fields else None
    _load().or_lb_run(C.byref(p), stage, _b(Sa), _d(c1a), _d(f), _d(g), nsteps,
                      None if fields is None else _d(fields))
    if want_fields:
        return f, g, dict(zip(FIELD_NAMES, fields.reshape(8, n)))
    return f, g


def lb_fields(p: Params, stage: int, c1, f, g, S=None):
    """Macroscopic fields at the current time level (dict of N-vectors)."""
    n = _n(p)
    f, g = _f64(f), _f64(g)
    c1a = _f64(c1 if c1 is not None else np.zeros(n)).ravel()
    Sa = None if S is None else np.ascontiguousarray(S, dtype=np.uint8).ravel()
    fields = np.zeros(8 * n)
    _load().or_lb_fields(C.byref(p), stage, _b(Sa), _d(c1a), _d(f), _d(g), _d(fields))
    return dict(zip(FIELD_NAMES, fields.reshape(8, n)))


def relax_solid(p: Params, S, c1, steps: int, beta: float, omega: float):
    """Stage-1 relaxation (Sec. II.B, solid initialisation): from C1 at rest,
    `steps` LB steps with confinement to the region S at strength beta and
    range penalty omega; returns the relaxed C1."""
    q = Params.from_buffer_copy(p)
    q.beta, q.omega = beta, omega
    S = np.ascontiguousarray(S, dtype=np.uint8).ravel()
    f, g = lb_init(q, 1, None, c1, S=S)
    f, g = lb_run(q, 1, None, f, g, steps, S=S)
    return lb_fields(q, 1, None, f, g, S=S)["C"]


def solid_two_step(p: Params, S, c1, steps1, beta1, omega1, steps2, beta2, omega2):
    """Two-step solid initialisation for sharp corners (Sec. II.B, after
    Eq. [frozen:poly-quadratic_lbm]): a short relaxation with larger beta and
    Omega, the region redefined as S := {C1 > 1/2}, then a further relaxation
    with the new S (from the relaxed C1, at rest).  Returns (C1, new S)."""
    c1a = relax_solid(p, S, c1, steps1, beta1, omega1)
    S2 = (c1a > 0.5).astype(np.uint8)
    return relax_solid(p, S2, c1a, steps2, beta2, omega2), S2


def energy_grad(p: Params, c1, c2, *, active=2, S=None, dP=0.0, kcs=0.0, V0=0.0, fg=0.0,
                want_grad=True):
    """Discrete free energy E, its gradient w.r.t. the active field, and the terms
    (bulk, gradient, confinement, constraint, gravity, V)."""
    n = _n(p)
    c1, c2 = _f64(c1).ravel(), _f64(c2).ravel()
    Sa = np.zeros(n, np.uint8) if S is None else np.ascontiguousarray(S, dtype=np.uint8).ravel()
    grad = np.empty(n) if want_grad else None
    terms = np.zeros(6)
    E = _load().or_energy_grad(C.byref(p), _d(c1), _d(c2), _b(Sa), active, dP, kcs, V0, fg,
                               None if grad is None else _d(grad), _d(terms))
    return E, grad, terms


def observables(p: Params, c1, f, g):
    out = np.zeros(6)
    _load().or_observables(C.byref(p), _d(_f64(c1).ravel()), _d(_f64(f)), _d(_f64(g)), _d(out))
    return dict(mass_c2=out[0], mass_c1=out[1], kinetic=out[2], max_u=out[3],
                nonfinite=int(out[4]), free_energy=out[5])
