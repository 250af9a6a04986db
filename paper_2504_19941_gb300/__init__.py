"""GB300-native Diffuse Solid Method: lattice Boltzmann step and free-energy twin.

The compute path is libdsm.so (hand-written CUDA for sm_103a, C ABI in
include/dsm.h).  This package only marshals arguments: ``_lib`` mirrors the C
entry points under the same names, ``Lattice`` owns a torch workspace tensor
for one lattice, ``energy`` holds the autograd function and the L-BFGS driver
of the energy minimisation, ``serving`` the request loop.  Importing the
package loads libdsm.so and fails loudly if it has not been built.
"""
from __future__ import annotations

from . import _lib
from ._lib import (DSM_BF16_STORE, DSM_D2Q9, DSM_D3Q19, DSM_F16_STORE, DSM_F32, DSM_F64,  # noqa
                   DSM_FIELD_C1, DSM_FIELD_C2, DSM_FIELD_C3, DSM_FIELD_MU, DSM_FIELD_PT,
                   DSM_FIELD_RHO, DSM_FIELD_TAU, DSM_FIELD_UX, DSM_FIELD_UY, DSM_FIELD_UZ,
                   DSM_FACE_MIRROR, DSM_FACE_PERIODIC, DSM_FACE_WALL, DSMError, dsm_params)

_lib.load()

PRECISIONS = {"f64": DSM_F64, "f32": DSM_F32, "bf16": DSM_BF16_STORE, "f16": DSM_F16_STORE}
LATTICES = {"D2Q9": DSM_D2Q9, "D3Q19": DSM_D3Q19}
FACES = {"periodic": DSM_FACE_PERIODIC, "mirror": DSM_FACE_MIRROR, "wall": DSM_FACE_WALL}
FIELDS = {"C1": DSM_FIELD_C1, "C2": DSM_FIELD_C2, "C3": DSM_FIELD_C3, "mu": DSM_FIELD_MU,
          "ux": DSM_FIELD_UX, "uy": DSM_FIELD_UY, "uz": DSM_FIELD_UZ, "pt": DSM_FIELD_PT,
          "rho": DSM_FIELD_RHO, "tau": DSM_FIELD_TAU}


def make_params(lattice: str, shape, precision: str = "f32", *, theta_deg=None, g12=2.5e-3,
                g13=None, g23=2.5e-3, alpha=1.0, alpha_s=0.0, rho2=1.0, rho3=1.0, tau2=1.0,
                tau3=1.0, tau_g=1.0, body=(0.0, 0.0, 0.0), beta=0.0, omega=0.0,
                faces=None) -> dsm_params:
    """dsm_params from keyword arguments.  Give either theta_deg (with g23, g12)
    or the three tensions g12, g13, g23.  faces: the boundary of the faces x-,
    x+, y-, y+, z-, z+, each "periodic", "mirror" (symmetry plane) or "wall"
    (halfway bounce-back); None: all periodic."""
    p = dsm_params()
    p.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    p.nx, p.ny = int(shape[0]), int(shape[1])
    p.nz = int(shape[2]) if len(shape) > 2 else 1
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.alpha, p.alpha_s = alpha, alpha_s
    if theta_deg is not None:
        p.tension_mode, p.theta_deg = 1, float(theta_deg)
    else:
        p.tension_mode = 0
    p.g12, p.g23 = g12, g23
    p.g13 = 0.0 if g13 is None else g13
    p.rho2, p.rho3, p.tau2, p.tau3, p.tau_g = rho2, rho3, tau2, tau3, tau_g
    for a in range(3):
        p.body_force[a] = float(body[a])
    p.beta, p.omega = beta, omega
    if faces is not None:
        if len(faces) != 6:
            raise ValueError("faces: six entries, x-, x+, y-, y+, z-, z+")
        for k, f in enumerate(faces):
            p.face[k] = FACES[f] if isinstance(f, str) else int(f)
    return p


def ring_records(rows, written: int, fields) -> list:
    """The records a ring of len(rows) slots holds after `written` appends
    (record k in slot k % len(rows)), oldest first, as dicts of `fields`."""
    cap = len(rows)
    out = []
    for k in range(max(0, written - cap), written):
        r = rows[k % cap]
        out.append({name: (int(v) if name in ("step", "nonfinite") else float(v))
                    for name, v in zip(fields, r)})
    return out


class Lattice:
    """One lattice on the device: a torch workspace tensor plus a libdsm handle.

    Every method is a direct call into libdsm on this lattice's stream."""

    def __init__(self, params: dsm_params, device="cuda", stream=None):
        import torch
        self.params = params
        self.shape = (params.nx, params.ny, params.nz)
        self.n = params.nx * params.ny * params.nz
        self.q = 9 if params.lattice == DSM_D2Q9 else 19
        self.real = torch.float64 if params.precision == DSM_F64 else torch.float32
        self.device = _lib.cuda_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.nbytes = _lib.dsm_workspace_bytes(params)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.h = _lib.dsm_create(params, self.workspace, self.nbytes, self.stream)
        self.ring = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            try:
                _lib.dsm_destroy(h)
            except Exception:
                pass
            self.h = None

    def _field_arg(self, t, what="field"):
        """A contiguous tensor of nx*ny*nz reals of the lattice's type on its device."""
        return _lib.tensor_arg(t, self.n, self.real, self.device, what)

    def set_solid_distance(self, sd):
        _lib.dsm_set_solid(self.h, self._field_arg(sd), 0)

    def set_solid_c1(self, c1):
        _lib.dsm_set_solid(self.h, self._field_arg(c1), 1)

    def relax_solid(self, mask, steps: int, beta: float, omega: float):
        mask = _lib.tensor_arg(mask, self.n, None, self.device, "mask", copy=True, itemsize=1)
        _lib.dsm_relax_solid(self.h, mask, steps, beta, omega)

    def solid_region(self, out=None):
        """S = {C1 > 1/2} of the current diffuse solid, a uint8 device tensor."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        out = _lib.tensor_arg(out, self.n, None, self.device, "out", itemsize=1)
        _lib.dsm_solid_region(self.h, out)
        return out

    def relax_solid_two_step(self, mask, steps1: int, beta1: float, omega1: float, steps2: int,
                             beta2: float, omega2: float):
        """The two-step solid initialisation for sharp corners (Sec. II.B): a
        short relaxation with larger beta and Omega, S := {C1 > 1/2}, then a
        further relaxation with the new S.  Returns the new S."""
        self.relax_solid(mask, steps1, beta1, omega1)
        region = self.solid_region()
        self.relax_solid(region, steps2, beta2, omega2)
        return region

    def set_fluid(self, c2):
        _lib.dsm_set_fluid(self.h, self._field_arg(c2))

    def step(self, nsteps: int = 1):
        _lib.dsm_step(self.h, int(nsteps))

    def observables(self, check=True) -> dict:
        return _lib.dsm_get_observables(self.h, check)

    RING_FIELDS = ("step", "mass_c2", "mass_c1", "kinetic", "max_u", "nonfinite")

    def set_observables_ring(self, capacity: int, every: int):
        """Record the observables on the device after every `every`-th step
        (dsm_set_observables_ring) into a ring of `capacity` records; every=0
        turns recording off."""
        import torch
        if every == 0:
            self.ring = None
            _lib.dsm_set_observables_ring(self.h, None, 0, 0)
            return
        # written only by the library's kernels on the lattice's stream
        self.ring = torch.empty((int(capacity), len(self.RING_FIELDS)), dtype=torch.float64,
                                device=self.device)
        _lib.dsm_set_observables_ring(self.h, self.ring, capacity, every)

    def observables_ring(self) -> list:
        """The records the ring still holds, oldest first, as dicts (waits for
        the lattice's stream)."""
        written = _lib.dsm_observables_ring_count(self.h)
        if self.ring is None or written == 0:
            return []
        self.stream.synchronize()
        return ring_records(self.ring.cpu().numpy(), written, self.RING_FIELDS)

    def field(self, name: str, out=None):
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=self.real, device=self.device)
        out = self._field_arg(out, "out")
        _lib.dsm_get_field(self.h, FIELDS[name], out)
        return out

    def populations(self):
        import torch
        f = torch.empty(self.q * self.n, dtype=self.real, device=self.device)
        g = torch.empty_like(f)
        _lib.dsm_get_populations(self.h, f, g)
        return f, g

    def set_populations(self, f, g):
        f = _lib.tensor_arg(f, self.q * self.n, self.real, self.device, "f", copy=True)
        g = _lib.tensor_arg(g, self.q * self.n, self.real, self.device, "g", copy=True)
        _lib.dsm_set_populations(self.h, f, g)

    def set_g_storage(self, form: str):
        """'auto' (g held as g_eq when tau_g = 1) or 'populations'."""
        _lib.dsm_set_g_storage(self.h, {"auto": _lib.DSM_G_AUTO,
                                        "populations": _lib.DSM_G_POPULATIONS}[form])

    def set_body_force(self, body):
        """Body force on the liquid (3 components) for the following steps."""
        _lib.dsm_set_body_force(self.h, body)

    def set_step_form(self, form: str, zrun: int = 0):
        """'auto' (one pass per step where the lattice allows it) or 'two_pass';
        zrun: z planes per block of the one-pass step (0: automatic)."""
        _lib.dsm_set_step_form(self.h, {"auto": _lib.DSM_STEP_AUTO,
                                        "two_pass": _lib.DSM_STEP_TWO_PASS}[form], int(zrun))

    @property
    def single_pass(self) -> bool:
        """True when dsm_step runs the one-pass step on this lattice."""
        return _lib.dsm_step_info(self.h)[0]

    @property
    def g_implicit(self) -> bool:
        """True when the current state holds g as g_eq (A, u) rather than populations."""
        return bool(_lib.dsm_get_g_storage(self.h)[1])

    def state(self):
        """Checkpoint of the current state (a device byte tensor)."""
        import torch
        nb = _lib.dsm_state_bytes(self.h)
        buf = torch.empty(nb, dtype=torch.uint8, device=self.device)
        _lib.dsm_get_state(self.h, buf, nb)
        return buf

    def set_state(self, buf):
        import torch
        buf = _lib.tensor_arg(buf, buf.numel(), torch.uint8, self.device, "state")
        _lib.dsm_set_state(self.h, buf, buf.numel())


class MultiLattice:
    """A lattice of N = nfluid fluid components (dsm_ml_*): kappa holds
    kappa_1 .. kappa_{N+1}, rho and tau the N fluids' densities and relaxation
    times (fluids 2 .. N + 1).  The workspace is a torch tensor it owns."""

    def __init__(self, params: dsm_params, nfluid: int, kappa, rho, tau, device="cuda",
                 stream=None):
        import torch
        self.params = params
        self.nfluid = int(nfluid)
        self.n = params.nx * params.ny * params.nz
        self.q = 9 if params.lattice == DSM_D2Q9 else 19
        self.real = torch.float64 if params.precision == DSM_F64 else torch.float32
        self.device = _lib.cuda_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.nbytes = _lib.dsm_ml_workspace_bytes(params, self.nfluid)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.h = _lib.dsm_ml_create(params, self.nfluid, kappa, rho, tau, self.workspace,
                                    self.nbytes, self.stream)

    @property
    def g_implicit(self) -> bool:
        """g held as g_eq (tau_g = 1 and every face periodic)."""
        return self.params.tau_g == 1.0 and not any(self.params.face)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            _lib.dsm_ml_destroy(h)
            self.h = None

    def _arg(self, t, count, what="field"):
        return _lib.tensor_arg(t, count, self.real, self.device, what, copy=True)

    def set_solid_distance(self, sd):
        _lib.dsm_ml_set_solid(self.h, self._arg(sd, self.n), 0)

    def set_solid_c1(self, c1):
        _lib.dsm_ml_set_solid(self.h, self._arg(c1, self.n), 1)

    def set_fluids(self, c):
        """The free fluids C_2 .. C_N, an (N - 1, nodes) tensor."""
        _lib.dsm_ml_set_fluids(self.h, self._arg(c, (self.nfluid - 1) * self.n))

    def step(self, nsteps: int = 1):
        _lib.dsm_ml_step(self.h, int(nsteps))

    def set_step_form(self, form: str, zrun: int = 0):
        """'auto' (one pass per step where the lattice allows it) or 'two_pass';
        zrun: z planes per block of the one-pass step (0: automatic)."""
        _lib.dsm_ml_set_step_form(self.h, {"auto": _lib.DSM_STEP_AUTO,
                                           "two_pass": _lib.DSM_STEP_TWO_PASS}[form], int(zrun))

    @property
    def single_pass(self) -> bool:
        """True when dsm_ml_step runs the one-pass step on this lattice."""
        return _lib.dsm_ml_step_info(self.h)[0]

    def field(self, name: str, index: int = 0, out=None):
        """name as for Lattice.field; "C" with index f is C_{2+f} (index N - 1:
        the dependent fluid), "mu" with index f is mu_{2+f}."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=self.real, device=self.device)
        out = _lib.tensor_arg(out, self.n, self.real, self.device, "out")
        code = DSM_FIELD_C2 if name == "C" else FIELDS[name]
        _lib.dsm_ml_get_field(self.h, code, index, out)
        return out

    def status(self) -> int:
        """0, or the status latched on the device (DSM_E_NONFINITE;
        DSM_E_TIMEOUT when a staged plane of the one-pass step never arrived;
        DSM_E_BOUNDS when the checked library caught an index outside its
        buffer)."""
        return _lib.dsm_ml_check(self.h, check=False)

    def populations(self):
        import torch
        f = torch.empty(self.q * self.n, dtype=self.real, device=self.device)
        g = torch.empty((self.nfluid - 1) * self.q * self.n, dtype=self.real, device=self.device)
        _lib.dsm_ml_get_populations(self.h, f, g)
        return f, g
