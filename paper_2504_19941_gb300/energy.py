"""Phase-field energy minimisation on the GPU (Sec. II.A of the paper).

``FreeEnergy`` evaluates the discrete free energy and its gradient with
``dsm_fe_energy_grad`` (FP32 fields, FP64 energy).  ``Energy`` exposes it to
autograd: the forward pass returns E and keeps the hand-written adjoint dE/dC,
the backward pass scales it by the incoming gradient (``dsm_vec_axpy_dev``).
``lbfgs`` minimises E over one component with the library's native L-BFGS loop
(``dsm_lbfgs_minimize``: the compact form of the L-BFGS matrix, a strong-Wolfe
line search, FP64 dot products; its readings are stated in ``include/dsm.h``).
"""
from __future__ import annotations

import torch

from . import _lib
from ._lib import dsm_params


class FreeEnergy:
    """Energy + gradient of one grid (shape and material fixed by ``params``)."""

    def __init__(self, params: dsm_params, device="cuda", stream=None):
        self.params = params
        self.device = _lib.cuda_device(device)
        self.stream = stream
        self.n = params.nx * params.ny * params.nz
        self.sb = _lib.dsm_fe_scratch_bytes(params.lattice, params.nx, params.ny, params.nz)
        self.scratch = torch.empty(self.sb, dtype=torch.uint8, device=self.device)
        self.terms = torch.zeros(6, dtype=torch.float64, device=self.device)

    def __call__(self, c1, c2, *, active=2, mask=None, dP=0.0, kcs=0.0, V0=0.0, fg=0.0,
                 energy=None, grad=None):
        """Returns (E as a 1-element float64 device tensor, gradient w.r.t. the
        active field as a float32 device tensor)."""
        if energy is None:
            energy = torch.empty(1, dtype=torch.float64, device=self.device)
        if grad is None:
            grad = torch.empty(self.n, dtype=torch.float32, device=self.device)
        arg = _lib.tensor_arg
        c1 = arg(c1, self.n, torch.float32, self.device, "c1", copy=True)
        c2 = arg(c2, self.n, torch.float32, self.device, "c2", copy=True)
        if mask is not None:
            mask = arg(mask, self.n, None, self.device, "mask", copy=True, itemsize=1)
        energy = arg(energy, 1, torch.float64, self.device, "energy")
        grad = arg(grad, self.n, torch.float32, self.device, "grad")
        _lib.dsm_fe_energy_grad(self.params, c1, c2, mask, active, dP, kcs, V0, fg, energy, grad,
                                self.terms, self.scratch, self.sb, self.stream)
        return energy, grad


    def decomposition(self) -> dict:
        """The last evaluation's energy by term (Sec. III.B reports the surface
        and gravitational parts of capillary rise): surface = bulk + gradient
        (the interfacial energy of every component pair), confinement,
        constraint (pressure or volume term), gravity, and the liquid volume V."""
        t = self.terms.cpu().tolist()
        return {"surface": t[0] + t[1], "bulk": t[0], "gradient": t[1], "confinement": t[2],
                "constraint": t[3], "gravity": t[4], "volume": t[5]}


class Energy(torch.autograd.Function):
    """E(C) with the hand-written adjoint.  Differentiable in the active field."""

    @staticmethod
    def forward(ctx, c_active, c_other, fe: FreeEnergy, active: int = 2, mask=None, dP=0.0,
                kcs=0.0, V0=0.0, fg=0.0):
        c1, c2 = (c_other, c_active) if active == 2 else (c_active, c_other)
        E, grad = fe(c1.detach().contiguous(), c2.detach().contiguous(), active=active,
                     mask=mask, dP=dP, kcs=kcs, V0=V0, fg=fg)
        ctx.save_for_backward(grad)
        ctx.fe = fe
        return E.reshape(())

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        out = torch.empty_like(grad)
        n = grad.numel()
        go = gout.detach().to(torch.float64).reshape(1).contiguous()
        _lib.dsm_vec_axpby(n, 0.0, grad, 0.0, out, ctx.fe.stream)          # out = 0
        _lib.dsm_vec_axpy_dev(n, 1.0, go, None, grad, out, ctx.fe.stream)  # out += gout grad
        return out, None, None, None, None, None, None, None, None


class _Vec:
    """Device vector helpers over libdsm (no torch arithmetic)."""

    def __init__(self, n, device, stream):
        self.n = n
        self.device = device
        self.stream = stream
        self.sb = _lib.dsm_vec_scratch_bytes(n)
        self.scratch = torch.empty(self.sb, dtype=torch.uint8, device=device)
        self.out = torch.zeros(4, dtype=torch.float64, device=device)

    def dot(self, x, y, slot=0):
        _lib.dsm_vec_dot(self.n, x, y, self.out[slot:slot + 1], self.scratch, self.sb, self.stream)
        return self.out[slot:slot + 1]

    def axpby(self, a, x, b, y):
        _lib.dsm_vec_axpby(self.n, a, x, b, y, self.stream)


def lbfgs(fe: FreeEnergy, x0, other, *, active=2, mask=None, dP=0.0, kcs=0.0, V0=0.0, fg=0.0,
          m=10, tol=1e-6, max_iter=10000):
    """Minimise E over the active field from x0 (FP32 device vector, not
    modified) with the library's native L-BFGS loop (dsm_lbfgs_minimize).  Stops
    when sqrt(mean(grad^2)) < tol.  Returns (x, E, info)."""
    n = fe.n
    x = _lib.tensor_arg(x0, n, torch.float32, fe.device, "x0", copy=True).detach().clone()
    other = _lib.tensor_arg(other, n, torch.float32, fe.device, "other", copy=True)
    if mask is not None:
        mask = _lib.tensor_arg(mask, n, None, fe.device, "mask", copy=True, itemsize=1)
    nb = _lib.dsm_lbfgs_workspace_bytes(fe.params, m)
    work = torch.empty(nb, dtype=torch.uint8, device=x.device)
    info = _lib.dsm_lbfgs_minimize(fe.params, other, mask, active, dP, kcs, V0, fg, x, m, tol,
                                   max_iter, work, nb, fe.stream)
    return x, info["energy"], info


class FreeEnergyMulti:
    """Energy + gradients of N fluid components on a frozen solid
    (dsm_fe_energy_grad_multi): kappa holds kappa_1 .. kappa_{N+1}; the free
    fluids C_2 .. C_N are the N - 1 planes of one (N - 1, nodes) FP32 tensor."""

    def __init__(self, params: dsm_params, nfluid: int, kappa, device="cuda", stream=None):
        self.params = params
        self.nfluid = int(nfluid)
        self.kappa = [float(k) for k in kappa]
        self.device = _lib.cuda_device(device)
        self.stream = stream
        self.n = params.nx * params.ny * params.nz
        self.sb = _lib.dsm_fe_multi_scratch_bytes(params.lattice, params.nx, params.ny,
                                                  params.nz, self.nfluid)
        self.scratch = torch.empty(self.sb, dtype=torch.uint8, device=self.device)
        self.terms = torch.zeros(2 + self.nfluid, dtype=torch.float64, device=self.device)

    def __call__(self, c1, c, *, dP=None, kcs=None, V0=None, energy=None, grad=None):
        """Returns (E as a 1-element float64 device tensor, gradients as an
        (N - 1, nodes) float32 device tensor)."""
        if energy is None:
            energy = torch.empty(1, dtype=torch.float64, device=self.device)
        if grad is None:
            grad = torch.empty((self.nfluid - 1, self.n), dtype=torch.float32, device=self.device)
        arg, nf = _lib.tensor_arg, self.nfluid - 1
        c1 = arg(c1, self.n, torch.float32, self.device, "c1", copy=True)
        c = arg(c, nf * self.n, torch.float32, self.device, "c", copy=True)
        energy = arg(energy, 1, torch.float64, self.device, "energy")
        grad = arg(grad, nf * self.n, torch.float32, self.device, "grad")
        _lib.dsm_fe_energy_grad_multi(self.params, self.nfluid, self.kappa, c1, c, dP, kcs, V0,
                                      energy, grad, self.terms, self.scratch, self.sb,
                                      self.stream)
        return energy, grad


def lbfgs_multi(fe: FreeEnergyMulti, x0, c1, *, dP=None, kcs=None, V0=None, m=10, tol=1e-6,
                max_iter=10000):
    """Minimise the N-fluid energy over the free fluid planes from x0 ((N - 1,
    nodes) FP32, not modified) with the native L-BFGS loop.  Returns (x, E, info)."""
    nf = fe.nfluid - 1
    x = _lib.tensor_arg(x0, nf * fe.n, torch.float32, fe.device, "x0", copy=True).detach().clone()
    c1 = _lib.tensor_arg(c1, fe.n, torch.float32, fe.device, "c1", copy=True)
    nb = _lib.dsm_lbfgs_multi_workspace_bytes(fe.params, fe.nfluid, m)
    work = torch.empty(nb, dtype=torch.uint8, device=x.device)
    info = _lib.dsm_lbfgs_minimize_multi(fe.params, fe.nfluid, fe.kappa, c1, dP, kcs, V0, x, m,
                                         tol, max_iter, work, nb, fe.stream)
    return x, info["energy"], info
