"""Helpers shared by the GPU parity tests: run the same seeded case through the
CUDA library and through the FP64 oracle, and compare.

Parity metric (per field): max |a - b| / max |b|, because velocities and most
populations are near zero in the bulk."""
from __future__ import annotations

import numpy as np

import oracle as O
import synthetic as S


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def direction_map(kind: int):
    """perm[i_gpu] = i_oracle with equal velocity vectors."""
    from paper_2504_19941_gb300 import _lib
    cg, _ = _lib.dsm_lattice_table(kind)
    co, _ = O.lattice(kind)
    perm = []
    for c in cg:
        hits = [j for j in range(len(co)) if tuple(co[j]) == tuple(c)]
        assert len(hits) == 1
        perm.append(hits[0])
    return np.array(perm)


def oracle_params(case: S.Case, kind: int):
    k, rc = O.kappa_from_angle(case.theta_deg, case.g23, case.g12, case.alpha)
    assert rc == 0
    return O.make_params(kind, case.shape, k, alpha=case.alpha, alpha_s=case.alpha_s,
                         rho2=case.rho2, rho3=case.rho3, tau2=case.tau2, tau3=case.tau3,
                         tau_g=case.tau_g, body=case.body, faces=case.faces)


def gpu_lattice(case: S.Case, precision: str, device="cuda", g_storage="auto"):
    import torch
    import paper_2504_19941_gb300 as P
    p = P.make_params(case.lattice, case.shape, precision, theta_deg=case.theta_deg, g12=case.g12,
                      g23=case.g23, alpha=case.alpha, alpha_s=case.alpha_s, rho2=case.rho2,
                      rho3=case.rho3, tau2=case.tau2, tau3=case.tau3, tau_g=case.tau_g,
                      body=case.body, faces=case.faces)
    lat = P.Lattice(p, device=device)
    lat.set_g_storage(g_storage)
    real = lat.real
    lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=real, device=device))
    lat.set_fluid(torch.as_tensor(case.c2, dtype=real, device=device))
    return lat


FIELDS = ("C", "mu", "ux", "uy", "uz", "pt", "rho")
GPU_NAME = {"C": "C2", "mu": "mu", "ux": "ux", "uy": "uy", "uz": "uz", "pt": "pt", "rho": "rho"}


def gpu_fields(lat):
    return {k: lat.field(GPU_NAME[k]).double().cpu().numpy() for k in FIELDS}


def gpu_pops(lat, perm):
    """GPU populations reordered to the oracle's direction order (q x N)."""
    f, g = lat.populations()
    q = lat.q
    f = f.double().cpu().numpy().reshape(q, -1)
    g = g.double().cpu().numpy().reshape(q, -1)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(q)
    return f[inv], g[inv]


def compare(gf, of, names=FIELDS):
    return {k: rel_err(gf[k], of[k]) for k in names}


# ---- N fluids (dsm_ml_*) against oracle/multi_lb.py
def ml_run(case, prec, steps, tau_g=0.9, form="auto", zrun=0):
    """One N-fluid case through MultiLattice and through the oracle's MultiLB.
    case: (shape, c1, C (free fluids), kappa, rho, tau, faces, body)."""
    import torch
    import paper_2504_19941_gb300 as P
    from oracle.multi_lb import MultiLB
    shape, c1, C, kappa, rho, tau, faces, body = case
    nf = C.shape[0]
    lat = "D2Q9" if len(shape) == 2 else "D3Q19"
    kind = O.D2Q9 if lat == "D2Q9" else O.D3Q19
    real = torch.float64 if prec == "f64" else torch.float32

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=real, device="cuda")
    p = P.make_params(lat, shape, prec, theta_deg=90.0, tau_g=tau_g, body=body, faces=faces,
                      alpha_s=1.0)
    ml = P.MultiLattice(p, nf + 1, kappa, rho, tau)
    ml.set_step_form(form, zrun)
    ml.set_solid_c1(t(c1))
    ml.set_fluids(t(C))
    ml.step(steps)
    po = O.make_params(kind, shape, kappa[:3], tau_g=tau_g, body=body, faces=faces, alpha_s=1.0)
    c1r = t(c1).double().cpu().numpy()
    m = MultiLB(po, kappa, rho, tau, c1r)
    f, g = m.init(t(C).double().cpu().numpy())
    f, g = m.run(f, g, steps)
    return ml, m, f, g, kind


def ml_compare(ml, m, f, g, kind, speed_scale=False):
    """Per-quantity errors of an N-fluid lattice against the oracle's state.
    Velocity components: against their own maximum, or (speed_scale, or a
    component zero by symmetry) against the maximum speed of all three."""
    perm = direction_map(kind)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    fg_, gg_ = ml.populations()
    q, n, nf = ml.q, ml.n, ml.nfluid - 1
    gf = fg_.double().cpu().numpy().reshape(q, n)[inv]
    gg = gg_.double().cpu().numpy().reshape(nf, q, n)[:, inv]
    errs = {"f": rel_err(gf, f), "g": rel_err(gg, g)}
    F = m.fields(f, g)
    for k in range(nf):
        errs[f"C{k}"] = rel_err(ml.field("C", k).double().cpu().numpy(), F["C"][k])
        errs[f"mu{k}"] = rel_err(ml.field("mu", k).double().cpu().numpy(), F["mu"][k])
    umax = np.abs(F["u"]).max()
    for a, name in enumerate(("ux", "uy", "uz")):
        got = ml.field(name).double().cpu().numpy()
        if not speed_scale and np.abs(F["u"][a]).max() > 1e-9 * umax:
            errs[name] = rel_err(got, F["u"][a])
        else:  # zero by symmetry up to rounding: compare against max |u|
            errs[name] = np.abs(got - F["u"][a]).max() / max(umax, 1e-300)
    errs["pt"] = rel_err(ml.field("pt").double().cpu().numpy(), F["pt"])
    errs["rho"] = rel_err(ml.field("rho").double().cpu().numpy(), F["rho"])
    errs["tau"] = rel_err(ml.field("tau").double().cpu().numpy(), F["tau"])
    return errs
