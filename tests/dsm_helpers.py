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
