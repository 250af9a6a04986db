"""Wetting observables of a lattice: the apparent contact angle of a drop.

The paper measures contact angles by fitting a circle (a sphere in 3D) to the
C2 = 1/2 level of the liquid-gas interface away from the solid and reading the
angle where the fit meets the wall (Sec. III.A, Liquid Contact Angle).  On a
rough surface (pillars, a sinusoidal wall, a packing of spheres) the angle
read against the plane through the top of the roughness is the apparent
angle of the drop.  Here:
  * the liquid fraction C2/(1 - C1) is sampled where it crosses 1/2 along grid
    lines (linear interpolation between the two nodes);
  * points within `margin` nodes of the top of the solid are left out (the
    interface bends into the wall there);
  * Kasa's algebraic least-squares circle/sphere, |p|^2 + D.p + F = 0;
  * theta = arccos(-(c_h - h_w)/R), h_w the height of the topmost C1 = 1/2
    crossing along the last axis (y in 2D, z in 3D).
Host code (numpy) run on fields the library returns.
"""
from __future__ import annotations

import math

import numpy as np


def level_points(field: np.ndarray, level: float = 0.5):
    """Crossings of `level` along the grid lines of every axis.  field: (ny, nx)
    or (nz, ny, nx).  Returns (points (k, d) in (x, y[, z]) order, index of
    the node of each crossing nearer to it (as a flat array index))."""
    d = field.ndim
    pts, near = [], []
    shape = field.shape
    for ax in range(d):
        lo = np.take(field, np.arange(shape[ax] - 1), axis=ax) - level
        hi = np.take(field, np.arange(1, shape[ax]), axis=ax) - level
        hit = lo * hi < 0.0
        idx = np.nonzero(hit)
        t = lo[idx] / (lo[idx] - hi[idx])
        coord = [i.astype(np.float64) for i in idx]
        coord[ax] = coord[ax] + t
        pts.append(np.stack(coord[::-1], axis=1))       # array order -> (x, y[, z])
        nidx = list(idx)
        nidx[ax] = idx[ax] + (t > 0.5)
        near.append(np.ravel_multi_index(tuple(nidx), shape))
    if not pts:
        return np.zeros((0, d)), np.zeros(0, dtype=np.int64)
    return np.concatenate(pts), np.concatenate(near)


def sphere_fit(pts: np.ndarray):
    """Algebraic least-squares circle / sphere through points (k, d): centre, R."""
    A = np.concatenate([pts, np.ones((pts.shape[0], 1))], axis=1)
    rhs = -np.einsum("ij,ij->i", pts, pts)
    sol, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    centre = -0.5 * sol[:-1]
    r2 = float(centre @ centre - sol[-1])
    return centre, math.sqrt(max(r2, 0.0))


def roughness_top(c1: np.ndarray) -> float:
    """Height (along the last coordinate) of the topmost C1 = 1/2 crossing."""
    col = c1.reshape(c1.shape[0], -1)                    # (nh, columns)
    solid = col >= 0.5
    rows = np.nonzero(solid.any(axis=1))[0]
    if rows.size == 0:
        return math.nan
    k = int(rows.max())
    if k + 1 >= col.shape[0]:
        return float(k)
    a = col[k][solid[k]]
    b = col[k + 1][solid[k]]
    frac = np.where(a > b, (a - 0.5) / np.where(a > b, a - b, 1.0), 0.0)
    return float(k + frac.max())


def apparent_contact_angle(c2: np.ndarray, c1: np.ndarray, margin: float = 3.0) -> float:
    """Apparent contact angle (degrees) of the drop in c2 on the solid c1 (both
    (ny, nx) or (nz, ny, nx)); nan when too few interface points remain."""
    den = 1.0 - c1
    phi = np.where(den > 1e-6, c2 / np.where(den > 1e-6, den, 1.0), 0.0)
    hw = roughness_top(c1)
    if not math.isfinite(hw):
        return math.nan
    pts, _ = level_points(phi, 0.5)
    pts = pts[pts[:, -1] > hw + margin]
    if pts.shape[0] < 4 * pts.shape[1]:
        return math.nan
    centre, R = sphere_fit(pts)
    if not R > 0.0:
        return math.nan
    cos_t = max(-1.0, min(1.0, -(centre[-1] - hw) / R))
    return math.degrees(math.acos(cos_t))
