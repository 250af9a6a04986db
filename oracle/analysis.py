"""Oracle analysis of fields -- TEST INFRASTRUCTURE ONLY.

Contact angle by a circle (sphere) fit of the liquid/gas interface, as the
paper measures it (Sec. III.A: fit the C2 = 1/2 line to a circle and read the
angle where it meets the solid; the distortion at the contact line is left
out).  Reading: interface points come from linear interpolation along grid
lines, points within 3 alpha of the wall are dropped, the fit is Kasa's
algebraic least-squares circle (Kasa 1976), and theta = arccos(-(y_c - y_w)/R)
with y_w the C1 = 1/2 wall plane.
"""
from __future__ import annotations

import math

import numpy as np


def iso_points(field: np.ndarray, level: float = 0.5) -> np.ndarray:
    """Points where `field` crosses `level` along grid lines (linear
    interpolation).  field has shape (ny, nx) or (nz, ny, nx); returns (k, d)
    coordinates ordered (x, y[, z])."""
    pts = []
    d = field.ndim
    for ax in range(d):
        a = np.moveaxis(field, ax, -1)
        v0, v1 = a[..., :-1] - level, a[..., 1:] - level
        hit = (v0 * v1 < 0.0)
        idx = np.nonzero(hit)
        t = v0[idx] / (v0[idx] - v1[idx])
        coords = [np.asarray(i, dtype=np.float64) for i in idx]
        coords[-1] = coords[-1] + t
        # coords are in the moved-axis order; move the last back to position ax
        order = list(range(d))
        order.remove(ax)
        full = [None] * d
        for k, o in enumerate(order):
            full[o] = coords[k]
        full[ax] = coords[-1]
        # array axes are (z, y, x) / (y, x): reverse to (x, y, z)
        pts.append(np.stack(full[::-1], axis=1))
    return np.concatenate(pts, axis=0) if pts else np.zeros((0, d))


def kasa_fit(pts: np.ndarray):
    """Algebraic least-squares circle / sphere: |p|^2 + D.p + F = 0."""
    A = np.concatenate([pts, np.ones((pts.shape[0], 1))], axis=1)
    b = -np.sum(pts * pts, axis=1)
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    centre = -0.5 * sol[:-1]
    R = math.sqrt(float(np.dot(centre, centre) - sol[-1]))
    return centre, R


def wall_plane(c1: np.ndarray, axis_from_end: int = 0) -> float:
    """Height of the C1 = 1/2 plane of a flat wall at the bottom of the last
    array axis' normal (y in 2D, z in 3D), from a column far from anything."""
    col = c1.reshape(c1.shape[0], -1)[:, 0] if c1.ndim == 2 else c1[:, 0, 0]
    for k in range(col.size - 1):
        if col[k] >= 0.5 > col[k + 1]:
            return k + (col[k] - 0.5) / (col[k] - col[k + 1])
    raise ValueError("no C1 = 1/2 crossing")


def contact_angle_flat(c2: np.ndarray, c1: np.ndarray, alpha: float = 1.0,
                       margin: float = 3.0) -> float:
    """Contact angle (degrees) of a drop on a flat wall normal to the last
    coordinate (y in 2D, z in 3D)."""
    yw = wall_plane(c1)
    pts = iso_points(c2, 0.5)
    h = pts[:, -1]
    keep = h > yw + margin * alpha
    pts = pts[keep]
    centre, R = kasa_fit(pts)
    cos_t = -(centre[-1] - yw) / R
    cos_t = max(-1.0, min(1.0, cos_t))
    return math.degrees(math.acos(cos_t))


def young_angle(kappa2: float, kappa3: float) -> float:
    """Young's angle cos(theta) = (k3 - k2)/(k2 + k3) (Sec. II.B, Eq. [eqn:st_ca])."""
    return math.degrees(math.acos((kappa3 - kappa2) / (kappa2 + kappa3)))


def width_10_90(profile: np.ndarray) -> float:
    """10-90 % span of a monotone profile sampled at unit spacing (linear interp.)."""
    p = np.asarray(profile, dtype=np.float64)
    if p[0] > p[-1]:
        p = p[::-1]

    def cross(level):
        for k in range(p.size - 1):
            if p[k] <= level < p[k + 1]:
                return k + (level - p[k]) / (p[k + 1] - p[k])
        raise ValueError("level not crossed")
    return cross(0.9) - cross(0.1)


def sample_bilinear(field: np.ndarray, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """Bilinear interpolation of a (ny, nx) field at points (px, py), node
    coordinates, clamped to the lattice."""
    ny, nx = field.shape
    px = np.clip(px, 0.0, nx - 1.0)
    py = np.clip(py, 0.0, ny - 1.0)
    x0 = np.minimum(np.floor(px).astype(int), nx - 2)
    y0 = np.minimum(np.floor(py).astype(int), ny - 2)
    fx, fy = px - x0, py - y0
    f00, f10 = field[y0, x0], field[y0, x0 + 1]
    f01, f11 = field[y0 + 1, x0], field[y0 + 1, x0 + 1]
    return (1 - fy) * ((1 - fx) * f00 + fx * f10) + fy * ((1 - fx) * f01 + fx * f11)


def meniscus_position(c2: np.ndarray, entrance, direction, length: float, ds: float = 0.25,
                      start: float = -5.0) -> float:
    """Distance along a channel's axis, from its entrance, of the liquid front:
    the first point past `start` where C2 along the axis drops below 1/2
    (bilinear interpolation of the field, linear between samples).  Returns
    `length` when the channel is full, `start` when it is empty."""
    s = np.arange(start, length + ds / 2, ds)
    v = sample_bilinear(c2, entrance[0] + s * direction[0], entrance[1] + s * direction[1])
    below = np.flatnonzero(v < 0.5)
    if below.size == 0:
        return float(length)
    k = below[0]
    if k == 0:
        return float(start)
    return float(s[k - 1] + ds * (v[k - 1] - 0.5) / (v[k - 1] - v[k]))


def lucas_washburn_fit(t: np.ndarray, L: np.ndarray):
    """Least-squares fit of L = L0 + k sqrt(t - t0) (Sec. IV, Eq. [eqn:cfilling],
    t0 and L0 the constants of the initial entry).  For each t0 the model is
    linear in (L0, k); t0 is found by a bounded scalar search below the first
    sample.  Returns (k, L0, t0, rms residual)."""
    from scipy.optimize import minimize_scalar
    t = np.asarray(t, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)

    def solve(t0):
        A = np.stack([np.ones_like(t), np.sqrt(t - t0)], axis=1)
        coef, *_ = np.linalg.lstsq(A, L, rcond=None)
        r = A @ coef - L
        return coef, float(np.sqrt(np.mean(r * r)))

    span = t[-1] - t[0]
    res = minimize_scalar(lambda t0: solve(t0)[1], bounds=(t[0] - 10.0 * span, t[0] - 1e-9),
                          method="bounded", options={"xatol": 1e-6 * span})
    (L0, k), rms = solve(res.x)
    return float(k), float(L0), float(res.x), rms


def washburn_angle(k: float, gamma: float, H: float, eta: float) -> float:
    """Contact angle (degrees) that makes the Lucas-Washburn prefactor
    sqrt(gamma H cos(theta) / (3 eta)) equal to k."""
    c = 3.0 * eta * k * k / (gamma * H)
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))
