"""Critical pressure of a liquid slab on a micropillar array under a body-force
ramp (the lattice Boltzmann counterpart of Sec. III, Critical Pressure on
Micropillared Surfaces, Eq. [frozen:critical-pressure-cyl-2d]; the body force
on the liquid of Sec. IV).

The liquid slab rests on the pillar tops (the suspended state) with gas in the
gaps below.  A body force on the liquid along -z, F_g = C2 f, grows linearly
from 0 to f_max over the ramp; on a slab of thickness H it presses with
dP = f H.  The slab stays pinned at the pillar edges until the meniscus in the
gaps reaches the advancing angle, then the contact line slides down the pillar
sides.

Reading: the gas in the gaps is sealed by the slab and, in this pseudo-
incompressible scheme, keeps its volume, so the mean interface height over a
whole gap cannot fall; the depinning shows at the contact line.  The detector
therefore watches the C2 = 1/2 height (of the liquid fraction C2/(1 - C1))
over the ring of gap columns next to the pillar sides, and the ramp's force
when that mean first falls `drop` nodes below the pillar tops is the critical
force (z_top - drop = 36 for pillars topping out at 38).

The detector gathers the ring columns of the liquid field the library returns
on the device and reads them on the host; every lattice Boltzmann step runs in
libdsm.
"""
from __future__ import annotations

import numpy as np

from . import Lattice


def pillar_ring(c1_plane: np.ndarray, width: int = 1) -> np.ndarray:
    """Gap columns within `width` nodes (in x and y, periodic) of a pillar,
    from a z plane of C1 through the pillars (ny, nx): the columns a pillar's
    contact line passes through."""
    solid = c1_plane >= 0.5
    near = np.zeros_like(solid)
    for dy in range(-width, width + 1):
        for dx in range(-width, width + 1):
            near |= np.roll(np.roll(solid, dy, axis=0), dx, axis=1)
    return near & ~solid


def column_heights(phi_cols: np.ndarray, z_start: int, z_floor: int = 0) -> np.ndarray:
    """Height of the C2 = 1/2 level in each column of the liquid fraction
    phi_cols (nz, ncols): scanning down from z_start (inside the slab) to the
    first node below 1/2, interpolated linearly between it and the node above;
    a column liquid all the way down to z_floor gives z_floor."""
    seg = phi_cols[z_floor:z_start + 1][::-1]        # rows: z_start, z_start - 1, ...
    below = seg < 0.5
    any_below = below.any(axis=0)
    j = np.where(any_below, below.argmax(axis=0), 0)
    z = z_start - j                                   # first node below 1/2
    h = np.full(phi_cols.shape[1], float(z_floor))
    top = any_below & (z >= z_start)
    h[top] = z_start
    mid = any_below & (z < z_start)
    k = np.nonzero(mid)[0]
    a = phi_cols[z[k], k]
    b = phi_cols[z[k] + 1, k]
    h[k] = z[k] + (0.5 - a) / (b - a)
    return h


def liquid_fraction(c2, c1):
    den = 1.0 - c1
    return np.where(den > 1e-6, c2 / np.where(den > 1e-6, den, 1.0), 0.0)


def interface_height(c2: np.ndarray, c1: np.ndarray, cols: np.ndarray, z_start: int,
                     z_floor: int = 0) -> float:
    """Mean height of the C2 = 1/2 level of the liquid fraction C2/(1 - C1)
    over the selected columns (cols: (ny, nx) bool) of c2, c1 (nz, ny, nx):
    see column_heights."""
    phi = liquid_fraction(c2[:, cols], c1[:, cols])
    return float(column_heights(phi, z_start, z_floor).mean())


def pressure_ramp(lat: Lattice, f_max: float, ramp_steps: int, c1: np.ndarray,
                  ring: np.ndarray, z_top: int, thickness: float, *, check_every: int = 100,
                  drop: float = 2.0, stop_at_depinning: bool = True, axis: int = 2):
    """Ramp the body force on the liquid along -axis linearly from 0 to f_max
    over ramp_steps steps (the force of step s is f_max s / ramp_steps, set
    before each step), checking the contact-line height every check_every
    steps.  c1: (nz, ny, nx) solid; ring: (ny, nx) columns next to the
    pillars; z_top: first node above the pillars.  Returns a dict with the
    critical force and pressure (None if the slab stayed pinned), the steps
    taken and the history (step, force, height).  Each check reads the liquid
    field once and copies only the ring columns up to the middle of the slab
    to the host."""
    import torch
    hist = []
    f_crit = None
    t = 0
    nz, ny, nx = c1.shape
    z_start = min(z_top + int(thickness) // 2, nz - 1)
    idx = torch.as_tensor(np.flatnonzero(ring.ravel()), device=lat.device)
    c1_cols = c1[: z_start + 1].reshape(z_start + 1, -1)[:, ring.ravel()]
    buf = torch.empty(lat.n, dtype=lat.real, device=lat.device)
    while t < ramp_steps:
        n = min(check_every, ramp_steps - t)
        for k in range(n):
            body = [0.0, 0.0, 0.0]
            body[axis] = -f_max * (t + k + 1) / ramp_steps
            lat.set_body_force(body)
            lat.step(1)
        t += n
        lat.field("C2", out=buf)
        cols = buf.view(nz, ny * nx)[: z_start + 1].index_select(1, idx)
        c2_cols = cols.double().cpu().numpy()
        h = float(column_heights(liquid_fraction(c2_cols, c1_cols), z_start).mean())
        hist.append((t, f_max * t / ramp_steps, h))
        if f_crit is None and h < z_top - drop:
            f_crit = f_max * t / ramp_steps
            if stop_at_depinning:
                break
    return {"f_crit": f_crit, "dp_crit": None if f_crit is None else f_crit * thickness,
            "steps": t, "history": hist}
