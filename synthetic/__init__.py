"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the Diffuse Solid Method.  It produces only
what a user hands to the method: a solid-geometry field (a signed distance,
positive inside the solid region S), an initial liquid field C2, the seeded
perturbation, the material parameters (tensions or a contact angle, densities,
relaxation times, body force) and the request stream of the served workload.
Turning a signed distance into the solid order parameter C1, tensions into
kappa, and everything that follows, is done separately by the oracle and by
the CUDA library.

Array convention: node n = x + nx*(y + ny*z); numpy arrays have shape
(nz, ny, nx) in 3D and (ny, nx) in 2D and are raveled in C order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) on uint64 states."""
    with np.errstate(over="ignore"):
        z = (x + _GOLDEN).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(30))) * _M1).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * _M2).astype(np.uint64)
        return z ^ (z >> np.uint64(31))


def perturbation(seed: int, n: int, amplitude: float = 1e-3) -> np.ndarray:
    """Uniform [-amplitude, amplitude) per node from SplitMix64(seed XOR index)."""
    idx = np.arange(n, dtype=np.uint64)
    z = splitmix64(idx ^ np.uint64(seed))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return amplitude * (2.0 * u - 1.0)


def width_to_alpha(w_10_90: float) -> float:
    """Tanh width parameter whose 10-90 % rise spans w_10_90 nodes.

    For 1/2 + tanh(x / (2a))/2 the 10-90 % span is 2 a ln 9."""
    return w_10_90 / (2.0 * math.log(9.0))


# --------------------------------------------------------------------------
# coordinates and geometry (signed distance, positive inside the solid)
# --------------------------------------------------------------------------
def _coords(shape):
    """Integer node coordinates, arrays broadcast to (nz, ny, nx) or (ny, nx)."""
    if len(shape) == 2:
        nx, ny = shape
        y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        return [x.astype(np.float64), y.astype(np.float64)]
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return [x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)]


def _pdist(a, centre, length):
    """Signed minimal-image offset a - centre on a periodic axis."""
    d = a - centre
    return d - length * np.round(d / length)


def slab_sd(shape, axis: int, lo: int, hi: int) -> np.ndarray:
    """Periodic slab of solid nodes lo..hi-1 along `axis`; faces mid-way between nodes."""
    X = _coords(shape)
    length = shape[axis]
    centre = 0.5 * (lo + hi - 1)
    half = 0.5 * (hi - lo)
    return half - np.abs(_pdist(X[axis], centre, length))


def box_sd(shape, lo, hi, periodic=True) -> np.ndarray:
    """Axis-aligned box of solid nodes lo[a]..hi[a]-1 (exact box distance)."""
    X = _coords(shape)
    q = []
    for a in range(len(shape)):
        centre = 0.5 * (lo[a] + hi[a] - 1)
        half = 0.5 * (hi[a] - lo[a])
        d = _pdist(X[a], centre, shape[a]) if periodic else X[a] - centre
        q.append(np.abs(d) - half)
    q = np.stack(q)
    outside = np.sqrt(np.sum(np.maximum(q, 0.0) ** 2, axis=0))
    inside = np.minimum(np.max(q, axis=0), 0.0)
    return -(outside + inside)


def sphere_sd(shape, centre, radius) -> np.ndarray:
    X = _coords(shape)
    r2 = sum(_pdist(X[a], centre[a], shape[a]) ** 2 for a in range(len(shape)))
    return radius - np.sqrt(r2)


def sinusoid_sd(shape, base: float, amplitude: float, wavelength: float,
                along: int = 0, normal: int = -1) -> np.ndarray:
    """Wall below h(s) = base + A sin(2 pi s / wavelength): first-order normal distance."""
    X = _coords(shape)
    normal = normal % len(shape)
    k = 2.0 * math.pi / wavelength
    h = base + amplitude * np.sin(k * X[along])
    slope = amplitude * k * np.cos(k * X[along])
    return (h - X[normal]) / np.sqrt(1.0 + slope * slope)


def pillars_sd(shape, base: int, width: int, pitch: int, height: int,
               offset: int = 0, vent: int = 0) -> np.ndarray:
    """Base plate (nodes z < base) plus square pillars width x width, z in
    [base, base + height), on an x-y grid of the given pitch (3D), or a row of
    rectangular pillars along x (2D, normal y).  vent > 0 (3D): the plate has a
    square hole vent x vent under the middle of each gap cell (centred half a
    pitch from the pillars), so gas below a liquid slab can leave through the
    plate (and the periodic z boundary)."""
    d = len(shape)
    X = _coords(shape)
    normal = d - 1
    sd = slab_sd(shape, normal, 0, base)
    if vent > 0 and d == 3:
        # distance outside the vent's square prism: the plate minus the hole
        hq = []
        for a in range(2):
            centre = offset + 0.5 * (width - 1) + 0.5 * pitch
            da = X[a] - centre
            da = da - pitch * np.round(da / pitch)
            hq.append(np.abs(da) - 0.5 * vent)
        inside_hole = np.maximum(hq[0], hq[1])   # < 0 inside the hole's footprint
        sd = np.minimum(sd, inside_hole)
    # pillar cells: distance to the nearest pillar via the pitch-periodic image
    q = []
    for a in range(d - 1):
        centre = offset + 0.5 * (width - 1)
        da = X[a] - centre
        da = da - pitch * np.round(da / pitch)
        q.append(np.abs(da) - 0.5 * width)
    zc = base + 0.5 * (height - 1)
    q.append(np.abs(X[normal] - zc) - 0.5 * height)
    q = np.stack(q)
    outside = np.sqrt(np.sum(np.maximum(q, 0.0) ** 2, axis=0))
    inside = np.minimum(np.max(q, axis=0), 0.0)
    return np.maximum(sd, -(outside + inside))


def union_sd(*sds) -> np.ndarray:
    out = sds[0]
    for s in sds[1:]:
        out = np.maximum(out, s)
    return out


def fluid_fraction(solid_sd: np.ndarray, width: float) -> np.ndarray:
    """Initial-condition helper: a smooth 0..1 factor that vanishes inside the solid."""
    return 0.5 * (1.0 - np.tanh(solid_sd / (2.0 * width)))


def drop_c2(shape, centre, radius, alpha=1.0, solid_sd=None, solid_width=1.0):
    """Initial liquid field: a round drop (disc or ball) of the given radius,
    cut off where the solid is."""
    X = _coords(shape)
    r = np.sqrt(sum((X[a] - centre[a]) ** 2 for a in range(len(shape))))
    c2 = 0.5 * (1.0 + np.tanh((radius - r) / (2.0 * alpha)))
    if solid_sd is not None:
        c2 = c2 * fluid_fraction(solid_sd, solid_width)
    return c2


def cap_c2(shape, wall: float, radius: float, theta_deg: float, alpha=1.0,
           solid_sd=None, solid_width=1.0, centre_x=None):
    """Initial liquid field: a circular cap (2D) or spherical cap (3D) of the given
    radius meeting the plane `wall` (along the last axis) at theta_deg."""
    centre = [(s - 1) / 2.0 for s in shape]
    if centre_x is not None:
        centre[0] = centre_x
    centre[-1] = wall - radius * math.cos(math.radians(theta_deg))
    return drop_c2(shape, centre, radius, alpha, solid_sd, solid_width)


def layer_c2(shape, axis, lo, hi, alpha=1.0, solid_sd=None, solid_width=1.0):
    """Initial liquid field: a layer lo <= coordinate < hi along `axis`."""
    X = _coords(shape)
    a = X[axis]
    c2 = 0.25 * (1.0 + np.tanh((a - lo + 0.5) / (2.0 * alpha))) * \
        (1.0 + np.tanh((hi - 0.5 - a) / (2.0 * alpha)))
    if solid_sd is not None:
        c2 = c2 * fluid_fraction(solid_sd, solid_width)
    return c2


# --------------------------------------------------------------------------
# workload recipes
# --------------------------------------------------------------------------
@dataclass
class Case:
    """One lattice Boltzmann (or energy minimisation) problem as a user states it."""
    name: str
    lattice: str                 # "D2Q9" or "D3Q19"
    shape: tuple                 # (nx, ny) or (nx, ny, nz)
    solid_sd: np.ndarray         # signed distance, positive in S (float64, raveled)
    c2: np.ndarray               # initial liquid field (float64, raveled)
    theta_deg: float = 90.0
    g23: float = 2.5e-3
    g12: float = 2.5e-3
    alpha: float = 1.0
    alpha_s: float = 1.0
    rho2: float = 1.0
    rho3: float = 1.0
    tau2: float = 1.0
    tau3: float = 1.0
    tau_g: float = 1.0
    body: tuple = (0.0, 0.0, 0.0)
    steps: int = 0
    extra: dict = field(default_factory=dict)
    faces: tuple = None          # x-, x+, y-, y+, z-, z+ ("periodic", "mirror", "wall")

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))


def wall_drop_2d(nx=128, ny=64, wall=8, radius=25.0, theta=60.0, width=4.0, seed=0,
                 g=2.5e-3, perturb=1e-3, steps=2000) -> Case:
    """Semicircular drop on a flat wall along y = 0 (D2Q9).  With the defaults this
    is the 128x64 FP64 plain-method case: wall 8 nodes thick, 10-90 width 4,
    drop radius 25 centred on the wall surface, 60 degrees, +-1e-3 seeded noise."""
    shape = (nx, ny)
    sd = slab_sd(shape, 1, 0, wall).ravel()
    a_s = width_to_alpha(width)
    c2 = drop_c2(shape, (nx / 2.0, wall - 0.5), radius, 1.0, sd.reshape(ny, nx), a_s).ravel()
    if perturb:
        c2 = c2 + perturbation(seed, c2.size, perturb)
    return Case("wall_drop_2d", "D2Q9", shape, sd, c2, theta_deg=theta, g23=g, g12=g,
                alpha_s=a_s, steps=steps)


def pillar_slab_3d(nx=256, ny=256, nz=192, seed=0, pitch=32, width=10, height=30,
                   base=8, liquid=(38, 98), diffuse_width=3.0, g=2.5e-3,
                   steps=10000, vent=0) -> Case:
    """Square micro-pillar array on a base plate with a liquid slab resting on the
    pillar tops (D3Q19).  Defaults: 256x256x192, pillars 10 wide and 30 high on an
    8-node base, 8 per axis at pitch 32 (the gap of 20 cannot tile 256 with
    width 10, so the gap is 22), 10-90 width 3, liquid z in [38, 98), contact
    angle drawn uniformly in [90, 150] degrees from the seed, body force ramp on
    the liquid along -z up to twice the square-pillar critical estimate."""
    shape = (nx, ny, nz)
    rng = np.random.default_rng(seed)
    theta = float(rng.uniform(90.0, 150.0))
    sd = pillars_sd(shape, base, width, pitch, height, offset=(pitch - width) // 2, vent=vent)
    a_s = width_to_alpha(diffuse_width)
    c2 = layer_c2(shape, 2, liquid[0], liquid[1], 1.0, sd, a_s).ravel()
    # square-pillar depinning estimate: dP ~ 4 a gamma |cos(theta)| / (p^2 - a^2)
    dp_est = 4.0 * width * g * abs(math.cos(math.radians(theta))) / (pitch ** 2 - width ** 2)
    f_max = 2.0 * dp_est / (liquid[1] - liquid[0])
    return Case("pillar_slab_3d", "D3Q19", shape, sd.ravel(), c2, theta_deg=theta, g23=g,
                g12=g, alpha_s=a_s, body=(0.0, 0.0, 0.0), steps=steps,
                extra={"f_max": f_max, "ramp_steps": 10000, "seed": seed})


def pillar_row_2d(nx=4096, ny=4096, seed=0, pitch=32, width=10, height=30, base=8,
                  liquid=(38, 98), theta=None, g=2.5e-3, width_10_90=3.0) -> Case:
    """The 2D analogue of pillar_slab_3d (D2Q9): base plate y < base, a row of
    rectangular pillars width x height at the given pitch along x, a liquid layer
    y in [liquid) on the pillar tops, theta drawn in [90, 150] from the seed when
    not given, +-1e-3 noise."""
    rng = np.random.default_rng(seed)
    if theta is None:
        theta = float(rng.uniform(90.0, 150.0))
    shape = (nx, ny)
    sd = pillars_sd(shape, base, width, pitch, height)
    a_s = width_to_alpha(width_10_90)
    c2 = layer_c2(shape, 1, liquid[0], liquid[1], 1.0, sd, a_s).ravel()
    c2 = c2 + perturbation(seed, c2.size) * fluid_fraction(sd, a_s).ravel()
    return Case("pillar_row_2d", "D2Q9", shape, sd.ravel(), c2, theta_deg=theta, g23=g, g12=g,
                alpha_s=a_s)


def plates_rise_3d(nx=384, ny=384, nz=256, gap=40, thick=8, theta=45.0, g=1e-2,
                   target_rise=120.0, x0=40, x1=340, reservoir=60, lid=8,
                   steps=50000) -> Case:
    """Capillary rise between two parallel plates (normal y) under gravity along -x
    (D3Q19).  Defaults: 384x384x256, gap 40, plates 8 thick spanning z over
    x in [40, 340), reservoir x < 60, solid lids at x < 8 and x >= 376, 45 degrees,
    gamma 1e-2, gravity chosen for a Jurin rise of 120 nodes."""
    shape = (nx, ny, nz)
    yc = ny // 2
    lo1, hi1 = yc - gap // 2 - thick, yc - gap // 2
    lo2, hi2 = yc + gap // 2, yc + gap // 2 + thick
    p1 = box_sd(shape, (x0, lo1, 0), (x1, hi1, nz))
    p2 = box_sd(shape, (x0, lo2, 0), (x1, hi2, nz))
    lids = union_sd(slab_sd(shape, 0, 0, lid), slab_sd(shape, 0, nx - lid, nx))
    # the plates span z: make them periodic in z by using the slab distance in z
    sd = union_sd(p1, p2, lids)
    a_s = width_to_alpha(3.0)
    c2 = layer_c2(shape, 0, lid, reservoir, 1.0, sd, a_s).ravel()
    fg = 2.0 * g * math.cos(math.radians(theta)) / (target_rise * gap)
    return Case("plates_rise_3d", "D3Q19", shape, sd.ravel(), c2, theta_deg=theta, g23=g,
                g12=g, alpha_s=a_s, body=(-fg, 0.0, 0.0), steps=steps,
                extra={"fg": fg, "gap": gap})


def em_sphere_interface(n=128, radius=20.0) -> Case:
    """Energy minimisation: a solid sphere of radius 20 adsorbed at a flat
    liquid/gas interface at z = n/2 (128^3)."""
    shape = (n, n, n)
    c = (n / 2.0, n / 2.0, n / 2.0)
    sd = sphere_sd(shape, c, radius)
    c2 = layer_c2(shape, 2, 0, n // 2, 1.0, sd, 1.0).ravel()
    return Case("em_sphere_interface", "D3Q19", shape, sd.ravel(), c2,
                theta_deg=90.0, g23=math.sqrt(8.0 / 9.0), g12=1.0, alpha_s=1.0)


def em_sinusoid_drop(n=128, amplitude=6.0, wavelength=32.0, base=16.0, radius=30.0,
                     theta=120.0) -> Case:
    """Energy minimisation: a drop of radius 30 on a sinusoidal wall
    z < 16 + 6 sin(2 pi x / 32) (128^3), volume-constrained."""
    shape = (n, n, n)
    sd = sinusoid_sd(shape, base, amplitude, wavelength, along=0, normal=2)
    c2 = drop_c2(shape, (n / 2.0, n / 2.0, base + amplitude), radius, 1.0, sd, 1.0).ravel()
    return Case("em_sinusoid_drop", "D3Q19", shape, sd.ravel(), c2, theta_deg=theta,
                g23=math.sqrt(8.0 / 9.0), g12=1.0, alpha_s=1.0,
                extra={"kcs": 1e-2})


def pillar_gap_2d(period=64, height=120, width=24, pillar=40, base=6, theta=112.0,
                  g23=math.sqrt(8.0 / 9.0), g12=1.0, solid_width=1.0) -> Case:
    """Energy minimisation, critical pressure on micropillars (Sec. III, 2D): one
    period of a row of rectangular pillars of width `width` and height `pillar`
    on a base plate y < `base` (the pillar split across the periodic x
    boundary, so the gap s = period - width is centred), gas in the gap and a
    liquid layer on the pillar tops up to the box top (periodic in y: the box
    top meets the underside of the base plate).  extra['gap'] holds the nodes of
    the lower half of the gap, extra['s'] the gap width."""
    shape = (period, height)
    half = width // 2
    sd = union_sd(slab_sd(shape, 1, 0, base),
                  box_sd(shape, (0, base), (half, base + pillar)),
                  box_sd(shape, (period - (width - half), base), (period, base + pillar)))
    top = base + pillar
    # liquid from the pillar tops through the periodic top to the base's underside
    c2 = layer_c2(shape, 1, top, height + 8, 1.0, sd, solid_width).ravel()
    x, y = _coords(shape)
    s = period - width
    lo_x, hi_x = half + s // 4, period - (width - half) - s // 4
    gap = ((x >= lo_x) & (x < hi_x) & (y >= base + 2) & (y < base + pillar // 2)).ravel()
    return Case("pillar_gap_2d", "D2Q9", shape, sd.ravel(), c2, theta_deg=theta, g23=g23, g12=g12,
                alpha_s=solid_width, extra={"gap": np.flatnonzero(gap), "s": s})


def capillary_channel_2d(nx=1750, ny=450, length=900.0, width=40.0, angle_deg=20.0,
                         entrance=(300.0, 71.0), reservoir=120.0, theta=60.0, g=2.5e-3,
                         seed=0) -> Case:
    """Lattice Boltzmann capillary filling (Sec. IV, "Capillary Filling
    Dynamics"): a solid slab crossed by a straight channel of the given length
    and width, its axis inclined by angle_deg to the x axis so that the solid
    does not align to the grid; a finite liquid reservoir against the slab's
    entrance face, gas elsewhere.  Periodic left/right, mirror top/bottom.
    Liquid viscosity 1/6, gas 2/300, equal densities, M = 1/6 (tau = 1,
    0.52 and tau_g = 1).

    Channel coordinates: s along the axis from the entrance point, t across
    it.  The solid is {0 <= s <= length} minus {|t| < width/2}; solid_sd is its
    signed distance (positive inside) as the smaller of the two constraints'
    distances, extra['mask'] the sharp region S from which the paper relaxes
    the solid first.  The reservoir is {-reservoir <= s < 0}: c2 is its tanh
    profile in s (the caller multiplies it by 1 - C1 once the solid is set).
    extra holds the axis (entrance, direction), the channel length and width."""
    shape = (nx, ny)
    x, y = _coords(shape)
    a = math.radians(angle_deg)
    d = (math.cos(a), math.sin(a))
    xe, ye = entrance
    sx = (x - xe) * d[0] + (y - ye) * d[1]
    tx = -(x - xe) * d[1] + (y - ye) * d[0]
    sd = np.minimum(np.minimum(sx, length - sx), np.abs(tx) - width / 2.0)
    c2 = 0.25 * (1.0 + np.tanh((sx + reservoir) / 2.0)) * (1.0 - np.tanh(sx / 2.0))
    c2 = c2.ravel() + perturbation(seed, nx * ny)
    return Case("capillary_channel_2d", "D2Q9", shape, sd.ravel(), c2, theta_deg=theta, g23=g,
                g12=g, alpha_s=1.0, tau2=1.0, tau3=0.5 + 3.0 * 2.0 / 300.0, tau_g=1.0,
                faces=("periodic", "periodic", "mirror", "mirror", "periodic", "periodic"),
                extra={"mask": (sd.ravel() > 0).astype(np.uint8), "entrance": (xe, ye),
                       "direction": d, "length": length, "width": width,
                       "beta": 1e-3, "omega": 2e-4, "solid_steps": 5000})


def random_fields(n, seed=0, lo=0.05, hi=0.95):
    """Independent uniform fields in [lo, hi) for finite-difference checks."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n), rng.uniform(lo, hi, n)


@dataclass
class Request:
    """One served wetting study; its fields are built on demand by ``case()``."""
    rid: int
    arrival: float
    lattice: str
    shape: tuple
    kind: int            # 0 pillars, 1 sinusoidal wall, 2 sphere packing
    theta_deg: float
    steps: int
    geom_seed: int

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    def case(self) -> Case:
        rng = np.random.default_rng(self.geom_seed)
        shape = self.shape
        d = len(shape)
        side = shape[0]
        if self.kind == 0:
            pitch = int(rng.integers(16, 33))
            width = int(rng.integers(4, pitch // 2 + 1))
            sd = pillars_sd(shape, 6, width, pitch, int(rng.integers(8, side // 4 + 9)))
        elif self.kind == 1:
            sd = sinusoid_sd(shape, 8.0, float(rng.uniform(2, 8)), float(rng.uniform(16, 64)))
        else:
            sds = [slab_sd(shape, d - 1, 0, 4)]
            for _ in range(int(rng.integers(2, 7))):
                c = [float(rng.uniform(0, s)) for s in shape]
                c[-1] = float(rng.uniform(8, side / 3))
                sds.append(sphere_sd(shape, c, float(rng.uniform(4, side / 8))))
            sd = union_sd(*sds)
        a_s = width_to_alpha(3.0)
        centre = [s / 2.0 for s in shape]
        centre[-1] = side / 3.0
        c2 = drop_c2(shape, centre, side / 5.0, 1.0, sd, a_s).ravel()
        return Case(f"req{self.rid}", self.lattice, shape, sd.ravel(), c2,
                    theta_deg=self.theta_deg, alpha_s=a_s, steps=self.steps)


def serving_stream(n_req=512, rate=20.0, seed=0, min_side=64, max_side_2d=512,
                   max_side_3d=160, steps=(2000, 20000), scale_steps=1.0):
    """Poisson arrivals (rate per second) of wetting-sweep requests: half 2D
    (side min_side..max_side_2d), half 3D (side min_side..max_side_3d); geometry =
    random pillars, sinusoidal wall or sphere packing; contact angle U[30, 150];
    step budget U[steps] scaled by scale_steps."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_req):
        t += float(rng.exponential(1.0 / rate))
        is3d = bool(rng.integers(0, 2))
        side = int(rng.integers(min_side, (max_side_3d if is3d else max_side_2d) + 1))
        kind = int(rng.integers(0, 3))
        theta = float(rng.uniform(30.0, 150.0))
        nsteps = max(1, int(round(float(rng.uniform(*steps)) * scale_steps)))
        shape = (side, side, side) if is3d else (side, side)
        out.append(Request(rid, t, "D3Q19" if is3d else "D2Q9", shape, kind, theta, nsteps,
                           int(rng.integers(0, 2**31))))
    return out
