"""Seeded synthetic inputs for the colour-gradient D3Q27 step.

This module holds no arithmetic of the method itself: it only draws initial
fields (per-colour densities, velocity, solid mask) and parameter sets shaped
like the paper's test problems.  The same arrays feed the CUDA path and the
CPU oracle, so both see identical inputs.

Recipe (the paper is silent on initial profiles; Sec. IV gives the setups):
  * interface profile  phi0(r) = tanh(2 (R - r) / W), W = 4 cells;
  * rho_r = rho_r0 (1 + phi0) / 2,  rho_b = rho_b0 (1 - phi0) / 2,
    which the order parameter of Sec. II.A maps back to phi0 exactly;
  * optional noise from a splitmix64 stream (top 53 bits -> [0, 1)).
Rest fractions follow the pressure balance of Sec. II.A: the lighter phase
takes alpha = 8/27 (c_s^2 = 1/3, as in the bubble test of Sec. IV.D), the
heavier one 1 - alpha = (1 - 8/27) / ratio.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import Optional, Sequence, Tuple

import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n uniform doubles in [0, 1) from the splitmix64 generator (Steele et al.)."""
    out = np.empty(n, dtype=np.float64)
    # vectorised: state_k = seed + (k+1) * golden
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed & _MASK64) + k * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    out[:] = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return out


def rest_fractions(rho_r0: float, rho_b0: float) -> Tuple[float, float]:
    """(alpha_r, alpha_b) for a density ratio: lighter phase 8/27."""
    light = 8.0 / 27.0
    gamma = rho_r0 / rho_b0
    if gamma >= 1.0:
        return 1.0 - (1.0 - light) / gamma, light
    return light, 1.0 - (1.0 - light) * gamma


@dataclass
class Workload:
    """Parameters of one domain in lattice units (mirrors the C struct)."""
    nx: int
    ny: int
    nz: int
    bc: Tuple[int, int, int] = (0, 0, 0)
    rho_r0: float = 1.0
    rho_b0: float = 1.0
    alpha_r: float = 8.0 / 27.0
    alpha_b: float = 8.0 / 27.0
    nu_r: float = 0.1
    nu_b: float = 0.1
    sigma: float = 0.01
    beta: float = 0.7
    omega: Tuple[float, ...] = (1.0,) * 11
    g: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    rho_ref: float = 0.0
    force_mode: int = 0
    model: int = 3
    use_Q: int = 1
    steps: int = 200
    name: str = ""

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def params(self) -> dict:
        d = asdict(self)
        d.pop("steps"); d.pop("name")
        return d


def droplet_fields(shape_zyx, center_xyz, radius, rho_r0, rho_b0, width=4.0,
                   u0=(0.0, 0.0, 0.0), semi_axes=None, noise=0.0, seed=0,
                   invert=False):
    """(rho_r, rho_b, u) for a red droplet (or blue bubble if invert) in a
    periodic box; arrays are [nz, ny, nx] and u is [3, nz, ny, nx]."""
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = center_xyz
    if semi_axes is None:
        r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        dist = radius - r
    else:
        ax, ay, az = semi_axes
        q = np.sqrt(((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2 + ((z - cz) / az) ** 2)
        dist = (1.0 - q) * min(ax, ay, az)
    phi0 = np.tanh(2.0 * dist / width)
    if invert:
        phi0 = -phi0
    rho_r = rho_r0 * (1.0 + phi0) / 2.0
    rho_b = rho_b0 * (1.0 - phi0) / 2.0
    u = np.empty((3, nz, ny, nx))
    for a in range(3):
        u[a] = u0[a]
    if noise > 0.0:
        n = nx * ny * nz
        rnd = splitmix64(seed, 5 * n).reshape(5, nz, ny, nx) * 2.0 - 1.0
        rho_r = rho_r * (1.0 + noise * rnd[0])
        rho_b = rho_b * (1.0 + noise * rnd[1])
        u = u + noise * rnd[2:5]
    return rho_r, rho_b, u


def layered_fields(nz, a, rho_r0, rho_b0, width=4.0):
    """Layered channel: red in |z - zc| <= a, blue outside; walls at z=0, nz-1.
    Returns fields of shape [nz, 1, 1]."""
    zc = (nz - 1) / 2.0
    z = np.arange(nz, dtype=np.float64)
    phi0 = np.tanh(2.0 * (a - np.abs(z - zc)) / width)
    rho_r = (rho_r0 * (1.0 + phi0) / 2.0).reshape(nz, 1, 1)
    rho_b = (rho_b0 * (1.0 - phi0) / 2.0).reshape(nz, 1, 1)
    u = np.zeros((3, nz, 1, 1))
    return rho_r, rho_b, u


# ---- the paper-shaped workloads (sizes, densities, viscosities) ---------------

def static_droplet_32() -> Workload:
    """32^3 periodic, R=8 centred, equal densities, nu=0.1, sigma=0.01."""
    return Workload(32, 32, 32, nu_r=0.1, nu_b=0.1, sigma=0.01, beta=0.7,
                    steps=200, name="static_droplet_32")


def translating_droplet(edge=128) -> Workload:
    """edge^3 periodic, ratio 10 (1 : 0.1), nu=0.05, sigma=0.005, u0=(0.05,0.05,0)."""
    ar, ab = rest_fractions(1.0, 0.1)
    return Workload(edge, edge, edge, rho_r0=1.0, rho_b0=0.1, alpha_r=ar, alpha_b=ab,
                    nu_r=0.05, nu_b=0.05, sigma=0.005, beta=0.7, steps=4000,
                    name="translating_droplet_%d" % edge)


def rising_bubble(nx=192, ny=192, nz=384) -> Workload:
    """Ratio 1000 bubble with z walls (liquid red rho=1, gas blue rho=0.001)."""
    ar, ab = rest_fractions(1.0, 0.001)
    return Workload(nx, ny, nz, bc=(0, 0, 1), rho_r0=1.0, rho_b0=0.001,
                    alpha_r=ar, alpha_b=ab, nu_r=0.005, nu_b=0.05, sigma=0.01,
                    beta=0.2, g=(0.0, 0.0, -1e-6), rho_ref=1.0, force_mode=3,
                    steps=20000, name="rising_bubble_%dx%dx%d" % (nx, ny, nz))


def rising_bubble_case2(nx=192, ny=192, nz=384) -> Workload:
    """Case 2 of the bubble test of Sec. IV.D (ratio 1000, viscosity ratio 100,
    Eo = 125, Re = 35, liquid Mach number 0.0548) in 3D with R = nx / 8 = 24:
    U = sqrt(g D) = 1e-3 lattice units, g = U^2 / D, sigma = rho_l g D^2 / Eo,
    nu_l = U D / Re, nu_g = 10 nu_l (dynamic ratio 100); z walls, buoyancy form."""
    ar, ab = rest_fractions(1.0, 0.001)
    D = nx / 4.0
    U = 1e-3
    g = U * U / D
    nu_l = U * D / 35.0
    return Workload(nx, ny, nz, bc=(0, 0, 1), rho_r0=1.0, rho_b0=0.001,
                    alpha_r=ar, alpha_b=ab, nu_r=nu_l, nu_b=10.0 * nu_l,
                    sigma=g * D * D / 125.0, beta=0.2, g=(0.0, 0.0, -g), rho_ref=1.0,
                    force_mode=3, steps=20000, name="rising_bubble_case2_%dx%dx%d" % (nx, ny, nz))


def rayleigh_taylor(W=128, Re=1024.0, model=3) -> Workload:
    """Sec. IV.E: W x W x 4W fluid layers between no-slip walls (two more solid
    z layers), heavy red (rho 1) over light blue (rho 1/3, Atwood 0.5),
    sqrt(W g) = 0.04, Re = sqrt(W g) W / nu, equal kinematic viscosities, no
    interfacial tension, F = (rho - (rho_r0 + rho_b0)/2) g with g = (0, 0, -g)."""
    ar, ab = rest_fractions(1.0, 1.0 / 3.0)
    g = 0.04 ** 2 / W
    nu = 0.04 * W / Re
    return Workload(W, W, 4 * W + 2, bc=(0, 0, 1), rho_r0=1.0, rho_b0=1.0 / 3.0, alpha_r=ar, alpha_b=ab,
                    nu_r=nu, nu_b=nu, sigma=0.0, beta=0.7, g=(0.0, 0.0, -g), rho_ref=(1.0 + 1.0 / 3.0) / 2.0,
                    force_mode=3, model=model, steps=int(3 * math.sqrt(W / g)),
                    name="rayleigh_taylor_%d_Re%g" % (W, Re))


def rayleigh_taylor_fields(wl: Workload, width=4.0):
    """Interface at the middle of the fluid layers displaced by
    h(x, y) = 0.05 W [cos(2 pi x / W) + cos(2 pi y / W)]; heavy fluid above."""
    W = wl.nx
    z, y, x = np.meshgrid(np.arange(wl.nz), np.arange(wl.ny), np.arange(wl.nx), indexing="ij")
    z_mid = (wl.nz - 1) / 2.0
    h = 0.05 * W * (np.cos(2.0 * math.pi * x / W) + np.cos(2.0 * math.pi * y / W))
    phi0 = np.tanh(2.0 * (z - (z_mid + h)) / width)
    rho_r = wl.rho_r0 * (1.0 + phi0) / 2.0
    rho_b = wl.rho_b0 * (1.0 - phi0) / 2.0
    return rho_r, rho_b, np.zeros((3,) + rho_r.shape)


def droplet_collision(edge=512) -> Workload:
    """Head-on binary collision: two droplets of radius 48/512 edge closing at a
    relative speed 0.2 along x, ratio 1, nu = 0.002, sigma = 0.005."""
    return Workload(edge, edge, edge, nu_r=0.002, nu_b=0.002, sigma=0.005, beta=0.7,
                    steps=10000, name="droplet_collision_%d" % edge)


def collision_fields(wl: Workload, z_range=None, noise=0.0, seed=0):
    """Two red droplets at x = c -+ 56/512 edge moving at +-0.1 along x.
    Filled plane by plane (a 512^3 domain needs no full-size temporaries);
    z_range = (z0, z1) returns only those planes of the domain.  noise > 0
    perturbs the whole domain as droplet_fields does (splitmix64 from seed),
    which breaks the mirror symmetry of the two droplets."""
    n = wl.nx
    R, d = 48.0 * n / 512.0, 56.0 * n / 512.0
    z0, z1 = (0, wl.nz) if z_range is None else z_range
    nzs = z1 - z0
    cx, cy, cz = n / 2.0, wl.ny / 2.0, wl.nz / 2.0
    y, x = np.meshgrid(np.arange(wl.ny), np.arange(wl.nx), indexing="ij")
    rho_r = np.empty((nzs, wl.ny, wl.nx))
    rho_b = np.empty((nzs, wl.ny, wl.nx))
    u = np.zeros((3, nzs, wl.ny, wl.nx))
    for k in range(nzs):
        z = z0 + k
        r1 = np.sqrt((x - (cx - d)) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        r2 = np.sqrt((x - (cx + d)) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        t1 = np.tanh(2.0 * (R - r1) / 4.0)
        t2 = np.tanh(2.0 * (R - r2) / 4.0)
        phi = np.maximum(t1, t2)
        rho_r[k] = wl.rho_r0 * (1.0 + phi) / 2.0
        rho_b[k] = wl.rho_b0 * (1.0 - phi) / 2.0
        u[0, k] = 0.1 * ((1.0 + t1) / 2.0) - 0.1 * ((1.0 + t2) / 2.0)
    if noise > 0.0:
        shape = (wl.nz, wl.ny, wl.nx)
        rnd = splitmix64(seed, 5 * wl.cells).reshape((5,) + shape)[:, z0:z1] * 2.0 - 1.0
        rho_r = rho_r * (1.0 + noise * rnd[0])
        rho_b = rho_b * (1.0 + noise * rnd[1])
        u = u + noise * rnd[2:5]
    return rho_r, rho_b, u


def workload_fields(wl: Workload, seed: int = 0, noise: float = 0.0):
    """Initial fields for a named workload (droplet/bubble placement)."""
    shape = (wl.nz, wl.ny, wl.nx)
    if wl.name.startswith("static_droplet"):
        c = (wl.nx / 2.0, wl.ny / 2.0, wl.nz / 2.0)
        return droplet_fields(shape, c, wl.nx / 4.0, wl.rho_r0, wl.rho_b0,
                              noise=noise, seed=seed)
    if wl.name.startswith("translating_droplet"):
        c = (wl.nx / 2.0, wl.ny / 2.0, wl.nz / 2.0)
        return droplet_fields(shape, c, 20.0 * wl.nx / 128.0, wl.rho_r0, wl.rho_b0,
                              u0=(0.05, 0.05, 0.0), noise=noise, seed=seed)
    if wl.name.startswith("rising_bubble"):
        c = (wl.nx / 2.0, wl.ny / 2.0, wl.nz / 6.0)
        return droplet_fields(shape, c, wl.nx / 8.0, wl.rho_r0, wl.rho_b0,
                              noise=noise, seed=seed, invert=True)
    if wl.name.startswith("droplet_collision"):
        return collision_fields(wl)
    if wl.name.startswith("rayleigh_taylor"):
        return rayleigh_taylor_fields(wl)
    raise ValueError("unknown workload " + wl.name)


# ---- serving workload: many independent droplet runs -------------------------------------

SERVING_EDGES = (32, 48, 64, 96, 128)


@dataclass
class Request:
    """One independent simulation request (a static or oscillating droplet in a
    periodic cube): arrival time in seconds after the start of the run."""
    rid: int
    arrival: float
    edge: int
    radius: float
    ratio: float
    sigma: float
    steps: int
    kind: str  # "static" (sphere) or "oscillating" (ellipsoid, equal volume)

    @property
    def cells(self) -> int:
        return self.edge ** 3

    def workload(self) -> Workload:
        ar, ab = rest_fractions(1.0, 1.0 / self.ratio)
        return Workload(self.edge, self.edge, self.edge, rho_r0=1.0, rho_b0=1.0 / self.ratio,
                        alpha_r=ar, alpha_b=ab, nu_r=0.1, nu_b=0.1, sigma=self.sigma, beta=0.7,
                        steps=self.steps, name="serving_%s_%d" % (self.kind, self.rid))

    def fields(self):
        n = self.edge
        c = (n / 2.0, n / 2.0, n / 2.0)
        semi = None
        if self.kind == "oscillating":
            R = self.radius
            semi = (R * 1.1, R * 0.95, R * 0.95)
        return droplet_fields((n, n, n), c, self.radius, 1.0, 1.0 / self.ratio, semi_axes=semi)


def serving_requests(n: int = 256, rate: float = 4.0, seed: int = 4):
    """n requests with Poisson arrivals at `rate` per second: edge uniform in
    {32, 48, 64, 96, 128}, radius uniform in [0.2, 0.35] edge, density ratio
    uniform in [1, 10], sigma uniform in [0.001, 0.02], steps uniform in
    500..5000, half static spheres and half oscillating ellipsoids."""
    u = splitmix64(seed, 8 * n).reshape(n, 8)
    out, t = [], 0.0
    for i in range(n):
        t += -math.log(1.0 - float(u[i, 0])) / rate
        out.append(Request(
            rid=i, arrival=t,
            edge=SERVING_EDGES[min(4, int(u[i, 1] * 5))],
            radius=0.0, ratio=float(1.0 + 9.0 * u[i, 3]), sigma=float(0.001 + 0.019 * u[i, 4]),
            steps=500 + min(4500, int(u[i, 5] * 4501)),
            kind="static" if u[i, 6] < 0.5 else "oscillating"))
        out[-1].radius = float((0.2 + 0.15 * u[i, 2]) * out[-1].edge)
    return out
