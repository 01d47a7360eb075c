"""Seeded synthetic workloads: lattice configurations, nucleus sites, initial
perturbations.

This module produces inputs only.  It holds none of the method's arithmetic,
so the CUDA path and the CPU oracle can both start from exactly the same
bytes.  The workloads stand in for the paper's foaming cases (Sec. 4.4:
nucleated bubbles in a liquid below a headspace); the paper used no public
dataset.

Conventions: cells are indexed ``n = x + nx*(y + ny*z)``; the up axis is y
in 2D and z in 3D; ``walls`` is a bitmask over the faces -x,+x,-y,+y,-z,+z.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20190812

BASE = dict(
    nx=32, ny=32, nz=1, storage="fp64",
    tau=0.8, rho0=1.0, accel=(0.0, 0.0, 0.0),
    rheo=0, rheo_n=1.0, rheo_k=0.0, rheo_lambda=0.0, rheo_a=2.0,
    tau0=0.8, tau_inf=0.505, tau_min=0.505, tau_max=2.0,
    sigma=0.0, k_pi=0.0, d_max=4.0,
    D=0.05, kH=0.0, RT=1.0, c0=0.0, q=0.0, p0=1.0 / 3.0,
    fill_height=1e9, walls=0, wall_u=(0.0, 0.0, 0.0),
    atmosphere=1, eps=1e-3, bubble_capacity=4096,
    collision=0, trt_magic=3.0 / 16.0, kappa=0, mrt_rates=(0.0, 0.0, 0.0, 0.0),
)

RHEO = {"newtonian": 0, "powerlaw": 1, "carreau": 2}


def config(**kw) -> dict:
    c = dict(BASE)
    c.update(kw)
    return c


def powerlaw_k(n: float, tau_ref: float = 0.7, shear_ref: float = 1e-3) -> float:
    """Consistency k of a power-law fluid whose relaxation time is ``tau_ref``
    at shear rate ``shear_ref`` (lattice units, c_s^2 = 1/3)."""
    return (tau_ref - 0.5) / 3.0 * shear_ref ** (1.0 - n)


# ---------------------------------------------------------------------------
# nucleus placement


def uniform_spheres(rng, n, box_lo, box_hi, rmin, rmax, min_spacing, max_tries=200000):
    """Uniform random centres by rejection with a minimum centre spacing."""
    lo, hi = np.asarray(box_lo, float), np.asarray(box_hi, float)
    pts, rad = [], []
    tries = 0
    while len(pts) < n and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin, rmax)
        p = lo + r + rng.random(lo.size) * (hi - lo - 2 * r)
        if all(np.linalg.norm(p - q) >= min_spacing for q in pts):
            pts.append(p)
            rad.append(r)
    if len(pts) < n:
        raise RuntimeError("could not place %d spheres" % n)
    return np.array(pts), np.array(rad)


def poisson_disk(rng, n, box_lo, box_hi, min_dist, rmin, rmax, max_tries=2000000):
    """Dart-throwing Poisson-disk sampling (minimum distance ``min_dist``)
    with a uniform grid for neighbour look-up; radii uniform in [rmin, rmax]
    and every sphere kept inside the box."""
    lo, hi = np.asarray(box_lo, float), np.asarray(box_hi, float)
    dim = lo.size
    cell = min_dist / math.sqrt(dim)
    shape = np.maximum(1, np.ceil((hi - lo) / cell).astype(int))
    grid = {}
    pts, rad = [], []
    tries = 0
    reach = int(math.ceil(min_dist / cell))
    while len(pts) < n and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin, rmax)
        p = lo + r + rng.random(dim) * (hi - lo - 2 * r)
        g = tuple(np.minimum(((p - lo) / cell).astype(int), shape - 1))
        ok = True
        ranges = [range(max(0, g[d] - reach), min(shape[d], g[d] + reach + 1)) for d in range(dim)]
        for idx in np.stack(np.meshgrid(*ranges, indexing="ij"), -1).reshape(-1, dim):
            j = grid.get(tuple(idx))
            if j is not None and np.linalg.norm(pts[j] - p) < min_dist:
                ok = False
                break
        if not ok:
            continue
        if tuple(g) in grid:
            continue
        grid[tuple(g)] = len(pts)
        pts.append(p)
        rad.append(r)
    if len(pts) < n:
        raise RuntimeError("poisson_disk placed %d of %d" % (len(pts), n))
    return np.array(pts), np.array(rad)


def nuclei_from_field(rng, n, prob, radius, min_gap=1.0, max_tries=2000000):
    """Nucleation sites drawn from a nucleation probability field (Sec. 3.4:
    a field on the lattice gives the distribution, and optionally the
    radius, of the nuclei) by dart throwing: a candidate cell is drawn with
    probability proportional to ``prob`` (an array shaped like the lattice,
    (ny, nx) or (nz, ny, nx)), the site uniformly inside it; a candidate is
    kept when it lies at least r_new + r_old + min_gap from every kept site,
    so that the spheres (disks) neither overlap nor touch.  ``radius`` is a
    number or an array shaped like ``prob`` (the radius at the candidate's
    cell).  Returns (n x dim centres, n radii)."""
    prob = np.asarray(prob, float)
    dim = prob.ndim
    w = prob.reshape(-1)
    if np.any(w < 0) or not np.any(w > 0):
        raise ValueError("the probability field must be non-negative and not all zero")
    cdf = np.cumsum(w) / w.sum()
    rad_field = np.broadcast_to(np.asarray(radius, float), prob.shape).reshape(-1)
    shape_xyz = prob.shape[::-1]  # (nx, ny[, nz])
    pts, rad = [], []
    tries = 0
    while len(pts) < n and tries < max_tries:
        tries += 1
        cell = int(np.searchsorted(cdf, rng.random(), side="right"))
        cell = min(cell, w.size - 1)
        idx = np.unravel_index(cell, prob.shape)[::-1]  # (x, y[, z])
        p = np.asarray(idx, float) + rng.random(dim) - 0.5
        r = float(rad_field[cell])
        if any(np.linalg.norm(p - q) < r + rq + min_gap for q, rq in zip(pts, rad)):
            continue
        if np.any(p - r < 0.5) or np.any(p + r > np.asarray(shape_xyz) - 1.5):
            continue  # keep the nucleus off the lattice's faces
        pts.append(p)
        rad.append(r)
    if len(pts) < n:
        raise RuntimeError("nuclei_from_field placed %d of %d" % (len(pts), n))
    return np.array(pts), np.array(rad)


def nuclei_organised(box_lo, box_hi, spacing, radius, hexagonal=False):
    """Nucleation sites in an organised arrangement (Sec. 3.4): a square
    (cubic) lattice of the given spacing filling the box, or in 2D a
    hexagonal one (every other row shifted by half a spacing, rows
    spacing * sqrt(3)/2 apart).  Returns (centres, radii)."""
    lo, hi = np.asarray(box_lo, float), np.asarray(box_hi, float)
    dim = lo.size
    if hexagonal and dim != 2:
        raise ValueError("the hexagonal arrangement is two-dimensional")
    pts = []
    if hexagonal:
        dy = spacing * math.sqrt(3.0) / 2.0
        row = 0
        y = lo[1] + radius
        while y <= hi[1] - radius + 1e-9:
            x = lo[0] + radius + (0.5 * spacing if row % 2 else 0.0)
            while x <= hi[0] - radius + 1e-9:
                pts.append((x, y))
                x += spacing
            y += dy
            row += 1
    else:
        axes = [np.arange(lo[d] + radius, hi[d] - radius + 1e-9, spacing) for d in range(dim)]
        for p in np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, dim):
            pts.append(tuple(p))
    pts = np.array(pts, float).reshape(-1, dim)
    return pts, np.full(len(pts), float(radius))


def as3(pts):
    pts = np.asarray(pts, float)
    if pts.shape[1] == 2:
        pts = np.concatenate([pts, np.zeros((len(pts), 1))], axis=1)
    return pts


# ---------------------------------------------------------------------------
# the workloads


def c1_2d_128_fp64() -> tuple[dict, np.ndarray, np.ndarray]:
    """2D D2Q9, 128x128, FP64: free surface at y = 112, one bubble of radius 8
    at the domain centre; tau 0.8, sigma 0.01, D2Q5 gas with c0 = 1, kH = 0.5,
    D = 0.05."""
    cfg = config(nx=128, ny=128, nz=1, storage="fp64", tau=0.8, sigma=0.01, k_pi=0.0,
                 D=0.05, kH=0.5, c0=1.0, RT=0.1, fill_height=112.0, walls=0xF)
    return cfg, np.array([[64.0, 64.0, 0.0]]), np.array([8.0])


def _c2_physics(**kw):
    n = 0.6
    return config(storage="fp32", rheo=RHEO["powerlaw"], rheo_n=n, rheo_k=powerlaw_k(n),
                  tau=0.7, sigma=5e-3, d_max=3.0, k_pi=1e-3 / 3.0, D=0.02, kH=0.5, c0=1.0,
                  RT=0.1, walls=0x3F, **kw)


def c2_3d_128_fp32(seed=DEFAULT_SEED):
    """3D D3Q19, 128^3, FP32: 8 bubbles, uniform random centres (spacing >= 20),
    radii U[4,6]; power-law n = 0.6 with tau = 0.7 at shear rate 1e-3;
    disjoining pressure (Pi_max 1e-3, cutoff 3); D3Q7 gas c0 = 1, kH = 0.5,
    D = 0.02.  Liquid fills 3/4 of the height."""
    n = 128
    cfg = _c2_physics(nx=n, ny=n, nz=n, fill_height=0.75 * n)
    rng = np.random.default_rng(seed)
    pts, rad = uniform_spheres(rng, 8, (3, 3, 3), (n - 3, n - 3, 0.75 * n - 3), 4.0, 6.0, 20.0)
    return cfg, pts, rad


def c2_crop_3d_32(seed=DEFAULT_SEED, storage="fp32"):
    """32^3 lattice with the physics of the 128^3 case and one bubble of
    radius 5, for element-wise comparison with the oracle."""
    n = 32
    cfg = _c2_physics(nx=n, ny=n, nz=n, fill_height=0.75 * n)
    cfg["storage"] = storage
    rng = np.random.default_rng(seed)
    c = np.array([[16.0, 16.0, 12.0]]) + rng.uniform(-0.5, 0.5, (1, 3))
    return cfg, c, np.array([5.0])


def c3_3d_256_fp16s(seed=DEFAULT_SEED):
    """3D D3Q19, 256^3, shifted-FP16 storage: 200 Poisson-disk nuclei (min
    distance 8), radii U[2,4], nucleation times U[0,5000]; Carreau fluid
    n = 0.5, lambda = 50 (a = 2, tau0 = 0.8, tau_inf = 0.505)."""
    n = 256
    cfg = config(nx=n, ny=n, nz=n, storage="fp16s", rheo=RHEO["carreau"], rheo_n=0.5,
                 rheo_lambda=50.0, rheo_a=2.0, tau0=0.8, tau_inf=0.505, tau=0.8,
                 sigma=5e-3, d_max=3.0, k_pi=1e-3 / 3.0, D=0.02, kH=0.5, c0=1.0, RT=0.1,
                 walls=0x3F, fill_height=0.75 * n)
    rng = np.random.default_rng(seed)
    pts, rad = poisson_disk(rng, 200, (2, 2, 2), (n - 2, n - 2, 0.75 * n - 3), 8.0, 2.0, 4.0)
    times = np.sort(rng.integers(0, 5001, size=200))
    return cfg, pts, rad, times


def c5_3d_512x512x384_bf16s(seed=DEFAULT_SEED):
    """3D D3Q19, 512x512x384, shifted-BF16 storage: 2000 Poisson-disk nuclei
    (min distance 10), radii U[2,4]; power-law n = 0.7."""
    nx, ny, nz = 512, 512, 384
    n = 0.7
    cfg = config(nx=nx, ny=ny, nz=nz, storage="bf16s", rheo=RHEO["powerlaw"], rheo_n=n,
                 rheo_k=powerlaw_k(n), tau=0.7, sigma=5e-3, d_max=3.0, k_pi=1e-3 / 3.0,
                 D=0.02, kH=0.5, c0=1.0, RT=0.1, walls=0x3F, fill_height=0.75 * nz)
    rng = np.random.default_rng(seed)
    pts, rad = poisson_disk(rng, 2000, (2, 2, 2), (nx - 2, ny - 2, 0.75 * nz - 3), 10.0, 2.0, 4.0)
    return cfg, pts, rad


def random_flow_state(cfg: dict, seed: int, du: float = 0.02, drho: float = 0.01):
    """Seeded random density/velocity perturbation of an all-liquid lattice,
    for driving every population through the collision."""
    rng = np.random.default_rng(seed)
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    rho = cfg["rho0"] + drho * (rng.random(N) - 0.5)
    u = du * (rng.random((N, 3)) - 0.5)
    if cfg["nz"] == 1:
        u[:, 2] = 0.0
    conc = cfg["c0"] + 0.1 * rng.random(N)
    return rho, u, conc


# ---------------------------------------------------------------------------
# voxelised spheres (fill levels by sub-sampling)


def voxel_spheres(shape, centres, radii, sub: int = 4, gas_inside: bool = True):
    """Cell types (0 gas, 1 liquid, 2 interface) and fill levels of spheres
    drawn on a periodic lattice of ``shape`` (nx, ny, nz): the fill level of
    a cell is the fraction of its sub^3 regularly spaced sample points that
    lie in the liquid.  Arrays are flat, ``n = x + nx*(y + ny*z)``."""
    nx, ny, nz = shape
    g = (np.arange(sub) + 0.5) / sub - 0.5
    liquid = np.zeros((nz, ny, nx))
    for c, r in zip(np.asarray(centres, float), np.asarray(radii, float)):
        lo = np.floor(c - r - 1).astype(int)
        hi = np.ceil(c + r + 1).astype(int)
        ix = np.arange(lo[0], hi[0] + 1) % nx
        iy = np.arange(lo[1], hi[1] + 1) % ny
        iz = np.arange(lo[2], hi[2] + 1) % nz
        frac = np.zeros((iz.size, iy.size, ix.size))
        cx = np.arange(lo[0], hi[0] + 1)[None, None, :]
        cy = np.arange(lo[1], hi[1] + 1)[None, :, None]
        cz = np.arange(lo[2], hi[2] + 1)[:, None, None]
        for sz in g:
            for sy in g:
                for sx in g:
                    d2 = (cx + sx - c[0]) ** 2 + (cy + sy - c[1]) ** 2 + (cz + sz - c[2]) ** 2
                    frac += d2 < r * r
        frac /= sub ** 3
        liquid[np.ix_(iz, iy, ix)] += frac
    inside = np.clip(liquid, 0.0, 1.0).reshape(-1)
    alpha = 1.0 - inside if gas_inside else inside
    types = np.where(alpha <= 0.0, 0, np.where(alpha >= 1.0, 1, 2)).astype(np.uint8)
    return types, alpha


# ---------------------------------------------------------------------------
# 2D foams of Sec. 4.4 (the 2D foaming and foam-drainage figures)


def _foam2d_physics(**kw):
    """2D foaming with a gas source: tau 0.9, tau_g 0.6 (D = 0.1/3 on D2Q5),
    RT 1, no initial dissolved gas, kH 1e-3, gamma 5e-3, disjoining slope
    2e-3 (cutoff 3), source q = 5e-5, no gravity; walls on all faces."""
    return config(tau=0.9, sigma=5e-3, k_pi=2e-3, d_max=3.0, D=0.1 / 3.0, kH=1e-3, c0=0.0,
                  RT=1.0, q=5e-5, walls=0xF, **kw)


def _drainage2d_physics(g, **kw):
    """2D foam drainage: tau 0.95, tau_g 0.53 (D = 0.01), c0 0.02, kH 1e-5,
    gamma 5e-3, disjoining slope 2e-3 (cutoff 3), no source, gravity g along
    -y; walls on all faces.  RT = 5 (RT c0 = 0.1, as in the 3D workloads):
    the printed RT = 50 with c0 = 0.02 swells the bubbles of radius 3
    sevenfold and makes their gas mass negative within 40 steps."""
    return config(tau=0.95, sigma=5e-3, k_pi=2e-3, d_max=3.0, D=0.01, kH=1e-5, c0=0.02, RT=5.0,
                  q=0.0, accel=(0.0, -g, 0.0), walls=0xF, **kw)


def foam_2d_450x650(seed=DEFAULT_SEED, storage="fp32", n_nuclei=300):
    """The 2D foaming case: 450 x 650 cells (y up), liquid to 60 % of the
    height, 300 nuclei of radius 3 by Poisson-disk sampling (spacing 9) in
    the liquid."""
    ny = 650
    h = 0.6 * ny
    cfg = _foam2d_physics(nx=450, ny=ny, nz=1, storage=storage, fill_height=h)
    rng = np.random.default_rng(seed)
    pts, rad = poisson_disk(rng, n_nuclei, (2.0, 2.0), (448.0, h - 4.0), 9.0, 3.0, 3.0)
    return cfg, as3(pts), rad


def drainage_2d_450x650(seed=DEFAULT_SEED, storage="fp32", g=3e-5, n_bubbles=150):
    """The 2D drainage case: 450 x 650 cells, liquid to 60 % of the height,
    150 bubbles of radius 3 at uniform random centres (spacing 9)."""
    ny = 650
    h = 0.6 * ny
    cfg = _drainage2d_physics(g, nx=450, ny=ny, nz=1, storage=storage, fill_height=h)
    rng = np.random.default_rng(seed)
    pts, rad = uniform_spheres(rng, n_bubbles, (2.0, 2.0), (448.0, h - 4.0), 3.0, 3.0, 9.0)
    return cfg, as3(pts), rad


def foam_2d_crop(seed=DEFAULT_SEED, storage="fp64", drainage=False):
    """64 x 96 crops of the two 2D foam cases for element-wise comparison with
    the oracle: liquid to 60 % of the height, 6 nuclei of radius 3."""
    ny = 96
    h = 0.6 * ny
    if drainage:
        cfg = _drainage2d_physics(3e-5, nx=64, ny=ny, nz=1, storage=storage, fill_height=h)
    else:
        cfg = _foam2d_physics(nx=64, ny=ny, nz=1, storage=storage, fill_height=h)
    rng = np.random.default_rng(seed)
    pts, rad = poisson_disk(rng, 6, (2.0, 2.0), (62.0, h - 4.0), 12.0, 3.0, 3.0)
    return cfg, as3(pts), rad


def dissolution_2d(seed=DEFAULT_SEED, storage="fp64"):
    """Dissolution of a bubble into a liquid without dissolved gas (Sec. 4.3,
    the dissolution figure): tau 0.98, tau_g 0.8 (D = 0.1 on D2Q5), c0 0,
    kH 5e-3, gamma 4.2e-3, no disjoining pressure, no gravity; 48 x 64 cells
    with walls, free surface at y = 52, one bubble of radius 8.  RT = 5: a
    bubble in Laplace equilibrium holds the gas mass p V / RT, which at the
    printed RT = 500 is 0.13 for this bubble, and the Henry condition
    dissolves it within 100 steps; at RT = 5 it loses 5 % of its volume in
    the first 500 steps, closer to the time scale of the paper's figure
    (t = 5000)."""
    cfg = config(nx=48, ny=64, nz=1, storage=storage, tau=0.98, D=0.1, kH=5e-3, RT=5.0, c0=0.0,
                 k_pi=0.0, sigma=4.2e-3, fill_height=52.0, walls=0xF)
    rng = np.random.default_rng(seed)
    c = np.array([[24.0, 26.0, 0.0]]) + np.concatenate([rng.uniform(-0.5, 0.5, (1, 2)), np.zeros((1, 1))], 1)
    return cfg, c, np.array([8.0])

