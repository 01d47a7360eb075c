"""Pins of the oracle's free-surface parts (Sec. 2.1-2.2): exact mass
conservation with conversions, the liquid/gas separation invariant, and the
Laplace pressure jump of a static bubble."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W


def _neighbour_offsets(dim):
    r = (-1, 0, 1)
    if dim == 2:
        return [(dx, dy, 0) for dx in r for dy in r if (dx, dy) != (0, 0)]
    return [(dx, dy, dz) for dx in r for dy in r for dz in r
            if 0 < abs(dx) + abs(dy) + abs(dz) <= 2]


def liquid_touches_gas(types, shape, dim, oracle_mod):
    t = types.reshape(shape)  # (nz, ny, nx)
    L = t == oracle_mod.LIQ
    G = t == oracle_mod.GAS
    for dx, dy, dz in _neighbour_offsets(dim):
        if np.any(L & np.roll(G, (dz, dy, dx), axis=(0, 1, 2))):
            return True
    return False


def _growing_bubble_2d(oracle_mod, n=40):
    cfg, _, _ = W.c1_2d_128_fp64()
    cfg.update(nx=n, ny=n, fill_height=n - 8)
    s = oracle_mod.OracleSim(cfg)
    s.nucleate([[n / 2 + 0.3, n / 2 - 3.2, 0.0]], [6.0])
    return s


def test_mass_conserved_through_conversions(oracle_mod):
    s = _growing_bubble_2d(oracle_mod)
    L0 = s.ledger()
    m0 = L0[0] + L0[1] + L0[2]
    t_prev = s.types().copy()
    changed = 0
    for _ in range(30):
        s.step(10)
        t = s.types()
        changed += int(np.sum(t != t_prev))
        t_prev = t.copy()
        L = s.ledger()
        assert abs(L[0] + L[1] + L[2] - m0) < 1e-12 * m0
        assert not liquid_touches_gas(t, (1, s.ny, s.nx), 2, oracle_mod)
    assert changed > 20  # conversions really happened


def test_mass_conserved_3d(oracle_mod):
    cfg, c, r = W.c2_crop_3d_32(storage="fp64")
    cfg.update(nx=16, ny=16, nz=16, fill_height=12)
    s = oracle_mod.OracleSim(cfg)
    s.nucleate([[8.2, 7.9, 6.1]], [3.5])
    L0 = s.ledger()
    m0 = L0[0] + L0[1] + L0[2]
    for _ in range(4):
        s.step(5)
        L = s.ledger()
        assert abs(L[0] + L[1] + L[2] - m0) < 1e-12 * m0
        assert not liquid_touches_gas(s.types(), (16, 16, 16), 3, oracle_mod)


def _laplace(oracle_mod, dim, n, R, sigma, steps, kappa=0):
    nz = 1 if dim == 2 else n
    cfg = W.config(nx=n, ny=n, nz=nz, tau=0.9, sigma=sigma, kH=0.0, c0=0.0, atmosphere=0, kappa=kappa)
    s = oracle_mod.OracleSim(cfg)
    c = [n / 2, n / 2, 0.0 if dim == 2 else n / 2]
    s.nucleate([c], [R])
    s.step(steps)
    b = s.bubbles()
    assert len(b["pressure"]) == 1
    t = s.types()
    rho = s.get("rho")
    pl = np.mean(rho[t == oracle_mod.LIQ]) / 3.0
    V = b["volume"][0]
    Reff = np.sqrt(V / np.pi) if dim == 2 else (3 * V / (4 * np.pi)) ** (1 / 3)
    return (b["pressure"][0] - pl) / ((dim - 1) * sigma / Reff)


def test_laplace_jump_2d(oracle_mod):
    """p_g - p_l = sigma / R for a disk (kappa = 1/(2R) in Eq. rhob)."""
    ratio = _laplace(oracle_mod, 2, 40, 9.0, 0.01, 3000)
    assert 0.92 < ratio < 1.08


def test_laplace_jump_3d(oracle_mod):
    """p_g - p_l = 2 sigma / R for a sphere (kappa = 1/R in Eq. rhob)."""
    ratio = _laplace(oracle_mod, 3, 16, 4.5, 0.01, 400)
    assert 0.9 < ratio < 1.1


def test_laplace_jump_height_function_2d(oracle_mod):
    """The same disk with the height-function curvature in the step (the
    second method Sec. 2.2 names, cfg kappa = 1)."""
    ratio = _laplace(oracle_mod, 2, 40, 9.0, 0.01, 3000, kappa=1)
    assert 0.92 < ratio < 1.08


def test_laplace_jump_height_function_3d(oracle_mod):
    ratio = _laplace(oracle_mod, 3, 16, 4.5, 0.01, 400, kappa=1)
    assert 0.9 < ratio < 1.1
