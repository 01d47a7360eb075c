"""Pins of the oracle's advection-diffusion step (Sec. 3.1-3.2)."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W


def test_gas_conserved_in_closed_box(oracle_mod):
    cfg = W.config(nx=6, ny=5, nz=4, walls=0x3F, tau=0.7, D=0.03)
    s = oracle_mod.OracleSim(cfg)
    rho, u, conc = W.random_flow_state(cfg, seed=11, du=0.05)
    t = s.types()
    s.set_cells(t, rho, u, np.ones(s.N), conc)
    c0 = s.ledger()[3]
    s.step(200)
    assert abs(s.ledger()[3] - c0) < 1e-13 * c0


def test_source_term_adds_q_per_cell(oracle_mod):
    q = 1e-4
    cfg = W.config(nx=5, ny=4, nz=3, walls=0x3F, q=q, c0=0.2)
    s = oracle_mod.OracleSim(cfg)
    fluid = np.sum(s.types() == oracle_mod.LIQ)
    c0 = s.ledger()[3]
    s.step(50)
    assert abs(s.ledger()[3] - c0 - 50 * q * fluid) < 1e-13


def _slab(oracle_mod, nx, x0, x1, kH, q, D):
    """Liquid slab x0..x1 (interface cells at both ends, alpha = 1) between
    two gas regions connected through the periodic x boundary; ny = 2 and
    the gas touches the top layer, so it is the atmosphere at p0."""
    cfg = W.config(nx=nx, ny=2, nz=1, tau=1.25, D=D, kH=kH, q=q, c0=0.0)
    s = oracle_mod.OracleSim(cfg)
    x = np.arange(s.N) % nx
    t = np.full(s.N, oracle_mod.GAS, np.uint8)
    t[(x > x0) & (x < x1)] = oracle_mod.LIQ
    t[(x == x0) | (x == x1)] = oracle_mod.IFC
    s.set_cells(t, np.ones(s.N), np.zeros((s.N, 3)), np.ones(s.N), np.zeros(s.N))
    return s, x


def test_henry_slab_steady_profile(oracle_mod):
    """Sec. 4.1 Eq. diffusionanalytical: steady dissolved gas in a liquid
    slab of length L with uniform source q and c = kH p_g at both interfaces.
    The steady solution of D c'' = -q is the parabola
    8D(c - kH p_g)/(q L^2) = 1 - x'^2, x' = 2 x / L from the slab centre
    (the printed right-hand side lost its exponent; the diffusion equation
    fixes it).  Parameters of Table validatonParameters: q = 1e-6, D = 0.06,
    kH = 0.01, p_g = 1/3, L = 40."""
    q, D, kH, L = 1e-6, 0.06, 0.01, 40
    nx = 60
    x0 = 10
    x1 = x0 + L - 1
    s, x = _slab(oracle_mod, nx, x0, x1, kH, q, D)
    s.step(30000)
    c = s.get("conc").reshape(2, nx)[0]
    pg = s.bubbles()["pressure"][0]
    assert abs(pg - 1 / 3) < 1e-15
    xs = np.arange(x0, x1 + 1)
    xc = 0.5 * (x0 - 0.5 + x1 + 0.5)
    lhs = 8 * D * (c[x0:x1 + 1] - kH * pg) / (q * L * L)
    rhs = 1 - (2 * (xs - xc) / L) ** 2
    assert np.max(np.abs(lhs - rhs)) < 5e-3


def test_gas_ledger_closes_for_static_interface(oracle_mod):
    """With a static interface the per-cell gas current of Eq. gascurrent is
    the exact link exchange with the gas, so dissolved + bubble gas +
    exchange with the outside - source stays constant to round-off."""
    s, _ = _slab(oracle_mod, 30, 5, 20, kH=0.3, q=2e-4, D=0.05)
    def total():
        L = s.ledger()
        return L[3] + L[4] + L[5] - L[6]
    t0 = total()
    s.step(300)
    assert abs(total() - t0) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_advection_moves_the_centroid_at_the_flow_velocity(oracle_mod, dim):
    """Sec. 3.1 Eq. diffusion with the equilibrium g_eq = w_i c (1 + e_i.u /
    c_s^2): in a uniform periodic liquid moving at u0 (no force, no walls,
    density 1.02) the flow stays uniform, and from g = g_eq(c, u0) the
    collision keeps the lattice-wide first moment at u0 sum(c) (the first
    moment of g_eq is c u0, and relaxing towards it keeps the sum there), so
    the centroid of a concentration pulse moves by exactly u0 per step as
    long as nothing crosses the periodic faces: the populations move one
    cell per step, so a pulse of radius 4 stays inside radius 14 for 10
    steps, inside the box of 32.  Fails for a flipped advective sign (-u0),
    a missing 1/c_s^2 (u0/3 in D2Q5) or the momentum rho u in place of u
    (1.02 u0)."""
    n = 32
    u0 = np.array([0.05, -0.03, 0.02]) * (np.arange(3) < dim)
    cfg = W.config(nx=n, ny=n, nz=n if dim == 3 else 1, tau=0.8, D=0.05, c0=0.0, kH=0.0, atmosphere=0)
    s = oracle_mod.OracleSim(cfg)
    t = s.types()
    assert np.all(t == oracle_mod.LIQ)
    idx = np.arange(s.N)
    X = np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1).astype(float)
    centre = np.array([n / 2 - 0.3, n / 2 + 0.2, (n / 2 + 0.1) if dim == 3 else 0.0])
    conc = np.maximum(0.0, 1.0 - np.sum((X - centre) ** 2, 1) / 16.0) ** 2
    s.set_cells(t, np.full(s.N, 1.02), np.tile(u0, s.N), np.ones(s.N), conc)

    def centroid():
        c = s.get("conc")
        return (c @ X) / c.sum()

    x0 = centroid()
    T = 10
    s.step(T)
    assert np.max(np.abs(s.get("u") - u0)) < 1e-14
    assert np.max(np.abs(centroid() - x0 - T * u0)) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_diffusion_spreads_the_pulse_by_the_lattice_closed_form(oracle_mod, dim):
    """Sec. 3.1 Eq. diffusion at rest, worked out on the lattice: with
    omega = 1 / tau_g, tau_g = 1/2 + D / c_s^2 (c_s^2 = 1/3 on D2Q5, 1/4 on
    D3Q7) and g = g_eq(c, 0) at the start, the lattice-wide second moment
    of the ADE populations stays c_s^2 sum(c) and K = sum x J_x obeys
    K(t+1) = (1 - omega) K(t) + c_s^2 C, K(0) = 0, so along every axis

        Var(t) - Var(0) = sum_{k<t} c_s^2 [1 + 2 (1 - omega) (1 - (1 - omega)^k) / omega]

    (slope 2 D for large t), exactly, while nothing crosses the periodic
    faces (a pulse of radius 4 for 10 steps in a box of 32).  Fails for a
    wrong c_s^2 of either lattice, a relaxation rate that misses the 1/2 of
    tau_g, or equilibrium weights with another second moment."""
    n, T, D = 32, 10, 0.05
    cs2 = 1.0 / 3.0 if dim == 2 else 0.25
    om = 1.0 / (0.5 + D / cs2)
    cfg = W.config(nx=n, ny=n, nz=n if dim == 3 else 1, tau=0.8, D=D, c0=0.0, kH=0.0, atmosphere=0)
    s = oracle_mod.OracleSim(cfg)
    t = s.types()
    assert np.all(t == oracle_mod.LIQ)
    idx = np.arange(s.N)
    X = np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1)[:, :dim].astype(float)
    centre = np.array([n / 2 - 0.3, n / 2 + 0.2, n / 2 + 0.1])[:dim]
    conc = np.maximum(0.0, 1.0 - np.sum((X - centre) ** 2, 1) / 16.0) ** 2
    s.set_cells(t, np.ones(s.N), np.zeros((s.N, 3)), np.ones(s.N), conc)

    def variance():
        c = s.get("conc")
        m = (c @ X) / c.sum()
        return (c @ (X - m) ** 2) / c.sum()

    v0 = variance()
    s.step(T)
    grow = sum(cs2 * (1.0 + 2.0 * (1.0 - om) * (1.0 - (1.0 - om) ** k) / om) for k in range(T))
    assert np.max(np.abs(variance() - v0 - grow)) < 1e-11
