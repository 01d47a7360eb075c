"""Radial "cell model" of one gas bubble growing (or dissolving) in a finite
liquid reservoir: the continuum problem behind the growth law of Sec. 4.2
(Eq. 1Danalytical), solved numerically.  Test infrastructure; written from
the physics, independent of the oracle and of the CUDA path.

Model (d = 2: a disk, d = 3: a sphere; k = d - 1; Omega = 2 pi or 4 pi):
  * the liquid is incompressible and moves radially, u = dR/dt (R/r)^k, so
    the liquid volume per unit solid angle between the bubble and a liquid
    particle, sigma = r^d/d - R^d/d, is a material coordinate;
  * the dissolved gas obeys dc/dt + u dc/dr = D r^-k d/dr(r^k dc/dr)
    (Sec. 3.1 without the source term), which in sigma has no advection
    term:  dc/dt = D d/dsigma( r(sigma, t)^(2k) dc/dsigma );
  * Henry's law holds at the interface, c(sigma = 0) = k_H p_g (Sec. 3.2
    Eq. henryslaw); the outer edge of the reservoir (liquid volume
    Omega * sigma_max) is closed;
  * the bubble gains the diffusive flux, dm/dt = Omega D R^(2k) dc/dsigma at
    sigma = 0, and holds an ideal gas, V = m RT / p_g (Eq. idealgas), with
    p_g = p0 + (d - 1) gamma / R the pressure of the surrounding liquid plus
    the Laplace jump.

For a sphere in an unbounded reservoir at small supersaturation the solution
tends to R^2 = R0^2 + 2 dc V_m D t with V_m = RT / p (Eq. 1Danalytical);
``epstein_plesset`` integrates the classical quasi-static equation
dR/dt = D dc V_m (1/R + 1/sqrt(pi D t)) that includes the early transient.

Discretisation: finite volumes on a geometric grid in sigma (fine at the
bubble), backward Euler in time with a step that grows from 1e-4; the
gas held by the liquid plus the bubble's is conserved to round-off, which
``solve`` checks.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_banded


def _stretch(h0: float, total: float, cells: int) -> float:
    """Ratio g of a geometric series of `cells` widths starting at h0 that
    sums to `total` (bisection; g = 1 if uniform widths already suffice)."""
    if h0 * cells >= total:
        return 1.0
    lo, hi = 1.0, 2.0
    while h0 * (hi ** cells - 1.0) / (hi - 1.0) < total:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if h0 * (mid ** cells - 1.0) / (mid - 1.0) < total:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def solve(d: int, R0: float, c_inf: float, D: float, kH: float, RT: float, p0: float, gamma: float,
          liquid_volume: float, t_out, cells: int = 400, dr0: float = 0.01, dt_max: float = 0.5):
    """Radius R(t) at the times t_out (increasing, > 0).  liquid_volume is
    the reservoir's liquid volume (area in 2D); the first cell next to the
    bubble is dr0 wide in r, the others grow geometrically."""
    k = d - 1
    Om = 2.0 * math.pi if d == 2 else 4.0 * math.pi

    def p_of(R):
        return p0 + (d - 1) * gamma / R

    smax = liquid_volume / Om
    # cell faces: geometric growth from the bubble outwards
    g = _stretch(R0 ** k * dr0, smax, cells)
    h = R0 ** k * dr0 * g ** np.arange(cells)
    faces = np.concatenate([[0.0], np.cumsum(h)])
    faces *= smax / faces[-1]
    width = np.diff(faces)
    centre = 0.5 * (faces[:-1] + faces[1:])
    c = np.full(cells, float(c_inf))
    V = Om * R0 ** d / d
    m = p_of(R0) * V / RT
    total0 = m + Om * np.sum(c * width)
    t = 0.0
    out = []
    t_out = list(t_out)
    j = 0
    dt = 1e-4
    while j < len(t_out):
        step = min(dt, t_out[j] - t)
        S = V / Om
        R = (d * S) ** (1.0 / d)
        cR = kH * p_of(R)
        # diffusion coefficients r^(2k) at the faces, with the current S
        r_face = (d * (faces + S)) ** (1.0 / d)
        a_face = D * r_face ** (2 * k)
        # interior faces between cells i-1 and i; face 0 is the interface
        # (Dirichlet c = cR at distance centre[0]); the last face is closed
        g_int = a_face[1:-1] / np.diff(centre)
        g0 = a_face[0] / centre[0]
        diag = width / step
        lower = np.zeros(cells)
        upper = np.zeros(cells)
        diag = diag.copy()
        diag[:-1] += g_int
        diag[1:] += g_int
        diag[0] += g0
        upper[1:] = -g_int
        lower[:-1] = -g_int
        rhs = width / step * c
        rhs[0] += g0 * cR
        ab = np.vstack([upper, diag, lower])
        c_new = solve_banded((1, 1), ab, rhs)
        flux = g0 * (c_new[0] - cR)  # per unit solid angle, into the bubble
        m += Om * flux * step
        c = c_new
        t += step
        # the ideal gas at the pressure of the surrounding liquid
        R_guess = R
        for _ in range(50):
            V = m * RT / p_of(R_guess)
            R_next = (d * V / Om) ** (1.0 / d)
            if abs(R_next - R_guess) < 1e-13 * R_next:
                break
            R_guess = R_next
        V = m * RT / p_of(R_guess)
        if t >= t_out[j] - 1e-12:
            out.append((d * V / Om) ** (1.0 / d))
            j += 1
        dt = min(dt_max, dt * 1.05)
    total = m + Om * np.sum(c * width)
    assert abs(total - total0) <= 1e-9 * abs(total0), (total, total0)
    return np.array(out)


def epstein_plesset(R0: float, dc: float, Vm: float, D: float, t_out):
    """Quasi-static growth of a sphere, dR/dt = D dc V_m (1/R + 1/sqrt(pi D t))
    (Epstein and Plesset, J. Chem. Phys. 18, 1950), integrated with RK4 in
    the variable s = sqrt(t) (the transient term is singular at t = 0)."""
    def f(s, R):
        # dR/ds = 2 s dR/dt
        return 2.0 * s * D * dc * Vm * (1.0 / R) + 2.0 * D * dc * Vm / math.sqrt(math.pi * D)

    out = []
    R, s = float(R0), 0.0
    for t in t_out:
        s1 = math.sqrt(t)
        n = max(1, int(math.ceil((s1 - s) / 0.01)))
        hs = (s1 - s) / n
        for _ in range(n):
            k1 = f(s, R)
            k2 = f(s + hs / 2, R + hs / 2 * k1)
            k3 = f(s + hs / 2, R + hs / 2 * k2)
            k4 = f(s + hs, R + hs * k3)
            R += hs / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            s += hs
        out.append(R)
    return np.array(out)
