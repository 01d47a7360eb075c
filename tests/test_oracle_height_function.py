"""Pins of the oracle's height-function curvature (the second classical
curvature Sec. 2.2 names): exact fill levels of planes and
parabolas, whose column heights are exact integrals, give the exact
curvature; voxelised disks and spheres give 1/(2R) and 1/R."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests.test_oracle_geometry import _gas_fraction_incl_excl


def _sim(oracle_mod, nx, ny, nz, alpha):
    """An oracle lattice (periodic, no walls) holding the fill levels alpha
    (1 liquid, 0 gas, interface in between)."""
    t = np.where(alpha <= 0.0, 0, np.where(alpha >= 1.0, 1, 2)).astype(np.uint8)
    s = oracle_mod.OracleSim(W.config(nx=nx, ny=ny, nz=nz, atmosphere=0))
    N = nx * ny * nz
    s.set_cells(t, np.ones(N), np.zeros((N, 3)), alpha, np.zeros(N))
    return s


def _column_fraction_2d(height, x_lo, y_cell):
    """Liquid fraction of the cell [x_lo, x_lo+1] x [y_cell-1/2, y_cell+1/2]
    above the curve y = height(x): the integral of
    clamp(y_cell + 1/2 - height(x), 0, 1), by Simpson's rule on 64 pieces
    between the points where the integrand's pieces change (exact for
    linear and quadratic curves)."""
    xs = np.linspace(x_lo, x_lo + 1.0, 4097)
    f = np.clip(y_cell + 0.5 - height(xs), 0.0, 1.0)
    # breakpoints where the clamp switches: refine there by splitting
    knots = [x_lo, x_lo + 1.0]
    for level in (y_cell - 0.5, y_cell + 0.5):
        sgn = np.sign(height(xs) - level)
        idx = np.flatnonzero(np.diff(sgn) != 0)
        for k in idx:
            a, b = xs[k], xs[k + 1]
            for _ in range(80):
                m = 0.5 * (a + b)
                if np.sign(height(m) - level) == np.sign(height(a) - level):
                    a = m
                else:
                    b = m
            knots.append(0.5 * (a + b))
    knots = np.sort(np.asarray(knots))
    total = 0.0
    for a, b in zip(knots[:-1], knots[1:]):
        if b - a <= 0:
            continue
        t = np.linspace(a, b, 129)
        g = np.clip(y_cell + 0.5 - height(t), 0.0, 1.0)
        h = (b - a) / 128
        total += h / 3 * (g[0] + g[-1] + 4 * g[1:-1:2].sum() + 2 * g[2:-1:2].sum())
    return total


def _curve_alpha_2d(nx, ny, height):
    alpha = np.zeros((ny, nx))
    for x in range(nx):
        for y in range(ny):
            alpha[y, x] = _column_fraction_2d(height, x - 0.5, y)
    return alpha.reshape(-1)


def test_hf_curvature_of_a_line_is_zero(oracle_mod):
    nx, ny = 24, 32
    s_, c_ = 0.37, 14.3
    s = _sim(oracle_mod, nx, ny, 1, _curve_alpha_2d(nx, ny, lambda x: s_ * (x - 12.0) + c_))
    t = s.types()
    k = s.hf_curvature().reshape(ny, nx)
    xs, ys = np.arange(nx)[None, :], np.arange(ny)[:, None]
    # interface cells of the line (not those the periodic wrap makes)
    near = np.abs(ys - (s_ * (xs - 12.0) + c_)) < 1.5
    inner = (t.reshape(ny, nx) == 2) & near & (xs >= 3) & (xs < nx - 3)
    assert inner.sum() > 10
    assert np.max(np.abs(k[inner])) < 1e-12


def test_hf_curvature_of_a_parabola_is_exact(oracle_mod):
    """Column heights are the cell averages of the liquid length, whose
    centred differences are exact for a quadratic: kappa equals half the
    curvature of y = a (x - x0)^2 + c at the column's centre."""
    nx, ny, a, x0, c = 26, 32, -0.04, 12.3, 17.2
    s = _sim(oracle_mod, nx, ny, 1, _curve_alpha_2d(nx, ny, lambda x: a * (x - x0) ** 2 + c))
    t = s.types().reshape(ny, nx)
    k = s.hf_curvature().reshape(ny, nx)
    xs = np.arange(nx)
    near = np.abs(xs - x0) <= 5
    checked = 0
    for x in xs[near]:
        for y in np.flatnonzero(t[:, x] == 2):
            if abs(y - (a * (x - x0) ** 2 + c)) >= 1.5:
                continue  # made by the periodic wrap, not by the parabola
            want = -a / (1.0 + (2 * a * (x - x0)) ** 2) ** 1.5
            assert abs(k[y, x] - want) < 1e-10, (x, y, k[y, x], want)
            checked += 1
    assert checked >= 11


def test_hf_curvature_of_a_tilted_plane_is_zero(oracle_mod):
    nx, ny, nz = 14, 14, 24
    s1, s2, c = 0.3, -0.45, 11.6
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    # gas below z = s1 x + s2 y + c: in the cell's unit coordinates u the gas
    # is m.u < r with m = (-s1, -s2, 1); flip the negative components
    r = c + s1 * (x - 0.5) + s2 * (y - 0.5) - (z - 0.5)
    m = np.array([-s1, -s2, 1.0])
    mp = np.abs(m)
    shift = np.sum(mp[m < 0])
    alpha = np.empty((nz, ny, nx))
    for idx in np.ndindex(nz, ny, nx):
        aa = r[idx] + shift
        gas = 0.0 if aa <= 0 else (1.0 if aa >= mp.sum() else _gas_fraction_incl_excl(mp, aa))
        alpha[idx] = 1.0 - gas
    s = _sim(oracle_mod, nx, ny, nz, alpha.reshape(-1))
    t = s.types().reshape(nz, ny, nx)
    k = s.hf_curvature().reshape(nz, ny, nx)
    near = np.abs(z - (s1 * x + s2 * y + c)) < 1.5
    inner = (t == 2) & near & (x >= 3) & (x < nx - 3) & (y >= 3) & (y < ny - 3)
    assert inner.sum() > 20
    assert np.max(np.abs(k[inner])) < 1e-12


def _disk_alpha(n, c, R, sub=64):
    g = (np.arange(sub) + 0.5) / sub - 0.5
    alpha = np.zeros((n, n))
    for y in range(n):
        for x in range(n):
            px = x + g[None, :] - c[0]
            py = y + g[:, None] - c[1]
            alpha[y, x] = 1.0 - np.mean(px * px + py * py < R * R)
    return alpha.reshape(-1)


@pytest.mark.parametrize("dim,n,R,tol", [(2, 40, 10.0, 0.03), (3, 36, 10.0, 0.03)])
def test_hf_curvature_of_voxelised_bubbles(oracle_mod, dim, n, R, tol):
    """A gas disk gives 1/(2R), a gas sphere 1/R (mean over the interface
    cells), the least-squares curvature's sign and scale."""
    if dim == 2:
        s = _sim(oracle_mod, n, n, 1, _disk_alpha(n, (n / 2 + 0.23, n / 2 - 0.17), R))
        want = 1.0 / (2 * R)
    else:
        c = np.array([[n / 2 + 0.23, n / 2 - 0.17, n / 2 + 0.11]])
        _, alpha = W.voxel_spheres((n, n, n), c, [R], sub=8)
        s = _sim(oracle_mod, n, n, n, alpha)
        want = 1.0 / R
    k = s.hf_curvature()[s.types() == 2]
    assert not np.any(np.isnan(k))
    assert abs(np.mean(k) / want - 1.0) < tol


def test_hf_curvature_of_a_quadric_is_exact(oracle_mod):
    """z = c + a (x-x0)^2 + b (y-y0)^2 + e (x-x0)(y-y0), liquid above: the
    fill levels hold, column by column, the cell average of the surface
    height (all that column sums can see), so the height function must give
    minus the mean curvature of the surface at the column's centre, taken
    here from its fundamental forms (E, F, G; L, M, N with the upward
    normal)."""
    nx, ny, nz = 16, 16, 24
    a, b, e, x0, y0, c = -0.03, -0.05, 0.02, 7.6, 8.3, 12.4
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    zs = c + a * ((i - x0) ** 2 + 1 / 12) + b * ((j - y0) ** 2 + 1 / 12) + e * (i - x0) * (j - y0)
    k = np.arange(nz)[:, None, None]
    alpha = np.clip(k + 0.5 - zs[None, :, :], 0.0, 1.0)
    s = _sim(oracle_mod, nx, ny, nz, alpha.reshape(-1))
    t = s.types().reshape(nz, ny, nx)
    kap = s.hf_curvature().reshape(nz, ny, nx)
    checked = 0
    for (kk, jj, ii) in zip(*np.nonzero(t == 2)):
        if abs(ii - x0) > 4 or abs(jj - y0) > 4 or abs(kk - zs[jj, ii]) >= 1.5:
            continue
        fx = 2 * a * (ii - x0) + e * (jj - y0)
        fy = 2 * b * (jj - y0) + e * (ii - x0)
        fxx, fyy, fxy = 2 * a, 2 * b, e
        w = np.sqrt(1 + fx * fx + fy * fy)
        E, F, G = 1 + fx * fx, fx * fy, 1 + fy * fy
        L, M, N = fxx / w, fxy / w, fyy / w
        H = (E * N - 2 * F * M + G * L) / (2 * (E * G - F * F))
        assert abs(kap[kk, jj, ii] - (-H)) < 1e-12, (ii, jj, kk, kap[kk, jj, ii], -H)
        checked += 1
    assert checked >= 40
