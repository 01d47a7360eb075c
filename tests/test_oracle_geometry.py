"""Pins of the oracle's geometry (Sec. 2.2 curvature, Sec. 3.3 PLIC and
disjoining pressure, Appendix A traversal)."""
import itertools
import math

import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests import films


def _gas_fraction_incl_excl(m, a):
    """Textbook volume of {x in [0,1]^3 : m.x < a} for m_i > 0 by
    inclusion-exclusion over the cube's vertices."""
    tot = 0.0
    for sset in itertools.product((0, 1), repeat=3):
        v = a - np.dot(m, sset)
        if v > 0:
            tot += (-1) ** sum(sset) * v ** 3
    return tot / (6 * m[0] * m[1] * m[2])


def test_plic_axis_aligned(oracle_mod):
    for s in np.linspace(-0.5, 0.5, 11):
        assert abs(oracle_mod.plic_liquid_fraction(3, [0, 0, 1], s) - (0.5 - s)) < 1e-15
        assert abs(oracle_mod.plic_liquid_fraction(2, [-1, 0], s) - (0.5 - s)) < 1e-15


def test_plic_against_inclusion_exclusion(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        if np.min(np.abs(n)) < 0.05:
            continue
        h = 0.5 * np.abs(n).sum()
        s = rng.uniform(-h, h)
        want = 1.0 - _gas_fraction_incl_excl(np.abs(n), s + h)
        assert abs(oracle_mod.plic_liquid_fraction(3, n, s) - want) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_plic_against_sampling(oracle_mod, dim):
    rng = np.random.default_rng(7 + dim)
    k = 1200 if dim == 2 else 120
    g = (np.arange(k) + 0.5) / k - 0.5
    P = np.stack(np.meshgrid(*([g] * dim), indexing="ij"), -1).reshape(-1, dim)
    for trial in range(6):
        n = rng.normal(size=dim)
        if trial == 0:
            n[0] = 1e-7  # nearly axis-aligned: no cancellation allowed
        n /= np.linalg.norm(n)
        s = rng.uniform(-0.3, 0.3)
        frac = np.mean(P @ n > s)
        assert abs(oracle_mod.plic_liquid_fraction(dim, n, s) - frac) < 3.0 / k


def test_plic_offset_round_trip(oracle_mod):
    rng = np.random.default_rng(9)
    for dim in (2, 3):
        for _ in range(100):
            n = rng.normal(size=dim)
            n /= np.linalg.norm(n)
            a = rng.uniform(0.0, 1.0)
            s = oracle_mod.plic_offset(dim, n, a)
            assert abs(oracle_mod.plic_liquid_fraction(dim, n, s) - a) < 1e-13


@pytest.mark.parametrize("dim,n,R,lo,hi", [(2, 48, 12.0, 0.85, 1.15), (3, 30, 9.0, 0.85, 1.15)])
def test_curvature_of_voxelised_bubble(oracle_mod, dim, n, R, lo, hi):
    """kappa = 1/(2R) on a disk, 1/R on a sphere (half the divergence of the
    unit normal, Eq. rhob reading)."""
    nz = 1 if dim == 2 else n
    s = oracle_mod.OracleSim(W.config(nx=n, ny=n, nz=nz, atmosphere=0))
    c = [n / 2 + 0.23, n / 2 - 0.17, 0.0 if dim == 2 else n / 2 + 0.11]
    s.nucleate([c], [R])
    t = s.types()
    k = s.get("kappa")[(t == oracle_mod.IFC) & (s.labels() >= 0)]
    want = 1.0 / (2 * R) if dim == 2 else 1.0 / R
    assert lo < np.mean(k) / want < hi
    nrm = s.get("normal")[t == oracle_mod.IFC]
    assert np.allclose(np.linalg.norm(nrm, axis=1), 1.0)


def _film(oracle_mod, L, aa, ab, kpi=2e-3, dmax=4.0, nz=16, sigma=0.0):
    """Planar lamella between two bubbles: walls at z = 0 and z = nz-1,
    gas A below, interface (alpha_a) at za, L liquid layers, interface
    (alpha_b) at zb = za + L + 1, gas B above."""
    cfg = W.config(nx=4, ny=4, nz=nz, walls=0x30, k_pi=kpi, d_max=dmax, atmosphere=0, sigma=sigma)
    s = oracle_mod.OracleSim(cfg)
    z = np.arange(s.N) // 16
    za = 4
    zb = za + L + 1
    t = np.full(s.N, oracle_mod.LIQ, np.uint8)
    t[(z >= 1) & (z < za)] = oracle_mod.GAS
    t[z == za] = oracle_mod.IFC
    t[z == zb] = oracle_mod.IFC
    t[(z > zb) & (z < nz - 1)] = oracle_mod.GAS
    t[(z == 0) | (z == nz - 1)] = oracle_mod.WALL
    alpha = np.where(z == za, aa, np.where(z == zb, ab, 1.0))
    s.set_cells(t, np.ones(s.N), np.zeros((s.N, 3)), alpha, np.zeros(s.N))
    return s, z, za, zb


@pytest.mark.parametrize("L,aa,ab", [(1, 0.3, 0.6), (2, 0.5, 0.5), (0, 0.2, 0.1), (3, 0.9, 0.8),
                                     (1, 0.05, 0.95)])
def test_planar_film_disjoining_pressure(oracle_mod, L, aa, ab):
    """PLIC is exact for planes, so the film thickness between the two
    reconstructed interfaces is d = L + alpha_a + alpha_b and
    Pi = k_Pi (d_max - d) for d < d_max, else 0 (Sec. 3.3)."""
    kpi, dmax = 2e-3, 4.0
    s, z, za, zb = _film(oracle_mod, L, aa, ab, kpi, dmax)
    b = s.bubbles()
    assert b["mass"].size == 2
    Pi = s.get("pi")
    d = L + aa + ab
    want = kpi * (dmax - d) if d < dmax else 0.0
    assert np.allclose(Pi[z == za], want, rtol=0, atol=1e-14)
    assert np.allclose(Pi[z == zb], want, rtol=0, atol=1e-14)
    assert np.all(Pi[(z != za) & (z != zb)] == 0.0)


@pytest.mark.parametrize("L,kpi", [(1, 2e-3), (2, 2e-3), (2, 4e-3)])
def test_film_liquid_settles_at_gas_pressure_minus_disjoining(oracle_mod, L, kpi):
    """Sec. 3.3 Eq. rhobplusdisjoining at rest: a symmetric planar film (3
    gas layers on either side, so both bubbles keep one pressure) with
    sigma = 0.01 -- a plane's curvature is 0, so the Laplace term drops out
    -- settles to a state with no flow in which the liquid's pressure
    c_s^2 rho equals p_g - Pi.  Fails for Pi added instead of subtracted
    (off by 2 Pi), Pi left out (off by Pi), or the gas density without its
    factor 1 / c_s^2."""
    s, z, za, zb = _film(oracle_mod, L, 0.5, 0.5, kpi, nz=4 + L + 1 + 3 + 2, sigma=0.01)
    s.step(500)
    t = s.types()
    assert np.sum(t == oracle_mod.IFC) == 32
    assert np.max(np.abs(s.get("u"))) < 1e-9
    p = s.bubbles()["pressure"]
    assert p.size == 2 and abs(p[0] - p[1]) < 1e-12
    Pi = s.get("pi")[t == oracle_mod.IFC]
    assert np.all(Pi > 0) and np.ptp(Pi) < 1e-12
    assert np.all(s.get("kappa")[t == oracle_mod.IFC] == 0.0)
    rho = s.get("rho")[t == oracle_mod.LIQ]
    assert np.max(np.abs(rho / 3.0 - (p[0] - Pi[0]))) < 1e-9


def test_disjoining_off_beyond_cutoff(oracle_mod):
    s, z, za, zb = _film(oracle_mod, 4, 0.5, 0.5)
    assert np.all(s.get("pi") == 0.0)


def test_plic_degenerate_normals(oracle_mod):
    """Components far below rounding of the others must not change the cut."""
    for tiny in (1e-17, 1e-12, 0.0):
        assert abs(oracle_mod.plic_liquid_fraction(3, [0.0, tiny, -1.0], 0.3) - 0.2) < 1e-12
        assert abs(oracle_mod.plic_liquid_fraction(3, [tiny, 1.0, tiny], -0.25) - 0.75) < 1e-12
        assert abs(oracle_mod.plic_liquid_fraction(2, [tiny, -1.0], 0.1) - 0.4) < 1e-12



@pytest.mark.parametrize("dim,axes", [(2, 2), (3, 2), (3, 3)])
def test_oblique_film_disjoining_pressure(oracle_mod, dim, axes):
    """A planar film along a lattice diagonal, w = x + y (axes = 2) or
    w = x + y + z (axes = 3): gas A for w in (1.3, 5.3), the film for
    (5.3, 8.7), gas B for (8.7, 12.7), liquid elsewhere (period 24 in w, as
    the periodic box gives).  Fill levels are exact cut volumes
    (Irwin-Hall over the axes the plane is oblique to), so the Parker-Youngs
    normal is the diagonal (by the symmetry of its weights) and every PLIC
    plane is exact.  The ray of Algorithm 1 steps diagonally (w + axes per
    cell) across the film (Sec. 3.3, Pi = k_Pi (d_max - d)):

    * axes = 2 (D2Q9, or D3Q19 with its xy edge links): every face cell has
      a gas lattice neighbour, hence a bubble, and its ray meets the other
      face's plane: d = 3.4 / sqrt(2), the film thickness;
    * axes = 3 (D3Q19 has no corner links): the face layers at 0.3 from a
      plane (w = 5, 9) and at 1.3 (w = 4, 10) touch their gas through
      lattice links, the layers at 0.7 (w = 6, 8) only through corners, so
      they belong to no bubble (Pi = 0) and rays pass through them.  From
      w = 4 the ray meets w = 10, a face cell of bubble B: d = 3.4 / sqrt(3).
      From w = 5 it passes w = 8 and enters B's gas at w = 11, 1.5 sqrt(3)
      along the ray, whose own plane lies 0.3 / sqrt(3) ahead of the
      centre: d = 1.5 sqrt(3) - 0.3 / sqrt(3) (and alike from B's side).

    Faces towards the thick liquid (12.6 / sqrt(axes) away, beyond d_max)
    get Pi = 0.  With axes = 2 in 3D the steps have no z offset, so a
    distance that mixes up the z component with another fails."""
    kpi, dmax, N = 2e-3, 4.0, 24
    cfg = W.config(nx=N, ny=N, nz=N if dim == 3 else 1, k_pi=kpi, d_max=dmax, atmosphere=0)
    s = oracle_mod.OracleSim(cfg)
    w, t, alpha = films.diagonal_film(N, dim, axes, oracle_mod.LIQ, oracle_mod.GAS, oracle_mod.IFC)
    s.set_cells(t, np.ones(s.N), np.zeros((s.N, 3)), alpha, np.zeros(s.N))
    assert s.bubbles()["mass"].size == 2
    ifc = t == oracle_mod.IFC
    face_a = ifc & (np.abs(w - 5.3) < axes / 2.0)
    face_b = ifc & (np.abs(w - 8.7) < axes / 2.0)
    assert face_a.sum() == face_b.sum() == axes * N ** (dim - 1)
    diag = np.ones(3) * (np.arange(3) < axes) / math.sqrt(axes)
    nrm = s.get("normal")
    assert np.allclose(nrm[face_a], diag, rtol=0, atol=1e-12)
    assert np.allclose(nrm[face_b], -diag, rtol=0, atol=1e-12)
    Pi, lab = s.get("pi"), s.labels()
    film = kpi * (dmax - 3.4 / math.sqrt(axes))
    want = np.zeros(s.N)
    if axes == 2:
        want[face_a | face_b] = film
    else:
        want[(w == 4) | (w == 10)] = film
        want[(w == 5) | (w == 9)] = kpi * (dmax - (1.5 * math.sqrt(3) - 0.3 / math.sqrt(3)))
        assert np.all(lab[(w == 6) | (w == 8)] == -1)
    assert np.allclose(Pi, want, rtol=1e-9, atol=0)
