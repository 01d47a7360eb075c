"""Pins of the oracle's multiple-relaxation-time collision (the variant Sec. 2
names beside BGK and TRT).

The moment basis is the published one (Lallemand and Luo 2000 for D2Q9,
d'Humieres et al. 2002 for D3Q19): its rows are orthogonal with the row norms
those papers list, and contain density and momentum.  The collision is then
fixed by what it must reproduce: with every even rate at 1/tau and every odd
rate at 1/tau_m it is the TRT collision, with all rates at 1/tau it is BGK;
the stress rate alone sets the shear viscosity, so body-force Poiseuille flow
stays exact at the TRT product 3/16 whatever the energy, energy-square and
fourth-order rates are, while a third-order rate away from the energy-flux
rate moves the wall; the energy rate sets the bulk viscosity, which a
standing sound wave measures."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests.test_oracle_lattice import _channel, _lattice, _poiseuille_profile

# row norms |m_k|^2 of the published bases, in the published row order
NORMS = {
    2: [9, 36, 36, 6, 12, 6, 12, 4, 4],
    3: [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8],
}
ODD_GROUPS = (3, 6)  # energy flux q, third-order m (momentum is odd too)


@pytest.mark.parametrize("dim", [2, 3])
def test_mrt_basis_orthogonal_published_norms(oracle_mod, dim):
    M, grp = oracle_mod.mrt_basis(dim)
    e = _lattice(dim)
    G = M @ M.T
    assert np.max(np.abs(G - np.diag(np.diag(G)))) == 0.0
    assert np.array_equal(np.diag(G), np.array(NORMS[dim], float))
    # the conserved rows are density and the momentum components
    cons = np.flatnonzero(grp == 0)
    assert len(cons) == dim + 1
    want = [np.ones(len(e))] + [e[:, a] for a in range(dim)]
    assert all(np.array_equal(M[k], w) for k, w in zip(cons, want))
    # every row is even or odd under e -> -e as its group says
    opp = np.array([int(np.flatnonzero((e == -v).all(1))[0]) for v in e])
    for k in range(len(M)):
        odd = grp[k] in ODD_GROUPS or (grp[k] == 0 and k > 0)
        assert np.array_equal(M[k][opp], -M[k] if odd else M[k]), k
    # 2D has no fourth-order anisotropic or third-order m moments
    if dim == 2:
        assert not np.isin(grp, (5, 6)).any()


def _random_periodic(dim, n=8, seed=7):
    rng = np.random.default_rng(seed)
    nz = 1 if dim == 2 else n
    N = n * n * nz
    rho = 1.0 + 0.005 * rng.standard_normal(N)
    u = 0.02 * rng.uniform(-1, 1, (N, 3))
    if dim == 2:
        u[:, 2] = 0.0
    base = W.config(nx=n, ny=n, nz=nz, storage="fp64", accel=(2e-5, -1e-5, 0.0 if dim == 2 else 1e-5),
                    rheo=W.RHEO["newtonian"], tau=0.9, walls=0)
    return base, np.ones(N, np.uint8), rho, u


def _run(oracle_mod, cfg, t, rho, u, steps=50):
    s = oracle_mod.OracleSim(cfg)
    s.set_cells(t, rho, u, np.ones(t.size), np.zeros(t.size))
    s.step(steps)
    return s.get("rho"), s.get("u")


@pytest.mark.parametrize("dim", [2, 3])
def test_mrt_reduces_to_trt_and_bgk(oracle_mod, dim):
    """Rates left at 0 follow 1/tau (even groups) and the energy-flux rate
    (third-order group): that is TRT.  TRT with tau_m = tau and every rate at
    1/tau is BGK.  Random periodic flow with a body force, 50 steps."""
    base, t, rho, u = _random_periodic(dim)
    trt = _run(oracle_mod, dict(base, collision=1, trt_magic=3.0 / 16.0), t, rho, u)
    mrt = _run(oracle_mod, dict(base, collision=2, trt_magic=3.0 / 16.0), t, rho, u)
    assert np.max(np.abs(trt[0] - mrt[0])) < 1e-13
    assert np.max(np.abs(trt[1] - mrt[1])) < 1e-14
    om = 1.0 / 0.9
    bgk = _run(oracle_mod, dict(base, collision=0), t, rho, u)
    mrt = _run(oracle_mod, dict(base, collision=2, trt_magic=(0.9 - 0.5) ** 2, mrt_rates=(om, om, om, om)), t, rho, u)
    assert np.max(np.abs(bgk[0] - mrt[0])) < 1e-13
    assert np.max(np.abs(bgk[1] - mrt[1])) < 1e-14
    # a rate away from its default changes the flow (the group is used)
    other = _run(oracle_mod, dict(base, collision=2, trt_magic=3.0 / 16.0, mrt_rates=(1.6, 0, 0, 0)), t, rho, u)
    assert np.max(np.abs(other[1] - trt[1])) > 1e-8


@pytest.mark.parametrize("dim", [2, 3])
def test_mrt_poiseuille_exact_with_free_even_rates(oracle_mod, dim):
    ny, g, tau = 18, 1e-6, 1.2
    nu = (tau - 0.5) / 3.0
    y = np.arange(1, ny - 1)
    H = ny - 2
    exact = g / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
    s = oracle_mod.OracleSim(_channel(dim, ny, tau=tau, accel=(g, 0.0, 0.0), collision=2,
                                      trt_magic=3.0 / 16.0, mrt_rates=(1.1, 1.3, 1.7, 0.0)))
    s.step(25000)
    u = _poiseuille_profile(s, ny, dim)
    assert np.max(np.abs(u - exact)) < 1e-9 * exact.max()
    if dim == 3:
        # the third-order moments carry part of the wall's non-equilibrium:
        # away from the energy-flux rate the half-way wall moves
        s = oracle_mod.OracleSim(_channel(dim, ny, tau=tau, accel=(g, 0.0, 0.0), collision=2,
                                          trt_magic=3.0 / 16.0, mrt_rates=(1.1, 1.3, 1.7, 1.0)))
        s.step(25000)
        u = _poiseuille_profile(s, ny, dim)
        assert np.max(np.abs(u - exact)) > 1e-4 * exact.max()


def _sound_decay(oracle_mod, dim, se, tau=0.8, ny=64, steps=1000, A=1e-4):
    nz = 1 if dim == 2 else 3
    cfg = W.config(nx=3, ny=ny, nz=nz, walls=0, tau=tau, collision=2, trt_magic=3.0 / 16.0,
                   mrt_rates=(se, 0.0, 0.0, 0.0))
    s = oracle_mod.OracleSim(cfg)
    y = (np.arange(s.N) // 3) % ny
    k = 2 * np.pi / ny
    s.set_cells(np.ones(s.N, np.uint8), 1.0 + A * np.sin(k * y), np.zeros((s.N, 3)), np.ones(s.N), np.zeros(s.N))
    ph = np.exp(-1j * k * y) / s.N
    ts, E = [], []
    for t in range(0, steps, 5):
        a, b = (s.get("rho") - 1.0) @ ph, s.get("u")[:, 1] @ ph
        # acoustic energy of the mode: no oscillation, decays at 2 Gamma k^2
        E.append(abs(a) ** 2 / 3.0 + abs(b) ** 2)
        ts.append(t)
        s.step(5)
    return -np.polyfit(ts, np.log(E), 1)[0] / (2 * k * k)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("se", [0.6, 1.8])
def test_mrt_sound_attenuation_follows_energy_rate(oracle_mod, dim, se):
    """A standing sound wave decays at Gamma k^2 with Gamma = (1/2)(2 nu
    (1 - 1/d) + zeta); the bulk viscosity zeta = (2/d) nu_e with
    nu_e = (1/s_e - 1/2)/3 comes from the energy rate alone."""
    tau = 0.8
    nu, nu_e = (tau - 0.5) / 3.0, (1.0 / se - 0.5) / 3.0
    zeta = 2.0 / dim * nu_e
    want = 0.5 * (2.0 * nu * (1.0 - 1.0 / dim) + zeta)
    got = _sound_decay(oracle_mod, dim, se, tau)
    assert abs(got / want - 1.0) < 0.005, (got, want)
