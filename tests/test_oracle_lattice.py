"""Pins of the oracle's lattice, equilibria and streaming (Sec. 2, Sec. 3.1).

Equilibrium moments are fixed by the mathematics (rho, rho u, rho(uu + cs^2 I)
for the flow; c, c u, c cs_A^2 I for the gas); Couette flow is reproduced
exactly by BGK with half-way bounce-back; body-force Poiseuille flow is exact
at tau = 1/2 + sqrt(3/16) (Ginzburg's magic parameter for BGK)."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W


def _lattice(dim):
    if dim == 2:
        e = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
                      [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0]])
    else:
        e = [[0, 0, 0]]
        for a in range(3):
            for s in (1, -1):
                v = [0, 0, 0]
                v[a] = s
                e.append(v)
        e = np.array(e + [[1, 1, 0], [-1, -1, 0], [1, 0, 1], [-1, 0, -1], [0, 1, 1], [0, -1, -1],
                          [1, -1, 0], [-1, 1, 0], [1, 0, -1], [-1, 0, 1], [0, 1, -1], [0, -1, 1]])
    return e


@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_moments(oracle_mod, dim):
    cfg = W.config(nx=5, ny=4, nz=1 if dim == 2 else 3, c0=0.3)
    s = oracle_mod.OracleSim(cfg)
    rho, u, conc = W.random_flow_state(cfg, seed=3, du=0.1, drho=0.2)
    t = np.full(s.N, oracle_mod.LIQ, np.uint8)
    s.set_cells(t, rho, u, np.ones(s.N), conc)
    f = s.get("fpop")
    g = s.get("gpop")
    e = _lattice(dim)
    assert np.allclose(f.sum(1), rho, rtol=0, atol=1e-14)
    assert np.allclose(f @ e, rho[:, None] * u, atol=1e-14)
    P = np.einsum("ni,ia,ib->nab", f, e, e)
    want = rho[:, None, None] * (np.einsum("na,nb->nab", u, u) + np.eye(3)[None] / 3.0)
    if dim == 2:
        P, want = P[:, :2, :2], want[:, :2, :2]
    assert np.allclose(P, want, atol=1e-14)
    ea = e[: (5 if dim == 2 else 7)]
    csa2 = 1 / 3 if dim == 2 else 1 / 4
    assert np.allclose(g.sum(1), conc, atol=1e-14)
    assert np.allclose(g @ ea, conc[:, None] * u, atol=1e-14)
    Pa = np.einsum("ni,ia,ib->nab", g, ea, ea)
    want = conc[:, None, None] * np.eye(3)[None] * csa2
    if dim == 2:
        Pa, want = Pa[:, :2, :2], want[:, :2, :2]
    assert np.allclose(Pa, want, atol=1e-14)
    # weights: rest populations of a fluid at rest
    s.set_cells(t, np.ones(s.N), np.zeros((s.N, 3)), np.ones(s.N), np.ones(s.N))
    f = s.get("fpop")
    w0 = 4 / 9 if dim == 2 else 1 / 3
    assert abs(f[0, 0] - w0) < 1e-15
    assert abs(f[0, 1] - (1 / 9 if dim == 2 else 1 / 18)) < 1e-15
    assert abs(f[0, -1] - 1 / 36) < 1e-15


def _channel(dim, ny, **kw):
    nz = 1 if dim == 2 else 3
    return W.config(nx=3, ny=ny, nz=nz, walls=0b1100, **kw)


@pytest.mark.parametrize("dim", [2, 3])
def test_couette_linear_profile(oracle_mod, dim):
    ny, U = 12, 0.05
    s = oracle_mod.OracleSim(_channel(dim, ny, tau=0.8, wall_u=(U, 0.0, 0.0)))
    s.step(6000)
    u = s.get("u")[:, 0].reshape(-1, ny, 3)[0 if dim == 2 else 1, :, 1]
    y = np.arange(1, ny - 1)
    exact = U * (y - 0.5) / (ny - 2)  # walls half-way between wall and fluid nodes
    assert np.max(np.abs(u[1:-1] - exact)) < 1e-10 * U


def _poiseuille_profile(s, ny, dim):
    u = s.get("u")[:, 0].reshape(s.nz, ny, s.nx)
    return u[0 if dim == 2 else 1, 1:-1, 1]


@pytest.mark.parametrize("dim", [2, 3])
def test_poiseuille_exact_at_magic_tau(oracle_mod, dim):
    ny, g = 10, 1e-5
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    s = oracle_mod.OracleSim(_channel(dim, ny, tau=tau, accel=(g, 0.0, 0.0)))
    s.step(8000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(1, ny - 1)
    H = ny - 2
    exact = g / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
    u = _poiseuille_profile(s, ny, dim)
    assert np.max(np.abs(u - exact)) < 1e-9 * exact.max()


def test_poiseuille_second_order_slip_away_from_magic_tau(oracle_mod):
    ny, g, tau = 18, 1e-6, 1.2
    s = oracle_mod.OracleSim(_channel(2, ny, tau=tau, accel=(g, 0.0, 0.0)))
    s.step(25000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(1, ny - 1)
    H = ny - 2
    exact = g / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
    u = _poiseuille_profile(s, ny, 2)
    err = np.max(np.abs(u - exact)) / exact.max()
    assert 1e-6 < err < 2e-2  # slip of order (tau-1/2)^2 / H^2, not zero


def _solve_channel_quadrature(ny, g, visc_of_rate):
    """Plane channel between half-way walls: shear stress is linear,
    sigma(y) = g (yc - y) (rho = 1); the local rate solves
    sigma = nu(rate) * rate; integrate du/dy = rate from the lower wall."""
    from scipy.optimize import brentq
    from scipy.integrate import quad

    H = ny - 2
    y0, y1 = 0.5, H + 0.5
    yc = 0.5 * (y0 + y1)

    def rate(y):
        sig = abs(g * (yc - y))
        if sig == 0:
            return 0.0
        return brentq(lambda r: visc_of_rate(r) * r - sig, 0.0, 10.0, xtol=1e-16, rtol=1e-14)

    def u_at(y):
        if y <= yc:
            return quad(rate, y0, y, epsabs=1e-14, limit=200)[0]
        return quad(rate, y0, yc, epsabs=1e-14, limit=200)[0] - quad(rate, yc, y, epsabs=1e-14, limit=200)[0]

    return np.array([u_at(y) for y in np.arange(1, ny - 1)])


def test_powerlaw_poiseuille_closed_form(oracle_mod):
    ny, g, n = 26, 2e-6, 0.8
    k = W.powerlaw_k(n, tau_ref=0.8, shear_ref=1e-4)
    cfg = _channel(2, ny, rheo=1, rheo_n=n, rheo_k=k, tau_min=0.505, tau_max=50.0,
                   accel=(g, 0.0, 0.0))
    s = oracle_mod.OracleSim(cfg)
    s.step(30000)
    u = _poiseuille_profile(s, ny, 2)
    H = ny - 2
    y = np.arange(1, ny - 1)
    yc = 0.5 * (0.5 + H + 0.5)
    a = (n + 1) / n
    exact = n / (n + 1) * (g / k) ** (1 / n) * ((H / 2) ** a - np.abs(y - yc) ** a)
    assert np.max(np.abs(u - exact)) < 0.02 * exact.max()


def test_carreau_poiseuille_against_quadrature(oracle_mod):
    ny, g = 26, 2e-5
    lam, nn, a, t0, tinf = 2000.0, 0.5, 2.0, 1.0, 0.55
    cfg = _channel(2, ny, rheo=2, rheo_n=nn, rheo_lambda=lam, rheo_a=a, tau0=t0, tau_inf=tinf,
                   tau_min=0.505, tau_max=2.0, accel=(g, 0.0, 0.0))
    s = oracle_mod.OracleSim(cfg)
    s.step(30000)
    u = _poiseuille_profile(s, ny, 2)

    def nu(r):
        tau = tinf + (t0 - tinf) * (1 + (lam * r) ** a) ** ((nn - 1) / a)
        return (tau - 0.5) / 3.0

    exact = _solve_channel_quadrature(ny, g, nu)
    shear_thin = exact.max() / (g * (ny - 2) ** 2 / (8 * (t0 - 0.5) / 3))
    assert shear_thin > 1.2  # the rheology really acts in this case
    assert np.max(np.abs(u - exact)) < 0.02 * exact.max()


# Two relaxation times (the collision variant Sec. 2 names besides BGK):
# with the product (tau - 1/2)(tau_m - 1/2) = 3/16 the half-way bounce-back
# wall sits exactly half-way for every tau, so body-force Poiseuille flow is
# exact where BGK slips (the test above); with tau_m = tau it is BGK.

@pytest.mark.parametrize("dim", [2, 3])
def test_trt_poiseuille_exact_at_any_tau(oracle_mod, dim):
    ny, g, tau = 18, 1e-6, 1.2
    s = oracle_mod.OracleSim(_channel(dim, ny, tau=tau, accel=(g, 0.0, 0.0), collision=1,
                                      trt_magic=3.0 / 16.0))
    s.step(25000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(1, ny - 1)
    H = ny - 2
    exact = g / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
    u = _poiseuille_profile(s, ny, dim)
    assert np.max(np.abs(u - exact)) < 1e-9 * exact.max()


@pytest.mark.parametrize("dim", [2, 3])
def test_trt_with_equal_rates_is_bgk(oracle_mod, dim):
    """tau_m = tau (trt_magic = (tau - 1/2)^2): the TRT path reproduces the
    BGK path on a random periodic flow state with a body force to
    round-off."""
    rng = np.random.default_rng(7)
    n = 8
    nz = 1 if dim == 2 else n
    base = W.config(nx=n, ny=n, nz=nz, storage="fp64", accel=(2e-5, -1e-5, 0.0), rheo=W.RHEO["newtonian"],
                    tau=0.9, walls=0)
    N = n * n * nz
    t = np.ones(N, np.uint8)
    rho = 1.0 + 0.005 * rng.standard_normal(N)
    u = 0.02 * rng.uniform(-1, 1, (N, 3))
    if dim == 2:
        u[:, 2] = 0.0
    runs = []
    for coll in (0, 1):
        cfg = dict(base, collision=coll, trt_magic=(0.9 - 0.5) ** 2)
        s = oracle_mod.OracleSim(cfg)
        s.set_cells(t, rho, u, np.ones(N), np.zeros(N))
        s.step(50)
        runs.append((s.get("rho"), s.get("u")))
    assert np.max(np.abs(runs[0][0] - runs[1][0])) < 1e-13
    assert np.max(np.abs(runs[0][1] - runs[1][1])) < 1e-14  # velocities O(1e-3)
