"""The 2D foam cases of Sec. 4.4 (foaming with a gas source; foam drainage
under gravity) on the oracle: the workload generator's nuclei, exact
liquid-mass conservation and the source term feeding bubble growth."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W


@pytest.mark.parametrize("which", ["foam", "drainage"])
def test_2d_foam_workloads_place_nuclei_in_the_liquid(which):
    if which == "foam":
        cfg, pts, rad = W.foam_2d_450x650()
        n, spacing = 300, 9.0
    else:
        cfg, pts, rad = W.drainage_2d_450x650()
        n, spacing = 150, 9.0
    assert (cfg["nx"], cfg["ny"], cfg["nz"]) == (450, 650, 1)
    assert len(pts) == n and np.all(rad == 3.0)
    h = cfg["fill_height"]
    assert np.all(pts[:, 0] - rad >= 1.0) and np.all(pts[:, 0] + rad <= cfg["nx"] - 1.0)
    assert np.all(pts[:, 1] - rad >= 1.0) and np.all(pts[:, 1] + rad <= h - 1.0)
    d = np.sqrt(((pts[:, None, :2] - pts[None, :, :2]) ** 2).sum(-1))
    assert np.min(d[np.triu_indices(n, 1)]) >= spacing
    # tau_g of the paper's captions from D on D2Q5 (c_s^2 = 1/3)
    assert abs(0.5 + 3.0 * cfg["D"] - (0.6 if which == "foam" else 0.53)) < 1e-12


@pytest.mark.parametrize("drainage", [False, True])
def test_2d_foam_crop_oracle_conserves_liquid_mass(oracle_mod, drainage):
    """Liquid mass (rho of liquid cells + M of interface cells + excess that
    found no interface neighbour + liquid removed by nucleation) is exact in
    FP64 through conversions, with the gas source or gravity on."""
    cfg, pts, rad = W.foam_2d_crop(drainage=drainage)
    s = oracle_mod.OracleSim(cfg)
    s.nucleate(pts, rad)
    L0 = s.ledger()
    b0 = s.bubbles()
    v0 = b0["volume"][~b0["atm"].astype(bool)]
    s.step(200)
    L = s.ledger()
    m0, m1 = L0[0] + L0[1] + L0[2], L[0] + L[1] + L[2]
    assert abs(m1 - m0) < 1e-12 * m0
    assert L[7] == 0
    b = s.bubbles()
    atm = b["atm"].astype(bool)
    if not drainage:
        # the source term (q > 0, no initial dissolved gas) makes every
        # nucleus grow
        assert L[6] > 0
        assert len(b["volume"][~atm]) == len(v0)
        assert np.all(b["volume"][~atm] > 1.02 * np.max(v0))
