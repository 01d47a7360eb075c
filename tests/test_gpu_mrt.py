"""The multiple-relaxation-time collision (the other variant Sec. 2 names
beside BGK) through the C ABI against the FP64 oracle: a random all-liquid
flow with walls, moving lid, Guo forcing and per-cell tau with every group
at its own rate; the 2D bubble-in-a-box free-surface case; the 32^3 crop in
FP32 and FP16S."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests._parity import compare_state, rel_err

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
RATES = (1.15, 1.3, 1.7, 1.85)  # s_e, s_eps, s_pi, s_m


@pytest.fixture(scope="module")
def lbf():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1908_04262_gb300 import build as B
    from paper_1908_04262_gb300 import lbf as L

    B.build()
    return L


@pytest.mark.parametrize("dim,rheo", [(2, 0), (3, 0), (3, 1)])
def test_mrt_flow_step_fp64(lbf, oracle_mod, dim, rheo):
    nz = 1 if dim == 2 else 11
    cfg = W.config(nx=37, ny=21, nz=nz, storage="fp64", walls=0b1100, tau=0.77,
                   accel=(2e-5, 0.0, 1e-5 if dim == 3 else 0.0), wall_u=(0.02, 0.0, 0.0),
                   rheo=rheo, rheo_n=0.6, rheo_k=W.powerlaw_k(0.6), D=0.04, c0=0.5, q=1e-4,
                   collision=2, trt_magic=3.0 / 16.0, mrt_rates=RATES)
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(cfg)
    rho, u, conc = W.random_flow_state(cfg, seed=23, du=0.05)
    t = ora.types()
    for s in (sim, ora):
        s.set_cells(t, rho, u, np.ones(t.size), conc)
    for _ in range(3):
        sim.step(7)
        ora.step(7)
        errs, nflag = compare_state(sim, ora, ("rho", "u", "conc"))
        assert nflag == 0
        for k, e in errs.items():
            assert e < FP64_TOL, (k, e)


def test_mrt_default_rates_match_trt_fp64(lbf, oracle_mod):
    """Rates left at 0 follow the TRT rates: the MRT sweep then gives the
    TRT sweep's state to round-off (both on the device)."""
    cfg = W.config(nx=37, ny=21, nz=11, storage="fp64", walls=0b1100, tau=0.77, accel=(2e-5, 0.0, 1e-5),
                   wall_u=(0.02, 0.0, 0.0), D=0.04, c0=0.5, trt_magic=3.0 / 16.0)
    rho, u, conc = W.random_flow_state(cfg, seed=5, du=0.05)
    t = oracle_mod.OracleSim(cfg).types()
    out = []
    for coll in (1, 2):
        sim = lbf.Sim(dict(cfg, collision=coll))
        sim.set_cells(t, rho, u, np.ones(t.size), conc)
        sim.step(20)
        out.append(sim.fields(["rho", "u"]))
    assert np.max(np.abs(out[0]["rho"] - out[1]["rho"])) < 1e-13
    assert np.max(np.abs(out[0]["u"] - out[1]["u"])) < 1e-14


def test_mrt_free_surface_fp64_2d(lbf, oracle_mod):
    cfg, _, _ = W.c1_2d_128_fp64()
    n = 48
    cfg.update(nx=n, ny=n, fill_height=n - 8, collision=2, trt_magic=3.0 / 16.0, mrt_rates=RATES)
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(cfg)
    for s in (sim, ora):
        s.nucleate([[n / 2 + 0.3, n / 2 - 3.2, 0.0]], [6.0])
    for _ in range(3):
        sim.step(20)
        ora.step(20)
        errs, nflag = compare_state(sim, ora)
        assert nflag == 0
        assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
        for k, e in errs.items():
            assert e < FP64_TOL, (k, e)
    bg, bo = sim.bubbles(), ora.bubbles()
    for k in ("volume", "mass", "pressure"):
        assert rel_err(bg[k], bo[k]) < FP64_TOL, k


# the bounds of the BGK crop test: the collision adds no storage roundoff
CROP_TOL = {
    "fp32": dict(rho=1e-4, u=1e-4, alpha=1e-4, mass=1e-4, conc=1e-4),
    "fp16s": dict(rho=1e-4, u=2e-3, alpha=1e-4, mass=1e-4, conc=2e-3),
}


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_mrt_crop(lbf, oracle_mod, storage):
    cfg, c, r = W.c2_crop_3d_32(storage=storage)
    cfg.update(collision=2, trt_magic=3.0 / 16.0, mrt_rates=RATES)
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(dict(cfg, storage="fp64"))
    for s in (sim, ora):
        s.nucleate(c, r)
    sim.step(20)
    ora.step(20)
    errs, nflag = compare_state(sim, ora)
    print("\nMRT %s: errors against the FP64 oracle %s" % (storage, errs))
    assert nflag == 0
    for k, bound in CROP_TOL[storage].items():
        assert errs[k] < bound, (storage, k, errs[k], bound)
