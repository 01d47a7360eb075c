"""The two-relaxation-time collision (the variant Sec. 2 names besides BGK)
through the C ABI against the FP64 oracle: a random all-liquid flow with
walls, moving lid, Guo forcing and per-cell tau; the 2D bubble-in-a-box
free-surface case; the 32^3 crop in FP32."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests._parity import compare_state, rel_err

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def lbf():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1908_04262_gb300 import build as B
    from paper_1908_04262_gb300 import lbf as L

    B.build()
    return L


@pytest.mark.parametrize("dim,rheo", [(2, 0), (3, 1)])
def test_trt_flow_step_fp64(lbf, oracle_mod, dim, rheo):
    nz = 1 if dim == 2 else 11
    cfg = W.config(nx=37, ny=21, nz=nz, storage="fp64", walls=0b1100, tau=0.77,
                   accel=(2e-5, 0.0, 1e-5 if dim == 3 else 0.0), wall_u=(0.02, 0.0, 0.0),
                   rheo=rheo, rheo_n=0.6, rheo_k=W.powerlaw_k(0.6), D=0.04, c0=0.5, q=1e-4,
                   collision=1, trt_magic=3.0 / 16.0)
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(cfg)
    rho, u, conc = W.random_flow_state(cfg, seed=17, du=0.05)
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


def test_trt_free_surface_fp64_2d(lbf, oracle_mod):
    cfg, _, _ = W.c1_2d_128_fp64()
    n = 48
    cfg.update(nx=n, ny=n, fill_height=n - 8, collision=1, trt_magic=3.0 / 16.0)
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


def test_trt_crop_fp32(lbf, oracle_mod):
    cfg, c, r = W.c2_crop_3d_32(storage="fp32")
    cfg.update(collision=1, trt_magic=3.0 / 16.0)
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(dict(cfg, storage="fp64"))
    for s in (sim, ora):
        s.nucleate(c, r)
    sim.step(20)
    ora.step(20)
    errs, nflag = compare_state(sim, ora)
    assert nflag == 0
    for k, e in errs.items():
        assert e < 1e-4, (k, e)
