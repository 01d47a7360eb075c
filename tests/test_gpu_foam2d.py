"""The 2D foam cases of Sec. 4.4 through the C ABI: the 64 x 96 crops
(foaming with a gas source; drainage under gravity) element-wise against
the FP64 oracle, and the full 450 x 650 cases in FP32 checked by the
properties that hold at any size (the MLUPS of each run are printed)."""
import time

import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests._parity import compare_state, rel_err
from tests.test_gpu_fullsize import _check_properties

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


@pytest.mark.parametrize("drainage", [False, True])
def test_2d_foam_crop_matches_oracle(lbf, oracle_mod, drainage):
    cfg, pts, rad = W.foam_2d_crop(drainage=drainage)
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(cfg)
    for s in (sim, ora):
        s.nucleate(pts, rad)
    for _ in range(4):
        sim.step(50)
        ora.step(50)
        errs, nflag = compare_state(sim, ora)
        assert nflag == 0
        assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
        for k, e in errs.items():
            assert e < FP64_TOL, (k, e)
    bg, bo = sim.bubbles(), ora.bubbles()
    assert np.array_equal(bg["id"], bo["id"])
    for k in ("volume", "mass", "pressure"):
        assert rel_err(bg[k], bo[k]) < FP64_TOL, k
    lg, lo = sim.ledger(), ora.ledger()
    for k in (0, 3, 4, 6):
        assert abs(lg[k] - lo[k]) <= 1e-10 * max(abs(lo[k]), 1e-30), (k, lg[k], lo[k])


@pytest.mark.parametrize("which", ["foam", "drainage"])
def test_2d_foam_450x650_fp32_full_size_properties(lbf, which):
    cfg, pts, rad = W.foam_2d_450x650() if which == "foam" else W.drainage_2d_450x650()
    sim = lbf.Sim(cfg)
    sim.nucleate(pts, rad)
    sim.step(20)
    steps = 400
    t0 = time.perf_counter()
    sim.step(steps)  # returns after the device has finished
    dt = time.perf_counter() - t0
    N = cfg["nx"] * cfg["ny"]
    print("\n2D %s 450x650 FP32: %.0f MLUPS (%d steps, wall clock around lbf_step)" % (which, N * steps / dt / 1e6, steps))
    n = _check_properties(sim, cfg)
    assert n >= 2
    L = sim.ledger()
    assert L[7] == 0
    if which == "foam":
        assert L[6] > 0  # the source term adds gas
