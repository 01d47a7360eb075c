"""The dissolution case of Sec. 4.3 through the C ABI against the FP64
oracle: a bubble in a liquid without dissolved gas, 300 steps, flags and
labels bit-exact, fields, bubble table and gas ledgers within 1e-10."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests._parity import compare_state, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbf():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1908_04262_gb300 import build as B
    from paper_1908_04262_gb300 import lbf as L

    B.build()
    return L


def test_dissolution_2d_matches_oracle(lbf, oracle_mod):
    cfg, c, r = W.dissolution_2d()
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(cfg)
    for s in (sim, ora):
        s.nucleate(c, r)
    for _ in range(3):
        sim.step(100)
        ora.step(100)
        errs, nflag = compare_state(sim, ora)
        assert nflag == 0
        assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
        for k, e in errs.items():
            assert e < 1e-10, (k, e)
    bg, bo = sim.bubbles(), ora.bubbles()
    for k in ("volume", "mass", "pressure"):
        assert rel_err(bg[k], bo[k]) < 1e-10, k
    lg, lo = sim.ledger(), ora.ledger()
    for k in (3, 4, 5):
        assert abs(lg[k] - lo[k]) <= 1e-10 * max(abs(lo[k]), 1e-30), (k, lg[k], lo[k])
