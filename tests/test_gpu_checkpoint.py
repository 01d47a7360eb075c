"""Checkpoint and resume through the C ABI (lbf_checkpoint_*): the 32^3
crop (FP64) with a nucleus still queued is saved after 20 steps; resumed in
a fresh sim, and in the same sim rewound, it continues as the uninterrupted
run (flags and labels bit-exact, fields, bubble table and ledgers to
round-off: per-bubble sums are FP64 atomics); a sim of another layout
refuses the checkpoint."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests._parity import rel_err

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


FIELDS = ["rho", "u", "alpha", "mass", "conc", "kappa", "pi"]


def _state(sim):
    return (sim.fields(["flags", "label"]), sim.fields(FIELDS), sim.bubbles(), sim.ledger(),
            sim.step_count())


def _same(a, b):
    (ia, fa, ba, la, sa), (ib, fb, bb, lb, sb) = a, b
    assert sa == sb
    for k in ("flags", "label"):
        assert np.array_equal(ia[k], ib[k]), k
    for k in FIELDS:
        assert rel_err(fb[k], fa[k]) < 1e-12, k
    assert np.array_equal(ba["id"], bb["id"])
    for k in ("volume", "mass", "pressure"):
        assert rel_err(bb[k], ba[k]) < 1e-12, k
    assert np.max(np.abs(lb - la)) <= 1e-12 * np.max(np.abs(la))


def test_checkpoint_resume(lbf):
    cfg, c, r = W.c2_crop_3d_32(storage="fp64")
    pts = np.concatenate([np.asarray(c, float), [[24.0, 22.0, 9.0]]])
    rad = np.concatenate([np.asarray(r, float), [3.0]])
    a = lbf.Sim(cfg)
    a.nucleate(pts, rad, [0, 30])  # the second nucleus is due after the save
    a.step(20)
    buf = a.checkpoint()
    a.step(40)
    ref = _state(a)
    assert len(ref[2]["id"]) >= 3  # both nuclei and the headspace

    b = lbf.Sim(cfg)
    b.restore(buf)
    assert b.step_count() == 20
    b.step(40)
    _same(ref, _state(b))

    a.restore(buf)  # rewind the same sim
    a.step(40)
    _same(ref, _state(a))

    other = lbf.Sim(dict(cfg, nx=cfg["nx"] + 2))
    with pytest.raises(lbf.LbfError):
        other.restore(buf)
    with pytest.raises(lbf.LbfError):
        b.restore(buf[:100])
    for s in (a, b, other):
        s.close()
