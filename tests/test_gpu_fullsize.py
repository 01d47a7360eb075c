"""The workloads at their full sizes, in the launch configuration the
benchmark times (step graphs in which consecutive steps overlap; a graph of
two steps for the 128^3 case, the library's own stream).

* 2D 128^2 FP64 and 3D 128^3 FP32: element-wise against the FP64 oracle
  (the oracle runs the whole lattice: 200 steps in 2D, two steps in 3D).
* 256^3 shifted FP16 and 512x512x384 shifted BF16: properties that hold at
  any size, checked on the whole lattice on the host: liquid never touches
  gas; gas labels are the connected components of the gas cells over the
  lattice links, ranked by their smallest linear index; every interface cell
  carries the smallest label of its gas neighbours; every bubble's volume
  is its gas cells plus the empty fraction of its interface cells.
"""
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


def test_2d_128_fp64_full_size_matches_oracle(lbf, oracle_mod):
    cfg, c, r = W.c1_2d_128_fp64()
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(cfg)
    for s in (sim, ora):
        s.nucleate(c, r)
    for _ in range(4):
        sim.step(50)
        ora.step(50)
        errs, nflag = compare_state(sim, ora)
        assert nflag == 0
        for k, e in errs.items():
            assert e < 1e-10, (k, e)
    assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
    bg, bo = sim.bubbles(), ora.bubbles()
    assert rel_err(bg["volume"], bo["volume"]) < 1e-10
    assert rel_err(bg["pressure"], bo["pressure"]) < 1e-10


def test_3d_128_fp32_full_size_matches_oracle(lbf, oracle_mod):
    """The benchmark's workload itself: two steps (one two-step graph)."""
    cfg, pts, rad = W.c2_3d_128_fp32()
    sim, ora = lbf.Sim(cfg), oracle_mod.OracleSim(cfg)
    for s in (sim, ora):
        s.nucleate(pts, rad)
    sim.step(2)
    ora.step(2)
    errs, nflag = compare_state(sim, ora)
    print("\n128^3 FP32 after 2 steps: errors against the FP64 oracle %s" % errs)
    assert nflag == 0
    for k, e in errs.items():
        assert e < 1e-4, (k, e)
    assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
    assert rel_err(sim.bubbles()["volume"], ora.bubbles()["volume"]) < 1e-4


def _links(dim):
    if dim == 2:
        return [(dx, dy, 0) for dx in (-1, 0, 1) for dy in (-1, 0, 1) if (dx, dy) != (0, 0)]
    return [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
            if 0 < abs(dx) + abs(dy) + abs(dz) <= 2]


def _check_properties(sim, cfg):
    from scipy import ndimage

    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    f = sim.fields(["flags", "label", "alpha"], dtype=np.float32)
    t = (f["flags"] & 3).reshape(nz, ny, nx)
    lab = f["label"].reshape(nz, ny, nx)
    alpha = f["alpha"].reshape(nz, ny, nx).astype(np.float64)
    gas, liq, ifc = t == 0, t == 1, t == 2
    links = _links(3 if nz > 1 else 2)
    # liquid never touches gas (periodic neighbours; the faces are walls)
    for dx, dy, dz in links:
        assert not np.any(liq & np.roll(gas, (-dz, -dy, -dx), axis=(0, 1, 2)))
    # gas components over the lattice links, ranked by smallest linear index
    st = np.zeros((3, 3, 3), bool)
    st[1, 1, 1] = True
    for dx, dy, dz in links:
        st[dz + 1, dy + 1, dx + 1] = True
    comp, ncomp = ndimage.label(gas, structure=st)
    flat = comp.reshape(-1)
    idx = np.nonzero(flat)[0]
    first = np.full(ncomp + 1, np.iinfo(np.int64).max)
    np.minimum.at(first, flat[idx], idx)
    rank = np.empty(ncomp + 1, np.int64)
    rank[np.argsort(first[1:]) + 1] = np.arange(ncomp)
    assert np.array_equal(lab.reshape(-1)[idx], rank[flat[idx]])
    # interface cells: the smallest label of their gas neighbours
    big = np.iinfo(np.int32).max
    gl = np.where(gas, lab, big)
    best = np.full(lab.shape, big)
    for dx, dy, dz in links:
        best = np.minimum(best, np.roll(gl, (-dz, -dy, -dx), axis=(0, 1, 2)))
    want = np.where(best == big, -1, best)
    assert np.array_equal(lab[ifc], want[ifc])
    # volumes: gas cells + empty fraction of interface cells, per label
    vol = np.bincount(lab[gas], minlength=ncomp).astype(np.float64)
    ii = ifc & (lab >= 0)
    vol += np.bincount(lab[ii], weights=1.0 - alpha[ii], minlength=ncomp)
    b = sim.bubbles()
    assert len(b["volume"]) == ncomp
    assert rel_err(b["volume"], vol[:ncomp]) < 1e-9
    return ncomp


def test_3d_256_fp16s_full_size_properties(lbf):
    cfg, pts, rad, times = W.c3_3d_256_fp16s()
    sim = lbf.Sim(cfg)
    sim.nucleate(pts, rad, times)
    sim.step(60)
    n = _check_properties(sim, cfg)
    assert n >= 3  # the atmosphere and the nuclei due by step 60


def test_3d_512x512x384_bf16s_full_size_properties(lbf):
    cfg, pts, rad = W.c5_3d_512x512x384_bf16s()
    sim = lbf.Sim(cfg)
    sim.nucleate(pts, rad)
    sim.step(4)
    n = _check_properties(sim, cfg)
    assert n > 1000
