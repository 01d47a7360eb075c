"""The allocation-free labelling entry point (lbf_label_gas_noalloc), for
callers that cannot call cudaMalloc, gives exactly the labels of the regular
path (lbf_set_cells + lbf_fields(LABEL)) -- checked on two calls in a row
that share the static scratch array."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _random_types(shape, pg, seed):
    rng = np.random.default_rng(seed)
    r = rng.random(int(np.prod(shape)))
    return np.where(r < pg, 0, np.where(r < pg + 0.15, 2, 1)).astype(np.uint8)


def test_noalloc_labels_match_regular_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1908_04262_gb300 import build as B
    from paper_1908_04262_gb300 import lbf

    B.build()
    cases = [((45, 37, 22), 0.18, 11), ((45, 37, 22), 0.24, 12), ((70, 50, 1), 0.4, 13)]
    for (nx, ny, nz), pg, seed in cases:
        cfg = W.config(nx=nx, ny=ny, nz=nz, storage="fp32", walls=0, sigma=0.01, atmosphere=0)
        sim = lbf.Sim(cfg)
        N = sim.N
        t = _random_types((nz, ny, nx), pg, seed)
        sim.set_cells(t, np.ones(N), np.zeros((N, 3)), np.full(N, 0.5), np.zeros(N))
        ref = sim.fields(["flags", "label"])
        nbub = len(sim.bubbles()["id"])
        sim.close()
        types = torch.tensor(ref["flags"].astype(np.uint8), device="cuda")
        labels = torch.full((N,), 7, dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int32, device="cuda")
        lbf.label_gas_noalloc(types, nx, ny, nz, labels, count)
        torch.cuda.synchronize()
        got = labels.cpu().numpy()
        assert np.array_equal(got, ref["label"]), (nx, ny, nz, int(np.sum(got != ref["label"])))
        assert int(count.item()) == nbub
        assert nbub > 3


def test_noalloc_rejects_oversized_lattice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1908_04262_gb300 import lbf

    t = torch.zeros(8, dtype=torch.uint8, device="cuda")
    lab = torch.zeros(8, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(lbf.LbfError) as e:
        lbf.label_gas_noalloc(t, 1024, 1024, 2, lab, cnt)
    assert e.value.code == -1
