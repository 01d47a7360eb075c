"""The error contract of the C ABI (include/lbf.h): every failure is a
negative LBF_E* code with a message, caused here from the host side only --
bad configurations, bad arguments, a host-built field holding a NaN, more
bubbles than the configured capacity.  Configuration errors are found before
any CUDA call, so those tests run without a GPU."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W

EINVAL, ENONFINITE, ECAPACITY = -1, -5, -6


def _lib_or_skip():
    from paper_1908_04262_gb300 import build as B
    from paper_1908_04262_gb300 import lbf

    try:
        B.build()
    except Exception as e:  # pragma: no cover - needs nvcc
        pytest.skip("library not built and nvcc unavailable: %s" % e)
    return lbf


BAD_CONFIGS = [
    ("zero extent", dict(nx=0)),
    ("negative extent", dict(ny=-4)),
    ("extent below 3", dict(nx=2)),
    ("more than 2^31-1 cells", dict(nx=2048, ny=2048, nz=1024)),
    ("tau at 1/2", dict(tau=0.5)),
    ("tau below 1/2", dict(tau=0.3)),
    ("bad storage", dict(storage=7)),
    ("bad rheology", dict(rheo=5)),
    ("tau_min at 1/2", dict(rheo=1, tau_min=0.5)),
    ("tau_max below tau_min", dict(rheo=2, tau_min=0.6, tau_max=0.55)),
    ("zero diffusivity", dict(D=0.0)),
    ("zero RT", dict(RT=0.0)),
    ("negative rho0", dict(rho0=-1.0)),
    ("capacity 0", dict(bubble_capacity=0)),
    ("capacity above 16384", dict(bubble_capacity=20000)),
    ("bad collision", dict(collision=3)),
    ("TRT without magic", dict(collision=1, trt_magic=0.0)),
    ("MRT without magic", dict(collision=2, trt_magic=-1.0)),
    ("MRT rate at 2", dict(collision=2, mrt_rates=(1.2, 2.0, 0.0, 0.0))),
    ("MRT rate negative", dict(collision=2, mrt_rates=(0.0, 0.0, 0.0, -0.5))),
    ("MRT rate NaN", dict(collision=2, mrt_rates=(float("nan"), 0.0, 0.0, 0.0))),
    ("disjoining range 0", dict(k_pi=1e-3, d_max=0.0)),
    ("bad curvature method", dict(kappa=2)),
]


@pytest.mark.parametrize("name,bad", BAD_CONFIGS, ids=[b[0] for b in BAD_CONFIGS])
def test_create_rejects_bad_configuration(name, bad):
    """lbf_create returns LBF_EINVAL (and no handle) for each configuration
    the header excludes; the check comes before any device work."""
    lbf = _lib_or_skip()
    cfg = W.config(nx=16, ny=16, nz=16, storage="fp32")
    cfg.update(bad)
    with pytest.raises(lbf.LbfError) as ei:
        lbf.Sim(cfg)
    assert ei.value.code == EINVAL, (name, str(ei.value))


def test_network_calls_reject_bad_arguments_on_the_host():
    """The learned-curvature entry points check their arguments before any
    CUDA call: NULL pointers, negative or empty counts, radii that are not
    positive and training configurations outside the header's ranges are
    LBF_EINVAL; an empty forward pass (n = 0) succeeds without a launch."""
    import ctypes

    lbf = _lib_or_skip()
    lib = lbf.load()
    d = ctypes.c_void_p(16)  # never dereferenced: every call below returns first
    assert lib.lbf_mlp_forward(None, d, 4, d, None) == EINVAL
    assert lib.lbf_mlp_forward(d, d, -1, d, None) == EINVAL
    assert lib.lbf_mlp_forward(d, d, 0, d, None) == 0
    assert lib.lbf_mlp_loss_grad(d, d, d, 0, d, d, None) == EINVAL
    assert lib.lbf_mlp_loss_grad(d, None, d, 8, d, d, None) == EINVAL
    assert lib.lbf_mlp_generate(1, 8, 0.0, 4.0, d, d, None) == EINVAL
    assert lib.lbf_mlp_generate(1, 8, 5.0, 4.0, d, d, None) == EINVAL
    assert lib.lbf_mlp_generate(1, -1, 2.0, 4.0, d, d, None) == EINVAL
    assert lib.lbf_mlp_stencils_from_params(d, 0, d, d, None) == EINVAL
    assert lib.lbf_mlp_attach(None, None) == EINVAL
    assert lib.lbf_mlp_harvest(None, d, d, None, 4, ctypes.byref(ctypes.c_int())) == EINVAL
    theta = (ctypes.c_float * lbf.MLP_NPARAM)()
    assert lib.lbf_mlp_train(None, theta, None) == EINVAL
    good = dict(seed=1, n_samples=4096, epochs=1, batch=256, lr=1e-3, rmin=2.0, rmax=20.0, noise=0.0,
                x_extra=None, y_extra=None, n_extra=0, stream=None)
    for bad in (dict(batch=8), dict(epochs=0), dict(n_samples=-1), dict(noise=-0.1), dict(n_samples=100),
                dict(n_extra=5)):
        cfg = lbf.MlpTrainCfg(**dict(good, **bad))
        assert lib.lbf_mlp_train(ctypes.byref(cfg), theta, None) == EINVAL, bad
    assert b"bad" in lib.lbf_last_error() or b"fewer" in lib.lbf_last_error()


def test_noalloc_labelling_rejects_bad_sizes_on_the_host():
    """The labelling entry point that allocates nothing checks its buffers
    and sizes before any CUDA call: NULL buffers, extents below 3, and
    lattices beyond its static scratch (1,048,576 cells) are LBF_EINVAL with
    a message naming the limit."""
    import ctypes

    lbf = _lib_or_skip()
    lib = lbf.load()
    d = ctypes.c_void_p(16)  # never dereferenced
    assert lib.lbf_label_gas_noalloc(None, 8, 8, 1, d, d, None) == EINVAL
    assert lib.lbf_label_gas_noalloc(d, 2, 8, 1, d, d, None) == EINVAL
    assert lib.lbf_label_gas_noalloc(d, 8, 8, 2, d, d, None) == EINVAL
    assert lib.lbf_label_gas_noalloc(d, 1024, 1025, 1, d, d, None) == EINVAL
    assert b"1,048,576" in lib.lbf_last_error()
    assert lib.lbf_label_gas_noalloc(d, 128, 128, 65, d, d, None) == EINVAL


def test_create_rejects_null_config():
    import ctypes

    lbf = _lib_or_skip()
    lib = lbf.load()
    h = ctypes.c_void_p()
    assert lib.lbf_create(None, ctypes.byref(h)) == EINVAL
    assert not h.value
    assert b"NULL" in lib.lbf_last_error()


def _gpu_or_fail():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")


def _box_2d(**kw):
    # an all-liquid closed 2D box: no headspace, so every bubble is a nucleus
    return W.config(nx=48, ny=40, nz=1, storage="fp64", walls=0b1111, fill_height=100.0, atmosphere=0,
                    sigma=0.01, **kw)


@pytest.mark.gpu
def test_capacity_exceeded_is_reported():
    """Two separate nuclei in a sim that holds one bubble: LBF_ECAPACITY from
    the call that made the second bubble (bubble_capacity = 1)."""
    _gpu_or_fail()
    lbf = _lib_or_skip()
    sim = lbf.Sim(_box_2d(bubble_capacity=1))
    sim.nucleate([[12.3, 20.1, 0.0]], [4.0])
    assert len(sim.bubbles()["id"]) == 1
    with pytest.raises(lbf.LbfError) as ei:
        sim.nucleate([[34.2, 19.7, 0.0]], [4.0])
    assert ei.value.code == ECAPACITY
    sim.close()
    # the same two nuclei fit a capacity of two
    sim = lbf.Sim(_box_2d(bubble_capacity=2))
    sim.nucleate([[12.3, 20.1, 0.0], [34.2, 19.7, 0.0]], [4.0, 4.0])
    sim.step(4)
    assert len(sim.bubbles()["id"]) == 2
    sim.close()


@pytest.mark.gpu
def test_set_cells_rejects_nan_and_bad_types_and_keeps_the_state():
    """A NaN in a host-built field gives LBF_ENONFINITE, a cell type 7 or a
    zero density in a liquid cell LBF_EINVAL; the rejected call leaves the
    state as it was."""
    _gpu_or_fail()
    lbf = _lib_or_skip()
    cfg = _box_2d()
    sim = lbf.Sim(cfg)
    sim.nucleate([[24.0, 20.0, 0.0]], [5.0])
    sim.step(3)
    before = sim.fields(["rho", "alpha", "flags", "label"])
    N = sim.N
    types = before["flags"].astype(np.uint8)
    rho = np.where(types == 1, 1.0, np.where(types == 2, 1.0, 0.0))
    u = np.zeros(3 * N)
    alpha = before["alpha"].copy()
    conc = np.full(N, 1.0)
    for field, idx, value, code in (("rho", 500, np.nan, ENONFINITE), ("u", 77, np.inf, ENONFINITE),
                                    ("alpha", 900, -np.inf, ENONFINITE), ("conc", 3, np.nan, ENONFINITE),
                                    ("types", 60, 7, EINVAL), ("rho", 200, 0.0, EINVAL)):
        args = dict(types=types.copy(), rho=rho.copy(), u=u.copy(), alpha=alpha.copy(), conc=conc.copy())
        if field == "rho" and value == 0.0:
            idx = int(np.flatnonzero(types == 1)[0])
        args[field][idx] = value
        with pytest.raises(lbf.LbfError) as ei:
            sim.set_cells(**args)
        assert ei.value.code == code, (field, str(ei.value))
        after = sim.fields(["rho", "alpha", "flags", "label"])
        for k in before:
            assert np.array_equal(before[k], after[k]), (field, k)
    # the untouched arrays are accepted
    sim.set_cells(types, rho, u, alpha, conc)
    sim.step(2)
    sim.close()


@pytest.mark.gpu
def test_bad_call_arguments():
    """Negative step counts, non-positive radii, nucleation in the past and
    unknown field bits are LBF_EINVAL."""
    import ctypes

    _gpu_or_fail()
    lbf = _lib_or_skip()
    sim = lbf.Sim(_box_2d())
    lib = sim.lib
    assert lib.lbf_step(sim.h, -1) == EINVAL
    with pytest.raises(lbf.LbfError) as ei:
        sim.nucleate([[24.0, 20.0, 0.0]], [0.0])
    assert ei.value.code == EINVAL
    sim.step(5)
    with pytest.raises(lbf.LbfError) as ei:
        sim.nucleate([[24.0, 20.0, 0.0]], [3.0], at_step=[2])
    assert ei.value.code == EINVAL
    dst = (ctypes.c_void_p * 1)()
    assert lib.lbf_fields(sim.h, 1 << 12, dst, 0, 1) == EINVAL
    assert lib.lbf_fields(sim.h, 1, dst, 0, 1) == EINVAL  # NULL destination
    assert lib.lbf_fields(sim.h, 1, dst, 0, 2) == EINVAL  # bad dtype
    cnt = ctypes.c_int()
    assert lib.lbf_bubbles(sim.h, None, -1, ctypes.byref(cnt)) == EINVAL
    assert sim.step_count() == 5
    sim.close()
