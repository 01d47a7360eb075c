"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (Sec. 2-3 of the paper; tolerances: FP64 storage 1e-10
relative, reduced-precision storage 1e-4 relative for FP32 and a stated
bound for the shifted 16-bit forms)."""
import numpy as np
import pytest

from paper_1908_04262_gb300 import workloads as W
from tests import films
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


def _pair(lbf, oracle_mod, cfg):
    return lbf.Sim(cfg), oracle_mod.OracleSim(cfg)


@pytest.mark.parametrize("dim,rheo", [(2, 0), (3, 0), (2, 1), (3, 2)])
def test_flow_step_fp64(lbf, oracle_mod, dim, rheo):
    """Streaming, bounce-back, Guo forcing, BGK and per-cell tau on a random
    all-liquid state (ragged sizes, several blocks)."""
    nz = 1 if dim == 2 else 11
    cfg = W.config(nx=37, ny=21, nz=nz, storage="fp64", walls=0b1100, tau=0.77,
                   accel=(2e-5, 0.0, 1e-5 if dim == 3 else 0.0), wall_u=(0.02, 0.0, 0.0),
                   rheo=rheo, rheo_n=0.6, rheo_k=W.powerlaw_k(0.6), rheo_lambda=50.0,
                   tau0=0.8, tau_inf=0.505, D=0.04, c0=0.5, q=1e-4)
    sim, ora = _pair(lbf, oracle_mod, cfg)
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


def _c1_small(n=48):
    cfg, _, _ = W.c1_2d_128_fp64()
    cfg.update(nx=n, ny=n, fill_height=n - 8)
    return cfg, [[n / 2 + 0.3, n / 2 - 3.2, 0.0]], [6.0]


def _check_bubbles(sim, ora, tol):
    bg, bo = sim.bubbles(), ora.bubbles()
    assert np.array_equal(bg["root"], bo["root"])
    assert np.array_equal(bg["id"], bo["id"])
    assert np.array_equal(bg["atm"], bo["atm"])
    for k in ("volume", "mass", "pressure"):
        assert rel_err(bg[k], bo[k]) < tol, (k, bg[k], bo[k])


def test_free_surface_fp64_2d(lbf, oracle_mod):
    """The 2D bubble-in-a-box workload (D2Q9 + D2Q5) for 120 steps: flags and
    labels bit-exact, fields and bubble table within 1e-10."""
    cfg, c, r = _c1_small()
    sim, ora = _pair(lbf, oracle_mod, cfg)
    for s in (sim, ora):
        s.nucleate(c, r)
    for _ in range(6):
        sim.step(20)
        ora.step(20)
        errs, nflag = compare_state(sim, ora)
        assert nflag == 0
        assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
        for k, e in errs.items():
            assert e < FP64_TOL, (k, e)
        _check_bubbles(sim, ora, FP64_TOL)
        g = sim.fields(["kappa", "pi"])
        assert rel_err(g["kappa"], ora.get("kappa")) < 1e-9


def test_free_surface_fp64_3d_crop(lbf, oracle_mod):
    """The 32^3 crop workload (power law, disjoining pressure, D3Q7 gas) in
    FP64 for 40 steps (both labelling branches run: growing bubbles add gas
    cells)."""
    cfg, c, r = W.c2_crop_3d_32(storage="fp64")
    sim, ora = _pair(lbf, oracle_mod, cfg)
    for s in (sim, ora):
        s.nucleate(c, r)
    for _ in range(4):
        sim.step(10)
        ora.step(10)
        errs, nflag = compare_state(sim, ora)
        assert nflag == 0
        assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
        for k, e in errs.items():
            assert e < FP64_TOL, (k, e)
        _check_bubbles(sim, ora, FP64_TOL)


@pytest.mark.parametrize("dim,n,pg,seed", [(2, 23, 0.5, 1), (3, 13, 0.4, 2)])
def test_labels_random_fields(lbf, oracle_mod, dim, n, pg, seed):
    rng = np.random.default_rng(seed)
    nz = 1 if dim == 2 else n
    cfg = W.config(nx=n, ny=n + 2, nz=nz, storage="fp64", walls=0, sigma=0.01, atmosphere=1)
    sim, ora = _pair(lbf, oracle_mod, cfg)
    N = sim.N
    r = rng.random(N)
    t = np.where(r < pg, 0, np.where(r < pg + 0.15, 2, 1)).astype(np.uint8)
    alpha = rng.uniform(0.05, 0.95, N)
    for s in (sim, ora):
        s.set_cells(t, np.ones(N), np.zeros((N, 3)), alpha, np.zeros(N))
    assert np.array_equal(sim.fields(["flags"])["flags"], ora.types())
    assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
    _check_bubbles(sim, ora, 1e-12)


def test_geometry_fp64(lbf, oracle_mod):
    """Normals, PLIC offsets, curvature and disjoining pressure on a
    voxelised bubble pair (analytic PLIC on the GPU vs bisection in the
    oracle)."""
    cfg = W.config(nx=30, ny=26, nz=22, storage="fp64", k_pi=2e-3, d_max=4.0, atmosphere=0)
    sim, ora = _pair(lbf, oracle_mod, cfg)
    for s in (sim, ora):
        s.nucleate([[10.3, 12.8, 11.1], [19.9, 13.4, 10.6]], [4.6, 4.1])
    t = ora.types()
    assert np.array_equal(sim.fields(["flags"])["flags"], t)
    g = sim.fields(["normal", "dstar", "kappa", "pi", "alpha"])
    I = t == 2
    assert rel_err(g["alpha"], ora.get("alpha")) < 1e-15
    assert rel_err(g["normal"][I], ora.get("normal")[I]) < 1e-12
    assert rel_err(g["dstar"][I], ora.get("dstar")[I]) < 1e-10
    assert rel_err(g["kappa"][I], ora.get("kappa")[I]) < 1e-9
    assert rel_err(g["pi"][I], ora.get("pi")[I]) < 1e-9
    assert np.max(ora.get("pi")) > 0  # the pair is within reach


@pytest.mark.parametrize("dim,axes", [(2, 2), (3, 2), (3, 3)])
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_disjoining_diagonal_films(lbf, oracle_mod, dim, axes, storage, tol):
    """Disjoining pressure of planar films along the lattice diagonals (the
    oracle's closed-form pin): diagonal ray steps, the hit plane's distance
    and, along (1,1,1), the corner-only face layers that belong to no bubble
    and that rays pass through."""
    N = 24
    cfg = W.config(nx=N, ny=N, nz=N if dim == 3 else 1, storage=storage, k_pi=2e-3, d_max=4.0, atmosphere=0)
    w, t, alpha = films.diagonal_film(N, dim, axes, 1, 0, 2)
    one, zero, zero3 = np.ones(t.size), np.zeros(t.size), np.zeros((t.size, 3))
    ora = oracle_mod.OracleSim(cfg)
    ora.set_cells(t, one, zero3, alpha, zero)
    sim = lbf.Sim(cfg)
    sim.set_cells(t, one, zero3, alpha, zero)
    g = sim.fields(["flags", "label", "pi"])
    assert np.array_equal(g["flags"], ora.types())
    assert np.array_equal(g["label"], ora.labels())
    ref = ora.get("pi")
    assert np.max(ref) > 0
    assert rel_err(g["pi"], ref) < tol
    assert np.array_equal(g["pi"] > 0, ref > 0)
    sim.close()


def test_mass_ledger_gpu(lbf):
    cfg, c, r = _c1_small(64)
    for storage in ("fp64", "fp32"):
        cfg["storage"] = storage
        sim = lbf.Sim(cfg)
        sim.nucleate(c, r)
        L0 = sim.ledger()
        sim.step(300)
        L = sim.ledger()
        m0, m1 = L0[0] + L0[1] + L0[2], L[0] + L[1] + L[2]
        assert abs(m1 - m0) < (1e-12 if storage == "fp64" else 2e-5) * m0, (storage, m0, m1)
        assert L[7] == 0


# Per-field bounds (norm-relative, max |gpu - oracle| / max |oracle| over
# cells liquid or interface in both) after 20 steps of the 32^3 crop.  FP32:
# the 1e-4 of the task for every field.  Shifted 16-bit storage keeps f - w_i
# (g - w_i c0) with unit roundoff 2^-11 (FP16) or 2^-8 (BF16): density, fill
# level, mass and bubble volume integrate many rounded populations with
# alternating signs and stay near the FP32 error; velocity (a small
# difference of populations, max |u| ~ 1e-2) and concentration (which
# departs from c0 by up to ~0.8 at the Henry interface, so the shifted g are
# O(w_i)) carry the storage roundoff itself.
REDUCED_TOL = {
    "fp32": dict(rho=1e-4, u=1e-4, alpha=1e-4, mass=1e-4, conc=1e-4, volume=1e-4),
    "fp16s": dict(rho=1e-4, u=2e-3, alpha=1e-4, mass=1e-4, conc=2e-3, volume=1e-4),
    "bf16s": dict(rho=1e-3, u=2e-2, alpha=2e-2, mass=2e-2, conc=2e-2, volume=1e-4),
}


@pytest.mark.parametrize("storage", ["fp32", "fp16s", "bf16s"])
def test_reduced_precision_crop(lbf, oracle_mod, storage):
    """32^3 crop in FP32 / shifted FP16 / shifted BF16 storage against the
    FP64 oracle after 20 steps; every field's error is printed and bounded
    (REDUCED_TOL); flags must agree exactly."""
    cfg, c, r = W.c2_crop_3d_32(storage=storage)
    sim, ora = _pair(lbf, oracle_mod, cfg)
    for s in (sim, ora):
        s.nucleate(c, r)
    sim.step(20)
    ora.step(20)
    errs, nflag = compare_state(sim, ora)
    bg, bo = sim.bubbles(), ora.bubbles()
    errs["volume"] = rel_err(bg["volume"], bo["volume"])
    print("\n%s: errors against the FP64 oracle %s, flag mismatches %d" % (storage, errs, nflag))
    assert nflag == 0
    for k, bound in REDUCED_TOL[storage].items():
        assert errs[k] < bound, (storage, k, errs[k], bound)


def test_reduced_precision_error_follows_storage_roundoff(lbf):
    """The shifted 16-bit forms differ from the FP32 form only in how the
    populations are stored (the arithmetic is FP32 in all three), so each
    field's deviation from the FP32 form is storage roundoff: after 10 steps
    of the 32^3 crop it stays below two unit roundoffs of the format (2^-11
    for FP16, 2^-8 for BF16) in every field, and the BF16 deviation is the
    FP16 one times the ratio of the unit roundoffs, 8, within a factor 2.5.
    This is what the derived per-field bounds of the 20-step test rest on."""
    fields = ("rho", "u", "alpha", "mass", "conc")
    sims = {}
    for st in ("fp32", "fp16s", "bf16s"):
        cfg, c, r = W.c2_crop_3d_32(storage=st)
        sims[st] = lbf.Sim(cfg)
        sims[st].nucleate(c, r)
        sims[st].step(10)
    ref = sims["fp32"].fields(list(fields) + ["flags"])
    unit = {"fp16s": 2.0 ** -11, "bf16s": 2.0 ** -8}
    err = {}
    for st in ("fp16s", "bf16s"):
        g = sims[st].fields(list(fields) + ["flags"])
        assert np.array_equal(g["flags"], ref["flags"]), st
        both = (ref["flags"] == 1) | (ref["flags"] == 2)
        err[st] = {f: rel_err(g[f], ref[f], both) for f in fields}
        print("\n%s against FP32 after 10 steps: %s" % (st, {f: "%.2e" % v for f, v in err[st].items()}))
        for f in fields:
            assert err[st][f] < 2.0 * unit[st], (st, f, err[st][f])
    for f in fields:
        q = err["bf16s"][f] / err["fp16s"][f]
        assert 8.0 / 2.5 < q < 8.0 * 2.5, (f, q)


@pytest.mark.parametrize("dim", [2, 3])
def test_height_function_curvature_fp64(lbf, oracle_mod, dim):
    """The height-function curvature in the step (cfg kappa = 1): the 2D
    bubble-in-a-box case and the 32^3 crop in FP64 -- flags and labels
    bit-exact, fields, bubble table and curvature within 1e-10 -- and the
    curvature of every interface cell equal to the oracle's height-function
    read-out (limited to [-1, 1]) wherever no column meets a wall."""
    if dim == 2:
        cfg, c, r = _c1_small()
        chunks, per = 4, 25
    else:
        cfg, c, r = W.c2_crop_3d_32(storage="fp64")
        chunks, per = 3, 10
    cfg = dict(cfg, kappa=1)
    sim, ora = _pair(lbf, oracle_mod, cfg)
    for s in (sim, ora):
        s.nucleate(c, r)
    for _ in range(chunks):
        sim.step(per)
        ora.step(per)
        errs, nflag = compare_state(sim, ora)
        assert nflag == 0
        assert np.array_equal(sim.fields(["label"])["label"], ora.labels())
        for k, e in errs.items():
            assert e < FP64_TOL, (k, e)
        _check_bubbles(sim, ora, FP64_TOL)
        kg = sim.fields(["kappa"])["kappa"]
        assert rel_err(kg, ora.get("kappa")) < FP64_TOL
        hf = ora.hf_curvature()
        ok = np.isfinite(hf) & (ora.types() == oracle_mod.IFC)
        assert ok.sum() > 20
        assert np.max(np.abs(kg[ok] - np.clip(hf[ok], -1, 1))) < 1e-10
