"""Pins of the oracle's bubble labelling and gas bookkeeping (Sec. 3.5,
Sec. 2.2 Eq. idealgas): connected components against scipy.ndimage.label
with the lattice-link structure, volumes by brute force, Laplace-equilibrium
initial pressure, and conservation of gas content through merge and split."""
import numpy as np
import pytest
from scipy import ndimage

from paper_1908_04262_gb300 import workloads as W


def _structure(dim):
    if dim == 2:
        return np.ones((3, 3), bool)  # D2Q9 links: 8 neighbours
    st = np.ones((3, 3, 3), bool)
    for c in [(0, 0, 0), (0, 0, 2), (0, 2, 0), (0, 2, 2), (2, 0, 0), (2, 0, 2), (2, 2, 0), (2, 2, 2)]:
        st[c] = False  # D3Q19 links: no corners
    return st


def _random_state(oracle_mod, dim, n, pg, seed):
    rng = np.random.default_rng(seed)
    nz = 1 if dim == 2 else n
    shape = (nz, n, n)
    walls = 0xF if dim == 2 else 0x3F
    cfg = W.config(nx=n, ny=n, nz=nz, walls=walls, sigma=0.01, atmosphere=0)
    s = oracle_mod.OracleSim(cfg)
    t = s.types().reshape(shape).copy()
    inner = t != oracle_mod.WALL
    r = rng.random(shape)
    t[inner & (r < pg)] = oracle_mod.GAS
    t[inner & (r >= pg) & (r < pg + 0.15)] = oracle_mod.IFC
    t[inner & (r >= pg + 0.15)] = oracle_mod.LIQ
    alpha = rng.uniform(0.05, 0.95, shape)
    s.set_cells(t.reshape(-1), np.ones(s.N), np.zeros((s.N, 3)), alpha.reshape(-1),
                np.zeros(s.N))
    return s, shape


@pytest.mark.parametrize("dim,n,pg,seed", [(2, 14, 0.45, 1), (2, 20, 0.55, 2), (3, 9, 0.35, 3),
                                           (3, 10, 0.45, 4)])
def test_labels_match_connected_components(oracle_mod, dim, n, pg, seed):
    s, shape = _random_state(oracle_mod, dim, n, pg, seed)
    t = s.types().reshape(shape)
    lab = s.labels().reshape(shape)
    G = t == oracle_mod.GAS
    st = _structure(dim)
    ref, ncomp = ndimage.label(G if dim == 3 else G[0], structure=st)
    if dim == 2:
        ref = ref[None]
    assert s.bubbles()["volume"].size == ncomp
    # canonical numbering: components ordered by their smallest linear index
    flat_ref = ref.reshape(-1)
    first = {}
    for idx in np.flatnonzero(flat_ref):
        first.setdefault(flat_ref[idx], idx)
    order = sorted(first, key=first.get)
    canon = np.full(ncomp + 1, -1)
    for k, c in enumerate(order):
        canon[c] = k
    want = np.where(flat_ref > 0, canon[flat_ref], -1)
    flat_lab = lab.reshape(-1)
    assert np.array_equal(flat_lab[G.reshape(-1)], want[G.reshape(-1)])
    assert np.array_equal(s.bubbles()["root"], np.array([first[c] for c in order]))
    # interface cells: smallest label among gas lattice neighbours, else -1
    nz, ny, nx = shape
    offs = np.argwhere(st) - 1
    for idx in np.flatnonzero(t.reshape(-1) == oracle_mod.IFC):
        z, y, x = np.unravel_index(idx, shape)
        best = -1
        for o in offs:
            zz, yy, xx = (z + (o[0] if dim == 3 else 0)) % nz, (y + o[-2]) % ny, (x + o[-1]) % nx
            if G[zz, yy, xx]:
                k = want.reshape(shape)[zz, yy, xx]
                best = k if best < 0 else min(best, k)
        assert flat_lab[idx] == best
    # volumes: gas cells plus (1 - alpha) of the interface cells
    alpha = s.get("alpha")
    V = np.zeros(ncomp)
    for idx in range(s.N):
        if flat_lab[idx] >= 0:
            V[flat_lab[idx]] += 1.0 if G.reshape(-1)[idx] else 1.0 - alpha[idx]
    assert np.allclose(s.bubbles()["volume"], V, rtol=0, atol=1e-12)


def test_new_bubble_starts_in_laplace_equilibrium(oracle_mod):
    cfg = W.config(nx=40, ny=40, nz=1, sigma=0.02, RT=0.5, atmosphere=0)
    s = oracle_mod.OracleSim(cfg)
    s.nucleate([[20.0, 20.0, 0.0]], [7.0])
    b = s.bubbles()
    Req = np.sqrt(b["volume"][0] / np.pi)
    assert abs(b["pressure"][0] - (1 / 3 + 0.02 / Req)) < 1e-14
    assert abs(b["mass"][0] - b["pressure"][0] * b["volume"][0] / 0.5) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_nucleated_volume_matches_the_disk_or_sphere(oracle_mod, dim):
    """Nucleation carves fill levels from 4^d sub-cell points per cell (the
    fraction outside the sphere is the liquid fraction): the bubble's
    volume (gas cells + sum of 1 - alpha over its interface cells) is the
    disk's or sphere's within a bound that falls like 1/R -- 0.05/R in 2D,
    0.03/R in 3D, against measured errors of 1.2 % (2D) and 0.16 % (3D) at
    R = 2.7.  Carving whole cells by their centres (no sub-points) breaks
    the bound in 8 of the 12 2D cases and 5 of the 12 3D cases below (up to
    0.14/R and 0.08/R); taking the sampled fraction inside the sphere as the
    liquid fraction misses by far more."""
    import math

    rng = np.random.default_rng(3)
    for R in (2.7, 4.3, 6.1, 9.4):
        for _ in range(3):
            n = int(2 * R + 8)
            cfg = W.config(nx=n, ny=n, nz=n if dim == 3 else 1, atmosphere=0)
            s = oracle_mod.OracleSim(cfg)
            c = n / 2 + rng.uniform(-0.5, 0.5, 3)
            if dim == 2:
                c[2] = 0.0
            s.nucleate([list(c)], [R])
            V = s.bubbles()["volume"][0]
            exact = math.pi * R * R if dim == 2 else 4.0 / 3.0 * math.pi * R ** 3
            assert abs(V / exact - 1.0) < (0.05 if dim == 2 else 0.03) / R, (dim, R, V, exact)


def _two_bubbles(oracle_mod, RT=0.2):
    """Two disks separated by a thin liquid lamella (2D, periodic)."""
    cfg = W.config(nx=40, ny=24, nz=1, sigma=0.01, RT=RT, atmosphere=0)
    s = oracle_mod.OracleSim(cfg)
    s.nucleate([[12.0, 12.0, 0.0], [27.5, 12.0, 0.0]], [6.0, 8.0])
    return s


def test_merge_conserves_gas_and_keeps_smallest_id(oracle_mod):
    s = _two_bubbles(oracle_mod)
    b0 = s.bubbles()
    assert b0["mass"].size == 2
    ext0 = s.ledger()[5]
    t = s.types().reshape(24, 40)
    t[10:15, 15:24] = oracle_mod.GAS  # open a channel through the lamella
    s.debug_set_types(t.reshape(-1))
    s.debug_relabel()
    b1 = s.bubbles()
    assert b1["mass"].size == 1
    assert abs(b1["mass"][0] - b0["mass"].sum()) < 1e-13
    assert b1["id"][0] == b0["id"].min()
    assert abs(b1["pressure"][0] - b1["mass"][0] * 0.2 / b1["volume"][0]) < 1e-14
    assert s.ledger()[5] == ext0


def test_split_shares_gas_in_proportion_to_volume(oracle_mod):
    cfg = W.config(nx=48, ny=20, nz=1, sigma=0.01, RT=0.2, atmosphere=0)
    s = oracle_mod.OracleSim(cfg)
    s.nucleate([[14.0, 10.0, 0.0], [22.0, 10.0, 0.0], [30.0, 10.0, 0.0]], [5.0, 5.0, 5.0])
    b0 = s.bubbles()
    assert b0["mass"].size == 1  # overlapping nuclei form one elongated bubble
    t = s.types().reshape(20, 48)
    t[:, 25] = oracle_mod.LIQ  # cut it (the hook ignores the separation rule)
    s.debug_set_types(t.reshape(-1))
    s.debug_relabel()
    b1 = s.bubbles()
    assert b1["mass"].size == 2
    assert abs(b1["mass"].sum() - b0["mass"][0]) < 1e-13
    share = b1["volume"] / b1["volume"].sum()
    assert np.allclose(b1["mass"], b0["mass"][0] * share, rtol=1e-14)
    big = int(np.argmax(b1["volume"]))
    assert b1["id"][big] == b0["id"][0]
    assert b1["id"][1 - big] != b0["id"][0]


def test_vanished_bubble_gas_goes_to_ledger(oracle_mod):
    s = _two_bubbles(oracle_mod)
    b0 = s.bubbles()
    ext0 = s.ledger()[5]
    t = s.types().reshape(24, 40)
    lab = s.labels().reshape(24, 40)
    t[lab == 0] = oracle_mod.LIQ
    s.debug_set_types(t.reshape(-1))
    s.debug_relabel()
    b1 = s.bubbles()
    assert b1["mass"].size == 1
    assert abs(s.ledger()[5] - ext0 - b0["mass"][0]) < 1e-13
