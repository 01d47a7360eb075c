"""Training recipe of the learned interface curvature, on top of the C ABI.

Every computation runs in the CUDA library: stencil generation, forward and
backward passes and Adam (``lbf_mlp_train``), the simulations the pairs are
harvested from (``lbf_step``) and the harvest itself (``lbf_mlp_harvest``).
This module only decides which runs to make and concatenates device
buffers.

Recipe (the network is 27-64-64-1 SiLU, BF16 on the tensor cores):

1. synthetic pairs: voxelised spheres and ellipsoids with their analytic
   mean curvature, radii log-uniform in [2, 40];
2. pairs harvested from relaxed static bubbles run with the least-squares
   curvature in FP64 storage (the form that reproduces the CPU reference to
   1e-10), target 4 / R_eq from each bubble's volume;
3. rounds of dataset aggregation: the same runs with the current network
   driving the curvature; their interface stencils join the data and the
   network is retrained.  Without step 3 the network is accurate on both
   kinds of stencil but the coupled run drifts to interface shapes it never
   saw and spurious currents grow.
"""
from __future__ import annotations

import numpy as np

from . import lbf as L
from . import workloads as W

HARVEST_RADII = (2.5, 3.0, 3.5, 4.2, 5.0, 5.8, 6.6, 7.5, 8.5, 10.0, 12.0, 14.0, 17.0)


def init_params(seed: int) -> np.ndarray:
    """Random start: weights N(0, 1/fan_in), zero biases (6017 float32)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, 27 ** -0.5, 64 * 27), np.zeros(64), rng.normal(0, 64 ** -0.5, 64 * 64),
             np.zeros(64), rng.normal(0, 64 ** -0.5, 64), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def static_bubble_config(R: float, storage: str = "fp64", sigma: float = 0.01, n: int | None = None) -> dict:
    """One gas bubble in a periodic box of liquid at rest, no dissolved gas."""
    n = n or int(2 * R + 16)
    return W.config(nx=n, ny=n, nz=n, storage=storage, walls=0, atmosphere=0, tau=0.8, sigma=sigma,
                    kH=0.0, D=0.05, c0=0.0, p0=1.0 / 3.0)


def harvest_static_bubbles(radii=HARVEST_RADII, snaps=(150, 300, 450, 600), theta=None, storage="fp64",
                           seed: int = 5, stream: int | None = None):
    """(x, y) device tensors of the interface cells of relaxing static
    bubbles at the given steps; the curvature is least squares, or the
    network ``theta`` when given."""
    import torch

    rng = np.random.default_rng(seed)
    xs, ys = [], []
    for R in radii:
        cfg = static_bubble_config(R, storage)
        n = cfg["nx"]
        sim = L.Sim(cfg, stream=stream)
        sim.nucleate([[n / 2 + rng.uniform(-0.5, 0.5) for _ in range(3)]], [R])
        if theta is not None:
            sim.mlp_attach(theta)
        done = 0
        cap = 24 * int(4 * np.pi * (R + 3) ** 2) + 1024
        for st in snaps:
            sim.step(st - done)
            done = st
            x = torch.empty((cap, 27), device="cuda")
            y = torch.empty(cap, device="cuda")
            cells = torch.empty(cap, dtype=torch.int32, device="cuda")
            k = sim.mlp_harvest(x, y, cells)
            # pairs in cell order: the training set does not depend on the
            # order in which the interface list was built
            o = torch.argsort(cells[:k].long())
            xs.append(x[:k][o])
            ys.append(y[:k][o])
        sim.close()
    return torch.cat(xs), torch.cat(ys)


def train(seed: int = 1, rounds: int = 3, n_synthetic: int = 1 << 20, repeat_lsq: int = 30,
          repeat_agg: int = 10, epochs: int = 20, batch: int = 2048, lr: float = 3e-3,
          stream: int | None = None):
    """The full recipe; returns (theta float32, info dict)."""
    import torch

    X, Y = harvest_static_bubbles(seed=seed + 4, stream=stream)
    X, Y = X.repeat(repeat_lsq, 1), Y.repeat(repeat_lsq)
    info = {"harvested_lsq": int(Y.numel()) // repeat_lsq, "rounds": []}
    th, curve = L.mlp_train(init_params(seed), n_samples=n_synthetic, epochs=epochs, batch=batch, lr=lr,
                            seed=seed, x_extra=X.contiguous(), y_extra=Y.contiguous(), stream=stream)
    info["loss"] = [float(curve[-1])]
    for r in range(rounds):
        Xd, Yd = harvest_static_bubbles(snaps=(100, 200, 300), theta=th, seed=seed + 100 + r, stream=stream)
        X = torch.cat([X, Xd.repeat(repeat_agg, 1)])
        Y = torch.cat([Y, Yd.repeat(repeat_agg)])
        th, curve = L.mlp_train(init_params(seed), n_samples=n_synthetic, epochs=epochs, batch=batch, lr=lr,
                                seed=seed + 1 + r, x_extra=X.contiguous(), y_extra=Y.contiguous(), stream=stream)
        info["rounds"].append(int(Yd.numel()))
        info["loss"].append(float(curve[-1]))
    return th.astype(np.float32), info
