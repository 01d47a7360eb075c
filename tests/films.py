"""Deterministic geometric inputs shared by the oracle pins and the GPU parity
tests: planar films along lattice diagonals with exact fill levels."""
import math

import numpy as np

GAS_BANDS = [(1.3, 5.3), (8.7, 12.7)]  # gas A, gas B in w; the film is (5.3, 8.7)


def cube_fraction_below(t, dim):
    """Volume of the unit cell [-1/2, 1/2]^dim where u_1 + ... + u_dim <= t:
    the Irwin-Hall distribution function of dim uniforms at t + dim/2."""
    x = t + dim / 2.0
    if x <= 0.0:
        return 0.0
    if x >= dim:
        return 1.0
    return sum((-1) ** k * math.comb(dim, k) * max(0.0, x - k) ** dim for k in range(dim + 1)) / math.factorial(dim)


def diagonal_film(N, dim, axes, liq, gas, ifc):
    """Cell types and fill levels of the film of GAS_BANDS along
    w = x + y (axes = 2) or x + y + z (axes = 3) on an N^dim periodic box
    (period N in w); returns (w per cell, types, alpha)."""
    size = N ** dim
    idx = np.arange(size)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    w = np.mod(x + y + (z if axes == 3 else 0), N).astype(float)
    alpha = np.ones(size)
    for i, wi in enumerate(w):
        g = 0.0
        for lo, hi in GAS_BANDS:
            for img in (-N, 0, N):
                g += cube_fraction_below(hi + img - wi, axes) - cube_fraction_below(lo + img - wi, axes)
        alpha[i] = 1.0 - g
    t = np.where(alpha >= 1.0, liq, np.where(alpha <= 0.0, gas, ifc)).astype(np.uint8)
    return w, t, alpha
