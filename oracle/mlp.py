"""FP64 CPU reference of the learned-curvature network and its data.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Shares no code with the
CUDA path.

The network maps the 3x3x3 fill-level stencil of an interface cell, turned
into a canonical orientation, to the cell's curvature (the quantity kappa of
Sec. 2.2 Eq. rhob): 27 -> 64 -> 64 -> 1 with SiLU, output y = 4 kappa.
Parameters, flat in this order (6017 values):
    W1 (64 x 27, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1).

Stencil index: q = (dz+1)*9 + (dy+1)*3 + (dx+1), offsets in {-1,0,1}.
Canonical orientation: reflect every axis along which the interface normal
(Parker-Youngs weights 4/2/1, pointing into the liquid) is negative, then
order the axes by increasing normal component (ties keep axis order); the
new x axis carries the smallest component.  Curvature is invariant under
these 48 isometries.
"""
from __future__ import annotations

import numpy as np

SIZES = [(64, 27), (64,), (64, 64), (64,), (64,), (1,)]
NPARAM = 6017
Y_SCALE = 4.0


def split(theta):
    out, k = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[k:k + n], dtype=np.float64).reshape(s))
        k += n
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x):
    """x: (B, 27) canonical stencils -> y (B,), y = 4 kappa."""
    W1, b1, W2, b2, W3, b3 = split(theta)
    z1 = x @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    return h2 @ W3 + b3[0]


def bf16(a):
    """Round to the nearest BF16 value (ties to even), via FP32; returned as
    FP64.  BF16 keeps the top 16 bits of an IEEE single."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, x):
    """The network with the operands of its two hidden-layer products and
    of the output dot product in BF16 (x, W1, W2 and both hidden
    activations rounded), biases and W3 kept, every sum exact: the stated
    BF16-operand / wide-accumulation form without accumulation rounding."""
    W1, b1, W2, b2, W3, b3 = split(theta)
    z1 = bf16(x) @ bf16(W1).T + b1
    h1 = bf16(silu(z1))
    z2 = h1 @ bf16(W2).T + b2
    h2 = bf16(silu(z2))
    return h2 @ np.asarray(W3, np.float32).astype(np.float64) + np.float32(b3[0])


def loss_and_grad(theta, x, t):
    """Mean squared error 0.5 * mean((y - t)^2) and its gradient."""
    W1, b1, W2, b2, W3, b3 = split(theta)
    B = x.shape[0]
    z1 = x @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    y = h2 @ W3 + b3[0]
    r = y - t
    loss = 0.5 * np.mean(r * r)
    d3 = r / B                         # dL/dy
    gW3 = h2.T @ d3
    gb3 = np.array([d3.sum()])
    d2 = np.outer(d3, W3) * dsilu(z2)  # dL/dz2
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * dsilu(z1)         # dL/dz1
    gW1 = d1.T @ x
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss, g


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, 1 / np.sqrt(27), (64, 27))
    W2 = rng.normal(0, 1 / np.sqrt(64), (64, 64))
    W3 = rng.normal(0, 1 / np.sqrt(64), 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3, [0.0]])


# ---------------------------------------------------------------------------
# orientation

OFFS = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)])  # (dx, dy, dz)


def py_normal(a):
    """Parker-Youngs normal of a (27,) stencil (unnormalised), into liquid."""
    dx, dy, dz = OFFS[:, 0], OFFS[:, 1], OFFS[:, 2]
    wx = np.where(dy == 0, 2, 1) * np.where(dz == 0, 2, 1)
    wy = np.where(dx == 0, 2, 1) * np.where(dz == 0, 2, 1)
    wz = np.where(dx == 0, 2, 1) * np.where(dy == 0, 2, 1)
    return np.array([np.sum(dx * wx * a), np.sum(dy * wy * a), np.sum(dz * wz * a)])


def canonical_map(n):
    """Source index of every canonical stencil position for normal n."""
    sign = np.where(np.asarray(n) < 0, -1, 1)
    absn = np.abs(np.asarray(n, dtype=np.float64))
    order = sorted(range(3), key=lambda d: (absn[d], d))  # new axis j <- old axis order[j]
    src = np.zeros(27, dtype=np.int64)
    for q in range(27):
        new = OFFS[q]
        old = np.zeros(3, dtype=np.int64)
        for j in range(3):
            old[order[j]] = sign[order[j]] * new[j]
        src[q] = (old[2] + 1) * 9 + (old[1] + 1) * 3 + (old[0] + 1)
    return src


def canonicalize(a):
    a = np.asarray(a, dtype=np.float64)
    return a[canonical_map(py_normal(a))]


# ---------------------------------------------------------------------------
# synthetic stencils with analytic curvature


def ellipsoid_stencil(centre, axes, rot, gas_inside, cell, sub=6):
    """Fill levels of the 27 cells around integer cell `cell` for the
    ellipsoid {x : |D^-1 R^T (x - centre)| < 1} (D = diag(axes)), gas inside
    if gas_inside else liquid inside; fill level = fraction of sub^3 points
    (at (i + 1/2)/sub - 1/2) that are liquid.  Also returns kappa at the
    surface point reached from the cell centre by Newton steps along grad F
    (kappa > 0 for convex gas)."""
    centre = np.asarray(centre, dtype=np.float64)
    axes = np.asarray(axes, dtype=np.float64)
    rot = np.asarray(rot, dtype=np.float64)
    A = rot @ np.diag(1.0 / axes ** 2) @ rot.T
    g = (np.arange(sub) + 0.5) / sub - 0.5
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    alpha = np.zeros(27)
    for q in range(27):
        c = np.asarray(cell, dtype=np.float64) + OFFS[q]
        d = c + P - centre
        inside = np.einsum("ni,ij,nj->n", d, A, d) < 1.0
        liquid = ~inside if gas_inside else inside
        alpha[q] = np.mean(liquid)
    x = np.asarray(cell, dtype=np.float64) - centre
    if not np.any(x):
        # a cell centred on the ellipsoid: the nearest surface points lie
        # along the shortest axis (the Newton direction is undefined there)
        k = int(np.argmin(axes))
        x = rot[:, k] * axes[k]
    for _ in range(8):
        F = x @ A @ x - 1.0
        gF = 2 * A @ x
        x = x - F * gF / (gF @ gF)
    gF = 2 * A @ x
    H = 2 * A
    gn = np.linalg.norm(gF)
    mean_outward = (gF @ H @ gF - gn * gn * np.trace(H)) / (2 * gn ** 3)
    kappa = -mean_outward if gas_inside else mean_outward
    return alpha, kappa
