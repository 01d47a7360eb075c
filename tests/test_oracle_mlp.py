"""Pins of the CPU reference of the learned-curvature network: gradients
against central finite differences, canonical orientation against the
symmetries it must respect, synthetic stencils against closed forms."""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(3) + 0.05 * rng.normal(size=mlp.NPARAM)
    x = rng.random((7, 27))
    t = rng.normal(size=7)
    L, g = mlp.loss_and_grad(theta, x, t)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 27 * 64, 27 * 64 + 64 + 4096 + 3]])
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.NPARAM)
        e[k] = h
        fd = (mlp.loss_and_grad(theta + e, x, t)[0] - mlp.loss_and_grad(theta - e, x, t)[0]) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])
    assert abs(L - 0.5 * np.mean((mlp.forward(theta, x) - t) ** 2)) < 1e-15


def _rotations():
    mats = []
    import itertools
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((-1, 1), repeat=3):
            M = np.zeros((3, 3))
            for i in range(3):
                M[i, perm[i]] = signs[i]
            mats.append(M)
    return mats


def _apply(M, a):
    """Stencil of the field rotated by the isometry M (x' = M x)."""
    out = np.zeros(27)
    for q in range(27):
        old = np.linalg.inv(M) @ mlp.OFFS[q]
        oq = int((old[2] + 1) * 9 + (old[1] + 1) * 3 + (old[0] + 1))
        out[q] = a[oq]
    return out


def test_canonical_form_is_invariant_under_the_octahedral_group():
    rng = np.random.default_rng(4)
    for _ in range(20):
        a = rng.random(27)
        n = mlp.py_normal(a)
        if np.min(np.abs(np.diff(np.sort(np.abs(n))))) < 1e-6 or np.min(np.abs(n)) < 1e-6:
            continue  # ties would make the orientation ambiguous
        c0 = mlp.canonicalize(a)
        for M in _rotations():
            assert np.allclose(mlp.canonicalize(_apply(M, a)), c0)
        cn = mlp.py_normal(c0)
        assert np.all(cn >= 0) and cn[0] <= cn[1] <= cn[2]


def test_sphere_stencil_fill_levels_and_curvature():
    # a cell far inside / outside is pure; the analytic curvature is 1/R
    alpha, k = mlp.ellipsoid_stencil([0.3, -0.2, 0.1], [6.0, 6.0, 6.0], np.eye(3), True, [0, 0, 6])
    assert abs(k - 1 / 6.0) < 1e-12
    a2, k2 = mlp.ellipsoid_stencil([0.3, -0.2, 0.1], [6.0, 6.0, 6.0], np.eye(3), False, [0, 0, 6])
    assert abs(k2 + 1 / 6.0) < 1e-12 and np.allclose(a2, 1 - alpha)
    a3, _ = mlp.ellipsoid_stencil([0.0, 0.0, 0.0], [3.0, 3.0, 3.0], np.eye(3), True, [0, 0, 0])
    assert np.all(a3 == 0.0)
    # total liquid volume near a plane-like large sphere: the cell with the
    # surface through its centre is half full
    a4, _ = mlp.ellipsoid_stencil([0.0, 0.0, -1000.0], [1000.0] * 3, np.eye(3), True, [0, 0, 0], sub=8)
    assert abs(a4[13] - 0.5) < 1e-12


def test_ellipsoid_curvature_closed_form():
    # at the tip of the longest semi-axis a of a spheroid (a, b, b): the two
    # principal curvatures are a/b^2, so the mean curvature is a/b^2
    a, b = 5.0, 3.0
    _, k = mlp.ellipsoid_stencil([0.0, 0.0, 0.0], [a, b, b], np.eye(3), True, [5, 0, 0])
    assert abs(k - a / b ** 2) < 1e-9
    # at the equator (0, b, 0): principal curvatures 1/b and b/a^2
    _, k = mlp.ellipsoid_stencil([0.0, 0.0, 0.0], [a, b, b], np.eye(3), True, [0, 3, 0])
    assert abs(k - 0.5 * (1 / b + b / a ** 2)) < 1e-9


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    a = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        # exact ties between two BF16 neighbours, both parities
                        1.0 + np.array([1, 3, 5, 7]) * 2.0 ** -8, [-(1.0 + 2.0 ** -8), 0.0, -0.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(a), ref)


def test_bf16_forward_equals_exact_forward_on_representable_operands():
    # when x, W1, W2 are already BF16 values and the activations happen to be
    # BF16-representable, the two forms coincide; in general they differ by
    # at most the BF16 rounding of the activations
    rng = np.random.default_rng(2)
    theta = mlp.init_params(5)
    W1, b1, W2, b2, W3, b3 = mlp.split(theta)
    theta_b = np.concatenate([mlp.bf16(W1).ravel(), b1, mlp.bf16(W2).ravel(), b2,
                              np.float32(W3).astype(np.float64), [np.float64(np.float32(b3[0]))]])
    x = mlp.bf16(rng.random((64, 27)))
    y = mlp.forward(theta_b, x)
    yb = mlp.forward_bf16(theta_b, x)
    # relative error of a BF16 rounding is at most 2^-9
    bound = 2.0 ** -9 * (np.abs(mlp.silu(mlp.silu(x @ theta_b[:1728].reshape(64, 27).T)
                                         @ np.abs(theta_b[1792:5888].reshape(64, 64)).T) + 1.0)
                         @ np.abs(theta_b[5952:6016])) * 4
    assert np.all(np.abs(y - yb) <= bound + 1e-12)
    assert not np.allclose(y, yb, atol=0, rtol=1e-12)
