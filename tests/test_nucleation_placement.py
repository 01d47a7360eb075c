"""Nucleation placement (Sec. 3.4): sites from a nucleation probability
field without overlap, and organised arrangements."""
import numpy as np

from paper_1908_04262_gb300 import workloads as W


def _min_clearance(pts, rad):
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    gap = d - (rad[:, None] + rad[None, :])
    np.fill_diagonal(gap, np.inf)
    return gap.min()


def test_field_sampling_follows_the_field_and_keeps_nuclei_apart():
    rng = np.random.default_rng(3)
    ny, nx = 120, 160
    x = np.arange(nx)[None, :]
    prob = np.where(x < nx // 2, 0.0, 1.0) * np.ones((ny, 1))  # nothing on the left half
    prob[:, 3 * nx // 4:] *= 3.0  # three times as likely on the right quarter
    pts, rad = W.nuclei_from_field(rng, 60, prob, 2.0, min_gap=1.0)
    assert np.all(pts[:, 0] >= nx // 2 - 0.5)
    assert _min_clearance(pts, rad) >= 1.0 - 1e-12
    # 3/4 of the weight sits on the right quarter (dart throwing rejects a
    # few more there, where sites are denser)
    frac = np.mean(pts[:, 0] >= 3 * nx // 4 - 0.5)
    assert 0.6 < frac < 0.88
    assert np.all(pts - rad[:, None] >= 0.5) and np.all(pts[:, 0] + rad <= nx - 1.5)


def test_field_radius_and_3d():
    rng = np.random.default_rng(4)
    nz, ny, nx = 30, 30, 30
    prob = np.ones((nz, ny, nx))
    radius = np.where(np.arange(nz)[:, None, None] < 15, 2.0, 3.0) * np.ones((1, ny, nx))
    pts, rad = W.nuclei_from_field(rng, 40, prob, radius)
    low = pts[:, 2] < 14.5
    assert np.all(rad[low] == 2.0) and np.all(rad[pts[:, 2] >= 14.5] == 3.0)
    assert _min_clearance(pts, rad) >= 1.0 - 1e-12


def test_organised_arrangements():
    pts, rad = W.nuclei_organised((0, 0), (40, 30), 10.0, 3.0)
    assert len(pts) == 4 * 3 and np.all(rad == 3.0)
    assert np.allclose(np.unique(pts[:, 0]), [3, 13, 23, 33])
    assert np.allclose(np.unique(pts[:, 1]), [3, 13, 23])
    hx, _ = W.nuclei_organised((0, 0), (40, 30), 10.0, 3.0, hexagonal=True)
    d = np.sqrt(((hx[:, None] - hx[None]) ** 2).sum(-1))
    np.fill_diagonal(d, np.inf)
    assert np.allclose(d.min(axis=1), 10.0)  # every site has a neighbour at one spacing
    assert _min_clearance(hx, np.full(len(hx), 3.0)) >= 10.0 - 6.0 - 1e-9
    p3, _ = W.nuclei_organised((0, 0, 0), (20, 20, 20), 7.0, 2.0)
    assert len(p3) == 3 ** 3
