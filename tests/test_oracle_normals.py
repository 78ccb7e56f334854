"""Pins of the oracle's finite-difference normals (normal of the displaced
surface p = (x + Dx, y + Dy, h)): central and one-sided differences are
exact on linear fields, so planes, stretched and sheared grids give the
closed-form normal at every texel, edges included."""
import numpy as np

from oracle.synth import normal_map


def _grid(H, W, cell):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64) * cell
    return x, y


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def test_flat_surface_points_up():
    n = normal_map(np.zeros((5, 7)), np.zeros((5, 7)), np.zeros((5, 7)), 0.5)
    assert np.allclose(n[0], 0) and np.allclose(n[1], 0) and np.allclose(n[2], 1)


def test_tilted_plane():
    x, y = _grid(6, 9, 0.25)
    a, b = 0.3, -0.7
    n = normal_map(a * x + b * y, 0 * x, 0 * x, 0.25)
    want = _unit([-a, -b, 1.0])
    for k in range(3):
        assert np.allclose(n[k], want[k], atol=1e-14)


def test_stretched_grid():
    # Dx = p x, Dy = q y: tangents (1 + p, 0, a) and (0, 1 + q, b)
    x, y = _grid(7, 5, 0.5)
    a, b, p, q = 0.4, 0.2, 0.3, -0.25
    n = normal_map(a * x + b * y, p * x, q * y, 0.5)
    want = _unit([-a * (1 + q), -b * (1 + p), (1 + p) * (1 + q)])
    for k in range(3):
        assert np.allclose(n[k], want[k], atol=1e-14)


def test_sheared_grid():
    # Dx = r y: tangents (1, 0, a) and (r, 1, b) -> n ~ (-a, a r - b, 1)
    x, y = _grid(8, 6, 1.0)
    a, b, r = 0.5, -0.1, 0.6
    n = normal_map(a * x + b * y, r * y, 0 * x, 1.0)
    want = _unit([-a, a * r - b, 1.0])
    for k in range(3):
        assert np.allclose(n[k], want[k], atol=1e-14)


def test_curved_surface_second_order():
    # h = A cos(k x): central differences converge to the analytic normal
    # (-h', 0, 1)/|.| at second order inside the patch
    errs = []
    for cell in (0.2, 0.1):
        x, y = _grid(4, int(round(8 / cell)) + 1, cell)
        A, k = 0.3, 1.1
        n = normal_map(A * np.cos(k * x), 0 * x, 0 * x, cell)
        hp = -A * k * np.sin(k * x)
        want = np.stack([-hp, 0 * hp, 1 + 0 * hp]) / np.sqrt(1 + hp * hp)
        errs.append(np.abs(n[:, :, 1:-1] - want[:, :, 1:-1]).max())
    assert errs[1] < errs[0] / 3.5 and errs[1] < 1e-3
