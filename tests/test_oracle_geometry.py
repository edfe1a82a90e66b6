"""Pins for the oracle's grid traversal and point location.

Brute force: the segment of a ray inside every cell box is found by the slab
method over all cells independently (no walking), then sorted by entry.
"""
import math

import numpy as np
import pytest

from paper_1410_1629_gb300 import workloads as W


def _problem(grid):
    p = W.uniform_cube(n_cells=2, n_packets=1)
    p.grid = grid
    return p


def _cart_boxes(bounds, shape):
    nx, ny, nz = shape
    b = np.asarray(bounds, dtype=np.float64)
    ex = np.linspace(b[0], b[1], nx + 1)
    ey = np.linspace(b[2], b[3], ny + 1)
    ez = np.linspace(b[4], b[5], nz + 1)
    lo, hi = [], []
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                lo.append([ex[ix], ey[iy], ez[iz]])
                hi.append([ex[ix + 1], ey[iy + 1], ez[iz + 1]])
    return np.array(lo), np.array(hi)


def _brute_segments(lo, hi, x, k):
    """(cell, t_in, t_out) with positive length for every box the ray crosses (t >= 0)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - x) / k
        t2 = (hi - x) / k
    tn = np.where(k == 0, np.where((x >= lo) & (x <= hi), -np.inf, np.inf), np.minimum(t1, t2))
    tf = np.where(k == 0, np.where((x >= lo) & (x <= hi), np.inf, -np.inf), np.maximum(t1, t2))
    t_in = np.maximum(tn.max(axis=1), 0.0)
    t_out = tf.min(axis=1)
    sel = np.nonzero(t_out - t_in > 1e-12)[0]
    order = np.argsort(t_in[sel])
    c = sel[order]
    return c, t_in[c], t_out[c]


def _check_against_brute(oracle, prob, lo, hi, x, k, start=-1):
    cells, s_in, s_out = oracle.path(prob, x, k, start)
    pos = s_out - s_in > 1e-12
    bc, bt_in, bt_out = _brute_segments(lo, hi, np.asarray(x, float), np.asarray(k, float))
    assert list(cells[pos]) == list(bc)
    np.testing.assert_allclose(s_in[pos], bt_in, rtol=0, atol=1e-12)
    np.testing.assert_allclose(s_out[pos], bt_out, rtol=0, atol=1e-12)
    # the walk is contiguous: every segment starts where the previous one ended
    if len(s_in):
        np.testing.assert_array_equal(s_in[1:], s_out[:-1])
    return cells, s_in, s_out


def _dirs(rng, n):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    extra = np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1, 0], [0.6, 0.8, 0.0], [0.0, -0.6, 0.8]])
    return np.concatenate([v, extra])


@pytest.mark.parametrize("shape,bounds", [((4, 4, 4), [-1, 1, -1, 1, -1, 1]),
                                          ((4, 3, 5), [-1.0, 2.0, 0.0, 1.0, -0.5, 0.5])])
def test_cartesian_path_matches_brute_force(oracle, shape, bounds):
    nx, ny, nz = shape
    grid = W.cartesian_grid(bounds, np.ones((nz, ny, nx), np.float32))
    prob = _problem(grid)
    lo, hi = _cart_boxes(bounds, shape)
    rng = np.random.default_rng(7)
    b = np.asarray(bounds, float)
    for k in _dirs(rng, 60):
        inside = b[[0, 2, 4]] + rng.uniform(0, 1, 3) * (b[[1, 3, 5]] - b[[0, 2, 4]])
        _check_against_brute(oracle, prob, lo, hi, inside, k)
        outside = b[[0, 2, 4]] + rng.uniform(-1.0, 2.0, 3) * (b[[1, 3, 5]] - b[[0, 2, 4]])
        _check_against_brute(oracle, prob, lo, hi, outside, k)


def test_cartesian_path_from_a_known_cell(oracle):
    grid = W.cartesian_grid([-1, 1] * 3, np.ones((4, 4, 4), np.float32))
    prob = _problem(grid)
    lo, hi = _cart_boxes([-1, 1] * 3, (4, 4, 4))
    # a point on the face between cells 0 and 1 (x = -0.5), stated to lie in cell 1
    x = np.array([-0.5, -0.9, -0.9])
    for k in ([-1.0, 0.0, 0.0], [0.8, 0.6, 0.0]):
        cells, s_in, s_out = oracle.path(prob, x, k, 1)
        assert cells[0] == 1
        if k[0] < 0:
            assert s_out[0] == 0.0 and cells[1] == 0  # zero-length segment, then the neighbour


def test_missed_grid_gives_no_segment(oracle):
    grid = W.cartesian_grid([-1, 1] * 3, np.ones((4, 4, 4), np.float32))
    prob = _problem(grid)
    cells, _, _ = oracle.path(prob, [3.0, 0.0, 0.0], [1.0, 0.0, 0.0])
    assert cells.size == 0
    cells, _, _ = oracle.path(prob, [3.0, 3.0, 0.0], [0.0, 0.0, 1.0])
    assert cells.size == 0


def test_uniform_cube_path_length_closed_form(oracle):
    """Sum of segment lengths = distance from x to the box along k."""
    grid = W.cartesian_grid([-1, 1] * 3, np.ones((32, 32, 32), np.float32))
    prob = _problem(grid)
    rng = np.random.default_rng(1)
    for k in _dirs(rng, 40):
        x = rng.uniform(-1, 1, 3)
        with np.errstate(divide="ignore"):
            t = np.where(k > 0, (1 - x) / k, np.where(k < 0, (-1 - x) / k, np.inf))
        cells, s_in, s_out = oracle.path(prob, x, k)
        assert abs((s_out - s_in).sum() - t.min()) < 1e-12


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_voxelised_sphere_optical_depth_converges(oracle, n):
    """Uniform sphere R = 0.8 voxelised by cell centres: tau(centre -> out) -> R,
    with an error below one cell diagonal."""
    R = 0.8
    xs, ys, zs = W.cell_centres([-1, 1] * 3, (n, n, n))
    inside = (xs[None, None, :] ** 2 + ys[None, :, None] ** 2 + zs[:, None, None] ** 2) < R * R
    grid = W.cartesian_grid([-1, 1] * 3, inside.astype(np.float32))
    prob = _problem(grid)
    rng = np.random.default_rng(n)
    errs = []
    for k in _dirs(rng, 40):
        x = rng.uniform(-1e-3, 1e-3, 3)
        cells, s_in, s_out = oracle.path(prob, x, k)
        tau = ((s_out - s_in) * grid.density.ravel()[cells]).sum()
        errs.append(abs(tau - R))
    h = 2.0 / n
    assert max(errs) <= math.sqrt(3) * h + 2e-3
    assert np.mean(errs) <= 0.75 * h


def _random_octree(seed, max_level=3, bounds=(-1, 1, -1, 1, -1, 1)):
    rng = np.random.default_rng(seed)
    return W.build_octree(list(bounds), lambda lo, hi, lvl: rng.uniform(size=len(lo)) < (0.9 if lvl == 0 else 0.45),
                          lambda lo, hi: 1.0 + np.arange(len(lo)) % 5, max_level)


@pytest.mark.parametrize("seed,bounds", [(0, (-1, 1, -1, 1, -1, 1)), (1, (-2.0, 2.0, 0.0, 1.0, -0.5, 0.5))])
def test_octree_locate_matches_brute_force(oracle, seed, bounds):
    grid, llo, lhi = _random_octree(seed, bounds=bounds)
    prob = _problem(grid)
    rng = np.random.default_rng(seed + 10)
    b = np.asarray(bounds, float)
    for _ in range(300):
        p = b[[0, 2, 4]] + rng.uniform(0, 1, 3) * (b[[1, 3, 5]] - b[[0, 2, 4]])
        c, box = oracle.locate(prob, p)
        expect = np.nonzero(np.all((llo <= p) & (p < lhi), axis=1))[0]
        assert list(expect) == [c]
        np.testing.assert_array_equal(box[[0, 2, 4]], llo[c])
        np.testing.assert_array_equal(box[[1, 3, 5]], lhi[c])


def test_octree_tie_rule_follows_direction(oracle):
    grid, llo, lhi = W.build_octree([-1, 1] * 3, lambda lo, hi, l: np.ones(len(lo), bool),
                                    lambda lo, hi: np.ones(len(lo)), 2)
    prob = _problem(grid)
    p = [0.0, 0.3, 0.3]
    c_up, box_up = oracle.locate(prob, p, (1.0, 1.0, 1.0))
    c_dn, box_dn = oracle.locate(prob, p, (-1.0, 1.0, 1.0))
    assert box_up[0] == 0.0 and box_dn[1] == 0.0


@pytest.mark.parametrize("seed,bounds", [(2, (-1, 1, -1, 1, -1, 1)), (3, (-2.0, 2.0, 0.0, 1.0, -0.5, 0.5)),
                                         (4, (-1, 1, -1, 1, -1, 1))])
def test_octree_path_matches_brute_force(oracle, seed, bounds):
    grid, llo, lhi = _random_octree(seed, bounds=bounds)
    prob = _problem(grid)
    rng = np.random.default_rng(seed)
    b = np.asarray(bounds, float)
    for k in _dirs(rng, 60):
        inside = b[[0, 2, 4]] + rng.uniform(0, 1, 3) * (b[[1, 3, 5]] - b[[0, 2, 4]])
        _check_against_brute(oracle, prob, llo, lhi, inside, k)
        outside = b[[0, 2, 4]] + rng.uniform(-1.0, 2.0, 3) * (b[[1, 3, 5]] - b[[0, 2, 4]])
        _check_against_brute(oracle, prob, llo, lhi, outside, k)


def test_full_octree_equals_cartesian_grid(oracle):
    """An octree refined uniformly to level 2 is the 4^3 cartesian grid: same
    optical depth along every ray."""
    rng = np.random.default_rng(9)
    dens = rng.uniform(0.1, 2.0, (4, 4, 4)).astype(np.float32)
    cart = _problem(W.cartesian_grid([-1, 1] * 3, dens))

    def leaf_density(lo, hi):
        c = 0.5 * (lo + hi)
        idx = np.floor((c + 1) / 0.5).astype(int)
        return dens[idx[:, 2], idx[:, 1], idx[:, 0]]

    grid, _, _ = W.build_octree([-1, 1] * 3, lambda lo, hi, l: np.ones(len(lo), bool), leaf_density, 2)
    octp = _problem(grid)
    for k in _dirs(rng, 40):
        x = rng.uniform(-1, 1, 3)
        c1, a1, b1 = oracle.path(cart, x, k)
        c2, a2, b2 = oracle.path(octp, x, k)
        t1 = ((b1 - a1) * cart.grid.density.ravel()[c1]).sum()
        t2 = ((b2 - a2) * octp.grid.density[c2]).sum()
        assert abs(t1 - t2) < 1e-12
