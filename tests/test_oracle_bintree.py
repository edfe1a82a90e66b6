"""Pins for the oracle's k-d tree grids (Table 1(d): BinTree; nodes halved at
the midpoint of one axis).  CPU only.

* Point location and the walk against brute force over the leaf boxes the
  builder computed independently (no walking, no tree descent).
* The tie rule on a splitting plane follows the direction of travel.
* A k-d tree refined uniformly (axes in turn) to depth 3k is the 2^k
  cartesian grid: the same optical depth along every ray, the same images
  and the same absorption per cell (leaf order mapped to cell order).
"""
import numpy as np
import pytest

from paper_1410_1629_gb300 import workloads as W
from test_oracle_geometry import _check_against_brute, _dirs, _problem


def _random_bintree(seed, max_depth=7, bounds=(-1, 1, -1, 1, -1, 1), axes="cycle"):
    rng = np.random.default_rng(seed)
    axis_of = None if axes == "cycle" else (lambda lo, hi, d: rng.integers(0, 3, len(lo)))
    return W.build_bintree(list(bounds), lambda lo, hi, d: rng.uniform(size=len(lo)) < (0.95 if d < 2 else 0.6),
                           lambda lo, hi: 1.0 + np.arange(len(lo)) % 5, max_depth, axis_of=axis_of)


@pytest.mark.parametrize("seed,bounds,axes", [(0, (-1, 1, -1, 1, -1, 1), "cycle"),
                                              (1, (-2.0, 2.0, 0.0, 1.0, -0.5, 0.5), "random")])
def test_bintree_locate_matches_brute_force(oracle, seed, bounds, axes):
    grid, llo, lhi = _random_bintree(seed, bounds=bounds, axes=axes)
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


def test_bintree_tie_rule_follows_direction(oracle):
    grid, llo, lhi = W.build_bintree([-1, 1] * 3, lambda lo, hi, d: np.ones(len(lo), bool),
                                     lambda lo, hi: np.ones(len(lo)), 3)
    prob = _problem(grid)
    p = [0.0, 0.3, 0.3]  # on the x split (depth 2)
    c_up, box_up = oracle.locate(prob, p, (1.0, 1.0, 1.0))
    c_dn, box_dn = oracle.locate(prob, p, (-1.0, 1.0, 1.0))
    assert box_up[0] == 0.0 and box_dn[1] == 0.0


@pytest.mark.parametrize("seed,bounds,axes", [(2, (-1, 1, -1, 1, -1, 1), "cycle"),
                                              (3, (-2.0, 2.0, 0.0, 1.0, -0.5, 0.5), "random"),
                                              (4, (-1, 1, -1, 1, -1, 1), "random")])
def test_bintree_path_matches_brute_force(oracle, seed, bounds, axes):
    grid, llo, lhi = _random_bintree(seed, bounds=bounds, axes=axes)
    prob = _problem(grid)
    rng = np.random.default_rng(seed)
    b = np.asarray(bounds, float)
    for k in _dirs(rng, 60):
        inside = b[[0, 2, 4]] + rng.uniform(0, 1, 3) * (b[[1, 3, 5]] - b[[0, 2, 4]])
        _check_against_brute(oracle, prob, llo, lhi, inside, k)
        outside = b[[0, 2, 4]] + rng.uniform(-1.0, 2.0, 3) * (b[[1, 3, 5]] - b[[0, 2, 4]])
        _check_against_brute(oracle, prob, llo, lhi, outside, k)


def test_full_bintree_transport_equals_cartesian(oracle):
    """Depth 12 with the axes in turn is the 16^3 cube of side 2."""
    cart = W.uniform_cube(n_cells=16, n_pix=16, channels=3)
    rng = np.random.default_rng(5)
    dens = rng.uniform(0.2, 2.0, (16, 16, 16)).astype(np.float32)
    cart = W.with_density(cart, dens)

    def leaf_density(lo, hi):
        idx = np.floor((0.5 * (lo + hi) + 1.0) * 8).astype(int)
        return dens[idx[:, 2], idx[:, 1], idx[:, 0]]

    grid, llo, lhi = W.build_bintree([-1, 1] * 3, lambda lo, hi, d: np.ones(len(lo), bool), leaf_density, 12)
    assert grid.n_cells == 16 ** 3
    kd = W.replace(cart, grid=grid)
    rc = oracle.run(cart, 1500)
    rk = oracle.run(kd, 1500)
    np.testing.assert_allclose(rk["images"][0], rc["images"][0], rtol=1e-12, atol=1e-18)
    idx = np.floor((0.5 * (llo + lhi) + 1.0) * 8).astype(int)
    cell = idx[:, 0] + 16 * (idx[:, 1] + 16 * idx[:, 2])
    np.testing.assert_allclose(rk["absorption"][0], rc["absorption"][0][cell], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(rk["stats"], rc["stats"], rtol=1e-12)
