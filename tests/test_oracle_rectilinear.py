"""Pins for the oracle's rectilinear grids (cuboidal cells between arbitrary
edges per axis; the PowCub grid of Table 1(d) spaces the edges by a power
law).  CPU only.

* The walk against brute force: every cell box intersected with the ray by
  the slab method, independently of the walk.
* A rectilinear grid whose edges are the cartesian planes gives the
  cartesian run bit for bit.
* Refinement: splitting cells without changing the density changes no
  image and no total (the optical depth is additive over segments); the
  absorption of each coarse cell is the sum over its parts.
* The power-law edges: strictly increasing, symmetric, outermost / innermost
  width = the requested ratio.
"""
import numpy as np
import pytest

from paper_1410_1629_gb300 import workloads as W
from test_oracle_geometry import _brute_segments, _dirs, _problem


def _boxes(edges):
    ex, ey, ez = edges
    lo, hi = [], []
    for iz in range(len(ez) - 1):
        for iy in range(len(ey) - 1):
            for ix in range(len(ex) - 1):
                lo.append([ex[ix], ey[iy], ez[iz]])
                hi.append([ex[ix + 1], ey[iy + 1], ez[iz + 1]])
    return np.array(lo), np.array(hi)


def _random_edges(rng, lo, hi, n):
    inner = np.sort(rng.uniform(lo, hi, n - 1))
    return np.concatenate([[lo], inner, [hi]])


@pytest.mark.parametrize("seed", [1, 2])
def test_rectilinear_path_matches_brute_force(oracle, seed):
    rng = np.random.default_rng(seed)
    edges = [_random_edges(rng, -1.0, 1.5, 4), _random_edges(rng, 0.0, 1.0, 3), _random_edges(rng, -0.5, 0.5, 5)]
    grid = W.rectilinear_grid(edges, np.ones((5, 3, 4), np.float32))
    prob = _problem(grid)
    lo, hi = _boxes(edges)
    b = np.asarray(grid.bounds)
    for k in _dirs(rng, 60):
        for x in (b[[0, 2, 4]] + rng.uniform(0, 1, 3) * (b[[1, 3, 5]] - b[[0, 2, 4]]),
                  b[[0, 2, 4]] - 0.3 * (b[[1, 3, 5]] - b[[0, 2, 4]]) * np.sign(k + 1e-9)):
            cells, s_in, s_out = oracle.path(prob, x, k)
            pos = s_out - s_in > 1e-12
            bc, bt_in, bt_out = _brute_segments(lo, hi, np.asarray(x, float), np.asarray(k, float))
            assert list(cells[pos]) == list(bc)
            np.testing.assert_allclose(s_in[pos], bt_in, rtol=0, atol=1e-12)
            np.testing.assert_allclose(s_out[pos], bt_out, rtol=0, atol=1e-12)
            if len(s_in):
                np.testing.assert_array_equal(s_in[1:], s_out[:-1])
    # point location: the cell whose box contains the point
    for p in rng.uniform(b[[0, 2, 4]], b[[1, 3, 5]], (200, 3)):
        c, box = oracle.locate(prob, p)
        inside = np.flatnonzero(np.all((lo <= p) & (p < hi), axis=1))
        assert c == inside[0]


def test_cartesian_planes_as_edges_give_the_cartesian_run(oracle):
    cart = W.disk_galaxy(n_cells=16, n_lambda=2, n_pix=16, channels=3)
    nx, ny, nz = cart.grid.shape
    b = np.asarray(cart.grid.bounds)
    # the cartesian planes lo + i (hi - lo) / n, as the oracle computes them
    edges = [b[2 * a] + np.arange(n + 1) * ((b[2 * a + 1] - b[2 * a]) / n) for a, n in enumerate((nx, ny, nz))]
    for a in range(3):
        edges[a][-1] = b[2 * a + 1]
    rect = W.replace(cart, grid=W.rectilinear_grid(edges, cart.grid.density))
    n = 2000
    r1 = oracle.run(cart, n, n_threads=1, counts=True)
    r2 = oracle.run(rect, n, n_threads=1, counts=True)
    for a, c in zip(r1["images"], r2["images"]):
        np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(r1["absorption"], r2["absorption"])
    np.testing.assert_array_equal(r1["stats"], r2["stats"])
    np.testing.assert_array_equal(r1["counters"], r2["counters"])


def test_refining_cells_with_equal_density_changes_no_tally(oracle):
    rng = np.random.default_rng(5)
    edges = [W.powcub_edges(-1.0, 1.0, 6, 4.0), W.powcub_edges(-1.0, 1.0, 5, 3.0), W.powcub_edges(-1.0, 1.0, 4, 2.0)]
    dens = rng.uniform(0.2, 2.0, (4, 5, 6)).astype(np.float32)
    coarse_grid = W.rectilinear_grid(edges, dens)
    # split every cell in two along x and along z
    fx = np.sort(np.concatenate([edges[0], 0.5 * (edges[0][1:] + edges[0][:-1])]))
    fz = np.sort(np.concatenate([edges[2], 0.5 * (edges[2][1:] + edges[2][:-1])]))
    fine = np.repeat(np.repeat(dens, 2, axis=2), 2, axis=0)
    fine_grid = W.rectilinear_grid([fx, edges[1], fz], fine)
    base = W.uniform_cube(albedo=0.7, g=0.4, channels=3, n_pix=8, source_pos=(0.13, -0.21, 0.07))
    coarse = W.replace(base, grid=coarse_grid, kappa=np.array([1.3]))
    fine_p = W.replace(base, grid=fine_grid, kappa=np.array([1.3]))
    n = 3000
    rc = oracle.run(coarse, n, n_threads=2)
    rf = oracle.run(fine_p, n, n_threads=2)
    np.testing.assert_allclose(rf["images"][0], rc["images"][0], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(rf["stats"], rc["stats"], rtol=1e-11)
    assert rf["counters"][1] == rc["counters"][1]  # same events
    ab = rf["absorption"].reshape(1, 8, 5, 12)
    merged = ab.reshape(1, 4, 2, 5, 6, 2).sum(axis=(2, 5)).reshape(1, -1)
    np.testing.assert_allclose(merged, rc["absorption"], rtol=1e-9, atol=1e-15 * rc["absorption"].max())


@pytest.mark.parametrize("n,ratio", [(6, 50.0), (7, 10.0), (101, 50.0), (100, 1.0)])
def test_powcub_edges(n, ratio):
    e = W.powcub_edges(-7.0, 7.0, n, ratio)
    w = np.diff(e)
    assert len(e) == n + 1 and np.all(w > 0) and e[0] == -7.0 and e[-1] == 7.0
    np.testing.assert_allclose(e, -e[::-1], atol=1e-12)
    np.testing.assert_allclose(w.max() / w.min(), ratio, rtol=1e-9)
    # the widths grow away from the centre
    half = w[n // 2:]
    assert np.all(np.diff(half) >= -1e-12)
