"""Pins for the oracle's Voronoi grids (Table 1(d): VoronoiDustGrid; Sect.
2.4: cell c holds the points nearest to its site).  CPU only.

* The walk against the lower envelope of the squared distances along the
  ray: |x + t k - s_c|^2 = a_c + b_c t + t^2, so the nearest site along the
  ray follows the lowest of the lines a_c + b_c t over all sites, with no
  planes and no neighbour lists involved.  This also pins the neighbour
  lists (a missing face would let the walk overshoot).
* Point location is the nearest site; points sampled along each segment are
  nearest to that segment's site.
* A walk meets each (convex) cell once.
* Sites on the cell centres of a cartesian grid with face neighbours give
  the cartesian grid: the same images, absorption and totals.
"""
import numpy as np
import pytest

from paper_1410_1629_gb300 import workloads as W
from test_oracle_geometry import _dirs, _problem


def _random_voronoi(seed, n=300, bounds=(-2.0, 2.0, 0.0, 1.0, -0.5, 0.5)):
    rng = np.random.default_rng(seed)
    b = np.asarray(bounds, float).reshape(3, 2)
    uni = b[:, 0] + rng.uniform(0.0, 1.0, (n // 2, 3)) * (b[:, 1] - b[:, 0])
    # a cluster, so that cell sizes vary by an order of magnitude
    clu = np.clip(rng.normal(b.mean(axis=1), 0.08 * (b[:, 1] - b[:, 0]), (n - n // 2, 3)),
                  b[:, 0] + 1e-6, b[:, 1] - 1e-6)
    sites = np.concatenate([uni, clu])
    return W.voronoi_grid(list(bounds), sites, 1.0 + np.arange(n) % 7)


def _envelope(sites, bounds, x, k):
    """(cells, t_in, t_out) of the ray x + t k (t >= 0) inside the box, from
    the lower envelope of the lines a_c + b_c t (lowest index on ties)."""
    b = np.asarray(bounds, float).reshape(3, 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (b[:, 0] - x) / k
        t2 = (b[:, 1] - x) / k
    inside_slab = (x >= b[:, 0]) & (x <= b[:, 1])
    tn = np.where(k == 0, np.where(inside_slab, -np.inf, np.inf), np.minimum(t1, t2))
    tf = np.where(k == 0, np.where(inside_slab, np.inf, -np.inf), np.maximum(t1, t2))
    t0, t_end = max(0.0, tn.max()), tf.min()
    if not t0 < t_end:
        return [], [], []
    a = ((x - sites) ** 2).sum(axis=1)
    bb = 2.0 * ((x - sites) @ k)
    c = int(np.argmin(a + bb * t0))
    cells, tin, tout = [c], [t0], []
    t = t0
    while True:
        faster = bb < bb[c]
        with np.errstate(divide="ignore", invalid="ignore"):
            tc = np.where(faster, (a - a[c]) / (bb[c] - bb), np.inf)
        tc[c] = np.inf
        tc[tc < t] = np.inf
        j = int(np.argmin(tc))
        if not tc[j] < t_end:
            tout.append(t_end)
            return cells, tin, tout
        t = tc[j]
        tout.append(t)
        cells.append(j)
        tin.append(t)
        c = j


def _check(oracle, prob, x, k, start=-1):
    g = prob.grid
    cells, s_in, s_out = oracle.path(prob, x, k, start)
    ec, et_in, et_out = (np.asarray(v) for v in _envelope(g.sites, g.bounds, np.asarray(x, float),
                                                         np.asarray(k, float)))
    keep = et_out - et_in > 1e-12
    ec, et_in, et_out = ec[keep], et_in[keep], et_out[keep]
    pos = s_out - s_in > 1e-12
    assert list(cells[pos]) == list(ec)
    np.testing.assert_allclose(s_in[pos], et_in, rtol=0, atol=1e-10)
    np.testing.assert_allclose(s_out[pos], et_out, rtol=0, atol=1e-10)
    if len(s_in):
        np.testing.assert_array_equal(s_in[1:], s_out[:-1])
        assert len(set(cells.tolist())) == len(cells)  # each convex cell once
        # points inside every positive segment are nearest to its site
        for c, a, b in zip(cells[pos], s_in[pos], s_out[pos]):
            for f in (0.25, 0.5, 0.75):
                p = np.asarray(x, float) + (a + f * (b - a)) * np.asarray(k, float)
                d2 = ((g.sites - p) ** 2).sum(axis=1)
                assert d2[c] <= d2.min() * (1 + 1e-12) + 1e-300
    return cells, s_in, s_out


@pytest.mark.parametrize("seed", [0, 1])
def test_voronoi_locate_is_the_nearest_site(oracle, seed):
    grid = _random_voronoi(seed)
    prob = _problem(grid)
    rng = np.random.default_rng(seed + 20)
    b = np.asarray(grid.bounds, float).reshape(3, 2)
    for _ in range(300):
        p = b[:, 0] + rng.uniform(0, 1, 3) * (b[:, 1] - b[:, 0])
        c, _ = oracle.locate(prob, p)
        assert c == int(np.argmin(((grid.sites - p) ** 2).sum(axis=1)))


@pytest.mark.parametrize("seed", [2, 3])
def test_voronoi_path_matches_the_distance_envelope(oracle, seed):
    grid = _random_voronoi(seed)
    prob = _problem(grid)
    rng = np.random.default_rng(seed)
    b = np.asarray(grid.bounds, float).reshape(3, 2)
    n_long = 0
    for k in _dirs(rng, 60):
        inside = b[:, 0] + rng.uniform(0, 1, 3) * (b[:, 1] - b[:, 0])
        cells, _, _ = _check(oracle, prob, inside, k)
        n_long += len(cells) > 5
        outside = b[:, 0] + rng.uniform(-1.0, 2.0, 3) * (b[:, 1] - b[:, 0])
        _check(oracle, prob, outside, k)
    assert n_long > 10


def test_voronoi_path_from_a_known_cell(oracle):
    """From its known cell the walk is the located walk; from a point a
    rounding error outside the known cell (beyond a face it shares with the
    point's true cell) it takes a zero-length segment there and then has the
    located walk's segments."""
    grid = _random_voronoi(4)
    prob = _problem(grid)
    rng = np.random.default_rng(4)
    S = grid.sites
    tested = 0
    for c in rng.permutation(grid.n_cells)[:40]:
        for j in grid.child[grid.offsets[c]:grid.offsets[c + 1]]:
            m = 0.5 * (S[c] + S[j])
            d2 = ((S - m) ** 2).sum(axis=1)
            others = np.delete(d2, [c, j])
            if others.min() < d2[c] * (1 + 1e-3) or np.any(np.abs(m - np.asarray(grid.bounds)[[0, 2, 4]]) < 1e-9):
                continue  # the midpoint is not on the common face
            x = m + 1e-13 * (S[c] - S[j]) / np.linalg.norm(S[c] - S[j])
            for k in _dirs(rng, 2)[:2]:
                cells, s_in, s_out = _check(oracle, prob, x, k, start=int(c))
                assert cells[0] == c
                cj, sj_in, sj_out = oracle.path(prob, x, k, int(j))
                assert cj[0] == j
                # segments beyond the rounding-level first one
                pos, posj = s_out - s_in > 1e-9, sj_out - sj_in > 1e-9
                assert list(cj[posj]) == list(cells[pos])
                np.testing.assert_allclose(sj_out[posj], s_out[pos], rtol=0, atol=1e-12)
                tested += 1
            break
    assert tested >= 10


def test_voronoi_lattice_equals_cartesian(oracle):
    """Sites on the cell centres of an 8^3 cube with face neighbours: every
    tally equals the cartesian grid's (the same planes, the same order)."""
    cart = W.uniform_cube(n_cells=8, n_pix=16, channels=3, source_pos=(0.1, 0.05, -0.07))
    rng = np.random.default_rng(9)
    dens = rng.uniform(0.2, 3.0, (8, 8, 8)).astype(np.float32)
    cart = W.with_density(cart, dens)
    vor = W.replace(cart, grid=W.voronoi_lattice(cart.grid))
    rc = oracle.run(cart, 3000)
    rv = oracle.run(vor, 3000)
    for a, b in zip(rv["images"], rc["images"]):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(rv["absorption"], rc["absorption"], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(rv["stats"], rc["stats"], rtol=1e-12)
    assert rv["counters"][1] == rc["counters"][1]


def test_voronoi_disk_conserves_luminosity(oracle):
    prob = W.voronoi_disk(n_sites=3000, n_lambda=2, n_pix=16)
    r = oracle.run(prob, 400, n_threads=4)
    emitted, escaped, absorbed, truncated = r["stats"]
    assert abs(emitted - escaped - absorbed - truncated) <= 1e-12 * emitted
    assert absorbed > 0.05 * emitted and r["counters"][1] > 0
    assert abs(r["absorption"].sum() - absorbed) <= 1e-9 * absorbed


def test_voronoi_neighbour_lists_are_symmetric():
    grid = _random_voronoi(5)
    n = grid.n_cells
    pairs = set()
    for c in range(n):
        for j in grid.child[grid.offsets[c]:grid.offsets[c + 1]]:
            assert j != c and 0 <= j < n
            pairs.add((c, int(j)))
    assert all((j, c) in pairs for c, j in pairs)
