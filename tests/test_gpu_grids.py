"""GPU parity on rectilinear grids (cells between arbitrary edges per axis;
the PowCub grid of Table 1(d)) and on the paper's worked spiral-galaxy
example (Sect. 2.5), through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from paper_1410_1629_gb300 import rt
from paper_1410_1629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)

import parity as PAR  # noqa: E402


def _assert_ok(rep):
    print(PAR.summary(rep))
    if not rep["ok"]:
        import json
        print("PARITY REPORT", json.dumps(rep, default=float))
    assert rep["ok"]


def _powcub_disk(nx=48, nz=32, n_lambda=3, n_pix=48):
    """The disk galaxy's dust and stars on a power-law spaced grid (ratio 20
    in x and y, 50 in z), three frames with direct and scattered channels and
    an SED instrument."""
    base = W.disk_galaxy(n_cells=nx, n_lambda=n_lambda, n_pix=n_pix, channels=3)
    edges = [W.powcub_edges(-25.0, 25.0, nx, 20.0), W.powcub_edges(-25.0, 25.0, nx, 20.0),
             W.powcub_edges(-3.0, 3.0, nz, 50.0)]
    xs, ys, zs = (0.5 * (e[1:] + e[:-1]) for e in edges)
    R = np.sqrt(xs[None, None, :] ** 2 + ys[None, :, None] ** 2)
    dens = np.exp(-R / 6.0 - np.abs(zs)[:, None, None] / 0.2)
    prob = W.replace(base, grid=W.rectilinear_grid(edges, dens))
    prob.instruments = prob.instruments + [W.sed_instrument(60.0)]
    return prob


def test_powcub_grid_parity():
    prob = _powcub_disk()
    n = 20000
    g = PAR.gpu_run(prob, n, records_cap=8_000_000)
    o = PAR.oracle_run(prob, n, records_cap=8_000_000)
    assert g["raw_stats"]["device_flags"] == 0
    rep = PAR.compare(g, o, prob, groups=PAR.cell_groups(prob.grid))
    _assert_ok(rep)
    assert rep["crossings_rel"] < 1e-5
    sed_g, sed_o = g["images"][3][:, :, 0, 0], o["images"][3][:, :, 0, 0]
    np.testing.assert_allclose(sed_g, sed_o, rtol=1e-6)


def test_rectilinear_grid_arguments_are_checked():
    prob = _powcub_disk(nx=8, nz=4, n_lambda=1, n_pix=8)
    ctx = rt.rt_context_create(0)
    try:
        d, keep = rt.grid_desc(prob.grid)
        bad = np.array(prob.grid.edges[2])
        bad[2] = bad[1]  # not strictly increasing
        keep.append(bad)
        d.edges[2] = bad.ctypes.data
        with pytest.raises(rt.RTError) as e:
            rt.rt_create_grid(ctx, d)
        assert e.value.status == rt.RT_ERR_ARG
        d, keep = rt.grid_desc(prob.grid)
        d.bounds[5] = 4.0  # last z edge is 3
        with pytest.raises(rt.RTError) as e:
            rt.rt_create_grid(ctx, d)
        assert e.value.status == rt.RT_ERR_ARG
    finally:
        rt.rt_context_destroy(ctx)


@pytest.mark.parametrize("grid", ["powcub", "cartesian"])
def test_spiral_example_first_packet_ids(grid):
    """The paper's spiral-galaxy example at full size (256 x 256 x 128
    power-law cells, or 256 x 256 x 72 equal cells; 1200 x 300 edge-on
    frame; 1e7-packet weights) on its first 1e5 packet ids: bins of at least
    1e3 oracle contributions (pixels, 20 x 20 blocks, cells, 4^3-cell
    blocks) within 1e-4, totals within 1e-6."""
    prob = W.spiral_example(grid) if grid == "powcub" else W.spiral_example("cartesian", n_z=72)
    prob.instruments[0].channels = 3
    n_ids = 100_000
    g = PAR.gpu_run(prob, n_ids, n_norm=prob.run.n_per_lambda, records_cap=40 * n_ids)
    o = PAR.oracle_run(prob, n_ids, n_norm=prob.run.n_per_lambda, records_cap=40 * n_ids)
    assert g["raw_stats"]["device_flags"] == 0
    rep = PAR.compare(g, o, prob, groups=PAR.cell_groups(prob.grid), block=20)
    _assert_ok(rep)
    assert rep["pixels"][0]["blocks"]["bins"] > 0 and rep["cell_groups"]["bins"] > 0


def test_powcub_column_sums_equal_walked_peel_offs():
    """On a power-law grid, peel-offs towards frames along the grid axes
    (face-on along +z, edge-on along -y) take their optical depth from
    per-line sums of density times cell width: the same paths, events,
    crossing counts and absorption as walking every peel-off, and images
    equal to FP32 rounding of the optical depth."""
    prob = _powcub_disk()
    n = 20000
    walked = PAR.gpu_run(prob, n, walk_peels=1)
    summed = PAR.gpu_run(prob, n)
    assert summed["raw_stats"]["column_peels"] > 0 and walked["raw_stats"]["column_peels"] == 0
    assert np.array_equal(walked["counters"], summed["counters"])
    np.testing.assert_allclose(summed["absorption"], walked["absorption"], rtol=1e-12, atol=1e-30)
    for a, b in zip(summed["images"], walked["images"]):
        np.testing.assert_allclose(a, b, rtol=2e-5, atol=1e-12 * b.max())


@pytest.mark.parametrize("case", ["random_axes", "clumpy"])
def test_bintree_parity(case):
    """k-d tree grids (Table 1(d): BinTree): a random tree with random split
    axes under a uniform-cube problem, and the clumpy medium refined by mass
    with the axes in turn (~2e4 leaves, Plummer bulge + exponential disk,
    four wavelengths, two frames), against the oracle."""
    if case == "random_axes":
        rng = np.random.default_rng(11)
        grid, _, _ = W.build_bintree([-1, 1] * 3, lambda lo, hi, d: rng.uniform(size=len(lo)) < (0.95 if d < 3 else 0.7),
                                     lambda lo, hi: rng.lognormal(0.0, 1.0, len(lo)), 12,
                                     axis_of=lambda lo, hi, d: rng.integers(0, 3, len(lo)))
        prob = W.replace(W.uniform_cube(axis_tau=2.0, channels=3), grid=grid)
        n = 50000
    else:
        prob = W.clumpy_bintree(channels=3)
        n = prob.run.n_per_lambda
    g = PAR.gpu_run(prob, n, records_cap=8_000_000)
    o = PAR.oracle_run(prob, n, records_cap=8_000_000)
    assert g["raw_stats"]["device_flags"] == 0
    rep = PAR.compare(g, o, prob, groups=PAR.cell_groups(prob.grid))
    _assert_ok(rep)
    assert rep["crossings_rel"] < 1e-4


@pytest.mark.parametrize("kind", ["bintree", "octree"])
def test_tree_leaf_ids_are_checked(kind):
    """Every leaf id of a tree appears once: a repeated id and a tree with
    fewer leaves than n_leaves are rejected; the unchanged tree is accepted."""
    if kind == "bintree":
        grid, _, _ = W.build_bintree([-1, 1] * 3, lambda lo, hi, d: np.ones(len(lo), bool),
                                     lambda lo, hi: np.ones(len(lo)), 4)
    else:
        grid, _, _ = W.build_octree([-1, 1] * 3, lambda lo, hi, l: np.ones(len(lo), bool),
                                    lambda lo, hi: np.ones(len(lo)), 2)
    ctx = rt.rt_context_create(0)
    try:
        leaves = np.flatnonzero(np.asarray(grid.child) < 0)
        dup = np.array(grid.child)
        dup[leaves[1]] = dup[leaves[0]]
        short = W.replace(grid, density=np.concatenate([grid.density, np.ones(3, np.float32)]))
        for bad in (W.replace(grid, child=dup), short):
            d, keep = rt.grid_desc(bad)
            with pytest.raises(rt.RTError) as e:
                rt.rt_create_grid(ctx, d)
            assert e.value.status == rt.RT_ERR_ARG
        d, keep = rt.grid_desc(grid)
        rt.rt_create_grid(ctx, d)
    finally:
        rt.rt_context_destroy(ctx)


def _chain_octree(depth):
    """An octree whose first child is split at every level down to `depth`."""
    n_nodes = 1 + 8 * depth
    child = np.empty(n_nodes, np.int32)
    leaf = 0
    for node in range(n_nodes):
        level_first = node == 0 or (node - 1) % 8 == 0
        if level_first and (node == 0 or (node - 1) // 8 + 1 < depth):
            child[node] = 1 + 8 * (0 if node == 0 else (node - 1) // 8 + 1)
        else:
            child[node] = -(leaf + 1)
            leaf += 1
    return W.Grid(kind="octree", bounds=[-1.0, 1.0] * 3, density=np.ones(leaf, np.float32), child=child)


def test_octree_depth_is_checked():
    """Octrees deeper than 21 levels (the walk's 3 path bits per level in 64
    bits) are rejected at grid creation; 21 levels are accepted."""
    ctx = rt.rt_context_create(0)
    try:
        d, keep = rt.grid_desc(_chain_octree(22))
        with pytest.raises(rt.RTError) as e:
            rt.rt_create_grid(ctx, d)
        assert e.value.status == rt.RT_ERR_ARG
        d, keep = rt.grid_desc(_chain_octree(21))
        rt.rt_create_grid(ctx, d)
    finally:
        rt.rt_context_destroy(ctx)
