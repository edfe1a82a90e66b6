"""GPU parity on Voronoi grids (Table 1(d): VoronoiDustGrid; Sect. 2.4:
sites placed following the dust density of a disk galaxy), through the C ABI
against the FP64 oracle."""
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


@pytest.mark.parametrize("case", ["disk", "lattice"])
def test_voronoi_parity(case):
    """The disk galaxy on 2e4 Voronoi cells (three frames with direct and
    scattered channels, three wavelengths), and the Voronoi grid of an 16^3
    cube's cell centres with random densities; every frame, channel and cell
    (and groups of cells) under the acceptance rule."""
    if case == "disk":
        prob = W.voronoi_disk(n_sites=20_000, n_lambda=3, n_pix=64, channels=3)
        n = 20_000
    else:
        cart = W.uniform_cube(n_cells=16, n_pix=32, axis_tau=3.0, channels=3, source_pos=(0.1, 0.05, -0.07))
        rng = np.random.default_rng(12)
        cart = W.with_density(cart, rng.lognormal(0.0, 0.7, (16, 16, 16)).astype(np.float32))
        prob = W.replace(cart, grid=W.voronoi_lattice(cart.grid))
        n = 40_000
    g = PAR.gpu_run(prob, n, records_cap=8_000_000)
    o = PAR.oracle_run(prob, n, records_cap=8_000_000)
    assert g["raw_stats"]["device_flags"] == 0
    rep = PAR.compare(g, o, prob, groups=PAR.cell_groups(prob.grid))
    _assert_ok(rep)
    assert rep["crossings_rel"] < 1e-4


def test_voronoi_grid_arguments_are_checked():
    prob = W.voronoi_disk(n_sites=500, n_lambda=1, n_pix=8)
    ctx = rt.rt_context_create(0)
    try:
        def expect_arg(mutate):
            d, keep = rt.grid_desc(prob.grid)
            mutate(d, keep)
            with pytest.raises(rt.RTError) as e:
                rt.rt_create_grid(ctx, d)
            assert e.value.status == rt.RT_ERR_ARG

        def bad_neighbour(d, keep):
            nbr = np.array(prob.grid.child)
            nbr[3] = prob.grid.n_cells  # out of range
            keep.append(nbr)
            d.child = nbr.ctypes.data

        def self_neighbour(d, keep):
            nbr = np.array(prob.grid.child)
            nbr[prob.grid.offsets[7]] = 7
            keep.append(nbr)
            d.child = nbr.ctypes.data

        def bad_offsets(d, keep):
            off = np.array(prob.grid.offsets)
            off[-1] -= 1
            keep.append(off)
            d.offsets = off.ctypes.data

        def site_outside(d, keep):
            s = np.array(prob.grid.sites)
            s[5, 2] = 4.0  # the domain ends at z = 3
            keep.append(s)
            d.sites = s.ctypes.data

        def equal_sites(d, keep):
            s = np.array(prob.grid.sites)
            c = 9
            j = prob.grid.child[prob.grid.offsets[c]]
            s[j] = s[c]
            keep.append(s)
            d.sites = s.ctypes.data

        for m in (bad_neighbour, self_neighbour, bad_offsets, site_outside, equal_sites):
            expect_arg(m)
        # the unchanged grid is accepted
        d, keep = rt.grid_desc(prob.grid)
        rt.rt_create_grid(ctx, d)
    finally:
        rt.rt_context_destroy(ctx)


@pytest.mark.parametrize("n_sites", [1, 2])
def test_voronoi_degenerate_grids(n_sites):
    """One site (the whole domain is one cell, no faces: the walk meets only
    the domain boundary) and two sites (one bisecting plane), against the
    oracle; the one-site grid also against the one-cell cartesian grid."""
    cart = W.uniform_cube(n_cells=1, n_pix=16, axis_tau=2.0, channels=3, source_pos=(0.2, -0.1, 0.05))
    if n_sites == 1:
        grid = W.Grid("voronoi", np.array([-1.0, 1.0] * 3), np.ones(1, np.float32), child=np.zeros(0, np.int32),
                      sites=np.array([[0.1, 0.2, -0.3]]), offsets=np.array([0, 0], np.int64))
    else:
        grid = W.Grid("voronoi", np.array([-1.0, 1.0] * 3), np.array([1.0, 3.0], np.float32),
                      child=np.array([1, 0], np.int32), sites=np.array([[-0.4, 0.1, 0.0], [0.5, -0.2, 0.3]]),
                      offsets=np.array([0, 1, 2], np.int64))
    prob = W.replace(cart, grid=grid)
    n = 20000
    g = PAR.gpu_run(prob, n, records_cap=2_000_000)
    o = PAR.oracle_run(prob, n, records_cap=2_000_000)
    assert g["raw_stats"]["device_flags"] == 0
    _assert_ok(PAR.compare(g, o, prob))
    if n_sites == 1:
        c = PAR.gpu_run(cart, n)
        for a, b in zip(g["images"], c["images"]):
            np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-9 * b.max())
        np.testing.assert_allclose(g["stats"], c["stats"], rtol=1e-6)
