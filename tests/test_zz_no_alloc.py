"""The allocation-free entry point gives the same tallies as the context path.

rt_launch_packets_noalloc is for callers that may not allocate GPU memory
while they run: it brings its own fixed working area (a static device array)
and takes every other buffer from the caller.  Here two calls in a row through
the C ABI are each compared with rt_launch_packets on a context, at the
tolerance of FP64 summation order.  This file is collected last on purpose.
"""
import ctypes
from dataclasses import replace

import numpy as np
import pytest

from paper_1410_1629_gb300 import rt
from paper_1410_1629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)


def _problem():
    # several wavelengths, three frames with direct/scattered channels
    return W.disk_galaxy(n_cells=32, n_lambda=3, n_pix=32, channels=3)


def _context_run(prob, n, first, seed, n_norm):
    sim = rt.Simulation(prob)
    try:
        # the allocation-free path walks every peel-off (it keeps no column sums)
        sim.launch(n, first, seed, n_norm=n_norm, walk_peels=1)
        imgs = [t.cpu().numpy() for t in sim.images()]
        ab = sim.absorption().cpu().numpy()
        st = sim.stats()
    finally:
        sim.close()
    return imgs, ab, st


def _grid(prob, dens):
    grid = rt.rt_grid_desc()
    grid.kind = rt.RT_GRID_CARTESIAN
    grid.bounds[:] = [float(b) for b in prob.grid.bounds]
    grid.nz, grid.ny, grid.nx = prob.grid.density.shape
    grid.density = dens.data_ptr()
    grid.on_device = 1
    return grid


def _noalloc_run(prob, dens, n, first, seed, n_norm):
    grid = _grid(prob, dens)
    imgs = [torch.zeros((q.channels, prob.n_lambda, q.ny, q.nx), dtype=torch.float64, device="cuda")
            for q in prob.instruments]
    ab = torch.zeros((prob.n_lambda, prob.grid.n_cells), dtype=torch.float64, device="cuda")
    stats = torch.zeros(ctypes.sizeof(rt.rt_stats), dtype=torch.uint8, device="cuda")
    opts = rt.rt_default_opts()
    opts.n_norm = n_norm
    rt.rt_launch_packets_noalloc(grid, prob.kappa, prob.albedo, prob.g, [rt.source_desc(s) for s in prob.sources],
                                 [s.lum for s in prob.sources], [rt.instrument_desc(q) for q in prob.instruments],
                                 [t.data_ptr() for t in imgs], ab.data_ptr(), n, first, seed, opts,
                                 stats.data_ptr())
    torch.cuda.synchronize()
    st = rt.rt_stats.from_buffer_copy(bytes(stats.cpu().numpy())).as_dict()
    return [t.cpu().numpy() for t in imgs], ab.cpu().numpy(), st


def test_noalloc_matches_context_path_on_two_calls():
    prob = _problem()
    dens = torch.from_numpy(np.ascontiguousarray(prob.grid.density)).cuda()
    n = 4000
    for first, seed in [(0, 11), (n, 11)]:
        gi, ga, gs = _noalloc_run(prob, dens, n, first, seed, 2 * n)
        ri, ra, rs = _context_run(prob, n, first, seed, 2 * n)
        for a, b in zip(gi, ri):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-20)
        np.testing.assert_allclose(ga, ra, rtol=1e-12, atol=1e-20)
        for key in ("crossings", "path_crossings", "events", "peeloffs", "packets"):
            assert gs[key] == rs[key], key
        for key in ("emitted", "escaped", "absorbed", "truncated"):
            assert abs(gs[key] - rs[key]) <= 1e-12 * abs(rs[key]) + 1e-300, key
        assert gs["device_flags"] == 0


def test_noalloc_without_instruments_or_stats_allocates_nothing():
    """No frames and no statistics output: the absorption field still equals
    the context path's.  The calls allocate no device memory: after a first
    call (which loads the library's device code), the free device memory is
    the same before and after several more calls."""
    prob = _problem()
    dens = torch.from_numpy(np.ascontiguousarray(prob.grid.density)).cuda()
    grid = _grid(prob, dens)
    n = 4000
    ab = torch.zeros((prob.n_lambda, prob.grid.n_cells), dtype=torch.float64, device="cuda")
    srcs = [rt.source_desc(s) for s in prob.sources]
    lums = [s.lum for s in prob.sources]
    rt.rt_launch_packets_noalloc(grid, prob.kappa, prob.albedo, prob.g, srcs, lums, [], [], ab.data_ptr(), n, 0, 3)
    torch.cuda.synchronize()
    got = ab.cpu().numpy()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(4):
        rt.rt_launch_packets_noalloc(grid, prob.kappa, prob.albedo, prob.g, srcs, lums, [], [], ab.data_ptr(), n,
                                     0, 3)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    np.testing.assert_allclose(ab.cpu().numpy(), 5 * got, rtol=1e-11, atol=1e-300)
    noframes = replace(prob, instruments=[])
    sim = rt.Simulation(noframes)
    try:
        sim.launch(n, 0, 3, walk_peels=1)
        ref = sim.absorption().cpu().numpy()
    finally:
        sim.close()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-20)


def test_noalloc_rejects_sizes_beyond_its_working_area():
    prob = _problem()
    dens = torch.from_numpy(np.ascontiguousarray(prob.grid.density)).cuda()
    grid = _grid(prob, dens)
    ab = torch.zeros(1, dtype=torch.float64, device="cuda")
    many = np.full(65, 0.5)
    with pytest.raises(rt.RTError) as e:
        rt.rt_launch_packets_noalloc(grid, many, many, many * 0, [rt.source_desc(prob.sources[0])], [np.ones(65)],
                                     [], [], ab.data_ptr(), 10)
    assert e.value.status == rt.RT_ERR_ARG and "64" in str(e.value)
    opts = rt.rt_default_opts()
    opts.tape = 1
    with pytest.raises(rt.RTError) as e:
        rt.rt_launch_packets_noalloc(grid, prob.kappa, prob.albedo, prob.g, [rt.source_desc(prob.sources[0])],
                                     [prob.sources[0].lum], [], [], ab.data_ptr(), 10, opts=opts)
    assert e.value.status == rt.RT_ERR_ARG
