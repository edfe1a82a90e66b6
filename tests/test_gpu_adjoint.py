"""GPU adjoint: against the oracle's forward-mode dual numbers on small grids,
and against central differences of the GPU forward under common random
numbers (bilinear deposit, termination by event count)."""
import numpy as np
import pytest

from paper_1410_1629_gb300 import rt
from paper_1410_1629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)


def _gpu_grad(prob, n, adj_img, adj_abs, **opts):
    sim = rt.Simulation(prob)
    try:
        a_img = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in adj_img]
        a_abs = torch.from_numpy(np.ascontiguousarray(adj_abs)).cuda() if adj_abs is not None else None
        grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device="cuda")
        o = sim.opts(**opts)
        rt.rt_adjoint(sim.ctx, [a.data_ptr() for a in a_img], a_abs.data_ptr() if a_abs is not None else 0,
                      grad.data_ptr(), n, 0, prob.run.seed, o)
        st = sim.stats()  # synchronises, reports device flags
        assert st["device_flags"] == 0
        return grad.cpu().numpy()
    finally:
        sim.close()


@pytest.mark.parametrize("n_cells,channels", [(4, 1), (6, 3)])
def test_adjoint_matches_oracle_dual_numbers(n_cells, channels):
    from oracle import oracle as O
    prob = W.lognormal_cube(n_cells=n_cells, n_pix=8, n_packets=400, max_events=6)
    prob.instruments[0].channels = channels
    rng = np.random.default_rng(n_cells)
    q = prob.instruments[0]
    adj_img = rng.standard_normal((q.channels, 1, q.ny, q.nx))
    adj_abs = rng.standard_normal((1, prob.grid.n_cells))
    n = prob.run.n_per_lambda
    g = _gpu_grad(prob, n, [adj_img], adj_abs, max_events=6, weight_cut=0)
    ref = O.vjp(prob, np.arange(prob.grid.n_cells), n, adj_images=[adj_img], adj_absorption=adj_abs,
                max_events=6, weight_cut=False, n_threads=O.default_threads())
    scale = np.abs(ref).max()
    err = np.abs(g - ref)
    print("max abs err / scale", err.max() / scale, "p99", np.quantile(err, 0.99) / scale)
    assert np.quantile(err, 0.99) <= 1e-4 * scale
    assert err.max() <= 1e-3 * scale


def _loss_problem(n_cells, n_pix, n_packets):
    prob = W.lognormal_cube(n_cells=n_cells, n_pix=n_pix, n_packets=n_packets, max_events=20)
    target = W.lognormal_cube(n_cells=n_cells, n_pix=n_pix, n_packets=n_packets, max_events=20, seed=104)
    return prob, target


def test_adjoint_matches_central_differences_and_duals():
    """Loss = sum (image - target)^2 on a 24^3 log-normal cube.

    The estimator is piecewise smooth in the densities: the optical depth
    along a ray is piecewise linear in the ray's start (kinks where the ray
    meets cell edges) and the bilinear deposit has kinks at pixel centres, so
    a central difference straddles kinks and converges only as fast as they
    allow.  Even the FP64 oracle's own central differences at steps 1e-2 to
    1e-3 of a density differ from its exact (dual-number) derivative by up to
    a few per cent on cells whose gradient is small.  The pin is therefore
    the oracle's dual-number derivative on every sampled cell; central
    differences of the GPU forward (step 1e-2, common random numbers) are
    held to the same derivative on the cells of largest gradient, where the
    kinks are negligible."""
    from oracle import oracle as O
    prob, target_prob = _loss_problem(24, 32, 50000)
    n = prob.run.n_per_lambda
    opts = dict(max_events=20, weight_cut=0)
    sim = rt.Simulation(prob)
    tsim = rt.Simulation(target_prob)
    try:
        tsim.launch(n, 0, 0, **opts)
        target = tsim.images()[0]

        def loss_of(dens):
            d = torch.from_numpy(np.ascontiguousarray(dens, dtype=np.float32)).cuda()
            rt.rt_update_density(sim.ctx, d.data_ptr(), 1)
            sim.reset()
            sim.launch(n, 0, 0, **opts)
            img = sim.images()[0]
            return float(((img - target) ** 2).sum().item()), img

        rho = prob.grid.density.ravel().copy()
        base, img = loss_of(rho)
        adj = (2.0 * (img - target)).contiguous()
        grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device="cuda")
        rt.rt_update_density(sim.ctx, torch.from_numpy(rho).cuda().data_ptr(), 1)
        rt.rt_adjoint(sim.ctx, [adj.data_ptr()], 0, grad.data_ptr(), n, 0, 0, sim.opts(**opts))
        assert sim.stats()["device_flags"] == 0
        g = grad.cpu().numpy()
        gmax = np.abs(g).max()
        top = np.argsort(-np.abs(g))[:6]
        rng = np.random.default_rng(4)
        rest = np.setdiff1d(np.arange(prob.grid.n_cells), top)
        cells = np.concatenate([top, rng.choice(rest, 10, replace=False)])
        for c in top:
            up, dn = rho.copy(), rho.copy()
            up[c] = np.float32(rho[c] * (1 + 1e-2))
            dn[c] = np.float32(rho[c] * (1 - 1e-2))
            fd = (loss_of(up)[0] - loss_of(dn)[0]) / (float(up[c]) - float(dn[c]))
            print("fd", c, fd, g[c])
            assert abs(fd - g[c]) <= 2e-3 * abs(g[c]) + 1e-5 * gmax, c

        # the exact derivative of the same estimator: the oracle's forward-mode
        # duals, with the oracle's own images in the adjoint
        kw = dict(max_events=20, weight_cut=False, n_threads=O.default_threads(), absorption=False)
        t_o = O.run(target_prob, n, **kw)["images"][0]
        i_o = O.run(prob, n, **kw)["images"][0]
        g_o = O.vjp(prob, cells, n, adj_images=[2.0 * (i_o - t_o)], max_events=20, weight_cut=False,
                    n_threads=O.default_threads())
        for c, go in zip(cells, g_o):
            print("dual", c, go, g[c])
        np.testing.assert_allclose(g[cells], g_o, rtol=5e-4, atol=1e-9 * gmax)
    finally:
        sim.close()
        tsim.close()


def test_adjoint_matches_duals_at_full_grid_size():
    """The 64^3 log-normal cube with its 128^2 bilinear detector (the
    differentiation workload at full grid and detector size; packets are
    independent, so 10^5 of them exercise the same per-packet arithmetic):
    the GPU adjoint against the oracle's dual-number derivative on the 4
    cells of largest gradient and 4 random cells, each to 5e-4 relative."""
    from oracle import oracle as O
    prob, target_prob = _loss_problem(64, 128, 100000)
    n = prob.run.n_per_lambda
    kw = dict(max_events=20, weight_cut=False, n_threads=O.default_threads(), absorption=False)
    t_o = O.run(target_prob, n, **kw)["images"][0]
    i_o = O.run(prob, n, **kw)["images"][0]
    adj_o = 2.0 * (i_o - t_o)
    g = _gpu_grad(prob, n, [adj_o], None, max_events=20, weight_cut=0)
    gmax = np.abs(g).max()
    top = np.argsort(-np.abs(g))[:4]
    rng = np.random.default_rng(4)
    cells = np.concatenate([top, rng.choice(np.setdiff1d(np.arange(prob.grid.n_cells), top), 4, replace=False)])
    g_o = O.vjp(prob, cells, n, adj_images=[adj_o], max_events=20, weight_cut=False, n_threads=O.default_threads())
    for c, go in zip(cells, g_o):
        print(c, go, g[c])
    np.testing.assert_allclose(g[cells], g_o, rtol=5e-4, atol=1e-12 * gmax)


def test_column_sums_equal_walked_peel_offs_in_the_adjoint():
    """Peel-offs towards a frame along a grid axis: the adjoint with column
    sums and per-line deposit differences equals the adjoint that walks every
    peel-off ray, to FP32 rounding, including an absorption adjoint."""
    prob = W.lognormal_cube(n_cells=16, n_pix=24, n_packets=20000, max_events=10)
    rng = np.random.default_rng(7)
    q = prob.instruments[0]
    adj_img = rng.standard_normal((q.channels, 1, q.ny, q.nx))
    adj_abs = rng.standard_normal((1, prob.grid.n_cells))
    n = prob.run.n_per_lambda
    for a_abs in (None, adj_abs):
        walked = _gpu_grad(prob, n, [adj_img], a_abs, max_events=10, weight_cut=0, walk_peels=1)
        summed = _gpu_grad(prob, n, [adj_img], a_abs, max_events=10, weight_cut=0)
        scale = np.abs(walked).max()
        np.testing.assert_allclose(summed, walked, rtol=0, atol=2e-5 * scale)


@pytest.mark.parametrize("n_cells,max_events", [(16, 10), (24, 20)])
def test_tape_equals_replay(n_cells, max_events):
    """A forward launch that records the adjoint tape lets rt_adjoint skip
    the replay of the forced paths; the gradient equals the replayed one to
    FP64 summation order (the forward writes every record field with the
    replay's own arithmetic).  A changed density invalidates the tape."""
    prob = W.lognormal_cube(n_cells=n_cells, n_pix=24, n_packets=6000, max_events=max_events)
    rng = np.random.default_rng(11)
    q = prob.instruments[0]
    a = torch.from_numpy(rng.standard_normal((q.channels, 1, q.ny, q.nx))).cuda()
    n = prob.run.n_per_lambda
    o = dict(max_events=max_events, weight_cut=0)
    sim = rt.Simulation(prob)
    try:
        grads = []
        for tape in (0, 1):
            sim.reset()
            sim.launch(n, 0, 5, tape=tape, **o)
            grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device="cuda")
            prof = torch.zeros(8, dtype=torch.int64, device="cuda")
            rt.rt_adjoint(sim.ctx, [a.data_ptr()], 0, grad.data_ptr(), n, 0, 5, sim.opts(profile=prof.data_ptr(), **o))
            grads.append((grad.cpu().numpy(), int(prof[0])))
            assert sim.stats()["device_flags"] == 0
        (g0, c0), (g1, c1) = grads
        np.testing.assert_allclose(g1, g0, rtol=1e-10, atol=1e-12 * np.abs(g0).max())
        assert c1 < c0  # the tape run walked fewer cells (no replay)
        # a new density invalidates the tape: the next adjoint replays
        d = torch.from_numpy(prob.grid.density.ravel().copy()).cuda()
        rt.rt_update_density(sim.ctx, d.data_ptr(), 1)
        prof = torch.zeros(8, dtype=torch.int64, device="cuda")
        grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device="cuda")
        rt.rt_adjoint(sim.ctx, [a.data_ptr()], 0, grad.data_ptr(), n, 0, 5, sim.opts(profile=prof.data_ptr(), **o))
        assert int(prof[0]) == c0
        np.testing.assert_allclose(grad.cpu().numpy(), g0, rtol=1e-10, atol=1e-12 * np.abs(g0).max())
    finally:
        sim.close()


def test_autograd_image_loss_uses_the_tape():
    """An image-only loss through the autograd Function: the forward records
    the tape and the backward uses it; the gradient equals a direct replayed
    adjoint of the same adjoint image."""
    from paper_1410_1629_gb300.autograd import transport
    prob = W.lognormal_cube(n_cells=12, n_pix=16, n_packets=5000, max_events=10)
    sim = rt.Simulation(prob)
    try:
        dens = torch.from_numpy(prob.grid.density.copy()).cuda().requires_grad_(True)
        imgs, _ = transport(dens, sim, max_events=10, weight_cut=0)
        w = torch.linspace(-1, 1, imgs[0].numel(), device="cuda", dtype=torch.float64).view_as(imgs[0])
        (w * imgs[0]).sum().backward()
        g_auto = dens.grad.double().cpu().numpy().ravel()
        sim.reset()
        sim.launch(prob.run.n_per_lambda, 0, prob.run.seed, max_events=10, weight_cut=0)  # no tape: replay
        grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device="cuda")
        rt.rt_adjoint(sim.ctx, [w.contiguous().data_ptr()], 0, grad.data_ptr(), prob.run.n_per_lambda, 0,
                      prob.run.seed, sim.opts(max_events=10, weight_cut=0))
        g_dir = grad.cpu().numpy()
        np.testing.assert_allclose(g_auto, g_dir.astype(np.float32), rtol=1e-5, atol=1e-6 * np.abs(g_dir).max())
    finally:
        sim.close()


def test_adjoint_tuner_keeps_gradients():
    """rt_adjoint_tune only chooses the deferral threshold: the gradient
    afterwards equals the untuned one to FP64 summation order."""
    prob = W.lognormal_cube(n_cells=16, n_pix=24, n_packets=8000, max_events=10)
    rng = np.random.default_rng(9)
    q = prob.instruments[0]
    adj_img = rng.standard_normal((q.channels, 1, q.ny, q.nx))
    n = prob.run.n_per_lambda
    ref = _gpu_grad(prob, n, [adj_img], None, max_events=10, weight_cut=0)
    sim = rt.Simulation(prob)
    try:
        a = torch.from_numpy(adj_img).cuda()
        lanes = rt.rt_adjoint_tune(sim.ctx, [a.data_ptr()], 0, 2000, 1, sim.opts(max_events=10, weight_cut=0))
        assert lanes in (12, 16, 20, 24, 28, 32)
        grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device="cuda")
        rt.rt_adjoint(sim.ctx, [a.data_ptr()], 0, grad.data_ptr(), n, 0, prob.run.seed,
                      sim.opts(max_events=10, weight_cut=0))
        g = grad.cpu().numpy()
    finally:
        sim.close()
    np.testing.assert_allclose(g, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def test_autograd_function_matches_direct_adjoint():
    from paper_1410_1629_gb300.autograd import transport
    prob = W.lognormal_cube(n_cells=8, n_pix=16, n_packets=5000, max_events=10)
    sim = rt.Simulation(prob)
    try:
        dens = torch.from_numpy(prob.grid.density.copy()).cuda().requires_grad_(True)
        imgs, ab = transport(dens, sim, max_events=10, weight_cut=0)
        w = torch.linspace(-1, 1, imgs[0].numel(), device="cuda", dtype=torch.float64).view_as(imgs[0])
        loss = (w * imgs[0]).sum() + 0.5 * ab.sum()
        loss.backward()
        g_auto = dens.grad.double().cpu().numpy().ravel()
        grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device="cuda")
        a_abs = torch.full_like(ab, 0.5)
        rt.rt_adjoint(sim.ctx, [w.contiguous().data_ptr()], a_abs.data_ptr(), grad.data_ptr(), prob.run.n_per_lambda,
                      0, 0, sim.opts(max_events=10, weight_cut=0))
        g_dir = grad.cpu().numpy()
        np.testing.assert_allclose(g_auto, g_dir.astype(np.float32), rtol=1e-5, atol=1e-6 * np.abs(g_dir).max())
    finally:
        sim.close()


def test_finite_differences_of_the_forward_on_64_random_cells():
    """Central differences at the workload's step (eps = 1e-3 of a cell's
    density) on 64 random cells (rng seed 4) of the 64^3 log-normal cube with
    its 128^2 bilinear detector (1e5 packets, common random numbers), of the
    linear functional sum_pixels a * image with a = 2 (image - target) taken
    from the oracle.

    * The GPU adjoint against central differences of the FP64 oracle forward
      at that step: the median cell within 1e-3, nine cells in ten within
      5e-2 (the estimator's kinks: the oracle's own differences depart from
      its dual-number derivative by as much on the same cells).
    * The GPU adjoint against the dual-number derivative (no step at all).
    * Central differences of the GPU forward against the oracle's at the same
      step: FP32 geometry and FP32 peel-off values round every contribution of
      a packet that crosses the perturbed cell afresh in each run; the change
      a step of 1e-3 makes is a few 1e-5 of a contribution, and where the
      functional's terms cancel (a changes sign) the rounding does not.  The
      GPU differences therefore follow the oracle's only to a few per cent
      (the median cell) and closely across cells (correlation above 0.98)."""
    from oracle import oracle as O
    prob, target_prob = _loss_problem(64, 128, 100000)
    n = prob.run.n_per_lambda
    eps = 1e-3
    kw = dict(max_events=20, weight_cut=False, n_threads=O.default_threads(), absorption=False)
    i_o = O.run(prob, n, **kw)["images"][0]
    t_o = O.run(target_prob, n, **kw)["images"][0]
    a = 2.0 * (i_o - t_o)
    cells = np.random.default_rng(4).choice(prob.grid.n_cells, 64, replace=False)
    rho = prob.grid.density.ravel().copy()
    opts = dict(max_events=20, weight_cut=0)
    sim = rt.Simulation(prob)
    try:
        def functional(dens):
            d = torch.from_numpy(np.ascontiguousarray(dens, dtype=np.float32)).cuda()
            rt.rt_update_density(sim.ctx, d.data_ptr(), 1)
            sim.reset()
            sim.launch(n, 0, 0, **opts)
            return float((a * sim.images()[0].cpu().numpy()).sum())

        fd_g = np.zeros(64)
        fd_o = np.zeros(64)
        for i, c in enumerate(cells):
            up, dn = rho.copy(), rho.copy()
            up[c] = np.float32(rho[c] * (1 + eps))
            dn[c] = np.float32(rho[c] * (1 - eps))
            h = float(up[c]) - float(dn[c])
            fd_g[i] = (functional(up) - functional(dn)) / h
            iu = O.run(W.with_density(prob, up.reshape(prob.grid.density.shape)), n, **kw)["images"][0]
            idn = O.run(W.with_density(prob, dn.reshape(prob.grid.density.shape)), n, **kw)["images"][0]
            fd_o[i] = float((a * (iu - idn)).sum() / h)
        rt.rt_update_density(sim.ctx, torch.from_numpy(rho).cuda().data_ptr(), 1)
        adj = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device="cuda")
        rt.rt_adjoint(sim.ctx, [adj.data_ptr()], 0, grad.data_ptr(), n, 0, 0, sim.opts(**opts))
        assert sim.stats()["device_flags"] == 0
        g = grad.cpu().numpy()[cells]
    finally:
        sim.close()
    dual = O.vjp(prob, cells, n, adj_images=[a], max_events=20, weight_cut=False, n_threads=O.default_threads())
    rel = lambda x, y: np.abs(x - y) / np.abs(y)
    q = lambda v: np.quantile(v, [0.5, 0.9, 1.0])
    print("GPU adjoint vs oracle FD: median, p90, max", q(rel(g, fd_o)))
    print("oracle FD vs duals:       median, p90, max", q(rel(fd_o, dual)))
    print("GPU adjoint vs duals:     median, p90, max", q(rel(g, dual)))
    print("GPU FD vs oracle FD:      median, p90, max", q(rel(fd_g, fd_o)),
          "abs / max|FD|", q(np.abs(fd_g - fd_o) / np.abs(fd_o).max()), "corr", np.corrcoef(fd_g, fd_o)[0, 1])
    print("GPU FD vs GPU adjoint:    median, p90, max", q(rel(fd_g, g)))
    assert np.median(rel(g, fd_o)) < 1e-3 and np.quantile(rel(g, fd_o), 0.9) < 5e-2
    scale = np.abs(dual).max()
    assert np.median(rel(g, dual)) < 1e-3
    assert np.all(np.abs(g - dual) <= 2e-3 * np.abs(dual) + 1e-3 * scale)
    assert np.median(rel(fd_g, fd_o)) < 0.1 and np.corrcoef(fd_g, fd_o)[0, 1] > 0.98
