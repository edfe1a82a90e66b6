"""The 4096-model batch workload has the stated distributions: cells per
side 8..48, half uniform / half exponential slabs, the central-row optical
depth log-uniform in 0.1..20, g and albedo uniform in their ranges, packets
log-uniform in 1e4..1e6 (about 8.9e8 in all)."""
import numpy as np

from paper_1410_1629_gb300 import workloads as W


def test_batch_models_distributions():
    ms = W.batch_models()
    assert len(ms) == 4096
    sides = np.array([m.grid.density.shape[0] for m in ms])
    assert sides.min() == 8 and sides.max() == 48
    assert all(m.grid.density.shape == (s, s, s) for m, s in zip(ms, sides))
    slab = np.array([m.meta["slab"] for m in ms])
    assert slab.sum() == 2048
    taus = np.array([m.meta["axis_tau"] for m in ms])
    assert taus.min() >= 0.1 and taus.max() <= 20.0
    # log-uniform: the mean of ln tau is the midpoint of the log range
    assert abs(np.log(taus).mean() - 0.5 * (np.log(0.1) + np.log(20.0))) < 0.1
    g = np.array([m.g[0] for m in ms])
    a = np.array([m.albedo[0] for m in ms])
    assert 0.0 <= g.min() and g.max() <= 0.9 and 0.3 <= a.min() and a.max() <= 0.8
    pk = np.array([m.run.n_per_lambda for m in ms])
    assert pk.min() >= 1e4 and pk.max() <= 1e6
    assert 8.0e8 < pk.sum() < 9.8e8
    for m in ms[:64]:
        d = m.grid.density.astype(np.float64)
        s = d.shape[0]
        # the stated optical depth along the full x axis through the centre (kappa = 1)
        assert abs(d[s // 2, s // 2, :].sum() * 2.0 / s - m.meta["axis_tau"]) <= 1e-6 * m.meta["axis_tau"]
        if m.meta["slab"]:
            # exp(-|z| / 0.4) at cell centres, constant in x and y
            z = -1.0 + (np.arange(s) + 0.5) * 2.0 / s
            prof = d[:, 0, 0] / d[:, 0, 0].max()
            np.testing.assert_allclose(prof, np.exp(-np.abs(z) / 0.4) / np.exp(-np.abs(z) / 0.4).max(), rtol=1e-6)
            assert np.all(d == d[:, :1, :1])
        else:
            assert np.all(d == d.flat[0])
        assert m.sources[0].kind == "point" and tuple(m.sources[0].center) == (0.0, 0.0, 0.0)
        assert m.instruments[0].nx == 64 and m.instruments[0].ny == 64
