"""Batched launches of many small models: each model of a batch equals the
single-model launch of the same problem (model_id = its index) up to the
order of FP64 additions, and matches the oracle; seeds, repeated launches,
the tuner and argument checks."""
import numpy as np
import pytest

from paper_1410_1629_gb300 import rt
from paper_1410_1629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)


def _models(idx, n_packets, bilinear=False):
    allm = W.batch_models()
    out = []
    for i in idx:
        p = allm[i]
        if bilinear:
            p.instruments[0].bilinear = True
        out.append(W.with_packets(p, n_packets))
    return out


# a spread of sizes, slab / uniform kinds and optical depths of the 4096-model workload
IDX = [0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144]


def _single(problem, model_id, seed, n):
    sim = rt.Simulation(problem)
    try:
        sim.launch(n, 0, seed, model_id=model_id)
        st = sim.stats()
        return sim.images(device=False)[0][0, 0], st
    finally:
        sim.close()


def test_batch_equals_single_model_launches():
    n = 3000
    probs = _models(IDX, n)
    b = rt.Batch(probs)
    try:
        b.launch(seed=7)
        imgs = b.images()
        tal = b.tallies()
        st = b.stats()
    finally:
        b.close()
    assert st["device_flags"] == 0
    tot = {k: 0 for k in ("crossings", "events", "peeloffs", "packets")}
    for m, p in enumerate(probs):
        img, s1 = _single(p, m, 7, n)
        np.testing.assert_allclose(imgs[m], img, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(tal[m], [s1["emitted"], s1["escaped"], s1["absorbed"], s1["truncated"]],
                                   rtol=1e-12, atol=1e-18)
        for k in tot:
            tot[k] += s1[k]
    for k in tot:
        assert st[k] == tot[k], k
    assert st["packets"] == n * len(probs)


def test_batch_matches_the_oracle():
    from oracle import oracle as O
    n = 20000
    idx = [0, 3, 8, 21]
    probs = _models(idx, n, bilinear=True)
    b = rt.Batch(probs)
    try:
        b.launch(seed=11)
        imgs = b.images()
        tal = b.tallies()
    finally:
        b.close()
    for m, p in enumerate(probs):
        o = O.run(p, n, seed=11, model_id=m, n_threads=O.default_threads(), counts=True)
        st = np.asarray(o["stats"])
        scale = np.array([st[0], st[1], st[2], st[0]])
        assert np.all(np.abs(tal[m] - st) <= 1e-6 * np.abs(scale)), (m, tal[m], st)
        ref = o["images"][0][0, 0]
        cnt = o["image_counts"][0][0, 0]
        assert abs(imgs[m].sum() - ref.sum()) <= 1e-6 * ref.sum()
        mask = cnt >= 1000
        assert mask.sum() > 0
        rel = np.abs(imgs[m][mask] - ref[mask]) / np.abs(ref[mask])
        assert rel.max() <= 1e-4, (m, rel.max())


def test_batch_seeds_and_repeated_launches():
    n = 2000
    probs = _models(IDX[:6], n)
    b = rt.Batch(probs)
    try:
        b.launch(seed=3)
        b.reset()
        b.launch(seed=9)  # the graph's kernel parameters change between launches
        one = b.images()
        b.launch(seed=9)
        two = b.images()
        tal = b.tallies()
    finally:
        b.close()
    for m, p in enumerate(probs):
        img, _ = _single(p, m, 9, n)
        np.testing.assert_allclose(one[m], img, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(two[m], 2 * img, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(tal[:, 0], 2.0)  # two launches of unit luminosity


def test_batch_tuner_keeps_results():
    n = 4000
    probs = _models(IDX, n)
    b = rt.Batch(probs)
    try:
        b.launch(seed=5)
        ref = b.images()
        b.reset()
        lanes, run = b.tune(seed=5, fraction=0.25)
        assert lanes in (8, 12, 16, 20, 24, 28, 32) and run in (64, 256, 1024, 4096)
        assert np.all(b.tallies() == 0.0)
        b.launch(seed=5)
        got = b.images()
        assert b.stats()["device_flags"] == 0
    finally:
        b.close()
    for a, r in zip(got, ref):
        np.testing.assert_allclose(a, r, rtol=1e-12, atol=1e-300)


def test_batch_rejects_bad_models():
    """The C ABI's checks, on descriptors the binding would not build."""
    p = _models([0], 100)[0]
    ctx = rt.rt_context_create(0)
    try:
        def descs(mutate):
            good, keep0 = rt.model_desc(p)
            bad, keep1 = rt.model_desc(p)
            mutate(bad)
            return [good, bad], (keep0, keep1)

        for mutate in (lambda d: setattr(d.instrument, "channels", 3), lambda d: setattr(d, "albedo", 1.5),
                       lambda d: setattr(d, "n_packets", 0), lambda d: setattr(d, "nx", 0),
                       lambda d: setattr(d, "luminosity", 0.0)):
            ds, keep = descs(mutate)
            with pytest.raises(rt.RTError) as e:
                rt.rt_batch_create(ctx, ds)
            assert e.value.status == rt.RT_ERR_ARG and "model 1" in str(e.value)
        with pytest.raises(rt.RTError):
            rt.rt_batch_launch(ctx, 7)
    finally:
        rt.rt_context_destroy(ctx)
