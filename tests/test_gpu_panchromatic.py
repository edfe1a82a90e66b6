"""GPU panchromatic mode (Sect. 2.1, 2.2): equilibrium dust temperatures,
the dust's thermal emission and the transport of dust-emission packets,
through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from paper_1410_1629_gb300 import rt
from paper_1410_1629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)

import parity as PAR  # noqa: E402


def _problem():
    # 32^3 cells over a flat box: stored with z unit-stride on the device
    return W.panchromatic_disk(n_cells=32, n_lambda=16, n_pix=32, channels=3)


def test_temperatures_and_emission_match_the_oracle():
    """From the same absorption field (the oracle's, and the GPU's own
    tallies read back) the temperatures agree to FP64 rounding, and so do
    the cells' thermal luminosities at the oracle's temperatures."""
    from oracle import oracle as O
    prob = _problem()
    S = prob.meta["emission_scale"]
    n = 4000
    ab_o = O.run(prob, n, n_threads=O.default_threads())["absorption"]
    T_o, cl_o = O.dust_temperature(prob, ab_o, S)
    sim = rt.Simulation(prob)
    try:
        T_g, cl_g = sim.dust_temperature(S, absorption=ab_o)
        np.testing.assert_allclose(T_g, T_o, rtol=1e-12, atol=0)
        assert cl_g == cl_o and np.count_nonzero(T_o) > 0.9 * T_o.size
        # the GPU's own tallies (storage order on the device) against the
        # oracle's temperatures of the same field read back row-major
        sim.launch(n, 0, 0)
        ab_g = sim.absorption().cpu().numpy()
        T_own, _ = sim.dust_temperature(S)
        T_ref, _ = O.dust_temperature(prob, ab_g, S)
        np.testing.assert_allclose(T_own, T_ref, rtol=1e-12, atol=0)
        # the chain's temperatures from GPU and oracle tallies
        rel = np.abs(T_own - T_o)[T_o > 0] / T_o[T_o > 0]
        print("T from GPU tallies vs oracle tallies: median, p99, max", np.quantile(rel, [0.5, 0.99, 1.0]))
        assert np.median(rel) < 1e-6
        sim.set_dust_emission(T_o, S)
        lum_g = sim.dust_emission()
    finally:
        sim.close()
    lum_o = O.dust_emission(prob, T_o, S)
    np.testing.assert_allclose(lum_g, lum_o, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(lum_o.sum(axis=0)[T_o > 1.0], ab_o.sum(axis=0)[T_o > 1.0], rtol=1e-12)


def test_dust_emission_transport_parity():
    """Packets emitted by the dust at the oracle's temperatures, on both
    sides: the acceptance rule on every frame and channel, the SED and the
    absorption field."""
    from oracle import oracle as O
    prob = _problem()
    S = prob.meta["emission_scale"]
    ab_o = O.run(prob, 4000, n_threads=O.default_threads())["absorption"]
    T_o, _ = O.dust_temperature(prob, ab_o, S)
    lum_o = O.dust_emission(prob, T_o, S)
    dusty = W.replace(prob, dust_lum=lum_o, sources=[])
    n = 20000
    sim = rt.Simulation(prob)
    try:
        sim.set_dust_emission(T_o, S)
        g = PAR.gpu_run(prob, n, sim=sim, records_cap=4_000_000, emitter=rt.RT_EMITTER_DUST)
    finally:
        sim.close()
    o = PAR.oracle_run(dusty, n, records_cap=4_000_000)
    assert g["raw_stats"]["device_flags"] == 0
    assert abs(g["stats"][0] - lum_o.sum()) <= 1e-12 * lum_o.sum()
    rep = PAR.compare(g, o, dusty, groups=PAR.cell_groups(prob.grid))
    print(PAR.summary(rep))
    assert rep["ok"], rep
    sed_g, sed_o = g["images"][3][:, :, 0, 0], o["images"][3][:, :, 0, 0]
    np.testing.assert_allclose(sed_g, sed_o, rtol=1e-6, atol=1e-300)


def test_dust_emitter_needs_emission():
    prob = _problem()
    sim = rt.Simulation(prob)
    try:
        with pytest.raises(rt.RTError) as e:
            sim.launch(10, 0, 0, emitter=rt.RT_EMITTER_DUST)
        assert e.value.status == rt.RT_ERR_STATE
        with pytest.raises(rt.RTError) as e:
            sim.dust_temperature(-1.0)
        assert e.value.status == rt.RT_ERR_ARG
    finally:
        sim.close()
