"""Pins for the oracle's panchromatic mode (Sect. 2.1, 2.2: dust temperature
from the absorbed energy integrated over the wavelengths, thermal dust
emission).  CPU only.

* The Planck function summed over a fine wavelength grid gives its integral
  pi^4 T^4 / (15 C2^4) (in units where the constant 2hc^2 is 1), times the
  cell's mass, the scale and kappa (1 - albedo) of a grey grain.
* The bin widths: for wavelengths 1 and 4 um the borders are 0.5, 2 and 8.
* Energy balance: each cell emits exactly what it absorbed (the bisection's
  own tolerance), and a grey grain's temperature has the closed form.
* Cells without absorption or dust stay at 0 and emit nothing; absorption
  beyond t_max or below t_min is held there and counted.
* Dust-emission packets: the emitted luminosity per wavelength is the sum
  of the cells'; the emitting cell follows the luminosities (binomial test);
  positions are uniform in the cell (chi-square over a frame's pixels);
  luminosity is conserved; a wavelength without emission launches nothing.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1410_1629_gb300 import workloads as W

C2 = 14387.768775039337


def _one_cell(lam, kappa=1.0, albedo=0.3, rho=2.0, side=1.5):
    """One cubic cell of side `side` with density rho: mass rho side^3."""
    n = len(lam)
    prob = W.uniform_cube(n_cells=1, half=0.5 * side, rho=rho, n_pix=4)
    return W.replace(prob, wavelengths=np.asarray(lam, float), kappa=np.full(n, kappa),
                     albedo=np.full(n, albedo), g=np.zeros(n),
                     sources=[W.Source("point", (0.0, 0.0, 0.0), np.ones(n))])


@pytest.mark.parametrize("T", [15.0, 300.0, 6000.0])
def test_planck_sum_is_the_stefan_boltzmann_integral(oracle, T):
    lam = np.geomspace(0.01, 1e5, 4000)
    prob = _one_cell(lam)
    S = 3.7
    lum = oracle.dust_emission(prob, np.array([T]), S)
    mass = 2.0 * 1.5 ** 3
    expect = S * mass * 1.0 * (1 - 0.3) * math.pi ** 4 * T ** 4 / (15.0 * C2 ** 4)
    assert abs(lum.sum() - expect) <= 1e-4 * expect


def test_bin_widths_follow_the_logarithmic_grid(oracle):
    prob = _one_cell([1.0, 4.0])
    T = 500.0
    lum = oracle.dust_emission(prob, np.array([T]), 1.0)[:, 0]
    mass = 2.0 * 1.5 ** 3
    beta = lambda l: 1.0 / (l ** 5 * math.expm1(C2 / (l * T)))
    assert abs(lum[0] - mass * 0.7 * 1.5 * beta(1.0)) <= 1e-13 * lum[0]   # bin [0.5, 2]
    assert abs(lum[1] - mass * 0.7 * 6.0 * beta(4.0)) <= 1e-13 * lum[1]   # bin [2, 8]


@pytest.mark.parametrize("L_abs", [1e-6, 1.0, 1e4])
def test_grey_grain_temperature_and_balance(oracle, L_abs):
    lam = np.geomspace(0.01, 1e5, 4000)
    prob = _one_cell(lam)
    S = 1e8
    ab = np.zeros((len(lam), 1))
    ab[100, 0] = L_abs
    T, clamped = oracle.dust_temperature(prob, ab, S, t_min=0.1, t_max=1e5)
    assert clamped == 0
    mass = 2.0 * 1.5 ** 3
    closed = (15.0 * C2 ** 4 * L_abs / (S * mass * 0.7 * math.pi ** 4)) ** 0.25
    assert abs(T[0] - closed) <= 1e-4 * closed
    emitted = oracle.dust_emission(prob, T, S).sum()
    assert abs(emitted - L_abs) <= 1e-12 * L_abs


def test_empty_and_clamped_cells(oracle):
    prob = W.panchromatic_disk(n_cells=4, n_lambda=8)
    nc = prob.grid.n_cells
    dens = prob.grid.density.copy().ravel()
    dens[5] = 0.0
    prob = W.with_density(prob, dens.reshape(prob.grid.density.shape))
    ab = np.full((8, nc), 1e-3)
    ab[:, 7] = 0.0      # nothing absorbed
    ab[:, 9] = 1e30     # more than any cell emits at t_max
    ab[:, 11] = 1e-300  # less than it emits at t_min
    S = prob.meta["emission_scale"]
    T, clamped = oracle.dust_temperature(prob, ab, S, t_min=1.0, t_max=1e4)
    assert T[5] == 0.0 and T[7] == 0.0
    assert T[9] == 1e4 and T[11] == 1.0 and clamped == 2
    lum = oracle.dust_emission(prob, T, S)
    assert np.all(lum[:, 5] == 0.0) and np.all(lum[:, 7] == 0.0)
    free = np.setdiff1d(np.arange(nc), [5, 7, 9, 11])
    np.testing.assert_allclose(lum[:, free].sum(axis=0), ab[:, free].sum(axis=0), rtol=1e-12)


def _emitting(prob, lum, kappa=None):
    lum = np.asarray(lum, float).reshape(prob.n_lambda, prob.grid.n_cells)
    out = W.replace(prob, dust_lum=lum, sources=[])
    if kappa is not None:
        out = W.replace(out, kappa=np.full(prob.n_lambda, kappa))
    return out


def test_dust_packets_follow_the_cell_luminosities(oracle):
    """Two cells side by side, luminosities 3:1, no extinction: a frame that
    sees each cell in its own half receives 3/4 of the packets in the first
    half (binomial), and the total of L/(4 pi) per packet."""
    base = W.uniform_cube(n_cells=2, n_pix=2)
    grid = W.cartesian_grid([-1, 1, -0.5, 0.5, -0.5, 0.5], np.ones((1, 1, 2), np.float32))
    prob = W.replace(base, grid=grid, instruments=[W.Instrument(0.0, -math.pi / 2, 0.0, 2, 1, 1.0, 0.5)])
    prob = _emitting(prob, [[3.0, 1.0]], kappa=0.0)
    n = 40000
    r = oracle.run(prob, n, n_threads=4, counts=True)
    assert abs(r["stats"][0] - 4.0) <= 1e-12 * 4.0
    img, cnt = r["images"][0][0, 0, 0], r["image_counts"][0][0, 0, 0]
    assert cnt.sum() == n
    assert abs(img.sum() - 4.0 / (4 * math.pi)) <= 1e-12
    p = stats.binomtest(int(cnt[0]), n, 0.75).pvalue
    assert p > 1e-4


def test_dust_packet_positions_are_uniform_in_the_cell(oracle):
    base = W.uniform_cube(n_cells=1, n_pix=8)
    prob = _emitting(base, [[1.0]], kappa=0.0)
    n = 64000
    r = oracle.run(prob, n, n_threads=4, counts=True)
    cnt = r["image_counts"][0][0, 0].ravel()
    assert cnt.sum() == n
    chi2 = ((cnt - n / 64) ** 2 / (n / 64)).sum()
    assert stats.chi2.sf(chi2, 63) > 1e-4


def test_dust_emission_transport_conserves_and_skips_dark_wavelengths(oracle):
    prob = W.panchromatic_disk(n_cells=16, n_lambda=12, n_pix=16)
    r = oracle.run(prob, 3000, n_threads=4)
    S = prob.meta["emission_scale"]
    T, _ = oracle.dust_temperature(prob, r["absorption"], S)
    lum = oracle.dust_emission(prob, T, S)
    dusty = _emitting(prob, lum)
    n = 2000
    d = oracle.run(dusty, n, n_threads=4)
    emitted, escaped, absorbed, truncated = d["stats"]
    assert abs(emitted - lum.sum()) <= 1e-12 * lum.sum()
    assert abs(emitted - escaped - absorbed - truncated) <= 1e-12 * emitted
    dark = np.flatnonzero(lum.sum(axis=1) == 0.0)
    assert len(dark) > 0  # the ultraviolet end: 20 K dust emits nothing there
    assert d["counters"][3] == n * prob.n_lambda
    assert np.all(d["absorption"][dark] == 0.0)
    for im in d["images"]:
        assert np.all(im[:, dark] == 0.0)
