"""Pins for the oracle's SED instrument (Sect. 2.2: the spectral energy
distribution of the flux received from a viewing direction, with direct and
scattered light recorded separately).  CPU only.

* Without dust every packet's only contribution is its emission peel-off,
  L0 / (4 pi) with nothing in the way: the SED is L_tot / (4 pi) per
  wavelength from any direction, all of it direct.
* Without scattering (albedo 0) a central point source seen along a grid
  axis of a uniform cube is dimmed by exactly exp(-tau) of the half-axis.
* The SED is a frame without a field of view: it equals the sum over all
  pixels of a frame that sees every peel-off position, per wavelength and
  channel, whatever the inclination.
"""
import math

import numpy as np
import pytest

from paper_1410_1629_gb300 import workloads as W

FOUR_PI = 4.0 * math.pi


def _with(prob, instruments):
    from dataclasses import replace
    return replace(prob, instruments=instruments)


@pytest.mark.parametrize("inc", [0.0, 33.0, 90.0])
def test_dust_free_sed_is_the_total_luminosity(oracle, inc):
    prob = _with(W.disk_galaxy(n_cells=16, n_lambda=3, n_pix=16, face_on_tau_v=0.0), [W.sed_instrument(inc)])
    n = 2000
    r = oracle.run(prob, n, n_threads=4)
    sed = r["images"][0][:, :, 0, 0]  # [channel, lambda]
    np.testing.assert_allclose(sed[0], np.ones(3) / FOUR_PI, rtol=1e-12)
    np.testing.assert_array_equal(sed[1], sed[0])
    assert np.all(sed[2] == 0.0)


def test_albedo_zero_point_source_is_dimmed_by_the_half_axis(oracle):
    prob = _with(W.uniform_cube(albedo=0.0, axis_tau=1.0), [W.sed_instrument(0.0), W.sed_instrument(90.0)])
    n = 3000
    r = oracle.run(prob, n, n_threads=4)
    for q in range(2):
        sed = r["images"][q][:, 0, 0, 0]
        assert abs(sed[1] - math.exp(-0.5) / FOUR_PI) <= 1e-12 * sed[1]
        assert sed[2] == 0.0 and abs(sed[0] - sed[1]) <= 1e-15 * sed[0]


@pytest.mark.parametrize("inc", [0.0, 41.0, 90.0])
def test_sed_equals_the_sum_of_an_enclosing_frame(oracle, inc):
    """Disk galaxy (several wavelengths, multiple scattering): a 300 kpc
    half-width frame sees every emission and scattering position (the disk's
    emission radius is below 200 kpc for any uniform of the generator)."""
    base = W.disk_galaxy(n_cells=24, n_lambda=3, n_pix=16)
    frame = W.Instrument(math.radians(inc), -math.pi / 2, 0.3, 16, 16, 300.0, 300.0, channels=3)
    prob = _with(base, [W.sed_instrument(inc), frame])
    n = 3000
    r = oracle.run(prob, n, n_threads=4)
    sed = r["images"][0][:, :, 0, 0]
    total = r["images"][1].sum(axis=(2, 3))
    np.testing.assert_allclose(sed, total, rtol=1e-12)
    assert np.all(sed[2] > 0) and np.all(sed[1] > 0)
    np.testing.assert_allclose(sed[0], sed[1] + sed[2], rtol=1e-12)
