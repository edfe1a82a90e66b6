"""Pins for emission sampling (Sect. 3.4: a source geometry draws positions from
its density; Table 1(a) lists point, exponential-disk and Plummer geometries)."""
import math

import numpy as np
from scipy import stats

from conftest import golden
from paper_1410_1629_gb300 import workloads as W

N = 6000


def _emit_many(oracle, prob, lam=0, n=N):
    xs, ks = [], []
    for p in range(n):
        x, k = oracle.emit(prob, p, lam)
        xs.append(x)
        ks.append(k)
    return np.array(xs), np.array(ks)


def test_point_source_isotropic(oracle):
    prob = W.uniform_cube(source_pos=(0.25, -0.5, 0.125))
    x, k = _emit_many(oracle, prob)
    assert np.all(x == np.array([0.25, -0.5, 0.125]))
    np.testing.assert_allclose(np.linalg.norm(k, axis=1), 1.0, atol=1e-14)
    # isotropy: each cosine is uniform on [-1, 1]
    for a in range(3):
        assert stats.kstest(k[:, a], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3


def test_exponential_disk_of_the_paper_example(oracle):
    """Stellar disk of the paper's example (hR = 4400 pc, hz = 500 pc): R has
    density R exp(-R/hR), |z| is exponential with scale hz, the azimuth is uniform."""
    G = golden("spiral_example.txt")
    hR, hz = float(G["star_radial_scale_pc"]), float(G["star_axial_scale_pc"])
    prob = W.uniform_cube()
    prob.sources = [W.Source("expdisk", (100.0, -50.0, 20.0), np.ones(1), scale_r=hR, scale_z=hz)]
    x, _ = _emit_many(oracle, prob)
    d = x - np.array([100.0, -50.0, 20.0])
    R = np.hypot(d[:, 0], d[:, 1])
    assert stats.kstest(R / hR, stats.gamma(2).cdf).pvalue > 1e-3
    assert stats.kstest(np.abs(d[:, 2]) / hz, stats.expon.cdf).pvalue > 1e-3
    assert stats.kstest(np.arctan2(d[:, 1], d[:, 0]), stats.uniform(loc=-math.pi, scale=2 * math.pi).cdf).pvalue > 1e-3
    assert abs(np.mean(d[:, 2] > 0) - 0.5) < 4 * 0.5 / math.sqrt(N)


def test_plummer_sphere(oracle):
    a = 1.5
    prob = W.uniform_cube()
    prob.sources = [W.Source("plummer", (0.0, 0.0, 0.0), np.ones(1), scale_r=a)]
    x, _ = _emit_many(oracle, prob)
    r = np.linalg.norm(x, axis=1)
    # enclosed mass fraction M(<r) = r^3 / (r^2 + a^2)^(3/2)
    assert stats.kstest(r, lambda s: s ** 3 / (s * s + a * a) ** 1.5).pvalue > 1e-3
    assert stats.kstest(x[:, 2] / r, stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3


def test_component_choice_follows_luminosity(oracle):
    prob = W.uniform_cube()
    prob.kappa = np.array([0.5, 0.5])
    prob.albedo = np.array([0.5, 0.5])
    prob.g = np.array([0.0, 0.0])
    prob.sources = [W.Source("point", (-0.5, 0, 0), np.array([1.0, 3.0])),
                    W.Source("point", (0.5, 0, 0), np.array([3.0, 1.0]))]
    for lam, p_first in [(0, 0.25), (1, 0.75)]:
        x, _ = _emit_many(oracle, prob, lam=lam, n=4000)
        frac = np.mean(x[:, 0] < 0)
        assert abs(frac - p_first) < 4 * math.sqrt(p_first * (1 - p_first) / 4000)
