"""Pins for the oracle's phase function, direction rotation and frame geometry."""
import math

import numpy as np
import pytest
from scipy import integrate

from conftest import golden
from paper_1410_1629_gb300 import workloads as W


@pytest.mark.parametrize("g", [-0.7, -0.2, 0.0, 0.3, 0.5, 0.9, 0.99])
def test_hg_phase_normalised(oracle, g):
    # mean of Phi over the sphere is 1: (1/2) int_{-1}^{1} Phi(mu) dmu = 1
    val, _ = integrate.quad(lambda mu: oracle.hg_phase(g, mu), -1.0, 1.0, epsabs=1e-14, epsrel=1e-13,
                            limit=200)
    assert abs(0.5 * val - 1.0) < 1e-11


@pytest.mark.parametrize("g", [0.5, 0.6, -0.4, 0.9])
def test_hg_sample_mean_cosine_equals_g(oracle, g):
    # E[mu] = g and E[mu^2] = (1 + 2 g^2)/3, by quadrature of the sampler over u
    m1, _ = integrate.quad(lambda u: oracle.hg_sample(g, u), 0.0, 1.0, epsabs=1e-14, limit=400)
    m2, _ = integrate.quad(lambda u: oracle.hg_sample(g, u) ** 2, 0.0, 1.0, epsabs=1e-14, limit=400)
    assert abs(m1 - g) < 1e-10
    assert abs(m2 - (1 + 2 * g * g) / 3) < 1e-10


@pytest.mark.parametrize("g", [0.5, -0.3, 0.85])
def test_hg_sample_inverts_the_cdf(oracle, g):
    # the sampled cosine is the u-quantile of the distribution Phi(mu)/2 on [-1, 1]
    for u in [1e-6, 0.01, 0.2, 0.5, 0.77, 0.999]:
        mu = oracle.hg_sample(g, u)
        cdf, _ = integrate.quad(lambda m: 0.5 * oracle.hg_phase(g, m), -1.0, mu, epsabs=1e-14, limit=200)
        assert abs(cdf - u) < 1e-10


def test_hg_isotropic_branch(oracle):
    for u in [0.1, 0.5, 0.9]:
        assert oracle.hg_sample(0.0, u) == 2 * u - 1
        assert oracle.hg_phase(0.0, 0.3) == 1.0


def _random_dirs(n, rng):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_rotation_angle_and_azimuth(oracle):
    rng = np.random.default_rng(3)
    ks = list(_random_dirs(200, rng)) + [np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -1.0]),
                                         np.array([1e-9, 0.0, math.sqrt(1 - 1e-18)]),
                                         np.array([1.0, 0.0, 0.0])]
    for k in ks:
        mu = rng.uniform(-1, 1)
        p1, p2 = rng.uniform(0, 2 * math.pi, 2)
        a = oracle.rotate(k, mu, p1)
        b = oracle.rotate(k, mu, p2)
        assert abs(np.linalg.norm(a) - 1) < 1e-14
        assert abs(a @ k - mu) < 1e-12
        # the azimuth difference is the angle between the components normal to k
        pa, pb = a - (a @ k) * k, b - (b @ k) * k
        if np.linalg.norm(pa) > 1e-6:
            cosd = pa @ pb / (np.linalg.norm(pa) * np.linalg.norm(pb))
            assert abs(cosd - math.cos(p1 - p2)) < 1e-9
            # turning by +phi is a right-handed rotation about k
            sind = np.cross(pa, pb) @ k / (np.linalg.norm(pa) * np.linalg.norm(pb))
            assert abs(sind - math.sin(p2 - p1)) < 1e-9


def test_frame_orthonormal_right_handed(oracle):
    rng = np.random.default_rng(5)
    for _ in range(50):
        q = W.Instrument(rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi), rng.uniform(-3, 3),
                         8, 8, 1.0, 1.0)
        kobs, ex, ey = oracle.frame(q)
        M = np.stack([ex, ey, kobs])
        np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-14)
        np.testing.assert_allclose(np.cross(ex, ey), kobs, atol=1e-14)


def test_frame_of_the_paper_example_is_the_xz_plane(oracle):
    """The paper's example frame, named "xz", has inclination 90 deg and
    azimuth -90 deg: image x runs along model x, image y along model z, and the
    observer looks from -y."""
    G = golden("spiral_example.txt")
    assert G["instrument_name"] == "xz"
    q = W.Instrument(math.radians(float(G["inclination_deg"])), math.radians(float(G["azimuth_deg"])),
                     math.radians(float(G["position_angle_deg"])), int(G["pixels_x"]), int(G["pixels_y"]),
                     float(G["extent_x_pc"]), float(G["extent_y_pc"]))
    kobs, ex, ey = oracle.frame(q)
    # exactly: the angles are multiples of pi/2, whose sines and cosines are
    # taken exact, so the observer looks exactly along -y
    assert list(ex) == [1, 0, 0] and list(ey) == [0, 0, 1] and list(kobs) == [0, -1, 0]


def test_face_on_frame_and_position_angle(oracle):
    kobs, ex, ey = oracle.frame(W.face_on(8, 1.0))
    assert list(kobs) == [0, 0, 1] and list(ex) == [1, 0, 0] and list(ey) == [0, 1, 0]
    # a position angle of 90 degrees turns image content counter-clockwise by 90 degrees:
    # the model +x axis then appears along image +y
    q = W.Instrument(0.0, -math.pi / 2, math.pi / 2, 8, 8, 1.0, 1.0)
    kobs, ex, ey = oracle.frame(q)
    np.testing.assert_allclose(np.array([1, 0, 0]) @ ey, 1.0, atol=1e-15)
    np.testing.assert_allclose(np.array([0, 1, 0]) @ ex, -1.0, atol=1e-15)


@pytest.mark.parametrize("g", [0.5, -0.3, 0.0])
def test_scattering_direction_mean_is_g_times_k(oracle, g):
    """Over the HG cosine and a uniform azimuth the mean new direction is g k:
    the azimuth average (midpoint rule, exact for the first harmonics) removes
    the transverse part and the cosine average is g."""
    k = np.array([0.36, -0.48, 0.8])
    n_az = 16
    u1 = (np.arange(2000) + 0.5) / 2000
    mean = np.zeros(3)
    for a in range(n_az):
        u2 = (a + 0.5) / n_az
        mean += np.mean([oracle.scatter_direction(k, g, x, u2) for x in u1], axis=0)
    mean /= n_az
    m_mu = np.mean([oracle.hg_sample(g, x) for x in u1])
    np.testing.assert_allclose(mean, m_mu * k, atol=1e-12)
    assert abs(m_mu - g) < 1e-5
