"""Pin of the oracle's multiple scattering against an analog Monte Carlo.

The oracle follows the paper's estimators (Sect. 1): forced scattering with
weights, continuous absorption and peel-off images.  An analog simulation of
the same medium, written here in numpy, uses none of them: each photon flies
an exponential free path, leaves the cube or interacts, is absorbed with
probability 1 - albedo or scattered with a Henyey-Greenstein angle, and is
counted where it escapes or is absorbed.  Both estimate the same
expectations: the escaped and absorbed fractions of the luminosity, the
intensity leaving the cube towards +z (the face-on frame), where on the frame
it comes from, and where in the cube luminosity is absorbed.  The medium is
thick enough (optical depth 1 from the centre to a face) that several orders
of scattering contribute, so a dropped or misweighted order, or light put in
the wrong place, in the oracle shows.
"""
import functools
import math

import numpy as np
import pytest

from paper_1410_1629_gb300 import workloads as W

# (extinction per unit length, albedo, g): optical depth 1 from the centre to
# a face with forward scattering, and 3 with isotropic scattering and a high
# albedo (many orders of scattering)
CASES = {"tau1": (1.0, 0.7, 0.5), "tau3": (3.0, 0.9, 0.0)}
CONE_COS = math.cos(math.radians(5.0))
NB = 4  # blocks per axis for the spatial comparisons


def _blocks(v):
    """Block index along an axis of [-1, 1] in NB blocks."""
    return np.clip(np.floor((v + 1.0) * 0.5 * NB).astype(np.int64), 0, NB - 1)


def _analog_cube(n, rng, kr, albedo, g, half=1.0):
    """Analog photons from the centre of the cube [-half, half]^3.  Returns
    (escaped, absorbed, photons escaping towards +z within the cone per image
    block of their last interaction point [NB, NB] (y, x), absorbed photons per
    cube block [NB, NB, NB] (z, y, x))."""
    mu = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(1.0 - mu * mu)
    k = np.stack([s * np.cos(phi), s * np.sin(phi), mu], axis=1)
    x = np.zeros((n, 3))
    escaped = absorbed = 0
    img = np.zeros((NB, NB))
    ab = np.zeros((NB, NB, NB))
    while len(x):
        # distance to the boundary along k
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(k > 0, (half - x) / k, np.where(k < 0, (-half - x) / k, np.inf))
        t_exit = t.min(axis=1)
        path = -np.log(rng.uniform(0.0, 1.0, len(x)) + 1e-300) / kr
        out = path >= t_exit
        escaped += int(out.sum())
        toward = out & (k[:, 2] > CONE_COS)
        np.add.at(img, (_blocks(x[toward, 1]), _blocks(x[toward, 0])), 1.0)
        stay = ~out
        x = x[stay] + path[stay, None] * k[stay]
        k = k[stay]
        scat = rng.uniform(0.0, 1.0, len(x)) < albedo
        gone = x[~scat]
        absorbed += len(gone)
        np.add.at(ab, (_blocks(gone[:, 2]), _blocks(gone[:, 1]), _blocks(gone[:, 0])), 1.0)
        x, k = x[scat], k[scat]
        if not len(x):
            break
        # Henyey-Greenstein polar angle (inverse of its cumulative distribution)
        u = rng.uniform(0.0, 1.0, len(x))
        if g == 0.0:
            ct = 2.0 * u - 1.0
        else:
            ct = (1.0 + g * g - ((1.0 - g * g) / (1.0 - g + 2.0 * g * u)) ** 2) / (2.0 * g)
        ct = np.clip(ct, -1.0, 1.0)
        st = np.sqrt(1.0 - ct * ct)
        ph = rng.uniform(0.0, 2.0 * math.pi, len(x))
        # an orthonormal pair perpendicular to k
        a = np.where(np.abs(k[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
        e1 = np.cross(k, a)
        e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
        e2 = np.cross(k, e1)
        k = ct[:, None] * k + st[:, None] * (np.cos(ph)[:, None] * e1 + np.sin(ph)[:, None] * e2)
    return escaped, absorbed, img, ab


@functools.lru_cache(maxsize=None)
def _analog(case):
    kr, albedo, g = CASES[case]
    rng = np.random.default_rng(20141006)
    n_chunk, n_chunks = 1_000_000, 12
    esc = absd = 0
    img = np.zeros((NB, NB))
    ab = np.zeros((NB, NB, NB))
    for _ in range(n_chunks):
        e, a, i, b = _analog_cube(n_chunk, rng, kr, albedo, g)
        esc, absd, img, ab = esc + e, absd + a, img + i, ab + b
    return n_chunk * n_chunks, esc, absd, img, ab


@pytest.fixture(scope="module", params=sorted(CASES))
def runs(oracle, request):
    """Oracle: K batches of packet ids, each an independent estimate."""
    kr, albedo, g = CASES[request.param]
    prob = W.uniform_cube(n_cells=16, axis_tau=2.0 * kr, albedo=albedo, g=g, n_pix=16)
    n_batches, per_batch = 24, 2000
    res = [oracle.run(prob, per_batch, first_id=b * per_batch, n_norm=n_batches * per_batch, n_threads=4)
           for b in range(n_batches)]
    return res, n_batches, request.param


def _sum_sigma(values, k):
    v = np.asarray(values, dtype=np.float64)
    return v.sum(axis=0), math.sqrt(k) * v.std(axis=0, ddof=1)


def test_escape_absorption_and_intensity_match_an_analog_simulation(runs):
    res, nb, case = runs
    kr = CASES[case][0]
    st, sig = _sum_sigma([r["stats"] for r in res], nb)  # emitted, escaped, absorbed, truncated
    i_o, i_sig = _sum_sigma([r["images"][0][0].sum() for r in res], nb)
    assert st[3] < 1e-3 * st[0]  # weight cut: little luminosity left over
    n, esc, absd, img, _ = _analog(case)
    f_esc, f_abs = esc / n, absd / n
    s_f = math.sqrt(f_esc * (1 - f_esc) / n)
    omega = 2.0 * math.pi * (1.0 - CONE_COS)
    i_a = img.sum() / n / omega
    s_i = math.sqrt(img.sum()) / n / omega
    assert abs(st[1] / st[0] - f_esc) < 4.0 * math.hypot(s_f, sig[1] / st[0]) + st[3] / st[0]
    assert abs(st[2] / st[0] - f_abs) < 4.0 * math.hypot(s_f, sig[2] / st[0]) + st[3] / st[0]
    # intensity towards +z: the cone average departs from the intensity on the
    # axis by about kr (5 deg)^2 / 4 = 0.2 % in the direct light
    assert abs(i_o - i_a) < 4.0 * math.hypot(s_i, i_sig) + 0.003 * i_a, (i_o, i_a, s_i, i_sig)
    # the comparison resolves the scattered light: more than a quarter of the
    # intensity is scattered, and the tolerance is below a tenth of it
    direct = math.exp(-kr) / (4.0 * math.pi)
    assert i_o - direct > 0.25 * i_o
    assert 4.0 * math.hypot(s_i, i_sig) < 0.1 * (i_o - direct)


def test_where_light_goes_matches_an_analog_simulation(runs):
    """Blocks of the face-on image (4 x 4 of 16^2 pixels) and of the absorption
    field (4 x 4 x 4 of 16^3 cells): the image per block against analog
    photons escaping in the cone, binned by their last interaction point (the
    point a peel-off projects); absorbed luminosity per block against analog
    absorptions there.  Only the image's inner 2 x 2 blocks are compared one
    by one: near the side faces the cone average over-weights directions that
    leave through a side face (less medium on the way) than the exact +z ray a
    peel-off follows (the border blocks still count in the total intensity)."""
    res, nb, case = runs
    m = 16 // NB
    imgs = [r["images"][0][0, 0].reshape(NB, m, NB, m).sum(axis=(1, 3)) for r in res]
    abss = [r["absorption"][0].reshape(NB, m, NB, m, NB, m).sum(axis=(1, 3, 5)) for r in res]
    emitted = sum(r["stats"][0] for r in res)
    i_o, i_sig = _sum_sigma(imgs, nb)
    a_o, a_sig = _sum_sigma(abss, nb)
    n, _, _, img, ab = _analog(case)
    omega = 2.0 * math.pi * (1.0 - CONE_COS)
    i_a, i_asig = img / n / omega, np.sqrt(img) / n / omega
    a_a, a_asig = ab / n * emitted, np.sqrt(ab) / n * emitted
    inner = (slice(1, 3), slice(1, 3))
    zi = np.abs(i_o - i_a)[inner] / np.hypot(i_sig, i_asig)[inner]
    za = np.abs(a_o - a_a) / np.hypot(a_sig, a_asig)
    assert np.all(zi < 4.5), zi.max()
    assert np.all(za < 4.5), za.max()  # 64 blocks
    # the blocks resolve the layout: the centre-to-corner contrasts are many
    # standard errors
    assert i_o[1:3, 1:3].mean() > 5.0 * i_o[0, 0] and i_o[0, 0] > 20.0 * i_sig[0, 0]
    assert a_o[1:3, 1:3, 1:3].mean() > 3.0 * a_o[0, 0, 0] and a_o[0, 0, 0] > 10.0 * a_sig[0, 0, 0]
