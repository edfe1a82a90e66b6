"""Pin of the oracle's multiple scattering against an analog Monte Carlo.

The oracle follows the paper's estimators (Sect. 1): forced scattering with
weights, continuous absorption and peel-off images.  An analog simulation of
the same medium, written here in numpy, uses none of them: each photon flies
an exponential free path, leaves the cube or interacts, is absorbed with
probability 1 - albedo or scattered with a Henyey-Greenstein angle, and is
counted where it escapes.  Both estimate the same expectations: the escaped
and absorbed fractions of the luminosity and the intensity leaving the cube
towards +z (the face-on frame, summed over its pixels).  The medium is thick
enough (optical depth 1 from the centre to a face) that several orders of
scattering contribute, so a dropped or misweighted order in the oracle shows.
"""
import math

import numpy as np

from paper_1410_1629_gb300 import workloads as W


def _analog_cube(n, kr, albedo, g, rng, cone_cos, half=1.0):
    """Analog photons from the centre of the cube [-half, half]^3 (extinction
    kr per unit length).  Returns (escaped, absorbed, escaped towards +z within
    the cone mu_z > cone_cos)."""
    mu = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(1.0 - mu * mu)
    k = np.stack([s * np.cos(phi), s * np.sin(phi), mu], axis=1)
    x = np.zeros((n, 3))
    escaped = absorbed = cone = 0
    while len(x):
        # distance to the boundary along k
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(k > 0, (half - x) / k, np.where(k < 0, (-half - x) / k, np.inf))
        t_exit = t.min(axis=1)
        path = -np.log(rng.uniform(0.0, 1.0, len(x)) + 1e-300) / kr
        out = path >= t_exit
        escaped += int(out.sum())
        cone += int((out & (k[:, 2] > cone_cos)).sum())
        stay = ~out
        x = x[stay] + path[stay, None] * k[stay]
        k = k[stay]
        scat = rng.uniform(0.0, 1.0, len(x)) < albedo
        absorbed += int((~scat).sum())
        x, k = x[scat], k[scat]
        if not len(x):
            break
        # Henyey-Greenstein polar angle (inverse of its cumulative distribution)
        u = rng.uniform(0.0, 1.0, len(x))
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
    return escaped, absorbed, cone


def test_multiple_scattering_matches_an_analog_simulation(oracle):
    kr, albedo, g = 1.0, 0.7, 0.5
    prob = W.uniform_cube(n_cells=16, axis_tau=2.0 * kr, albedo=albedo, g=g, n_pix=16)
    # oracle: K batches of packet ids give the standard error of each tally
    n_batches, per_batch = 24, 2000
    res = [oracle.run(prob, per_batch, first_id=b * per_batch, n_norm=n_batches * per_batch, n_threads=4,
                      absorption=False) for b in range(n_batches)]
    st = np.array([r["stats"] for r in res])          # emitted, escaped, absorbed, truncated per batch
    img = np.array([r["images"][0][0].sum() for r in res])
    sums = st.sum(axis=0)
    sig = math.sqrt(n_batches) * st.std(axis=0, ddof=1)
    i_o, i_sig = img.sum(), math.sqrt(n_batches) * img.std(ddof=1)
    assert sums[3] < 1e-3 * sums[0]                     # weight cut: little luminosity left over
    # analog photons, in chunks
    rng = np.random.default_rng(20141006)
    cone_cos = math.cos(math.radians(5.0))
    n_chunk, n_chunks = 1_000_000, 12
    esc = ab = cone = 0
    for _ in range(n_chunks):
        e, a, c = _analog_cube(n_chunk, kr, albedo, g, rng, cone_cos)
        esc, ab, cone = esc + e, ab + a, cone + c
    n = n_chunk * n_chunks
    f_esc, f_abs = esc / n, ab / n
    omega = 2.0 * math.pi * (1.0 - cone_cos)
    i_a = cone / n / omega
    s_esc = math.sqrt(f_esc * (1 - f_esc) / n)
    s_i = math.sqrt(cone) / n / omega
    tol_esc = 4.0 * math.hypot(s_esc, sig[1] / sums[0]) + sums[3] / sums[0]
    assert abs(sums[1] / sums[0] - f_esc) < tol_esc, (sums[1] / sums[0], f_esc, tol_esc)
    assert abs(sums[2] / sums[0] - f_abs) < 4.0 * math.hypot(s_esc, sig[2] / sums[0]) + sums[3] / sums[0]
    # intensity towards +z: the cone average departs from the intensity on the
    # axis by about kr (5 deg)^2 / 4 = 0.2 % in the direct light
    assert abs(i_o - i_a) < 4.0 * math.hypot(s_i, i_sig) + 0.003 * i_a, (i_o, i_a, s_i, i_sig)
    # the comparison resolves the scattered light: more than a quarter of the
    # intensity is scattered, and the tolerance is below a tenth of it
    direct = math.exp(-kr) / (4.0 * math.pi)
    assert i_o - direct > 0.25 * i_o
    assert 4.0 * math.hypot(s_i, i_sig) < 0.1 * (i_o - direct)
