"""Pins for the oracle's packet transport: conservation, closed forms,
quadratures of the expected tallies, special cases, symmetry and scale
invariance, and the dual-number gradient against central finite differences.

Monte Carlo comparisons use the batch method: a run of K packet-id batches
gives K independent estimates whose scatter measures the standard error.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_1410_1629_gb300 import workloads as W

FOUR_PI = 4.0 * math.pi


def _conservation(stats):
    emitted, escaped, absorbed, truncated = stats
    return abs(emitted - escaped - absorbed - truncated) / emitted


def _batches(oracle, prob, n_batches, per_batch, **kw):
    """Run K batches of packet ids with a common normalisation; return the list of results."""
    out = []
    for b in range(n_batches):
        out.append(oracle.run(prob, per_batch, first_id=b * per_batch, n_norm=n_batches * per_batch,
                              n_threads=4, **kw))
    return out


def _sum_and_sigma(values):
    v = np.asarray(values, dtype=np.float64)
    k = v.shape[0]
    return v.sum(axis=0), np.sqrt(k) * v.std(axis=0, ddof=1)


# ---------------------------------------------------------------- conservation
@pytest.mark.parametrize("which", ["cube", "cube_thick", "disk", "octree", "no_scatter"])
def test_luminosity_is_conserved(oracle, which):
    if which == "cube":
        prob, n = W.uniform_cube(), 3000
    elif which == "cube_thick":
        prob, n = W.uniform_cube(axis_tau=20.0, albedo=0.9, g=-0.3), 1000
    elif which == "disk":
        prob, n = W.disk_galaxy(n_cells=32, n_lambda=3, n_pix=32), 500
    elif which == "octree":
        rng = np.random.default_rng(2)
        grid, _, _ = W.build_octree([-1, 1] * 3, lambda lo, hi, l: rng.uniform(size=len(lo)) < 0.6,
                                    lambda lo, hi: rng.uniform(0.0, 2.0, len(lo)), 4)
        prob = W.uniform_cube()
        prob.grid = grid
        n = 2000
    else:
        prob, n = W.uniform_cube(albedo=0.0), 3000
    r = oracle.run(prob, n, n_threads=4)
    assert _conservation(r["stats"]) < 1e-12
    assert abs(r["absorption"].sum() - r["stats"][2]) <= 1e-12 * r["stats"][0]


# ---------------------------------------------------------------- emission peel-off
def test_direct_image_of_central_source_is_exact(oracle):
    """Face-on view of the central source: only pixel (32, 32) receives direct
    light, N * (L0/4pi) exp(-0.5) = exp(-0.5)/(4 pi) (centre-to-face tau 0.5)."""
    prob = W.uniform_cube(channels=3)
    r = oracle.run(prob, 2000, n_threads=2)
    direct = r["images"][0][1, 0]
    expect = math.exp(-0.5) / FOUR_PI
    assert abs(direct[32, 32] - expect) < 1e-12 * expect
    direct[32, 32] = 0.0
    assert np.all(direct == 0.0)


def test_direct_image_of_offset_source(oracle):
    """Source at (0.3, -0.5, 0.2): pixel (ix, iy) = (floor(1.3 * 32), floor(0.5 * 32))
    = (41, 16); the path to the top face is 0.8 long, tau = 0.5 * 0.8."""
    prob = W.uniform_cube(channels=3, source_pos=(0.3, -0.5, 0.2))
    r = oracle.run(prob, 500)
    direct = r["images"][0][1, 0]
    expect = math.exp(-0.4) / FOUR_PI
    assert abs(direct[16, 41] - expect) < 1e-12 * expect
    assert np.count_nonzero(direct) == 1


# ---------------------------------------------------------------- quadratures
def _face_quadrature(f):
    """(1/4pi) * integral over directions from the cube centre of f(d, kz, r), with
    the unit cube [-1, 1]^3 boundary at distance r along each direction."""
    def integrand(v, u):
        r = math.sqrt(u * u + v * v + 1.0)
        return (f(1.0 / r, r) + f(-1.0 / r, r) + 4.0 * f(v / r, r)) / r ** 3
    val, _ = integrate.dblquad(integrand, -1, 1, -1, 1, epsabs=1e-13, epsrel=1e-11)
    return val / FOUR_PI


def test_first_step_escape_matches_quadrature(oracle):
    """Escaped luminosity after the first forced step: E[L0 exp(-tau(k))] over
    isotropic directions from the centre of a cube with kappa rho = 0.5."""
    kr = 0.5
    m1 = _face_quadrature(lambda kz, r: math.exp(-kr * r))
    prob = W.uniform_cube()
    res = _batches(oracle, prob, 32, 1000, max_events=1, absorption=False)
    esc, sig = _sum_and_sigma([r["stats"][1] for r in res])
    assert abs(esc - m1) < 4 * sig
    assert sig < 2e-3


def test_no_scattering_case(oracle):
    """Albedo 0: no scattered light at all; the absorbed luminosity is
    1 - E[exp(-tau)] per unit emitted."""
    kr = 0.5
    m1 = _face_quadrature(lambda kz, r: math.exp(-kr * r))
    prob = W.uniform_cube(albedo=0.0, channels=3)
    res = _batches(oracle, prob, 32, 1000)
    for r in res:
        assert np.all(r["images"][0][2] == 0.0)
        assert r["stats"][3] == 0.0
        assert _conservation(r["stats"]) < 1e-12
    ab, sig = _sum_and_sigma([r["stats"][2] for r in res])
    assert abs(ab - (1 - m1)) < 4 * sig


def test_absorption_field_without_scattering_matches_quadrature(oracle):
    """Albedo 0 on an 8^3 grid: the expected absorption in a cell is the
    integral over the cell of kappa rho exp(-kappa rho r) / (4 pi r^2).  Cells
    are folded over the 8 octants; the cell touching the source is skipped."""
    kr = 0.5
    prob = W.uniform_cube(n_cells=8, albedo=0.0)
    res = _batches(oracle, prob, 32, 2000, peel_emission=False, peel_scatter=False)
    fold = []
    for r in res:
        a = r["absorption"][0].reshape(8, 8, 8)
        f = np.zeros((4, 4, 4))
        for sx in (slice(4, 8), slice(3, None, -1)):
            for sy in (slice(4, 8), slice(3, None, -1)):
                for sz in (slice(4, 8), slice(3, None, -1)):
                    f += a[sz, sy, sx]
        fold.append(f)
    tot, sig = _sum_and_sigma(fold)
    xg, wg = np.polynomial.legendre.leggauss(12)
    z = []
    for iz in range(4):
        for iy in range(4):
            for ix in range(4):
                if ix == iy == iz == 0:
                    continue
                lo = np.array([ix, iy, iz]) * 0.25
                p = [lo[a] + 0.125 * (xg + 1) for a in range(3)]
                X, Y, Z = np.meshgrid(p[0], p[1], p[2], indexing="ij")
                Wt = wg[:, None, None] * wg[None, :, None] * wg[None, None, :] * 0.125 ** 3
                R2 = X * X + Y * Y + Z * Z
                val = 8.0 * np.sum(Wt * kr * np.exp(-kr * np.sqrt(R2)) / (FOUR_PI * R2))
                z.append((tot[iz, iy, ix] - val) / sig[iz, iy, ix])
    z = np.array(z)
    assert np.max(np.abs(z)) < 5.0
    assert np.mean(z * z) < 2.0


@pytest.mark.parametrize("axis_tau", [1.0, 0.02])
def test_single_scattering_flux_matches_quadrature(oracle, axis_tau):
    """Total scattered light on the face-on frame after one forced scattering:
    (albedo kappa rho / 4 pi) * E_k[ Phi(k_z) int_0^d exp(-kr s) exp(-kr (1 - s k_z)) ds ]."""
    kr, albedo, g = axis_tau / 2.0, 0.6, 0.5
    prob = W.uniform_cube(axis_tau=axis_tau, albedo=albedo, g=g, channels=3)

    def f(kz, r):
        a = kr * (1.0 - kz)
        inner = r if a * r < 1e-12 else -math.expm1(-a * r) / a
        phi = (1 - g * g) / (1 + g * g - 2 * g * kz) ** 1.5
        return phi * math.exp(-kr) * inner

    expect = albedo * kr / FOUR_PI * _face_quadrature(f)
    res = _batches(oracle, prob, 32, 1000, max_events=1, absorption=False)
    sca, sig = _sum_and_sigma([r["images"][0][2].sum() for r in res])
    assert abs(sca - expect) < 4 * sig
    assert sig < 0.02 * expect


# ---------------------------------------------------------------- special cases
def test_dust_free_medium(oracle):
    prob = W.uniform_cube(rho=0.0, channels=3)
    r = oracle.run(prob, 1000)
    emitted, escaped, absorbed, truncated = r["stats"]
    assert escaped == emitted and absorbed == 0.0 and truncated == 0.0
    assert int(r["counters"][1]) == 0
    img = r["images"][0]
    assert abs(img[0, 0, 32, 32] - 1 / FOUR_PI) < 1e-12
    assert np.count_nonzero(img[0]) == 1 and np.all(img[2] == 0)


def test_face_on_image_has_the_symmetry_of_the_square(oracle):
    prob = W.uniform_cube(channels=3)
    res = _batches(oracle, prob, 16, 1500, absorption=False)
    imgs = np.array([r["images"][0][2, 0].reshape(8, 8, 8, 8).sum(axis=(1, 3)) for r in res])
    for T in (lambda a: a.T, lambda a: a[::-1], lambda a: a[:, ::-1], lambda a: np.rot90(a)):
        d = np.array([im - T(im) for im in imgs])
        tot, sig = _sum_and_sigma(d)
        mask = sig > 0
        z = tot[mask] / sig[mask]
        assert np.max(np.abs(z)) < 5.0
        assert np.mean(z * z) < 2.0


def test_scale_invariance_is_exact(oracle):
    """Lengths x 4 and kappa / 4 leave every tally bitwise unchanged."""
    a = W.uniform_cube(channels=3, source_pos=(0.25, -0.125, 0.5))
    b = W.uniform_cube(channels=3, source_pos=(1.0, -0.5, 2.0), half=4.0)
    assert b.kappa[0] == a.kappa[0] / 4
    ra = oracle.run(a, 1500)
    rb = oracle.run(b, 1500)
    np.testing.assert_array_equal(ra["images"][0], rb["images"][0])
    np.testing.assert_array_equal(ra["absorption"], rb["absorption"])
    np.testing.assert_array_equal(ra["stats"], rb["stats"])
    np.testing.assert_array_equal(ra["counters"], rb["counters"])


def test_full_octree_transport_equals_cartesian(oracle):
    """An octree refined uniformly to level 5 is the 32^3 cube: same images,
    same absorption per cell (leaf order mapped to cell order)."""
    cart = W.uniform_cube(channels=3)
    grid, llo, lhi = W.build_octree([-1, 1] * 3, lambda lo, hi, l: np.ones(len(lo), bool),
                                    lambda lo, hi: np.ones(len(lo)), 5)
    octp = W.uniform_cube(channels=3)
    octp.grid = grid
    rc = oracle.run(cart, 800)
    ro = oracle.run(octp, 800)
    np.testing.assert_allclose(ro["images"][0], rc["images"][0], rtol=1e-12, atol=1e-18)
    idx = np.floor((0.5 * (llo + lhi) + 1.0) * 16).astype(int)
    cell = idx[:, 0] + 32 * (idx[:, 1] + 32 * idx[:, 2])
    np.testing.assert_allclose(ro["absorption"][0], rc["absorption"][0][cell], rtol=1e-12, atol=1e-18)


# ---------------------------------------------------------------- gradient
def test_dual_gradient_matches_central_differences(oracle):
    """Pathwise derivative of a linear functional of the image and the absorption
    field (bilinear deposit, termination by event count) against central
    differences of the FP64 forward run under common random numbers."""
    prob = W.lognormal_cube(n_cells=4, n_pix=8, n_packets=300, max_events=5)
    rng = np.random.default_rng(0)
    adj_img = rng.standard_normal((1, 1, 8, 8))
    adj_abs = rng.standard_normal((1, 64))
    kw = dict(max_events=5, weight_cut=False)

    def loss(p):
        r = oracle.run(p, 300, **kw)
        return float((adj_img * r["images"][0]).sum() + (adj_abs * r["absorption"]).sum())

    cells = np.array([0, 21, 42, 63, 5])
    grad = oracle.vjp(prob, cells, 300, adj_images=[adj_img], adj_absorption=adj_abs, n_threads=4, **kw)
    rho = prob.grid.density.ravel().copy()
    for c, gval in zip(cells, grad):
        up, dn = rho.copy(), rho.copy()
        up[c] = np.float32(rho[c] * (1 + 1e-4))
        dn[c] = np.float32(rho[c] * (1 - 1e-4))
        h = float(up[c]) - float(dn[c])
        fd = (loss(W.with_density(prob, up.reshape(4, 4, 4))) - loss(W.with_density(prob, dn.reshape(4, 4, 4)))) / h
        assert abs(fd - gval) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max())
