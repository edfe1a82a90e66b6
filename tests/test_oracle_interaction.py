"""Pins for the oracle's forced-scattering interaction (steps a and c of the
per-packet algorithm): the inverted optical depth, the rounding fallback at
the top end of the uniform, and the move of the interaction point into its
cell.

In a uniform medium the inversion has a closed form: from x along k the path
to the boundary has length D and optical depth kappa rho D, the drawn depth is
tau* = -ln(1 - u (1 - exp(-kappa rho D))) and the interaction lies at
s* = tau* / (kappa rho).  Every case below is checked against that, whatever
the segments the walk cut the path into.  CPU only.
"""
import math

import numpy as np
import pytest

from paper_1410_1629_gb300 import workloads as W

KR = 1.5  # kappa rho of the uniform cube (kappa 1)


def _cube(n=8, tail_free_from=None):
    prob = W.uniform_cube(n_cells=n, rho=KR, axis_tau=2.0 * KR)
    assert abs(prob.kappa[0] - 1.0) < 1e-15
    if tail_free_from is not None:
        dens = prob.grid.density.copy()
        dens[:, :, tail_free_from:] = 0.0
        prob = W.with_density(prob, dens)
    return prob


def _exit_length(x, k, lo=-1.0, hi=1.0):
    d = np.inf
    for a in range(3):
        if k[a] > 0:
            d = min(d, (hi - x[a]) / k[a])
        elif k[a] < 0:
            d = min(d, (lo - x[a]) / k[a])
    return d


def _closed_form(x, k, u, D):
    tau_path = KR * D
    tau_star = -math.log1p(-u * -math.expm1(-tau_path))
    return tau_path, tau_star, np.asarray(x) + (tau_star / KR) * np.asarray(k)


def _box(prob, cell):
    b = np.asarray(prob.grid.bounds, dtype=np.float64)
    nx, ny, nz = prob.grid.shape
    idx = (cell % nx, (cell // nx) % ny, cell // (nx * ny))
    lo = np.array([b[2 * a] + idx[a] * ((b[2 * a + 1] - b[2 * a]) / n) for a, n in zip(range(3), (nx, ny, nz))])
    hi = np.array([b[2 * a] + (idx[a] + 1) * ((b[2 * a + 1] - b[2 * a]) / n) for a, n in zip(range(3), (nx, ny, nz))])
    return lo, hi


def _rays(n, seed):
    rng = np.random.default_rng(seed)
    xs = rng.uniform(-0.95, 0.95, (n, 3))
    ks = rng.standard_normal((n, 3))
    ks /= np.linalg.norm(ks, axis=1)[:, None]
    return xs, ks


def test_interaction_matches_the_closed_form(oracle):
    prob = _cube()
    xs, ks = _rays(200, 31)
    us = np.random.default_rng(32).uniform(0.0, 1.0, len(xs))
    for x, k, u in zip(xs, ks, us):
        xi, cell, tau_path, tau_star, flags = oracle.interaction(prob, x, k, u)
        D = _exit_length(x, k)
        tp, ts, xe = _closed_form(x, k, u, D)
        assert flags & 4 == 0 and flags & 1 == 0
        assert abs(tau_path - tp) <= 1e-12 * tp
        assert abs(tau_star - ts) <= 1e-12 * max(ts, 1e-300) + 1e-15
        assert np.max(np.abs(xi - xe)) <= 1e-12
        lo, hi = _box(prob, cell)
        assert np.all(xi >= lo) and np.all(xi <= hi)


def test_fallback_takes_the_end_of_the_last_dusty_segment(oracle):
    """A uniform just above 1 makes tau* exceed the path's optical depth (the
    situation rounding can create at u -> 1): the interaction is the limit of
    the inversion, the end of the dust along the path.  With the last cells
    along the ray empty that is where the dust ends, not the grid boundary."""
    for tail in (None, 6):
        prob = _cube(tail_free_from=tail)
        x = np.array([-0.9, 0.1, 0.2])
        k = np.array([1.0, 0.0, 0.0])
        D = 1.9 if tail is None else 1.4  # dust from x = -0.9 to 1.0, or to 0.5
        xi, cell, tau_path, tau_star, flags = oracle.interaction(prob, x, k, 1.0 + 2.0 ** -50)
        assert flags & 1, "the fallback branch did not act"
        assert abs(tau_path - KR * D) <= 1e-12 * KR * D
        assert np.max(np.abs(xi - (x + D * k))) <= 1e-12
        lo, hi = _box(prob, cell)
        assert np.all(xi >= lo) and np.all(xi <= hi) and abs(hi[0] - x[0] - D) <= 1e-12
        # continuity: below u = 1 the ordinary inversion approaches the same point
        prev = np.inf
        for e in (10, 20, 30, 40):
            u = 1.0 - 2.0 ** -e
            xu, _, _, _, fu = oracle.interaction(prob, x, k, u)
            assert fu & 1 == 0
            dist = np.max(np.abs(xu - xi))
            _, _, xe = _closed_form(x, k, u, D)
            assert np.max(np.abs(xu - xe)) <= 1e-12
            assert dist <= prev
            prev = dist
        assert prev < 1e-10


def test_interaction_point_is_moved_into_its_cell(oracle):
    """Uniforms that put tau* on a cell boundary of the path, where rounding of
    x + s* k can leave the point an ulp outside the interaction cell: the
    returned point always lies in the returned cell's box and within rounding
    of the closed-form point, and the move into the cell does act."""
    prob = _cube()
    xs, ks = _rays(300, 41)
    moved = 0
    cases = 0
    for x, k in zip(xs, ks):
        cells, s_in, s_out = oracle.path(prob, x, k)
        D = _exit_length(x, k)
        one_minus_E = -math.expm1(-KR * D)
        for s_b in s_out[:-1]:
            u0 = -math.expm1(-KR * s_b) / one_minus_E
            for u in (np.nextafter(u0, 0.0), u0, np.nextafter(u0, 2.0)):
                xi, cell, _, _, flags = oracle.interaction(prob, x, k, u)
                cases += 1
                moved += (flags >> 1) & 1
                lo, hi = _box(prob, cell)
                assert np.all(xi >= lo) and np.all(xi <= hi), (x, k, u)
                _, _, xe = _closed_form(x, k, u, D)
                assert np.max(np.abs(xi - xe)) <= 1e-12
    assert cases > 1000
    assert moved > 0, "no case exercised the move into the interaction cell"
