"""The parity rule itself (tests/parity.py), exercised on the CPU with the
oracle standing in for both sides: identical runs pass, and planted
differences of the kinds the rule must not let through fail it -- invented
records, a swapped direct/scattered channel, a changed absorption cell, a
pixel moved without a record to explain it."""
import copy

import numpy as np
import pytest

import parity as PAR
from paper_1410_1629_gb300 import workloads as W


@pytest.fixture(scope="module")
def runs(oracle):
    prob = W.uniform_cube(n_cells=16, n_pix=16, channels=3)
    n = 20000
    r = PAR.oracle_run(prob, n, records_cap=400_000, n_threads=4)
    return prob, r


def _gpu_like(r):
    g = copy.deepcopy(r)
    g["records"] = r["records"].copy()
    return g


def test_identical_runs_pass(runs):
    prob, r = runs
    rep = PAR.compare(_gpu_like(r), r, prob)
    assert rep["ok"], rep
    assert rep["corrections"] == 0 and rep["flip_total"] == 0 and rep["raw_unexplained"] == 0
    assert {p["channel"] for p in rep["pixels"]} == {0, 1, 2}
    assert all(p["corrected"]["bins"] > 0 for p in rep["pixels"])
    assert rep["cells"]["bins"] > 0 and rep["cells_all_lambda"]["bins"] > 0


def test_records_that_only_one_side_has_are_bounded(runs):
    """Dropping many oracle records from the 'GPU' side (and their values
    from its images) is repaired by the correction, but the number of such
    corrections exceeds the bound and the rule fails."""
    prob, r = runs
    g = _gpu_like(r)
    drop = np.arange(0, len(g["records"]), 50)
    for i in drop:
        rec = g["records"][i]
        for ch in (0, 1 if rec["event"] == 0 else 2):
            g["images"][rec["instr"]][ch, rec["lam"]].reshape(-1)[rec["pixel"]] -= rec["value"]
    g["records"] = np.delete(g["records"], drop)
    g["records_total"] = len(g["records"])
    rep = PAR.compare(g, r, prob)
    assert rep["oracle_only"] == len(drop) and rep["corrections"] > rep["corrections_limit"]
    assert not rep["ok"]


def test_swapped_channels_fail(runs):
    prob, r = runs
    g = _gpu_like(r)
    g["images"][0] = g["images"][0][[0, 2, 1]]
    rep = PAR.compare(g, r, prob)
    assert not rep["ok"]
    assert any(p["corrected"]["violations"] for p in rep["pixels"] if p["channel"] in (1, 2))


def test_unexplained_pixel_difference_fails(runs):
    """A pixel value changed with no record moved: the raw violation is not
    one the correction touched."""
    prob, r = runs
    g = _gpu_like(r)
    counts = r["image_counts"][0][0, 0]
    iy, ix = np.unravel_index(np.argmax(counts), counts.shape)
    g["images"][0][0, 0, iy, ix] *= 1.001
    rep = PAR.compare(g, r, prob)
    assert not rep["ok"] and rep["raw_unexplained"] >= 1


def test_changed_cell_fails(runs):
    prob, r = runs
    g = _gpu_like(r)
    c = int(np.argmax(r["absorption_counts"][0]))
    g["absorption"][0, c] *= 1.001
    rep = PAR.compare(g, r, prob)
    assert not rep["ok"] and rep["cells"]["violations"] == 1


def test_far_pixel_moves_are_bounded(runs):
    """Records whose GPU pixel is far from the oracle's (parted paths) are
    repaired like flips, but only up to 1e-4 of the records plus 10."""
    prob, r = runs
    g = _gpu_like(r)
    nx = prob.instruments[0].nx
    n_far = int(1e-4 * len(g["records"]) + 10) + 5
    sel = np.argsort(g["records"]["value"])[::-1][:n_far]
    for i in sel:
        rec = g["records"][i]
        old = int(rec["pixel"])
        new = (old + 5 * nx + 5) % (nx * nx)
        for ch in (0, 1 if rec["event"] == 0 else 2):
            img = g["images"][rec["instr"]][ch, rec["lam"]].reshape(-1)
            img[old] -= rec["value"]
            img[new] += rec["value"]
        g["records"]["pixel"][i] = new
    rep = PAR.compare(g, r, prob)
    assert rep["far_flips"] == n_far and rep["far_flips"] > rep["far_flip_limit"] and not rep["ok"]


def test_value_flips_are_bounded(runs):
    """Records whose values differ by more than 1e-2 are taken as cell flips
    (repaired per record), but only up to 2e-3 of the records."""
    prob, r = runs
    g = _gpu_like(r)
    sel = np.arange(0, len(g["records"]), 200)
    for i in sel:
        rec = g["records"][i]
        for ch in (0, 1 if rec["event"] == 0 else 2):
            g["images"][rec["instr"]][ch, rec["lam"]].reshape(-1)[rec["pixel"]] += 0.5 * rec["value"]
    g["records"]["value"][sel] *= 1.5
    rep = PAR.compare(g, r, prob)
    assert rep["value_flips"] == len(sel) and rep["flip_total"] > rep["flip_limit"] and not rep["ok"]


def test_pixel_and_value_flips_take_the_oracle_value(runs):
    """A record whose pixel and value both differ (a packet whose FP32 path
    parted) is moved to the oracle's pixel with the oracle's value: a few of
    them pass and are counted as value flips as well; the uncorrected image
    total is kept beside the corrected one."""
    prob, r = runs
    g = _gpu_like(r)
    nx = g["images"][0].shape[-1]
    sel = np.arange(7, len(g["records"]), 4000)[:5]
    for i in sel:
        rec = g["records"][i]
        old, new = int(rec["pixel"]), int(rec["pixel"]) ^ 1  # the horizontal neighbour
        for ch in (0, 1 if rec["event"] == 0 else 2):
            img = g["images"][rec["instr"]][ch, rec["lam"]].reshape(-1)
            img[old] -= rec["value"]
            img[new] += 3.0 * rec["value"]
        g["records"]["pixel"][i] = new
        g["records"]["value"][i] *= 3.0
    rep = PAR.compare(g, r, prob)
    assert rep["pixel_and_value_flips"] == len(sel) and rep["flips"] == len(sel)
    assert rep["image_total_rel"] < 1e-12 < rep["image_total_rel_raw"]
    assert all(p["corrected"]["max_rel"] < 1e-12 for p in rep["pixels"])
    assert nx > 1
