"""Host-side helpers of bench.py: the count of column-sum tables a launch
builds (part of the reported launch count), the kernel-source hash that keys
the stored DRAM traffic capture, and when that capture applies."""
import math

import numpy as np

import bench
from paper_1410_1629_gb300 import workloads as W


def test_column_tables_follow_the_frames():
    # frames at 0, 60 and 90 degrees: face-on (+z) and edge-on look along axes
    assert bench.column_tables(W.disk_galaxy(n_cells=8, n_lambda=1, n_pix=8)) == 2
    assert bench.column_tables(W.uniform_cube(n_cells=4, n_pix=8)) == 1
    prob = W.uniform_cube(n_cells=4, n_pix=8)
    prob.instruments[0].inclination = 0.3
    assert bench.column_tables(prob) == 0
    # two frames along the same axis and direction share one table
    prob = W.uniform_cube(n_cells=4, n_pix=8)
    prob.instruments.append(W.Instrument(0.0, 0.5 * math.pi, 0.0, 8, 8, 1.0, 1.0))
    assert bench.column_tables(prob) == 1
    # the opposite direction is a table of its own
    prob.instruments.append(W.Instrument(math.pi, 0.0, 0.0, 8, 8, 1.0, 1.0))
    assert bench.column_tables(prob) == 2


def test_octree_has_no_column_tables():
    grid, _, _ = W.build_octree([-1, 1] * 3, lambda lo, hi, l: np.full(len(lo), l < 1),
                                lambda lo, hi: np.ones(len(lo)), 3)
    prob = W.uniform_cube(n_cells=4, n_pix=8)
    prob.grid = grid
    assert bench.column_tables(prob) == 0


def test_traffic_capture_applies_to_its_kernel_and_workload_only():
    h = bench.kernel_sources_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    cap = bench.TRAFFIC_CAPTURE
    got = bench.captured_traffic(1e8)
    if h == cap["sources_sha256_16"]:
        assert got == cap["bytes_per_packet"] * 1e8
    else:
        assert got is None
    assert bench.captured_traffic(1e8, "clumpy_octree") is None
    assert bench.captured_traffic(1e8, "disk_galaxy", "k_peel_sorted") is None


def test_kernel_hash_ignores_comments_only():
    a = "int x;  // one\n\n// a whole line\nint y;\n"
    b = "int x;\nint y;  // two\n"
    assert bench.source_code(a, "k.cu") == bench.source_code(b, "k.cu")
    assert bench.source_code("int x;\nint z;\n", "k.cu") != bench.source_code(a, "k.cu")
    # other files are hashed whole
    assert bench.source_code("x = 1  # c\n", "build.py") == "x = 1  # c\n"


def test_leaf_depths_of_an_octree():
    """Leaf depths from the child array: a full octree of depth 2, and one
    whose lowest octant alone is refined on to depth 3."""
    full, _, _ = W.build_octree([-1, 1] * 3, lambda lo, hi, l: np.ones(len(lo), bool),
                                lambda lo, hi: np.ones(len(lo)), 2)
    d = bench.leaf_depths(full.child)
    assert len(d) == 64 and np.all(d == 2)
    mixed, _, _ = W.build_octree([-1, 1] * 3, lambda lo, hi, l: (l == 0) | np.all(hi <= 0.0, axis=1),
                                 lambda lo, hi: np.ones(len(lo)), 3)
    d = bench.leaf_depths(mixed.child)
    assert np.bincount(d).tolist() == [0, 7, 0, 64]
