"""Benchmark: photon-packet Monte Carlo transport on the edge-on disk galaxy.

Workload (one step): 1e8 photon packets (1e7 at each of 10 wavelengths) through
a 256^3 cartesian dust grid (double-exponential dust disk), double-exponential
stellar disk, three 512^2 frames at inclinations 0/60/90 degrees, forced
scattering, continuous absorption and peel-off (FP32 geometry, FP64
accumulators).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the baseline arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon packets/s & cell crossings/s at 1e-4 vs FP64 oracle; adjoint/forward ratio"
UNIT = "packets/s"
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes: forced-path crossing = 4 B density + 16 B FP64 absorption RMW;
# peel-off crossing = 4 B density; peel-off deposit = 16 B FP64 pixel RMW
BYTES_PATH_CROSSING, BYTES_PEEL_CROSSING, BYTES_DEPOSIT = 20, 4, 16
# a peel-off along a grid axis reads 4 B of density and 4 B of column sum
BYTES_COLUMN_PEEL = 8
# DRAM bytes (read + write) per packet of the transport kernel, from an ncu
# capture of one 2e6-packet launch of this workload (dram__bytes_read.sum
# 32.522 GB + dram__bytes_write.sum 13.386 GB), valid only for the kernel
# code whose hash is given (kernel_sources_hash: the sources without their
# comments); the per-launch traffic is this figure times the packets.
TRAFFIC_CAPTURE = {"sources_sha256_16": "67f73aa7b8b72c0a", "kernel": "k_forward_cartesian",
                   "bytes_per_packet": (32522363904 + 13386474752) / 2e6}
KERNEL_SOURCES = ["paper_1410_1629_gb300/csrc/rt_forward.cu", "paper_1410_1629_gb300/csrc/rt_device.cuh",
                  "paper_1410_1629_gb300/csrc/rt_internal.h", "paper_1410_1629_gb300/csrc/rt_transport.cuh",
                  "paper_1410_1629_gb300/build.py"]


def column_tables(prob):
    """Column-sum tables a cartesian or rectilinear launch builds: one per
    distinct grid axis and direction among the frames that look exactly along
    an axis (sines and cosines within 1e-15 of 0 or 1 taken as exact, as the
    library does)."""
    import math
    if prob.grid.kind not in ("cartesian", "rectilinear"):
        return 0

    def snap(v):
        if abs(v) < 1e-15:
            return 0.0
        if abs(abs(v) - 1.0) < 1e-15:
            return math.copysign(1.0, v)
        return v

    seen = set()
    for q in prob.instruments:
        st, ct = snap(math.sin(q.inclination)), snap(math.cos(q.inclination))
        sp, cp = snap(math.sin(q.azimuth)), snap(math.cos(q.azimuth))
        k = (st * cp, st * sp, ct)
        nz = [a for a in range(3) if k[a] != 0.0]
        if len(nz) == 1:
            seen.add((nz[0], k[nz[0]] > 0))
    return len(seen)


def source_code(text, name):
    """The code of a CUDA source without its // comments and blank lines (a
    comment edit leaves the kernel, and so its traffic, unchanged); other
    files whole."""
    if not name.endswith((".cu", ".cuh", ".h")):
        return text
    out = []
    for line in text.splitlines():
        i = line.find("//")
        line = (line if i < 0 else line[:i]).rstrip()
        if line:
            out.append(line)
    return "\n".join(out)


def kernel_sources_hash(read=None):
    """Hash of the code of the transport kernel's sources; read(name) -> text
    reads another version of them (default: the working tree)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(source_code(text, f).encode("utf-8"))
    return h.hexdigest()[:16]


def captured_traffic(packets, workload_name="disk_galaxy", kernel="k_forward_cartesian"):
    """Per-launch DRAM traffic of `kernel` from the stored capture
    (disk-galaxy workload), or None if the kernel changed since, another
    kernel is asked for or another workload runs."""
    if (workload_name != "disk_galaxy" or kernel != TRAFFIC_CAPTURE["kernel"]
            or kernel_sources_hash() != TRAFFIC_CAPTURE["sources_sha256_16"]):
        return None
    return TRAFFIC_CAPTURE["bytes_per_packet"] * packets


def workload(packets=None, name="disk_galaxy"):
    """The headline workload, or another one for profiling runs (the grid
    kinds of the extra bench blocks at their sizes there)."""
    from paper_1410_1629_gb300 import workloads as W
    kw = {"n_packets_total": int(packets)} if packets else {}
    if name == "clumpy_octree":
        return W.clumpy_octree(**kw)
    if name == "clumpy_bintree":
        kw.setdefault("n_packets_total", 8_000_000)
        return W.clumpy_bintree(n_particles=100_000, n_samples=5_000_000, target_leaves=200_000, max_level=8,
                                n_lambda=8, n_pix=512, **kw)
    if name == "voronoi_disk":
        kw.setdefault("n_packets_total", 3_000_000)
        return W.voronoi_disk(n_sites=100_000, n_lambda=3, n_pix=256, **kw)
    if name == "spiral_powcub":
        return W.spiral_example("powcub", n_packets=int(packets) if packets else 10_000_000)
    return W.disk_galaxy(**kw)


def workload_config(prob, world):
    packets = prob.run.n_per_lambda * prob.n_lambda
    if prob.grid.kind == "octree":
        return {"workload": f"clumpy medium on an adaptive octree: {prob.grid.n_cells} leaves "
                            f"({prob.meta['nodes']} nodes, max level 10, delta {prob.meta['delta']:.2e}), "
                            f"Plummer bulge + exponential disk, {prob.n_lambda} wavelengths, {packets:.0e} "
                            f"packets/step per GPU, 2 frames 1024^2 at i=0/90 deg",
                "grid": "octree float32 leaves", "n_lambda": prob.n_lambda,
                "packets_per_step_per_gpu": int(packets),
                "l2": "flushed between timed steps (256 MiB write)",
                "parallelism": f"packet-id ranges sharded over {world} GPU(s), no collective on the data path"}
    if prob.grid.kind != "cartesian":
        return {"workload": f"{prob.name}: {prob.grid.kind} grid of {prob.grid.n_cells} cells, {prob.n_lambda} "
                            f"wavelengths, {packets:.0e} packets/step per GPU",
                "grid": prob.grid.kind, "n_lambda": prob.n_lambda, "packets_per_step_per_gpu": int(packets),
                "l2": "flushed between timed steps (256 MiB write)",
                "parallelism": f"packet-id ranges sharded over {world} GPU(s), no collective on the data path"}
    return {"workload": f"edge-on disk galaxy: 256^3 cartesian grid, 10 wavelengths 0.15-2.2 um, {packets:.0e} "
                        f"packets/step ({prob.run.n_per_lambda:.0e} per wavelength) per GPU, 3 frames 512^2 at "
                        f"i=0/60/90 deg",
            "grid": "cartesian 256x256x256 float32", "n_lambda": prob.n_lambda,
            "packets_per_step_per_gpu": int(prob.run.n_per_lambda * prob.n_lambda),
            "detectors": "3 x 512x512 x 10 lambda, float64",
            "l2": "flushed between timed steps (256 MiB write); absorption tallies (1.34 GB) exceed L2",
            "parallelism": f"packet-id ranges sharded over {world} GPU(s), no collective on the data path"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(prob, seconds, threads):
    """Time the oracle (as it stands) on a bounded sample of the workload: the
    sample grows until one run takes about `seconds` (runs include the
    oracle's fixed set-up, so the rate is measured on the final run only)."""
    from oracle import oracle as O
    O.build()
    n = 50
    while True:
        t0 = time.perf_counter()
        r = O.run(prob, n, n_threads=threads, n_norm=prob.run.n_per_lambda)
        dt = time.perf_counter() - t0
        if dt >= 0.6 * seconds or n >= prob.run.n_per_lambda:
            break
        n = int(min(prob.run.n_per_lambda, max(2 * n, n * 0.9 * seconds / max(dt, 1e-3))))
    packets = n * prob.n_lambda
    return packets / dt, packets, dt, int(r["counters"][0])


def run_reference(args, prob, world, rank):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    per_step = []
    total_packets = 0
    for i in range(args.warmup + args.steps):
        rate, packets, dt, _ = oracle_sample(prob, args.reference_step_seconds, threads)
        if i >= args.warmup:
            per_step.append(dt)
            total_packets += packets
    value = total_packets / sum(per_step)
    sample = (f"first {total_packets // (args.steps * prob.n_lambda)} packet ids per wavelength of the "
              f"workload per step (all 10 wavelengths), FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(per_step) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(prob, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def launch_bytes(st, with_absorption=True):
    """Algorithmic bytes of a launch from its counters (the unit costs
    above); forced-path crossings move no absorption bytes when the launch
    keeps no absorption field (batches)."""
    path_cross, column_cross, column_peels = st["path_crossings"], st["column_crossings"], st["column_peels"]
    peel_cross = st["crossings"] - path_cross - column_cross
    return ((BYTES_PATH_CROSSING if with_absorption else BYTES_PEEL_CROSSING) * path_cross
            + BYTES_PEEL_CROSSING * peel_cross + BYTES_COLUMN_PEEL * column_peels + BYTES_DEPOSIT * st["peeloffs"])


def workload_rate(prob, device, stream, flush, warmup, timed, tune_fraction=0.05, cpu_seconds=0.0, peak=None,
                  kernel="k_forward_cartesian"):
    """Packets/s, crossings/s and the transport kernel's roofline for one
    workload: tuned on a sample (another seed), `warmup` untimed and `timed`
    timed launches (CUDA events on the launching stream, L2 flushed before
    each), optionally the oracle on a bounded sample of the same workload."""
    import torch
    from paper_1410_1629_gb300 import rt
    n = prob.run.n_per_lambda
    sim = rt.Simulation(prob, device=device)
    try:
        lanes = sim.tune(max(1, int(n * tune_fraction)), seed=prob.run.seed + 1, stream=stream.cuda_stream)
        blocks_per_sm = sim.tuned()[1]
        times, parts = [], []
        for i in range(warmup + timed):
            with torch.cuda.stream(stream):
                flush.zero_()
                sim.reset(stream=stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.launch(n, 0, prob.run.seed, stream=stream, time_parts=1)
                e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                times.append(e0.elapsed_time(e1) / 1e3)
                parts.append(sim.launch_times())
        st = sim.stats()
    finally:
        sim.close()
    t = sum(times) / len(times)
    packets = n * prob.n_lambda
    kern_ms = statistics.mean(p["transport"] for p in parts)
    walks_ms = statistics.mean(p["peel_walks"] for p in parts)
    sorted_peels = st["sorted_peels"]
    walked = st["peeloffs"] - st["column_peels"]
    peel_cross = st["crossings"] - st["path_crossings"] - st["column_crossings"]
    sorted_cross = peel_cross * sorted_peels / walked if walked else 0
    bytes_all = launch_bytes(st)
    bytes_kernel = bytes_all - (BYTES_PEEL_CROSSING * sorted_cross + BYTES_DEPOSIT * sorted_peels)
    out = {"packets": int(packets), "seconds_per_launch": t, "packets_per_s": packets / t,
           "crossings_per_s": st["crossings"] / t,
           "walked_crossings_per_s": (st["crossings"] - st["column_crossings"]) / t,
           "timed_launches": len(times),
           "tuned": {"control_lanes": lanes, "blocks_per_sm": blocks_per_sm or "as many as fit"},
           "kernel_ms": kern_ms, "peel_walks_ms": walks_ms,
           "conservation_rel": abs(st["emitted"] - st["escaped"] - st["absorbed"] - st["truncated"]) / st["emitted"],
           "device_flags": int(st["device_flags"]), "l2": "flushed before each timed launch (256 MiB write)"}
    if peak:
        ach = bytes_kernel / (kern_ms / 1e3) / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peak[0], "unit": "GB/s",
                           "frac": ach / peak[0], "peak_source": f"{peak[1]} hbm_gbs",
                           "algorithmic_bytes_per_launch": int(bytes_kernel), "traffic": None}
    if cpu_seconds > 0:
        threads = os.cpu_count() or 1
        rate, cpackets, dt, _ = oracle_sample(prob, cpu_seconds, threads)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"first {cpackets // prob.n_lambda} packet ids per wavelength "
                                         f"({cpackets} packets, {dt:.1f} s), FP64 oracle, all host threads"}
    return out


def octree_rate(args, device, stream, flush, peak):
    """The clumpy medium on the adaptive octree: 1e6 Gaussian clumps binned
    to ~5e6 leaves (max level 10), Plummer bulge + exponential disk, 20
    wavelengths, 2e8 packets, two 1024^2 frames."""
    from paper_1410_1629_gb300 import workloads as W
    t0 = time.time()
    kw = {"n_packets_total": int(args.octree_packets)} if args.octree_packets else {}
    prob = W.clumpy_octree(**kw)
    gen_s = time.time() - t0
    out = workload_rate(prob, device, stream, flush, warmup=1, timed=1, tune_fraction=0.01,
                        cpu_seconds=args.cpu_seconds / 2, peak=peak, kernel="k_forward_octree")
    out["workload"] = (f"clumpy_octree: {prob.grid.n_cells} leaves ({prob.meta['nodes']} nodes, max level 10, "
                       f"delta {prob.meta['delta']:.3e} of the total mass), Plummer bulge + exponential disk, "
                       f"{prob.n_lambda} wavelengths, {out['packets']:.0e} packets, 2 frames 1024^2 at i=0/90 deg")
    out["leaves"] = int(prob.grid.n_cells)
    out["nodes"] = int(prob.meta["nodes"])
    out["delta"] = float(prob.meta["delta"])
    out["generation_s"] = gen_s
    depth = leaf_depths(prob.grid.child)
    out["leaf_depth"] = {"mean": float(depth.mean()), "max": int(depth.max()),
                         "share_by_depth": {int(d): float(c) / len(depth)
                                            for d, c in zip(*np.unique(depth, return_counts=True))}}
    out["roofline"]["note"] = ("algorithmic bytes count no tree-node loads: a walk's re-descent reads one 4 B "
                               "child word per level below the common ancestor, the first 1024 words (the top "
                               "three levels) from shared memory")
    return out


def leaf_depths(child):
    """Depth of every leaf of an octree given as its child array (children
    after their parents)."""
    child = np.asarray(child, dtype=np.int64)
    depth = np.zeros(len(child), dtype=np.int64)
    inner = np.flatnonzero(child >= 0)
    for node in inner:  # parents first, so each parent's depth is final
        depth[child[node]:child[node] + 8] = depth[node] + 1
    return depth[child < 0]


def grid_kinds_rate(args, device, stream, flush, peak):
    """The adaptive grids of Table 1(d) beside the octree: the clumpy medium
    on a k-d tree (BinTree: ~2e5 leaves, 8 wavelengths, 8e6 packets, two
    512^2 frames) and the disk galaxy on a Voronoi grid whose sites follow
    its dust (1e5 sites, 3 wavelengths, 3e6 packets, three 256^2 frames).
    Algorithmic bytes as for the other grids (density and absorption per
    crossing); the Voronoi walk also reads each crossed cell's face planes
    (site, offsets and ~15 faces of 20 B), reported beside it."""
    from paper_1410_1629_gb300 import workloads as W
    out = {}
    t0 = time.time()
    kd = W.clumpy_bintree(n_particles=100_000, n_samples=5_000_000, target_leaves=200_000, max_level=8, n_lambda=8,
                          n_pix=512, n_packets_total=8_000_000)
    gen = time.time() - t0
    r = workload_rate(kd, device, stream, flush, warmup=2, timed=2, tune_fraction=0.2, peak=peak,
                      kernel="k_forward_bintree")
    r["workload"] = (f"clumpy_bintree: {kd.grid.n_cells} leaves ({kd.meta['nodes']} nodes, delta "
                     f"{kd.meta['delta']:.2e}), Plummer bulge + exponential disk, {kd.n_lambda} wavelengths, "
                     f"{r['packets']:.0e} packets, 2 frames 512^2 at i=0/90 deg")
    r["generation_s"] = gen
    out["bintree"] = r
    t0 = time.time()
    vor = W.voronoi_disk(n_sites=100_000, n_lambda=3, n_pix=256, n_packets_total=3_000_000)
    gen = time.time() - t0
    r = workload_rate(vor, device, stream, flush, warmup=2, timed=2, tune_fraction=0.2, peak=peak,
                      kernel="k_forward_voronoi")
    nb = vor.meta["neighbours_per_cell"]
    r["workload"] = (f"voronoi_disk: {vor.grid.n_cells} sites (90 % following the dust, {nb:.1f} neighbours per "
                     f"cell), disk galaxy stars and optics, {vor.n_lambda} wavelengths, {r['packets']:.0e} packets, "
                     f"3 frames 256^2 at i=0/60/90 deg")
    r["neighbours_per_cell"] = nb
    r["face_bytes_per_crossing"] = 16 + 8 + 20 * nb
    r["generation_s"] = gen
    out["voronoi"] = r
    return out


def spiral_rate(args, device, stream, flush, peak):
    """The paper's worked example (Sect. 2.5): spiral galaxy at 0.55 um, 1e7
    packets, one 1200 x 300 edge-on frame, on a 256 x 256 x 128 power-law
    (PowCub) grid and on a 256 x 256 x 72 equal-cell grid."""
    from paper_1410_1629_gb300 import workloads as W
    out = {}
    for name, prob in (("powcub", W.spiral_example("powcub")), ("cartesian", W.spiral_example("cartesian", n_z=72))):
        r = workload_rate(prob, device, stream, flush, warmup=3, timed=3, tune_fraction=0.1,
                          cpu_seconds=args.cpu_seconds / 3 if name == "powcub" else 0.0, peak=peak,
                          kernel="k_forward_rect" if name == "powcub" else "k_forward_cartesian")
        nz, ny, nx = prob.grid.density.shape
        r["workload"] = (f"spiral_example_{name}: {nx}x{ny}x{nz} cells, exponential stellar disk (4400 / 500 pc, "
                         f"1e11 Lsun) and dust disk (6600 / 250 pc, 4e7 Msun, edge-on tau_V "
                         f"{prob.meta['edge_on_tau_v']:.1f}), 0.55 um, {r['packets']:.0e} packets, 1200x300 frame "
                         f"at i=90 deg")
        out[name] = r
    return out


def panchromatic_rate(args, device, stream, flush):
    """Panchromatic mode on the disk galaxy (256^3 cells, 24 wavelengths
    0.1-1000 um, a 5800 K stellar spectrum): a stellar launch, the
    equilibrium dust temperatures from its absorption tallies, the thermal
    emission table, and a launch of dust-emission packets; device times of
    each step (CUDA events) and the energy balance."""
    import torch
    from paper_1410_1629_gb300 import rt
    from paper_1410_1629_gb300 import workloads as W
    prob = W.panchromatic_disk(n_cells=args.panchromatic_cells, n_pix=512,
                               n_packets_total=int(args.panchromatic_packets))
    S = prob.meta["emission_scale"]
    n = prob.run.n_per_lambda
    sim = rt.Simulation(prob, device=device)
    try:
        lanes = sim.tune(max(1, n // 20), seed=1, stream=stream.cuda_stream)
        T = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device=f"cuda:{device}")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        times = {}
        for i in range(2):  # a warm-up pass, then the timed one
            with torch.cuda.stream(stream):
                flush.zero_()
                sim.reset(stream=stream)
                ev[0].record(stream)
                sim.launch(n, 0, 0, stream=stream)
                ev[1].record(stream)
            clamped = rt.rt_dust_temperature(sim.ctx, S, 1.0, 1e4, 0, 0, T.data_ptr(), 1, stream.cuda_stream)
            with torch.cuda.stream(stream):
                ev[2].record(stream)
            rt.rt_set_dust_emission(sim.ctx, T.data_ptr(), 1, S, stream.cuda_stream)
            with torch.cuda.stream(stream):
                ev[3].record(stream)
                absorbed_stars = sim.stats()["absorbed"]
                sim.reset(stream=stream)
                flush.zero_()
            e_dust0 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e_dust0.record(stream)
                sim.launch(n, 0, 1, stream=stream, emitter=rt.RT_EMITTER_DUST)
                ev[4].record(stream)
            ev[4].synchronize()
            times = {"stellar_ms": ev[0].elapsed_time(ev[1]), "temperature_ms": ev[1].elapsed_time(ev[2]),
                     "emission_table_ms": ev[2].elapsed_time(ev[3]), "dust_launch_ms": e_dust0.elapsed_time(ev[4])}
        st = sim.stats()
        Tn = T.cpu().numpy()
    finally:
        sim.close()
    hot = Tn[Tn > 0]
    packets = n * prob.n_lambda
    return {"workload": f"panchromatic_disk_{args.panchromatic_cells}: {args.panchromatic_cells}^3 cells, "
                        f"{prob.n_lambda} wavelengths 0.1-1000 um, 5800 K stars, {packets:.1e} packets per launch, "
                        "three 512^2 frames and an SED instrument",
            "packets": int(packets), **times,
            "stellar_packets_per_s": packets / (times["stellar_ms"] / 1e3),
            "dust_packets_per_s": packets / (times["dust_launch_ms"] / 1e3),
            "temperature_K": {"min": float(hot.min()), "median": float(np.median(hot)), "max": float(hot.max())},
            "cells_held_at_limits": int(clamped),
            "dust_emitted_over_absorbed": float(st["emitted"] / absorbed_stars),
            "dust_conservation_rel": abs(st["emitted"] - st["escaped"] - st["absorbed"] - st["truncated"]) / st["emitted"],
            "tuned": {"control_lanes": lanes}, "device_flags": int(st["device_flags"])}


def plain_cube_rate(args, device, stream, flush):
    """The plain method: 32^3 uniform cube, axis tau 1, albedo 0.6, g 0.5,
    central point source, 1e5 packets, one 64^2 face-on frame."""
    from paper_1410_1629_gb300 import workloads as W
    prob = W.uniform_cube()
    r = workload_rate(prob, device, stream, flush, warmup=3, timed=5, tune_fraction=0.2,
                      cpu_seconds=min(5.0, args.cpu_seconds), peak=None)
    r["workload"] = ("uniform_cube_32: 32^3 cells of side 2/32 pc, axis tau 1, albedo 0.6, g 0.5, central point "
                     "source, 1e5 packets, one 64^2 face-on frame")
    r["note"] = "the grid (128 KB) and its tallies stay in L2; a launch this small is bound by its own latency"
    return r


def adjoint_ratio(args, device, stream, flush):
    """Adjoint/forward time on the differentiation workload: 64^3 log-normal
    cube, 10^7 packets, 128^2 bilinear detector, termination after 20 events;
    the adjoint of the L2 image loss against the image of an independent
    field.  CUDA events on the launching stream, L2 flushed before each."""
    import torch
    from paper_1410_1629_gb300 import rt
    from paper_1410_1629_gb300 import workloads as W
    prob = W.lognormal_cube(n_packets=int(args.adjoint_packets))
    target_prob = W.lognormal_cube(seed=104, n_packets=int(args.adjoint_packets))
    n = prob.run.n_per_lambda
    opts = dict(max_events=prob.run.max_events, weight_cut=0)
    sim = rt.Simulation(prob, device=device)
    tsim = rt.Simulation(target_prob, device=device)
    try:
        with torch.cuda.stream(stream):
            tsim.launch(n, 0, prob.run.seed, stream=stream, **opts)
            target = tsim.images(stream=stream)[0]
            sim.launch(n, 0, prob.run.seed, stream=stream, **opts)
            adj = (2.0 * (sim.images(stream=stream)[0] - target)).contiguous()
            grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device=f"cuda:{device}")
            prof = torch.zeros(8, dtype=torch.int64, device=f"cuda:{device}")
        sim.tune(max(1, n // 10), seed=prob.run.seed + 1, stream=stream.cuda_stream, **opts)
        o = sim.opts(**opts)
        o_prof = sim.opts(profile=prof.data_ptr(), **opts)

        def fwd():
            sim.reset(stream=stream)
            sim.launch(n, 0, prob.run.seed, stream=stream, **opts)

        rt.rt_adjoint_tune(sim.ctx, [adj.data_ptr()], 0, max(1, n // 10), prob.run.seed + 1, o, stream.cuda_stream)

        def bwd(o_):
            grad.zero_()
            rt.rt_adjoint(sim.ctx, [adj.data_ptr()], 0, grad.data_ptr(), n, 0, prob.run.seed, o_, stream.cuda_stream)

        def timed(f):
            ts = []
            for i in range(args.warmup + min(args.steps, 3)):
                with torch.cuda.stream(stream):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    f()
                    e1.record(stream)
                e1.synchronize()
                if i >= args.warmup:
                    ts.append(e0.elapsed_time(e1) / 1e3)
            return sum(ts) / len(ts)

        t_f = timed(fwd)
        st = sim.stats()
        with torch.cuda.stream(stream):
            t_b = timed(lambda: bwd(o))
            bwd(o_prof)
        torch.cuda.synchronize()
        adj_cross, dep_cross = int(prof[0].item()), int(prof[1].item())
        # with the adjoint tape: the forward launch records its events and the
        # adjoint of the same packets needs no replay (each timed adjoint
        # follows its own taped forward launch, both timed separately)
        tf, tb = [], []
        for i in range(args.warmup + min(args.steps, 3)):
            with torch.cuda.stream(stream):
                flush.zero_()
                e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
                e0.record(stream)
                sim.reset(stream=stream)
                sim.launch(n, 0, prob.run.seed, stream=stream, tape=1, **opts)
                e1.record(stream)
                flush.zero_()
                e2.record(stream)
                bwd(o)
                e3.record(stream)
            e3.synchronize()
            if i >= args.warmup:
                tf.append(e0.elapsed_time(e1) / 1e3)
                tb.append(e2.elapsed_time(e3) / 1e3)
        t_tf, t_tb = sum(tf) / len(tf), sum(tb) / len(tb)
        flags = sim.stats()["device_flags"]
        fd = fd_check(prob, sim, adj, opts, args.fd_packets, stream) if not args.skip_fd else None
    finally:
        sim.close()
        tsim.close()
    return {"workload": f"lognormal_cube_64: 64^3 cells, {n:.3g} packets, 128^2 bilinear detector, 20 events, "
                        "L2 image loss against an independent field",
            "forward_ms": 1e3 * t_f, "adjoint_ms": 1e3 * t_b, "ratio": t_b / t_f,
            "tape": {"forward_ms": 1e3 * t_tf, "adjoint_ms": 1e3 * t_tb, "ratio": t_tb / t_tf,
                     "note": "forward launch recording the adjoint tape, then the adjoint without replay"},
            "forward_crossings": int(st["crossings"]), "adjoint_crossings": adj_cross,
            "adjoint_deposit_crossings": dep_cross, "adjoint_crossings_per_s": adj_cross / t_b,
            "adjoint_algorithmic_bytes": int(BYTES_PEEL_CROSSING * adj_cross + BYTES_DEPOSIT * dep_cross),
            "fd_check": fd, "device_flags": int(flags), "l2": "flushed before each timed launch"}


def fd_check(prob, sim, adj, opts, n, stream):
    """Central differences of the GPU forward (eps = 1e-3 of a density, 64
    random cells, rng seed 4, common random numbers) against the GPU adjoint
    of the same packets and adjoint image: the relative deviation per cell
    (median, p90).  The forward's FP32 rounding puts a noise floor under the
    differences of cells whose gradient is small (the loss's adjoint changes
    sign over the image, so the rounding does not cancel); the tests compare
    the differences with the oracle's at the same step."""
    import torch
    from paper_1410_1629_gb300 import rt
    n = int(n)
    eps = 1e-3
    cells = np.random.default_rng(4).choice(prob.grid.n_cells, 64, replace=False)
    rho = prob.grid.density.ravel().copy()
    dev = adj.device

    def functional(dens):
        # the copy runs on torch's stream, where the buffer was made, and is
        # waited for before the buffer can be released
        d = torch.from_numpy(np.ascontiguousarray(dens, dtype=np.float32)).to(dev)
        rt.rt_update_density(sim.ctx, d.data_ptr(), 1, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        sim.reset(stream=stream)
        sim.launch(n, 0, prob.run.seed, stream=stream, **opts)
        with torch.cuda.stream(stream):
            v = (adj * sim.images(stream=stream)[0]).sum()
            # read on the stream that computed it (outside this block the
            # copy would run on torch's default stream, ahead of the sum)
            return float(v.item())

    t0 = time.time()
    fd = np.zeros(64)
    for i, c in enumerate(cells):
        up, dn = rho.copy(), rho.copy()
        up[c] = np.float32(rho[c] * (1 + eps))
        dn[c] = np.float32(rho[c] * (1 - eps))
        fd[i] = (functional(up) - functional(dn)) / (float(up[c]) - float(dn[c]))
    d = torch.from_numpy(rho).to(dev)
    rt.rt_update_density(sim.ctx, d.data_ptr(), 1, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    grad = torch.zeros(prob.grid.n_cells, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    rt.rt_adjoint(sim.ctx, [adj.data_ptr()], 0, grad.data_ptr(), n, 0, prob.run.seed, sim.opts(**opts),
                  stream.cuda_stream)
    torch.cuda.synchronize()
    g = grad.cpu().numpy()[cells]
    rel = np.abs(fd - g) / np.abs(g)
    big = np.abs(g) >= 0.1 * np.abs(g).max()
    return {"cells": 64, "eps": eps, "packets": n, "median_rel_dev": float(np.median(rel)),
            "p90_rel_dev": float(np.quantile(rel, 0.9)),
            "median_rel_dev_cells_above_tenth_of_max": float(np.median(rel[big])) if big.any() else None,
            "abs_dev_over_max_gradient_p90": float(np.quantile(np.abs(fd - g) / np.abs(g).max(), 0.9)),
            "seconds": time.time() - t0,
            "loss": "image L2 loss against the image of an independent field (the adjoint image of the timing)"}


def batch_rate(args, device, stream):
    """Packets/s of one batched launch of the 4096-model workload (8^3-48^3
    cubes, 1e4-1e6 packets each, 64^2 frame each): tuned once, then warm-up
    and timed graph launches with CUDA events on the launching stream.  The
    batch's densities (0.55 GB) and images (0.13 GB) exceed L2."""
    import torch
    from paper_1410_1629_gb300 import rt
    from paper_1410_1629_gb300 import workloads as W
    models = W.batch_models(n_models=args.batch_models)
    scale = args.batch_packet_scale
    counts = None if scale == 1.0 else [max(1, int(round(m.run.n_per_lambda * scale))) for m in models]
    b = rt.Batch(models, device=device, n_packets=counts)
    try:
        lanes, run = b.tune(seed=0, fraction=0.02, stream=stream.cuda_stream)
        ts = []
        for i in range(args.warmup + 2):
            b.reset(stream=stream.cuda_stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                b.launch(seed=0, stream=stream.cuda_stream)
                e1.record(stream)
            e1.synchronize()
            if i >= args.warmup:
                ts.append(e0.elapsed_time(e1) / 1e3)
        st = b.stats()
    finally:
        b.close()
    t = sum(ts) / len(ts)
    return {"workload": f"{len(models)} models: 8^3-48^3 cells, half uniform / half exponential slab, axis tau 0.1-20, "
                        f"g 0-0.9, albedo 0.3-0.8, {scale:g} x (1e4-1e6) packets, one 64^2 frame each",
            "models": len(models), "packets": int(st["packets"]), "seconds_per_launch": t,
            "algorithmic_bytes": int(launch_bytes(dict(st, path_crossings=0), with_absorption=False)),
            "packets_per_s": st["packets"] / t, "crossings_per_s": st["crossings"] / t,
            "tuned": {"control_lanes": lanes, "run_packets": run}, "launch": "CUDA graph",
            "timed_launches": len(ts), "device_flags": int(st["device_flags"]),
            "l2": "inputs larger than L2"}


def run_gpu(args, prob, world, rank, local_rank):
    import torch
    from paper_1410_1629_gb300 import rt

    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
    device = local_rank
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device)
    from paper_1410_1629_gb300.sharding import shard
    first, n, n_norm = shard(rank, world, prob.run.n_per_lambda)
    sim = rt.Simulation(prob, device=device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{device}")
    # set-up: the per-event deferral threshold, timed on a 5 % sample with
    # another seed (the tallies are zeroed afterwards)
    lanes = sim.tune(max(1, n // 20), seed=prob.run.seed + 1, stream=stream.cuda_stream)
    blocks_per_sm = sim.tuned()[1]

    def step(ev0, ev1):
        with torch.cuda.stream(stream):
            flush.zero_()
            sim.reset(stream=stream)
            ev0.record(stream)
            sim.launch(n, first, prob.run.seed, stream=stream, n_norm=n_norm, time_parts=1)
            ev1.record(stream)

    for _ in range(args.warmup):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        step(e0, e1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    times, counts, parts = [], [], []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        step(e0, e1)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        counts.append(sim.stats())
        parts.append(sim.launch_times())
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_total = sum(times)
    if dist:
        t = torch.tensor([t_total], dtype=torch.float64, device=f"cuda:{device}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total = float(t.item())
    packets_step = n * prob.n_lambda
    value = world * packets_step * args.steps / t_total
    st = counts[-1]
    crossings_step = st["crossings"]
    path_cross = st["path_crossings"]
    # peel-off rays along grid axes read two numbers (the cell's density and
    # its column sum) instead of walking; their crossings count as the walk's
    column_cross, column_peels = st["column_crossings"], st["column_peels"]
    peel_cross = crossings_step - path_cross - column_cross
    deposits = st["peeloffs"]
    bytes_launch = (BYTES_PATH_CROSSING * path_cross + BYTES_PEEL_CROSSING * peel_cross
                    + BYTES_COLUMN_PEEL * column_peels + BYTES_DEPOSIT * deposits)
    mean_launch = t_total / args.steps
    peak, peak_kind = peaks()
    # per kernel: the transport kernel's share of the bytes and the sorted
    # peel-off walks' share (walked peel-offs it could not hold stay in the
    # transport kernel; their crossings are apportioned by count)
    sorted_peels = st["sorted_peels"]
    walked_peels = deposits - column_peels
    sorted_cross = peel_cross * sorted_peels / walked_peels if walked_peels else 0
    bytes_walks = BYTES_PEEL_CROSSING * sorted_cross + BYTES_DEPOSIT * sorted_peels
    bytes_transport = bytes_launch - bytes_walks
    part_ms = {k: statistics.mean(p[k] for p in parts) for k in parts[0]}
    part_bytes = {"column_sums": 0, "transport": bytes_transport, "peel_order": 0, "peel_walks": bytes_walks}
    kernel_of = {"octree": "octree", "bintree": "bintree", "voronoi": "voronoi", "rectilinear": "rect"}
    names = {"column_sums": "k_columns", "transport": "k_forward_" + kernel_of.get(prob.grid.kind, "cartesian"),
             "peel_order": "k_peel_scan_tiles + k_peel_scan_sums + k_peel_scatter", "peel_walks": "k_peel_sorted"}
    top = max(part_ms, key=part_ms.get)
    achieved = part_bytes[top] / (part_ms[top] / 1e3) / 1e9
    launches_step = column_tables(prob) + 1 + (4 if sorted_peels else 0)
    conservation = abs(st["emitted"] - st["escaped"] - st["absorbed"] - st["truncated"]) / st["emitted"]

    # end to end through the C ABI with host buffers: upload the grid, set up,
    # launch, read every image and the absorption field back to pinned memory
    e2e = None
    if not args.skip_e2e:
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        dens_host = torch.from_numpy(np.ascontiguousarray(prob.grid.density)).pin_memory()
        img_host = [torch.empty(sim.image_shape(q), dtype=torch.float64).pin_memory()
                    for q in range(len(prob.instruments))]
        ab_host = torch.empty((prob.n_lambda, prob.grid.n_cells), dtype=torch.float64).pin_memory()
        ctx = rt.rt_context_create(device)
        try:
            e2e_times = []
            for i in range(e2e_steps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                d, keep = rt.grid_desc(prob.grid)
                d.density = dens_host.data_ptr()
                rt.rt_create_grid(ctx, d)
                rt.rt_set_optics(ctx, 0, prob.kappa, prob.albedo, prob.g, prob.wavelengths)
                rt.rt_add_sources(ctx, [rt.source_desc(s) for s in prob.sources], [s.lum for s in prob.sources])
                rt.rt_add_instruments(ctx, [rt.instrument_desc(q) for q in prob.instruments])
                o = rt.rt_default_opts()
                o.n_norm = n_norm
                o.control_lanes = lanes
                rt.rt_launch_packets(ctx, n, first, prob.run.seed, o, stream.cuda_stream)
                for q, buf in enumerate(img_host):
                    rt.rt_read_images(ctx, q, buf.data_ptr(), buf.numel(), 0, stream.cuda_stream)
                rt.rt_read_absorption(ctx, ab_host.data_ptr(), ab_host.numel(), 0, stream.cuda_stream)
                torch.cuda.synchronize()
                if i > 0:  # the first pass is a warm-up
                    e2e_times.append(time.perf_counter() - t0)
        finally:
            rt.rt_context_destroy(ctx)
        te = sum(e2e_times)
        if dist:
            t = torch.tensor([te], dtype=torch.float64, device=f"cuda:{device}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        h2d = dens_host.numel() * 4 + 8 * prob.n_lambda * (3 + len(prob.sources))
        d2h = sum(b.numel() for b in img_host) * 8 + ab_host.numel() * 8
        e2e = {"value": world * packets_step * len(e2e_times) / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": len(e2e_times),
               "step_seconds": [round(x, 4) for x in e2e_times],
               "includes": "rt_create_grid from pinned host density, optics, sources, instruments, launch, "
                           "rt_read_images and rt_read_absorption to pinned host memory"}
    sim.close()

    adjoint = None
    if rank == 0 and world == 1 and not args.skip_adjoint:
        adjoint = adjoint_ratio(args, device, stream, flush)
    batch = None
    if rank == 0 and world == 1 and not args.skip_batch:
        batch = batch_rate(args, device, stream)
    # the L2 read bandwidth of the library's own probe kernel (32 MiB buffer):
    # the roofline of the kernels whose working set stays in L2
    l2 = None
    if rank == 0 and world == 1:
        sizes = {f"{m}MiB": rt.rt_probe_bandwidth(device, m << 20, 40, 5) for m in (8, 16, 32, 48)}
        l2 = {"gb_per_s": max(sizes.values()), "by_buffer": sizes,
              "how": "rt_probe_bandwidth: L2-cached float4 loads over buffers of 8-48 MiB, 40 passes, best of 5, "
                     "CUDA events; the best buffer", "hbm_read_gb_per_s": rt.rt_probe_bandwidth(device, 4 << 30, 2, 3)}
        for block, secs_key in ((adjoint, "adjoint_ms"), (batch, "seconds_per_launch")):
            if not block:
                continue
            b = block["adjoint_algorithmic_bytes"] if secs_key == "adjoint_ms" else block["algorithmic_bytes"]
            secs = block[secs_key] / 1e3 if secs_key == "adjoint_ms" else block[secs_key]
            ach = b / secs / 1e9
            block["roofline"] = {"bound": "l2", "kernel": "k_adjoint" if secs_key == "adjoint_ms" else "k_batch",
                                 "achieved": ach, "peak": l2["gb_per_s"], "unit": "GB/s", "frac": ach / l2["gb_per_s"],
                                 "peak_source": "builder-measured L2 read bandwidth (rt_probe_bandwidth)",
                                 "time": "the whole call (its kernels back to back)"}
    octree = spiral = plain = grids = None
    if rank == 0 and world == 1 and not args.skip_octree:
        octree = octree_rate(args, device, stream, flush, (peak, peak_kind))
    if rank == 0 and world == 1 and not args.skip_grids:
        grids = grid_kinds_rate(args, device, stream, flush, (peak, peak_kind))
    if rank == 0 and world == 1 and not args.skip_spiral:
        spiral = spiral_rate(args, device, stream, flush, (peak, peak_kind))
    if rank == 0 and world == 1 and not args.skip_plain:
        plain = plain_cube_rate(args, device, stream, flush)
    panchro = None
    if rank == 0 and world == 1 and not args.skip_panchromatic:
        panchro = panchromatic_rate(args, device, stream, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        threads = os.cpu_count() or 1
        rate, packets, dt, _ = oracle_sample(prob, args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {packets // prob.n_lambda} packet ids per wavelength of the workload "
                         f"({packets} packets, {dt:.1f} s), FP64 oracle, all host threads"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": workload_config(prob, world),
                "crossings_per_s": world * crossings_step * args.steps / t_total,
                "walked_crossings_per_s": world * (crossings_step - column_cross) * args.steps / t_total,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak,
                             "traffic": (args.traffic if args.traffic is not None
                                         else captured_traffic(packets_step, args.workload, names[top])),
                             "peak_source": f"{peak_kind} hbm_gbs",
                             "kernel": names[top], "kernel_ms": part_ms[top],
                             "algorithmic_bytes_per_launch": int(part_bytes[top]),
                             "parts": {k: {"kernel": names[k], "ms": part_ms[k],
                                           "algorithmic_bytes": int(part_bytes[k]),
                                           "GB_per_s": part_bytes[k] / (part_ms[k] / 1e3) / 1e9 if part_ms[k] else 0.0}
                                       for k in part_ms},
                             "whole_launch": {"ms": 1e3 * mean_launch, "algorithmic_bytes": int(bytes_launch),
                                              "GB_per_s": bytes_launch / mean_launch / 1e9}},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_step * args.steps, "adjoint": adjoint,
                "tuned": {"control_lanes": lanes, "blocks_per_sm": blocks_per_sm or "as many as fit",
                          "sample": "5 % of the packets, another seed, before the warm-up"},
                "batch": batch, "octree": octree, "grids": grids, "spiral_example": spiral, "plain_cube": plain,
                "panchromatic": panchro, "l2_peak": l2,
                "clocks": clk,
                "checks": {"conservation_rel": conservation, "path_crossings": int(path_cross),
                           "walked_peel_crossings": int(peel_cross), "column_peels": int(column_peels),
                           "column_crossings": int(column_cross), "peeloffs": int(deposits),
                           "events": int(st["events"]), "sorted_peels": int(sorted_peels)}}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--only", choices=["adjoint", "batch"], default=None,
                    help="run one sub-measurement alone and print its object (profiling)")
    ap.add_argument("--adjoint-packets", type=float, default=1e7,
                    help="packets of the adjoint/forward measurement (default 1e7, the workload's size)")
    ap.add_argument("--batch-models", type=int, default=4096, help="models of the batch measurement (default 4096)")
    ap.add_argument("--batch-packet-scale", type=float, default=1.0,
                    help="scale of every batch model's packet count (default 1, the workload's size)")
    ap.add_argument("--skip-batch", action="store_true",
                    help="skip the batched 4096-model measurement")
    ap.add_argument("--skip-adjoint", action="store_true",
                    help="skip the adjoint/forward measurement on the 64^3 differentiation workload")
    ap.add_argument("--skip-octree", action="store_true", help="skip the clumpy-octree workload (2e8 packets)")
    ap.add_argument("--octree-packets", type=float, default=None,
                    help="packets of the clumpy-octree measurement (default 2e8, the workload's size)")
    ap.add_argument("--skip-grids", action="store_true",
                    help="skip the k-d tree and Voronoi workloads")
    ap.add_argument("--skip-spiral", action="store_true", help="skip the paper's spiral-galaxy example")
    ap.add_argument("--skip-plain", action="store_true", help="skip the plain-method 32^3 cube")
    ap.add_argument("--skip-panchromatic", action="store_true", help="skip the panchromatic disk galaxy")
    ap.add_argument("--panchromatic-cells", type=int, default=256, help="cells per axis of the panchromatic disk")
    ap.add_argument("--panchromatic-packets", type=float, default=2.4e7,
                    help="packets per launch of the panchromatic disk (stellar and dust launches)")
    ap.add_argument("--skip-fd", action="store_true", help="skip the finite-difference check of the adjoint")
    ap.add_argument("--fd-packets", type=float, default=1e6,
                    help="packets of the finite-difference check (64 cells x 2 forward launches)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--reference-step-seconds", type=float, default=8.0)
    ap.add_argument("--workload", default="disk_galaxy",
                    choices=["disk_galaxy", "clumpy_octree", "clumpy_bintree", "voronoi_disk", "spiral_powcub"],
                    help="disk_galaxy (the headline workload); the others are for profiling runs")
    ap.add_argument("--packets", type=float, default=None,
                    help="packets per step (default 1e8, the workload's size); smaller values are for profiling")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the forward kernel from an ncu capture (scaled)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.only:
        # one sub-measurement alone (for profiling): its JSON object only
        import torch
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream(0)
        if args.only == "adjoint":
            flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda:0")
            out = adjoint_ratio(args, 0, stream, flush)
        else:
            out = batch_rate(args, 0, stream)
        print(json.dumps({"only": args.only, args.only: out}), flush=True)
        return
    prob = workload(args.packets, args.workload)
    if args.impl == "reference":
        run_reference(args, prob, world, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    try:
        run_gpu(args, prob, world, rank, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
