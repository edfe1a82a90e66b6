"""Helpers for comparing the CUDA library with the FP64 oracle.

The acceptance rule: per pixel and per cell within 1e-4 relative wherever the
oracle's bin holds at least 1e3 contributions; totals within 1e-6 relative.

FP32 geometry places a peel-off a few 1e-7 away from the FP64 position; when
that straddles a pixel edge the contribution lands in the neighbouring pixel
(a "flip").  Flips are identified exactly from per-peel-off records of both
sides, keyed by (packet, wavelength, event, instrument), and each flipped
contribution is moved back to the oracle's pixel before the per-pixel check;
the check then allows no violation at all.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_1410_1629_gb300 import rt


def gpu_run(problem, n_per_lambda, first_id=0, seed=0, records_cap=0, record_stride=0, n_norm=0, sim=None,
            **opts):
    import torch
    own = sim is None
    if own:
        sim = rt.Simulation(problem)
    recs = None
    if records_cap:
        recs = torch.zeros(int(records_cap) * rt.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        opts.update(records=recs.data_ptr(), records_capacity=int(records_cap), record_stride=int(record_stride))
    if n_norm:
        opts["n_norm"] = int(n_norm)
    sim.launch(n_per_lambda, first_id, seed, **opts)
    st = sim.stats()
    out = {
        "images": [t.cpu().numpy() for t in sim.images()],
        "absorption": sim.absorption().cpu().numpy(),
        "stats": np.array([st["emitted"], st["escaped"], st["absorbed"], st["truncated"]]),
        "counters": np.array([st["crossings"], st["events"], st["peeloffs"], st["packets"]], dtype=np.uint64),
        "raw_stats": st,
    }
    if records_cap:
        n = min(int(st["records"]), int(records_cap))
        out["records"] = recs.cpu().numpy().view(rt.RECORD_DTYPE)[:n].copy()
        out["records_total"] = int(st["records"])
    if own:
        sim.close()
    return out


def oracle_run(problem, n_per_lambda, first_id=0, seed=0, records_cap=0, n_threads=None, **kw):
    run = problem.run
    kw.setdefault("w_min", run.w_min)
    kw.setdefault("max_events", run.max_events)
    kw.setdefault("weight_cut", run.weight_cut)
    return O.run(problem, n_per_lambda, first_id=first_id, seed=seed, n_threads=n_threads or O.default_threads(),
                 counts=True, records_cap=records_cap, **kw)


def _keys(rec):
    return (rec["pid"].astype(np.uint64) * np.uint64(1 << 20) + rec["lam"].astype(np.uint64) * np.uint64(1 << 12)
            + rec["event"].astype(np.uint64)) * np.uint64(64) + rec["instr"].astype(np.uint64)


def _channel_of(event):
    """Channel of a peel-off in a 3-channel frame: 1 direct (emission), 2 scattered."""
    return np.where(np.asarray(event) == 0, 1, 2)


def flip_corrected_images(gpu, ora, problem, value_flip_rtol=1e-2):
    """GPU images (every channel) with the FP32 flips undone, per record:

    * a pixel flip (the record's pixel differs from the oracle's) has its
      contribution moved to the oracle's pixel, with the oracle's value when
      the values also differ by more than value_flip_rtol (the packet's FP32
      path parted from the FP64 one: counted as a value flip too);
    * a value flip (same pixel, value off by more than value_flip_rtol: the
      FP32 position fell on the other side of a cell face, so the peel-off
      ray runs through other cells) has its contribution replaced by the
      oracle's value;
    * a GPU-only record is removed and an oracle-only record added.

    Returns (images, report); report["touched"] lists, per instrument, the
    flat bins (channel, lambda * ny * nx + pixel) a correction changed, and
    report["far_flips"] counts pixel flips to a pixel that is not a
    neighbour of the oracle's (Chebyshev distance above 1)."""
    g, o = gpu["records"], ora["records"]
    assert gpu["records_total"] == len(g) and ora["records_total"] == len(o), "record buffer overflow"
    kg, ko = _keys(g), _keys(o)
    assert len(np.unique(kg)) == len(kg) and len(np.unique(ko)) == len(ko)
    common, ig, io = np.intersect1d(kg, ko, return_indices=True)
    flip = g["pixel"][ig] != o["pixel"][io]
    rel = np.abs(g["value"][ig] - o["value"][io]) / np.maximum(np.abs(o["value"][io]), 1e-300)
    vflip = ~flip & (rel > value_flip_rtol)
    both = flip & (rel > value_flip_rtol)
    only_g = np.setdiff1d(np.arange(len(g)), ig)
    only_o = np.setdiff1d(np.arange(len(o)), io)
    imgs = [im.copy() for im in gpu["images"]]  # [channels, n_lambda, ny, nx]
    touched = [set() for _ in imgs]

    def add(q, lam, event, pix, value):
        im = imgs[q]
        plane = im.shape[-2] * im.shape[-1]
        chans = (0, int(_channel_of(event))) if im.shape[0] == 3 else (0,)
        for ch in chans:
            im[ch, lam].reshape(-1)[pix] += value
            touched[q].add((ch, int(lam) * plane + int(pix)))

    far = 0
    for a, b, both_ab in zip(ig[flip], io[flip], both[flip]):
        q, lam, ev = g["instr"][a], g["lam"][a], g["event"][a]
        nx = imgs[q].shape[-1]
        pg, po = int(g["pixel"][a]), int(o["pixel"][b])
        far += max(abs(pg % nx - po % nx), abs(pg // nx - po // nx)) > 1
        add(q, lam, ev, pg, -g["value"][a])
        add(q, lam, ev, po, o["value"][b] if both_ab else g["value"][a])
    for a, b in zip(ig[vflip], io[vflip]):
        add(g["instr"][a], g["lam"][a], g["event"][a], g["pixel"][a], o["value"][b] - g["value"][a])
    for a in only_g:
        add(g["instr"][a], g["lam"][a], g["event"][a], g["pixel"][a], -g["value"][a])
    for b in only_o:
        add(o["instr"][b], o["lam"][b], o["event"][b], o["pixel"][b], o["value"][b])
    worst = np.argsort(rel)[::-1][:3]
    report = {"worst_records": [{"pid": int(o["pid"][io[w]]), "lam": int(o["lam"][io[w]]),
                                 "event": int(o["event"][io[w]]), "instr": int(o["instr"][io[w]]),
                                 "gpu": float(g["value"][ig[w]]), "oracle": float(o["value"][io[w]])}
                                for w in worst if rel[w] > 1e-3],
              "records": int(len(o)), "flips": int(flip.sum()), "value_flips": int(vflip.sum()),
              "pixel_and_value_flips": int(both.sum()),
              "far_flips": int(far), "gpu_only": int(len(only_g)), "oracle_only": int(len(only_o)),
              "record_rel_p999": float(np.quantile(rel, 0.999)) if len(rel) else 0.0,
              "record_rel_max": float(rel.max()) if len(rel) else 0.0, "touched": touched}
    return imgs, report


def bin_check(gpu_vals, ora_vals, counts, min_count=1000, rtol=1e-4):
    """Bins with at least min_count oracle contributions must agree within rtol
    (relative); returns the number of such bins, of violations and their flat
    indices, and the largest relative difference."""
    mask = counts >= min_count
    g, o = gpu_vals[mask], ora_vals[mask]
    diff = np.abs(g - o)
    rel = np.where(diff == 0, 0.0, diff / np.maximum(np.abs(o), 1e-300))
    bad = np.flatnonzero(mask.reshape(-1))[rel > rtol]
    return {"bins": int(mask.sum()), "violations": int((rel > rtol).sum()),
            "max_rel": float(rel.max()) if rel.size else 0.0, "violating": bad}


def block_sum(a, b):
    """Sum over b x b pixel blocks of the last two axes."""
    ny, nx = a.shape[-2:]
    return a.reshape(a.shape[:-2] + (ny // b, b, nx // b, b)).sum(axis=(-3, -1))


def cell_groups(grid, block=4, level=None):
    """Group id of every cell for coarser absorption bins: cartesian and
    rectilinear grids in block^3 cubes of cells; trees (octree, k-d tree) by
    the leaf's ancestor at depth `level` (the parent node when level is
    None; a leaf shallower than `level` is its own group); Voronoi grids by
    the box of a coarse 8^3 (or `level`^3) division of the domain that holds
    the cell's site."""
    if grid.kind == "voronoi":
        bins = 8 if level is None else int(level)
        b = np.asarray(grid.bounds, dtype=np.float64).reshape(3, 2)
        idx = np.floor((grid.sites - b[:, 0]) / (b[:, 1] - b[:, 0]) * bins).astype(np.int64).clip(0, bins - 1)
        return idx[:, 0] + bins * (idx[:, 1] + bins * idx[:, 2])
    if grid.kind in ("cartesian", "rectilinear"):
        nx, ny, nz = grid.shape
        iz, iy, ix = np.meshgrid(np.arange(nz) // block, np.arange(ny) // block, np.arange(nx) // block,
                                 indexing="ij")
        gx, gy = (nx + block - 1) // block, (ny + block - 1) // block
        return (ix + gx * (iy + gy * iz)).reshape(-1)
    child = np.asarray(grid.child, dtype=np.int64)
    kids = 2 if grid.kind == "bintree" else 8
    n = len(child)
    parent = np.full(n, -1, dtype=np.int64)
    depth = np.zeros(n, dtype=np.int64)
    # children follow their parents in the node array: one pass in order
    inner = np.flatnonzero(child >= 0)
    for o in range(kids):
        parent[child[inner] + o] = inner
    for node in inner:  # depths, parents first
        depth[child[node]:child[node] + kids] = depth[node] + 1
    leaves = np.flatnonzero(child < 0)
    anc = leaves.copy() if level is not None else parent[leaves].clip(0)
    if level is not None:
        for _ in range(int(depth.max())):
            up = depth[anc] > level
            if not up.any():
                break
            anc = np.where(up, parent[anc], anc)
    groups = np.zeros(grid.n_cells, dtype=np.int64)
    groups[-child[leaves] - 1] = anc
    return groups


def _grouped(a, groups):
    n = int(groups.max()) + 1
    return np.stack([np.bincount(groups, weights=np.asarray(a[l], dtype=np.float64), minlength=n)
                     for l in range(a.shape[0])])


def compare(gpu, ora, problem, min_count=1000, rtol=1e-4, tot_rtol=1e-6, use_records=True, block=8,
            groups=None):
    """The acceptance rule, applied to every channel of every frame and to the
    absorption field (per cell and wavelength, per cell summed over the
    wavelengths, and per group of cells when `groups` is given).  With
    records, the corrections are bounded: at most 1e-4 of the records plus
    10 may be GPU-only or oracle-only, at most 2e-3 plus 10 may be FP32 flips
    (pixel or value), of which at most 1e-4 plus 10 land beyond the
    neighbouring pixel, and every bin that violates the rule before the
    correction must be one the correction changed."""
    rep = {}
    st_g, st_o = gpu["stats"], ora["stats"]
    # emitted, escaped and absorbed relative to themselves; the truncated
    # remainder (a small fraction) relative to the emitted luminosity
    scale = np.array([st_o[0], st_o[1], st_o[2], st_o[0]])
    rep["totals_rel"] = (np.abs(st_g - st_o) / np.abs(scale).clip(1e-300)).tolist()
    img_tot_o = sum(im[0].sum() for im in ora["images"])

    def image_total_rel(images):
        tot = sum(im[0].sum() for im in images)
        return float(abs(tot - img_tot_o) / img_tot_o) if img_tot_o else float(tot != 0)
    rep["image_total_rel"] = image_total_rel(gpu["images"])
    rep["absorption_total_rel"] = float(abs(gpu["absorption"].sum() - ora["absorption"].sum())
                                        / ora["absorption"].sum()) if ora["absorption"].sum() > 0 else 0.0
    rep["conservation_gpu"] = float(abs(st_g[0] - st_g[1] - st_g[2] - st_g[3]) / st_g[0])
    cg, co = gpu["counters"].astype(np.float64), ora["counters"].astype(np.float64)
    rep["crossings_rel"] = float(abs(cg[0] - co[0]) / co[0])
    rep["events_diff"] = int(cg[1] - co[1])
    touched = None
    if use_records:
        imgs, rrep = flip_corrected_images(gpu, ora, problem)
        touched = rrep.pop("touched")
        rep.update(rrep)
        # the image total after the corrections (the uncorrected one stays in
        # image_total_rel_raw): a packet whose path parted moves its later
        # records' values, which the records repair
        rep["image_total_rel_raw"] = rep["image_total_rel"]
        rep["image_total_rel"] = image_total_rel(imgs)
        # records one side lacks: at most 1e-4 of them (plus 10); FP32 flips
        # (pixel or value): at most 2e-3 (plus 10; a packet that interacts
        # close to a cell face flips with the FP32 position, and the clumpy
        # octree's dense, deep leaves give 1.1e-3 of its records), every
        # pixel flip to a neighbouring pixel
        rep["corrections"] = rep["gpu_only"] + rep["oracle_only"]
        rep["corrections_limit"] = 1e-4 * rep["records"] + 10
        rep["flip_total"] = rep["flips"] + rep["value_flips"]
        rep["flip_limit"] = 2e-3 * rep["records"] + 10
        # pixel flips beyond the neighbouring pixel: a packet whose FP32 path
        # parted from the FP64 one (an interaction in a near-empty cell after
        # dense ones moves far for a small optical-depth difference)
        rep["far_flip_limit"] = 1e-4 * rep["records"] + 10
    else:
        imgs = gpu["images"]
    rep["pixels"] = []
    unexplained = 0
    for q, im in enumerate(imgs):
        for ch in range(im.shape[0]):
            counts = ora["image_counts"][q][ch]
            raw = bin_check(gpu["images"][q][ch], ora["images"][q][ch], counts, min_count, rtol)
            cor = bin_check(im[ch], ora["images"][q][ch], counts, min_count, rtol)
            entry = {"instrument": q, "channel": ch, "raw": raw, "corrected": cor}
            if touched is not None:
                entry["raw_unexplained"] = sum(1 for b in raw["violating"] if (ch, int(b)) not in touched[q])
                unexplained += entry["raw_unexplained"]
            for r in (raw, cor):
                r["violating"] = r["violating"][:16].tolist()
            ny, nx = im.shape[-2:]
            if block and ny % block == 0 and nx % block == 0:
                entry["blocks"] = bin_check(block_sum(im[ch], block), block_sum(ora["images"][q][ch], block),
                                            block_sum(counts, block), min_count, rtol)
            rep["pixels"].append(entry)
    rep["raw_unexplained"] = unexplained
    rep["cells"] = bin_check(gpu["absorption"], ora["absorption"], ora["absorption_counts"], min_count, rtol)
    rep["cells_all_lambda"] = bin_check(gpu["absorption"].sum(axis=0), ora["absorption"].sum(axis=0),
                                        ora["absorption_counts"].sum(axis=0), min_count, rtol)
    if groups is not None:
        rep["cell_groups"] = bin_check(_grouped(gpu["absorption"], groups), _grouped(ora["absorption"], groups),
                                       _grouped(ora["absorption_counts"], groups), min_count, rtol)
    for key in ("cells", "cells_all_lambda", "cell_groups"):
        if key not in rep:
            continue
        rep[key]["violating"] = rep[key]["violating"][:16].tolist()
    for p in rep["pixels"]:
        if "blocks" in p:
            p["blocks"]["violating"] = p["blocks"]["violating"][:16].tolist()
    ok = (max(rep["totals_rel"]) <= tot_rtol and rep["image_total_rel"] <= tot_rtol
          and rep["absorption_total_rel"] <= tot_rtol and rep["cells"]["violations"] == 0
          and rep["cells_all_lambda"]["violations"] == 0
          and rep.get("cell_groups", {"violations": 0})["violations"] == 0
          and all(p["corrected"]["violations"] == 0 for p in rep["pixels"])
          and all(p.get("blocks", {"violations": 0})["violations"] == 0 for p in rep["pixels"])
          and unexplained == 0
          and (not use_records or (rep["corrections"] <= rep["corrections_limit"]
                                   and rep["flip_total"] <= rep["flip_limit"]
                                   and rep["far_flips"] <= rep["far_flip_limit"])))
    rep["ok"] = bool(ok)
    return rep


def summary(rep):
    """One line of the counts a parity test checked (for the test log)."""
    px = rep["pixels"]
    return (f"bins: pixels {sum(p['corrected']['bins'] for p in px)} "
            f"(channels {sorted({p['channel'] for p in px})}), blocks {sum(p.get('blocks', {'bins': 0})['bins'] for p in px)}, "
            f"cells {rep['cells']['bins']}, cells over all wavelengths {rep['cells_all_lambda']['bins']}, "
            f"cell groups {rep.get('cell_groups', {'bins': 0})['bins']}; "
            f"records {rep.get('records', 0)}, flips {rep.get('flips', 0)} + value flips {rep.get('value_flips', 0)} "
            f"(limit {rep.get('flip_limit', 0):.0f}, far {rep.get('far_flips', 0)}), gpu-only {rep.get('gpu_only', 0)}, "
            f"oracle-only {rep.get('oracle_only', 0)} (limit {rep.get('corrections_limit', 0):.0f}); "
            f"max rel: pixels {max((p['corrected']['max_rel'] for p in px), default=0):.2e}, "
            f"cells {rep['cells']['max_rel']:.2e}; totals {max(rep['totals_rel']):.2e}")
