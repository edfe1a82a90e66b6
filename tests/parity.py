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


def flip_corrected_images(gpu, ora, problem):
    """GPU total-channel images with every contribution whose pixel differs from
    the oracle's moved to the oracle's pixel.  Returns (images, report)."""
    g, o = gpu["records"], ora["records"]
    assert gpu["records_total"] == len(g) and ora["records_total"] == len(o), "record buffer overflow"
    kg, ko = _keys(g), _keys(o)
    assert len(np.unique(kg)) == len(kg) and len(np.unique(ko)) == len(ko)
    common, ig, io = np.intersect1d(kg, ko, return_indices=True)
    flip = g["pixel"][ig] != o["pixel"][io]
    only_g = np.setdiff1d(np.arange(len(g)), ig)
    only_o = np.setdiff1d(np.arange(len(o)), io)
    imgs = [im[0].copy() for im in gpu["images"]]  # total channel [n_lambda, ny, nx]
    for sel_g, sel_o in ((ig[flip], io[flip]),):
        for a, b in zip(sel_g, sel_o):
            q, lam = g["instr"][a], g["lam"][a]
            im = imgs[q][lam].reshape(-1)
            im[g["pixel"][a]] -= g["value"][a]
            im[o["pixel"][b]] += g["value"][a]
    for a in only_g:
        imgs[g["instr"][a]][g["lam"][a]].reshape(-1)[g["pixel"][a]] -= g["value"][a]
    for b in only_o:
        imgs[o["instr"][b]][o["lam"][b]].reshape(-1)[o["pixel"][b]] += o["value"][b]
    rel = np.abs(g["value"][ig] - o["value"][io]) / np.maximum(np.abs(o["value"][io]), 1e-300)
    worst = np.argsort(rel)[::-1][:3]
    report = {"worst_records": [{"pid": int(o["pid"][io[w]]), "lam": int(o["lam"][io[w]]),
                                 "event": int(o["event"][io[w]]), "instr": int(o["instr"][io[w]]),
                                 "gpu": float(g["value"][ig[w]]), "oracle": float(o["value"][io[w]])}
                                for w in worst if rel[w] > 1e-3],
              "records": int(len(o)), "flips": int(flip.sum()), "gpu_only": int(len(only_g)),
              "oracle_only": int(len(only_o)), "record_rel_p999": float(np.quantile(rel, 0.999)) if len(rel) else 0.0,
              "record_rel_max": float(rel.max()) if len(rel) else 0.0}
    return imgs, report


def bin_check(gpu_vals, ora_vals, counts, min_count=1000, rtol=1e-4):
    mask = counts >= min_count
    diff = np.abs(gpu_vals[mask] - ora_vals[mask])
    rel = np.where(diff == 0, 0.0, diff / np.maximum(np.abs(ora_vals[mask]), 1e-300))
    return {"bins": int(mask.sum()), "violations": int((rel > rtol).sum()),
            "max_rel": float(rel.max()) if rel.size else 0.0}


def block_sum(a, b):
    """Sum over b x b pixel blocks of the last two axes."""
    ny, nx = a.shape[-2:]
    return a.reshape(a.shape[:-2] + (ny // b, b, nx // b, b)).sum(axis=(-3, -1))


def compare(gpu, ora, problem, min_count=1000, rtol=1e-4, tot_rtol=1e-6, use_records=True, block=8):
    rep = {}
    st_g, st_o = gpu["stats"], ora["stats"]
    # emitted, escaped and absorbed relative to themselves; the truncated
    # remainder (a small fraction) relative to the emitted luminosity
    scale = np.array([st_o[0], st_o[1], st_o[2], st_o[0]])
    rep["totals_rel"] = (np.abs(st_g - st_o) / np.abs(scale).clip(1e-300)).tolist()
    img_tot_g = sum(im[0].sum() for im in gpu["images"])
    img_tot_o = sum(im[0].sum() for im in ora["images"])
    rep["image_total_rel"] = float(abs(img_tot_g - img_tot_o) / img_tot_o)
    rep["absorption_total_rel"] = float(abs(gpu["absorption"].sum() - ora["absorption"].sum())
                                        / ora["absorption"].sum()) if ora["absorption"].sum() > 0 else 0.0
    rep["conservation_gpu"] = float(abs(st_g[0] - st_g[1] - st_g[2] - st_g[3]) / st_g[0])
    cg, co = gpu["counters"].astype(np.float64), ora["counters"].astype(np.float64)
    rep["crossings_rel"] = float(abs(cg[0] - co[0]) / co[0])
    rep["events_diff"] = int(cg[1] - co[1])
    if use_records:
        imgs, rrep = flip_corrected_images(gpu, ora, problem)
        rep.update(rrep)
    else:
        imgs = [im[0] for im in gpu["images"]]
    rep["pixels"] = []
    for q, im in enumerate(imgs):
        raw = bin_check(gpu["images"][q][0], ora["images"][q][0], ora["image_counts"][q][0], min_count, rtol)
        cor = bin_check(im, ora["images"][q][0], ora["image_counts"][q][0], min_count, rtol)
        entry = {"raw": raw, "corrected": cor}
        ny, nx = im.shape[-2:]
        if block and ny % block == 0 and nx % block == 0:
            entry["blocks"] = bin_check(block_sum(im, block), block_sum(ora["images"][q][0], block),
                                        block_sum(ora["image_counts"][q][0], block), min_count, rtol)
        rep["pixels"].append(entry)
    rep["cells"] = bin_check(gpu["absorption"], ora["absorption"], ora["absorption_counts"], min_count, rtol)
    ok = (max(rep["totals_rel"]) <= tot_rtol and rep["image_total_rel"] <= tot_rtol
          and rep["absorption_total_rel"] <= tot_rtol and rep["cells"]["violations"] == 0
          and all(p["corrected"]["violations"] == 0 for p in rep["pixels"])
          and all(p.get("blocks", {"violations": 0})["violations"] == 0 for p in rep["pixels"]))
    rep["ok"] = bool(ok)
    return rep
