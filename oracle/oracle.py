"""Python wrapper around the FP64 CPU oracle (``rt_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
benchmark's CPU-baseline leg.  The CUDA transport library never imports it.

The problem object is duck-typed: any object with the attributes of
``paper_1410_1629_gb300.workloads.Problem`` (grid, kappa, albedo, g, sources,
instruments) works; this module imports nothing from the CUDA package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_rt.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no FMA contraction) and return the .so path.

    ``RT_ORACLE_LIB`` names an already-built library to load instead (used to
    run the pins against deliberately broken builds of the oracle)."""
    override = os.environ.get("RT_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrGrid(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("bounds", ctypes.c_double * 6),
                ("density", ctypes.POINTER(ctypes.c_float)), ("n_nodes", ctypes.c_int64),
                ("child", ctypes.POINTER(ctypes.c_int32)), ("n_leaves", ctypes.c_int64),
                ("edges", ctypes.POINTER(ctypes.c_double) * 3), ("split_axis", ctypes.POINTER(ctypes.c_int8)),
                ("sites", ctypes.POINTER(ctypes.c_double)), ("offsets", ctypes.POINTER(ctypes.c_int64))]


class OrSource(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("center", ctypes.c_double * 3),
                ("scale_r", ctypes.c_double), ("scale_z", ctypes.c_double)]


class OrInstrument(ctypes.Structure):
    _fields_ = [("inclination", ctypes.c_double), ("azimuth", ctypes.c_double),
                ("position_angle", ctypes.c_double), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("half_x", ctypes.c_double), ("half_y", ctypes.c_double),
                ("center_x", ctypes.c_double), ("center_y", ctypes.c_double),
                ("bilinear", ctypes.c_int32), ("channels", ctypes.c_int32), ("sed", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class OrProblem(ctypes.Structure):
    _fields_ = [("grid", OrGrid), ("n_lambda", ctypes.c_int32), ("n_sources", ctypes.c_int32),
                ("n_instr", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("kappa", ctypes.POINTER(ctypes.c_double)), ("albedo", ctypes.POINTER(ctypes.c_double)),
                ("g", ctypes.POINTER(ctypes.c_double)), ("sources", ctypes.POINTER(OrSource)),
                ("lum", ctypes.POINTER(ctypes.c_double)), ("instr", ctypes.POINTER(OrInstrument)),
                ("dust_lum", ctypes.POINTER(ctypes.c_double))]


class OrOpts(ctypes.Structure):
    _fields_ = [("n_per_lambda", ctypes.c_uint64), ("first_id", ctypes.c_uint64),
                ("n_norm", ctypes.c_uint64), ("seed", ctypes.c_uint32), ("model_id", ctypes.c_uint32),
                ("w_min", ctypes.c_double), ("max_events", ctypes.c_int32),
                ("weight_cut", ctypes.c_int32), ("peel_emission", ctypes.c_int32),
                ("peel_scatter", ctypes.c_int32), ("n_threads", ctypes.c_int32), ("pad", ctypes.c_int32)]


class OrRecord(ctypes.Structure):
    _fields_ = [("pid", ctypes.c_uint64), ("lam", ctypes.c_int32), ("event", ctypes.c_int32),
                ("instr", ctypes.c_int32), ("pad", ctypes.c_int32), ("pixel", ctypes.c_int64),
                ("value", ctypes.c_double)]


class OrOutput(ctypes.Structure):
    _fields_ = [("images", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("image_counts", ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))),
                ("absorption", ctypes.POINTER(ctypes.c_double)),
                ("absorption_counts", ctypes.POINTER(ctypes.c_int64)),
                ("stats", ctypes.c_double * 4), ("counters", ctypes.c_uint64 * 4),
                ("records", ctypes.POINTER(OrRecord)), ("records_cap", ctypes.c_int64),
                ("records_n", ctypes.c_int64)]


TRACE_DTYPE = np.dtype([("event", "<i4"), ("pad", "<i4"), ("cell", "<i8"), ("x", "<f8", 3), ("k", "<f8", 3),
                        ("L", "<f8"), ("tau_path", "<f8"), ("tau_star", "<f8")])
RECORD_DTYPE = np.dtype([("pid", "<u8"), ("lam", "<i4"), ("event", "<i4"), ("instr", "<i4"),
                         ("pad", "<i4"), ("pixel", "<i8"), ("value", "<f8")])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            L.or_draw4.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]
            L.or_hg_sample.restype = ctypes.c_double
            L.or_hg_sample.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_hg_phase.restype = ctypes.c_double
            L.or_hg_phase.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_rotate.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_double)]
            L.or_scatter_direction.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_double)]
            L.or_frame.argtypes = [ctypes.POINTER(OrInstrument), ctypes.POINTER(ctypes.c_double)]
            L.or_emit.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(OrOpts), ctypes.c_uint64,
                                  ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
            L.or_path.restype = ctypes.c_int64
            L.or_path.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int64]
            L.or_locate.restype = ctypes.c_int64
            L.or_locate.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.or_run.restype = ctypes.c_int32
            L.or_run.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(OrOpts), ctypes.POINTER(OrOutput)]
            L.or_trace.restype = ctypes.c_int64
            L.or_trace.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(OrOpts), ctypes.c_uint64,
                                   ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64]
            L.or_interaction.restype = ctypes.c_int32
            L.or_interaction.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
            L.or_dust_temperature.restype = ctypes.c_int32
            L.or_dust_temperature.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
            L.or_dust_emission.restype = ctypes.c_int32
            L.or_dust_emission.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double)]
            L.or_vjp.restype = ctypes.c_int32
            L.or_vjp.argtypes = [ctypes.POINTER(OrProblem), ctypes.POINTER(OrOpts),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                 ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
            _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


_SOURCE_KIND = {"point": 0, "expdisk": 1, "plummer": 2}


class _Marshalled:
    """Keeps the numpy buffers referenced by an OrProblem alive."""

    def __init__(self, problem):
        grid = problem.grid
        self.keep = []
        og = OrGrid()
        og.bounds[:] = [float(b) for b in np.asarray(grid.bounds, dtype=np.float64)]
        dens = np.ascontiguousarray(grid.density, dtype=np.float32).ravel()
        self.keep.append(dens)
        og.density = _ptr(dens, ctypes.c_float)
        if grid.kind in ("cartesian", "rectilinear"):
            og.kind = 0 if grid.kind == "cartesian" else 2
            nz, ny, nx = np.asarray(grid.density).shape
            og.nx, og.ny, og.nz = nx, ny, nz
            if grid.kind == "rectilinear":
                for a in range(3):
                    e = np.ascontiguousarray(grid.edges[a], dtype=np.float64)
                    self.keep.append(e)
                    og.edges[a] = _ptr(e, ctypes.c_double)
        elif grid.kind == "voronoi":
            og.kind = 4
            sites = np.ascontiguousarray(grid.sites, dtype=np.float64)
            offsets = np.ascontiguousarray(grid.offsets, dtype=np.int64)
            nbr = np.ascontiguousarray(grid.child, dtype=np.int32)
            self.keep += [sites, offsets, nbr]
            og.sites = _ptr(sites, ctypes.c_double)
            og.offsets = _ptr(offsets, ctypes.c_int64)
            og.child = _ptr(nbr, ctypes.c_int32)
            og.n_nodes = nbr.size
            og.n_leaves = dens.size
        else:
            og.kind = 1 if grid.kind == "octree" else 3
            child = np.ascontiguousarray(grid.child, dtype=np.int32)
            self.keep.append(child)
            og.child = _ptr(child, ctypes.c_int32)
            og.n_nodes = child.size
            og.n_leaves = dens.size
            if grid.kind == "bintree":
                axis = np.ascontiguousarray(grid.split_axis, dtype=np.int8)
                self.keep.append(axis)
                og.split_axis = _ptr(axis, ctypes.c_int8)
        nl = len(problem.kappa)
        kappa = np.ascontiguousarray(problem.kappa, dtype=np.float64)
        albedo = np.ascontiguousarray(problem.albedo, dtype=np.float64)
        g = np.ascontiguousarray(problem.g, dtype=np.float64)
        srcs = (OrSource * len(problem.sources))()
        lum = np.zeros((len(problem.sources), nl), dtype=np.float64)
        for i, s in enumerate(problem.sources):
            srcs[i].kind = _SOURCE_KIND[s.kind]
            srcs[i].center[:] = [float(c) for c in s.center]
            srcs[i].scale_r = float(s.scale_r)
            srcs[i].scale_z = float(s.scale_z)
            lum[i] = np.asarray(s.lum, dtype=np.float64)
        instr = (OrInstrument * max(1, len(problem.instruments)))()
        for i, q in enumerate(problem.instruments):
            instr[i] = make_instrument(q)
        self.keep += [kappa, albedo, g, lum, srcs, instr]
        p = OrProblem()
        p.grid = og
        p.n_lambda = nl
        p.n_sources = len(problem.sources)
        p.n_instr = len(problem.instruments)
        p.kappa = _ptr(kappa, ctypes.c_double)
        p.albedo = _ptr(albedo, ctypes.c_double)
        p.g = _ptr(g, ctypes.c_double)
        p.sources = srcs
        p.lum = _ptr(lum, ctypes.c_double)
        p.instr = instr
        dust = getattr(problem, "dust_lum", None)
        if dust is not None:
            dl = np.ascontiguousarray(dust, dtype=np.float64).reshape(nl, dens.size)
            self.keep.append(dl)
            p.dust_lum = _ptr(dl, ctypes.c_double)
        self.problem = p
        self.n_lambda = nl
        self.n_cells = dens.size


def make_instrument(q) -> OrInstrument:
    oi = OrInstrument()
    oi.inclination = float(q.inclination)
    oi.azimuth = float(q.azimuth)
    oi.position_angle = float(q.position_angle)
    oi.nx, oi.ny = int(q.nx), int(q.ny)
    oi.half_x, oi.half_y = float(q.half_x), float(q.half_y)
    oi.center_x, oi.center_y = float(q.center_x), float(q.center_y)
    oi.bilinear = int(bool(q.bilinear))
    oi.channels = int(q.channels)
    oi.sed = int(bool(getattr(q, "sed", False)))
    return oi


def _opts(n_per_lambda, first_id, n_norm, seed, model_id, w_min, max_events, weight_cut,
          peel_emission, peel_scatter, n_threads) -> OrOpts:
    o = OrOpts()
    o.n_per_lambda = int(n_per_lambda)
    o.first_id = int(first_id)
    o.n_norm = int(n_norm if n_norm is not None else n_per_lambda)
    o.seed = int(seed)
    o.model_id = int(model_id)
    o.w_min = float(w_min)
    o.max_events = int(max_events)
    o.weight_cut = int(bool(weight_cut))
    o.peel_emission = int(bool(peel_emission))
    o.peel_scatter = int(bool(peel_scatter))
    o.n_threads = int(n_threads)
    return o


def run(problem, n_per_lambda, first_id=0, seed=0, model_id=0, n_norm=None, w_min=1e-4,
        max_events=1000, weight_cut=True, peel_emission=True, peel_scatter=True, n_threads=1,
        absorption=True, counts=False, records_cap=0):
    """Run the oracle.  Returns a dict with images (list of [ch, nl, ny, nx]),
    absorption [nl, n_cells], stats (emitted, escaped, absorbed, truncated),
    counters (crossings, events, peeloffs, packets), optional counts and records."""
    L = lib()
    m = _Marshalled(problem)
    o = _opts(n_per_lambda, first_id, n_norm, seed, model_id, w_min, max_events, weight_cut,
              peel_emission, peel_scatter, n_threads)
    nl = m.n_lambda
    images = [np.zeros((q.channels, nl, q.ny, q.nx), dtype=np.float64) for q in problem.instruments]
    img_ptrs = (ctypes.POINTER(ctypes.c_double) * max(1, len(images)))(*[_ptr(a, ctypes.c_double) for a in images])
    out = OrOutput()
    out.images = img_ptrs
    result = {"images": images}
    if counts:
        icounts = [np.zeros(a.shape, dtype=np.int64) for a in images]
        cptrs = (ctypes.POINTER(ctypes.c_int64) * max(1, len(icounts)))(*[_ptr(a, ctypes.c_int64) for a in icounts])
        out.image_counts = cptrs
        result["image_counts"] = icounts
    if absorption:
        ab = np.zeros((nl, m.n_cells), dtype=np.float64)
        out.absorption = _ptr(ab, ctypes.c_double)
        result["absorption"] = ab
        if counts:
            ac = np.zeros((nl, m.n_cells), dtype=np.int64)
            out.absorption_counts = _ptr(ac, ctypes.c_int64)
            result["absorption_counts"] = ac
    if records_cap:
        recs = np.zeros(int(records_cap), dtype=RECORD_DTYPE)
        out.records = recs.ctypes.data_as(ctypes.POINTER(OrRecord))
        out.records_cap = int(records_cap)
    rc = L.or_run(ctypes.byref(m.problem), ctypes.byref(o), ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"or_run failed with status {rc}")
    result["stats"] = np.array(out.stats[:], dtype=np.float64)
    result["counters"] = np.array(out.counters[:], dtype=np.uint64)
    if records_cap:
        n = min(int(out.records_n), int(records_cap))
        result["records"] = recs[:n].copy()
        result["records_total"] = int(out.records_n)
    return result


def vjp(problem, cells, n_per_lambda, adj_images=None, adj_absorption=None, first_id=0, seed=0,
        model_id=0, n_norm=None, w_min=1e-4, max_events=1000, weight_cut=True, peel_emission=True,
        peel_scatter=True, n_threads=1):
    """sum_bins adj[bin] * d(bin)/d(rho[c]) for each c in ``cells`` (forward-mode dual numbers)."""
    L = lib()
    m = _Marshalled(problem)
    o = _opts(n_per_lambda, first_id, n_norm, seed, model_id, w_min, max_events, weight_cut,
              peel_emission, peel_scatter, n_threads)
    keep = []
    adj_ptrs = None
    if adj_images is not None:
        arrs = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None for a in adj_images]
        keep += arrs
        adj_ptrs = (ctypes.POINTER(ctypes.c_double) * len(arrs))(
            *[(_ptr(a, ctypes.c_double) if a is not None else ctypes.POINTER(ctypes.c_double)()) for a in arrs])
    adj_abs = None
    if adj_absorption is not None:
        adj_abs = np.ascontiguousarray(adj_absorption, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    grad = np.zeros(cells.size, dtype=np.float64)
    rc = L.or_vjp(ctypes.byref(m.problem), ctypes.byref(o), adj_ptrs,
                  _ptr(adj_abs, ctypes.c_double) if adj_abs is not None else None,
                  _ptr(cells, ctypes.c_int64), cells.size, _ptr(grad, ctypes.c_double))
    if rc != 0:
        raise ValueError(f"or_vjp failed with status {rc}")
    return grad


def trace(problem, pid, lam=0, seed=0, model_id=0, n_norm=1, w_min=1e-4, max_events=1000, weight_cut=True,
          peel_emission=True, peel_scatter=True):
    """Per-event state (position, direction, cell, weight, tau_path, tau*) of one packet."""
    m = _Marshalled(problem)
    o = _opts(1, 0, n_norm, seed, model_id, w_min, max_events, weight_cut, peel_emission, peel_scatter, 1)
    rows = np.zeros(max_events + 2, dtype=TRACE_DTYPE)
    n = lib().or_trace(ctypes.byref(m.problem), ctypes.byref(o), int(pid), int(lam), rows.ctypes.data, rows.size)
    return rows[:min(n, rows.size)].copy()


# ---------------------------------------------------------------- unit entry points
def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def draw4(pid, lam, event, block, seed=0, model=0):
    o = (ctypes.c_double * 4)()
    lib().or_draw4(pid, lam, event, block, seed, model, o)
    return np.array(o[:])


def hg_sample(g, u):
    return lib().or_hg_sample(float(g), float(u))


def hg_phase(g, mu):
    return lib().or_hg_phase(float(g), float(mu))


def rotate(k, mu, phi):
    kk = (ctypes.c_double * 3)(*[float(v) for v in k])
    o = (ctypes.c_double * 3)()
    lib().or_rotate(kk, float(mu), float(phi), o)
    return np.array(o[:])


def scatter_direction(k, g, u1, u2):
    kk = (ctypes.c_double * 3)(*[float(v) for v in k])
    o = (ctypes.c_double * 3)()
    lib().or_scatter_direction(kk, float(g), float(u1), float(u2), o)
    return np.array(o[:])


def frame(instrument):
    oi = make_instrument(instrument)
    o = (ctypes.c_double * 9)()
    lib().or_frame(ctypes.byref(oi), o)
    a = np.array(o[:])
    return a[0:3], a[3:6], a[6:9]


def emit(problem, pid, lam, seed=0, model_id=0):
    m = _Marshalled(problem)
    o = _opts(1, 0, 1, seed, model_id, 1e-4, 1000, True, True, True, 1)
    x = (ctypes.c_double * 3)()
    k = (ctypes.c_double * 3)()
    lib().or_emit(ctypes.byref(m.problem), ctypes.byref(o), int(pid), int(lam), x, k)
    return np.array(x[:]), np.array(k[:])


def path(problem, x, k, start_cell=-1, cap=1 << 16):
    m = _Marshalled(problem)
    xx = (ctypes.c_double * 3)(*[float(v) for v in x])
    kk = (ctypes.c_double * 3)(*[float(v) for v in k])
    cells = np.zeros(cap, dtype=np.int64)
    s_in = np.zeros(cap, dtype=np.float64)
    s_out = np.zeros(cap, dtype=np.float64)
    n = lib().or_path(ctypes.byref(m.problem), xx, kk, int(start_cell), _ptr(cells, ctypes.c_int64),
                      _ptr(s_in, ctypes.c_double), _ptr(s_out, ctypes.c_double), cap)
    n = min(n, cap)
    return cells[:n].copy(), s_in[:n].copy(), s_out[:n].copy()


def locate(problem, p, k=(1.0, 1.0, 1.0)):
    m = _Marshalled(problem)
    pp = (ctypes.c_double * 3)(*[float(v) for v in p])
    kk = (ctypes.c_double * 3)(*[float(v) for v in k])
    box = (ctypes.c_double * 6)()
    c = lib().or_locate(ctypes.byref(m.problem), pp, kk, box)
    return int(c), np.array(box[:])


def default_threads() -> int:
    return os.cpu_count() or 1


def interaction(problem, x, k, u, lam=0, start_cell=-1):
    """One forced path from x along k and its interaction for the uniform u
    (steps a and c): returns (x_interaction, cell, tau_path, tau_star, flags),
    flags bit 0 = the inversion's rounding fallback acted, bit 1 = the point
    was moved into the interaction cell, bit 2 = no dust on the path."""
    m = _Marshalled(problem)
    xx = (ctypes.c_double * 3)(*[float(v) for v in x])
    kk = (ctypes.c_double * 3)(*[float(v) for v in k])
    ox = (ctypes.c_double * 3)()
    oc = ctypes.c_int64(-1)
    ot = (ctypes.c_double * 2)()
    f = lib().or_interaction(ctypes.byref(m.problem), xx, kk, int(start_cell), int(lam), float(u), ox,
                             ctypes.byref(oc), ot)
    return np.array(ox[:]), int(oc.value), float(ot[0]), float(ot[1]), int(f)


def dust_temperature(problem, absorption, scale, t_min=1.0, t_max=1e4):
    """Equilibrium dust temperature per cell from the absorbed luminosity
    [n_lambda, n_cells] (panchromatic mode).  Returns (T [n_cells], cells
    held at t_min or t_max)."""
    m = _Marshalled(problem)
    lam = np.ascontiguousarray(problem.wavelengths, dtype=np.float64)
    ab = np.ascontiguousarray(absorption, dtype=np.float64)
    T = np.zeros(m.n_cells, dtype=np.float64)
    rc = lib().or_dust_temperature(ctypes.byref(m.problem), _ptr(lam, ctypes.c_double), _ptr(ab, ctypes.c_double),
                                   float(scale), float(t_min), float(t_max), _ptr(T, ctypes.c_double))
    if rc < 0:
        raise ValueError("or_dust_temperature: bad arguments")
    return T, int(rc)


def dust_emission(problem, T, scale):
    """Thermal emission [n_lambda, n_cells] of the cells at temperatures T."""
    m = _Marshalled(problem)
    lam = np.ascontiguousarray(problem.wavelengths, dtype=np.float64)
    TT = np.ascontiguousarray(T, dtype=np.float64)
    out = np.zeros((m.n_lambda, m.n_cells), dtype=np.float64)
    rc = lib().or_dust_emission(ctypes.byref(m.problem), _ptr(lam, ctypes.c_double), _ptr(TT, ctypes.c_double),
                                float(scale), _ptr(out, ctypes.c_double))
    if rc < 0:
        raise ValueError("or_dust_emission: bad arguments")
    return out
