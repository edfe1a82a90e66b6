"""Thin ctypes binding of the C ABI in ``include/rt.h`` (``librt_gb300.so``).

Every function here has the name of the C function it wraps and only
marshals arguments: all transport work runs in the library's CUDA kernels.
A non-zero status raises :class:`RTError` with the library's message.  If the
library is missing and cannot be built, :func:`lib` raises: there is no CPU
fallback.

PyTorch is used for device memory (output tensors) and streams
(``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

RT_OK, RT_ERR_ARG, RT_ERR_STATE, RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_TIMEOUT, RT_ERR_DEVICE_FLAG = 0, -1, -2, -3, -4, -5, -6
RT_GRID_CARTESIAN, RT_GRID_OCTREE, RT_GRID_RECTILINEAR, RT_GRID_BINTREE, RT_GRID_VORONOI = 0, 1, 2, 3, 4
RT_SOURCE_POINT, RT_SOURCE_EXPDISK, RT_SOURCE_PLUMMER = 0, 1, 2
RT_DEPOSIT_NEAREST, RT_DEPOSIT_BILINEAR, RT_DEPOSIT_SED = 0, 1, 2
RT_LAYOUT_AUTO, RT_LAYOUT_ROW_MAJOR = 0, 1
RT_EMITTER_SOURCES, RT_EMITTER_DUST = 0, 1
TRACE_DTYPE = np.dtype([("event", "<i4"), ("reserved", "<i4"), ("cell", "<i8"), ("x", "<f8", 3), ("k", "<f8", 3),
                        ("L", "<f8"), ("tau_path", "<f8"), ("tau_star", "<f8")])

_SOURCE_KIND = {"point": RT_SOURCE_POINT, "expdisk": RT_SOURCE_EXPDISK, "plummer": RT_SOURCE_PLUMMER}


class RTError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"rt status {status}: {message}")
        self.status = status


class rt_grid_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("bounds", ctypes.c_double * 6), ("density", ctypes.c_void_p), ("n_nodes", ctypes.c_int64),
                ("child", ctypes.c_void_p), ("n_leaves", ctypes.c_int64), ("on_device", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("edges", ctypes.c_void_p * 3), ("split_axis", ctypes.c_void_p),
                ("sites", ctypes.c_void_p), ("offsets", ctypes.c_void_p)]


class rt_source_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("center", ctypes.c_double * 3),
                ("scale_r", ctypes.c_double), ("scale_z", ctypes.c_double),
                ("luminosity", ctypes.POINTER(ctypes.c_double))]


class rt_instrument_desc(ctypes.Structure):
    _fields_ = [("inclination", ctypes.c_double), ("azimuth", ctypes.c_double), ("position_angle", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("half_x", ctypes.c_double),
                ("half_y", ctypes.c_double), ("center_x", ctypes.c_double), ("center_y", ctypes.c_double),
                ("deposit", ctypes.c_int32), ("channels", ctypes.c_int32)]


class rt_record(ctypes.Structure):
    _fields_ = [("packet", ctypes.c_uint64), ("lambda_", ctypes.c_int32), ("event", ctypes.c_int32),
                ("instrument", ctypes.c_int32), ("reserved", ctypes.c_int32), ("pixel", ctypes.c_int64),
                ("value", ctypes.c_double)]


RECORD_DTYPE = np.dtype([("pid", "<u8"), ("lam", "<i4"), ("event", "<i4"), ("instr", "<i4"),
                         ("pad", "<i4"), ("pixel", "<i8"), ("value", "<f8")])


class rt_trace_row(ctypes.Structure):
    _fields_ = [("event", ctypes.c_int32), ("reserved", ctypes.c_int32), ("cell", ctypes.c_int64),
                ("x", ctypes.c_double * 3), ("k", ctypes.c_double * 3), ("L", ctypes.c_double),
                ("tau_path", ctypes.c_double), ("tau_star", ctypes.c_double)]


TRACE_DTYPE = np.dtype([("event", "<i4"), ("pad", "<i4"), ("cell", "<i8"), ("x", "<f8", 3), ("k", "<f8", 3),
                        ("L", "<f8"), ("tau_path", "<f8"), ("tau_star", "<f8")])


class rt_launch_opts(ctypes.Structure):
    _fields_ = [("w_min", ctypes.c_double), ("max_events", ctypes.c_int32), ("weight_cut", ctypes.c_int32),
                ("peel_emission", ctypes.c_int32), ("peel_scatter", ctypes.c_int32), ("n_norm", ctypes.c_uint64),
                ("model_id", ctypes.c_uint32), ("walk_peels", ctypes.c_int32), ("records", ctypes.c_void_p),
                ("records_capacity", ctypes.c_int64), ("record_stride", ctypes.c_uint64),
                ("trace", ctypes.c_void_p), ("trace_capacity", ctypes.c_int64), ("trace_packet", ctypes.c_uint64),
                ("trace_lambda", ctypes.c_int32), ("control_lanes", ctypes.c_int32),
                ("profile", ctypes.c_void_p), ("tape", ctypes.c_int32), ("inline_peels", ctypes.c_int32),
                ("time_parts", ctypes.c_int32), ("emitter", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class rt_stats(ctypes.Structure):
    _fields_ = [("emitted", ctypes.c_double), ("escaped", ctypes.c_double), ("absorbed", ctypes.c_double),
                ("truncated", ctypes.c_double), ("crossings", ctypes.c_uint64), ("path_crossings", ctypes.c_uint64), ("events", ctypes.c_uint64),
                ("peeloffs", ctypes.c_uint64), ("packets", ctypes.c_uint64), ("records", ctypes.c_uint64),
                ("column_peels", ctypes.c_uint64), ("column_crossings", ctypes.c_uint64),
                ("sorted_peels", ctypes.c_uint64), ("device_flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class rt_model_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("bounds", ctypes.c_double * 6), ("density", ctypes.c_void_p), ("kappa", ctypes.c_double),
                ("albedo", ctypes.c_double), ("g", ctypes.c_double), ("luminosity", ctypes.c_double),
                ("source", ctypes.c_double * 3), ("instrument", rt_instrument_desc), ("n_packets", ctypes.c_uint64)]


# name -> (restype, argtypes): the exported symbols of include/rt.h
SIGNATURES = {
    "rt_version": (ctypes.c_char_p, []),
    "rt_context_create": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "rt_context_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "rt_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "rt_default_opts": (None, [ctypes.POINTER(rt_launch_opts)]),
    "rt_create_grid": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(rt_grid_desc), ctypes.POINTER(ctypes.c_int32)]),
    "rt_set_optics": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 4),
    "rt_add_sources": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(rt_source_desc)]),
    "rt_add_instruments": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(rt_instrument_desc),
                                            ctypes.POINTER(ctypes.c_int32)]),
    "rt_launch_packets": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.POINTER(rt_launch_opts), ctypes.c_void_p]),
    "rt_reset_tallies": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p]),
    "rt_adjoint_tune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(rt_launch_opts),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "rt_tune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(rt_launch_opts),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "rt_tuned": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "rt_read_absorption": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32,
                                            ctypes.c_void_p]),
    "rt_read_images": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_int32, ctypes.c_void_p]),
    "rt_read_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(rt_stats)]),
    "rt_synchronize": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p]),
    "rt_read_launch_times": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "rt_update_density": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "rt_adjoint": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(rt_launch_opts),
                                    ctypes.c_void_p]),
    "rt_launch_packets_noalloc": (ctypes.c_int32, [ctypes.POINTER(rt_grid_desc), ctypes.c_int32, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                   ctypes.POINTER(rt_source_desc), ctypes.c_int32,
                                                   ctypes.POINTER(rt_instrument_desc), ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                                   ctypes.POINTER(rt_launch_opts), ctypes.c_void_p, ctypes.c_void_p]),
    "rt_batch_create": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(rt_model_desc),
                                         ctypes.POINTER(ctypes.c_int32)]),
    "rt_batch_destroy": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "rt_batch_launch": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(rt_launch_opts),
                                         ctypes.c_void_p]),
    "rt_batch_reset": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "rt_batch_read_images": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                              ctypes.c_int32, ctypes.c_void_p]),
    "rt_batch_read_tallies": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                               ctypes.c_int32, ctypes.c_void_p]),
    "rt_batch_read_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(rt_stats)]),
    "rt_batch_tune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint32), ctypes.c_void_p]),
    "rt_probe_bandwidth": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_double)]),
    "rt_dust_temperature": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "rt_set_dust_emission": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_void_p]),
    "rt_read_dust_emission": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32,
                                               ctypes.c_void_p]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB_PATH


def lib():
    """Load librt_gb300.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_PATH
            if not _build.up_to_date():
                try:
                    path = _build.build()
                except Exception as exc:  # no toolkit: the extension does not exist
                    raise RuntimeError(f"librt_gb300.so is not built and cannot be built: {exc}") from exc
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(ctx, status):
    if status != RT_OK:
        msg = lib().rt_last_error(ctx)
        raise RTError(status, msg.decode() if msg else "")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- C functions
def rt_version() -> str:
    return lib().rt_version().decode()


def rt_context_create(device: int = 0):
    h = ctypes.c_void_p()
    st = lib().rt_context_create(int(device), ctypes.byref(h))
    if st != RT_OK:
        raise RTError(st, lib().rt_last_error(None).decode())
    return h


def rt_context_destroy(ctx):
    lib().rt_context_destroy(ctx)


def rt_last_error(ctx) -> str:
    return lib().rt_last_error(ctx).decode()


def rt_default_opts() -> rt_launch_opts:
    o = rt_launch_opts()
    lib().rt_default_opts(ctypes.byref(o))
    return o


def rt_create_grid(ctx, desc: rt_grid_desc) -> int:
    gid = ctypes.c_int32()
    _check(ctx, lib().rt_create_grid(ctx, ctypes.byref(desc), ctypes.byref(gid)))
    return gid.value


def rt_set_optics(ctx, grid_id, kappa, albedo, g, wavelengths=None):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (kappa, albedo, g)]
    wl = np.ascontiguousarray(wavelengths, dtype=np.float64) if wavelengths is not None else None
    n = arrs[0].size
    _check(ctx, lib().rt_set_optics(ctx, int(grid_id), n, wl.ctypes.data if wl is not None else None,
                                    arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data))


def rt_add_sources(ctx, descs, luminosities):
    n = len(descs)
    arr = (rt_source_desc * max(1, n))()
    keep = []
    for i, (d, lum) in enumerate(zip(descs, luminosities)):
        la = np.ascontiguousarray(lum, dtype=np.float64)
        keep.append(la)
        d.luminosity = la.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i] = d
    _check(ctx, lib().rt_add_sources(ctx, n, arr))


def rt_add_instruments(ctx, descs):
    n = len(descs)
    arr = (rt_instrument_desc * max(1, n))(*descs)
    ids = (ctypes.c_int32 * max(1, n))()
    _check(ctx, lib().rt_add_instruments(ctx, n, arr, ids))
    return list(ids[:n])


def rt_launch_packets(ctx, n_per_lambda, first_packet_id=0, seed=0, opts=None, stream=None):
    o = opts if opts is not None else rt_default_opts()
    _check(ctx, lib().rt_launch_packets(ctx, int(n_per_lambda), int(first_packet_id), int(seed), ctypes.byref(o),
                                        _stream_ptr(stream)))


def rt_tune(ctx, n_per_lambda, seed=0, opts=None, stream=None) -> int:
    o = opts if opts is not None else rt_default_opts()
    lanes = ctypes.c_int32()
    _check(ctx, lib().rt_tune(ctx, int(n_per_lambda), int(seed), ctypes.byref(o), ctypes.byref(lanes),
                              _stream_ptr(stream)))
    return lanes.value


def rt_tuned(ctx):
    """(control_lanes, blocks_per_sm) that untuned-field launches use (blocks 0: as many as fit)."""
    lanes, blocks = ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, lib().rt_tuned(ctx, ctypes.byref(lanes), ctypes.byref(blocks)))
    return lanes.value, blocks.value


def rt_reset_tallies(ctx, stream=None):
    _check(ctx, lib().rt_reset_tallies(ctx, _stream_ptr(stream)))


def rt_read_absorption(ctx, dst_ptr, n_elems, on_device, stream=None):
    _check(ctx, lib().rt_read_absorption(ctx, dst_ptr, int(n_elems), int(on_device), _stream_ptr(stream)))


def rt_read_images(ctx, instrument_id, dst_ptr, n_elems, on_device, stream=None):
    _check(ctx, lib().rt_read_images(ctx, int(instrument_id), dst_ptr, int(n_elems), int(on_device),
                                     _stream_ptr(stream)))


def rt_read_stats(ctx) -> rt_stats:
    s = rt_stats()
    _check(ctx, lib().rt_read_stats(ctx, ctypes.byref(s)))
    return s


LAUNCH_PARTS = ("column_sums", "transport", "peel_order", "peel_walks")


def rt_read_launch_times(ctx) -> dict:
    """Milliseconds per part of the last launch made with time_parts=1."""
    ms = (ctypes.c_float * 4)()
    _check(ctx, lib().rt_read_launch_times(ctx, ms, 4))
    return dict(zip(LAUNCH_PARTS, (float(v) for v in ms)))


def rt_synchronize(ctx, stream=None):
    _check(ctx, lib().rt_synchronize(ctx, _stream_ptr(stream)))


def rt_update_density(ctx, density_ptr, on_device, stream=None):
    _check(ctx, lib().rt_update_density(ctx, int(density_ptr), int(on_device), _stream_ptr(stream)))


def rt_adjoint(ctx, adj_image_ptrs, adj_absorption_ptr, grad_ptr, n_per_lambda, first_packet_id=0, seed=0,
               opts=None, stream=None):
    """Accumulate into grad (device float64 [n_cells]) the gradient of
    sum(adj_images * images) + sum(adj_absorption * absorption) w.r.t. the
    cell densities.  adj_image_ptrs: device addresses (or None) per instrument."""
    ptrs = [int(p) if p else 0 for p in (adj_image_ptrs or [])]
    arr = (ctypes.c_void_p * max(1, len(ptrs)))(*[p or None for p in ptrs])
    o = opts if opts is not None else rt_default_opts()
    _check(ctx, lib().rt_adjoint(ctx, arr, len(ptrs), int(adj_absorption_ptr) if adj_absorption_ptr else None,
                                 int(grad_ptr), int(n_per_lambda), int(first_packet_id), int(seed), ctypes.byref(o),
                                 _stream_ptr(stream)))


def rt_adjoint_tune(ctx, adj_image_ptrs, adj_absorption_ptr, n_per_lambda, seed=0, opts=None, stream=None) -> int:
    ptrs = [int(p) if p else 0 for p in (adj_image_ptrs or [])]
    arr = (ctypes.c_void_p * max(1, len(ptrs)))(*[p or None for p in ptrs])
    o = opts if opts is not None else rt_default_opts()
    lanes = ctypes.c_int32()
    _check(ctx, lib().rt_adjoint_tune(ctx, arr, len(ptrs), int(adj_absorption_ptr) if adj_absorption_ptr else None,
                                      int(n_per_lambda), int(seed), ctypes.byref(o), ctypes.byref(lanes),
                                      _stream_ptr(stream)))
    return lanes.value


def rt_launch_packets_noalloc(grid_desc_, kappa, albedo, g, sources, luminosities, instruments, image_ptrs,
                              absorption_ptr, n_per_lambda, first_packet_id=0, seed=0, opts=None, stats_ptr=None,
                              stream=None):
    """Forward transport without device allocation: every device buffer
    (grid density, images, absorption, optional rt_stats output) comes from
    the caller as a device address."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (kappa, albedo, g)]
    n_src = len(sources)
    src = (rt_source_desc * max(1, n_src))()
    keep = []
    for i, (d, lum) in enumerate(zip(sources, luminosities)):
        la = np.ascontiguousarray(lum, dtype=np.float64)
        keep.append(la)
        d.luminosity = la.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        src[i] = d
    n_ins = len(instruments)
    ins = (rt_instrument_desc * max(1, n_ins))(*instruments)
    imgs = (ctypes.c_void_p * max(1, n_ins))(*[int(p) for p in image_ptrs])
    o = opts if opts is not None else rt_default_opts()
    st = lib().rt_launch_packets_noalloc(ctypes.byref(grid_desc_), arrs[0].size, arrs[0].ctypes.data,
                                         arrs[1].ctypes.data, arrs[2].ctypes.data, n_src, src, n_ins, ins, imgs,
                                         int(absorption_ptr), int(n_per_lambda), int(first_packet_id), int(seed),
                                         ctypes.byref(o), stats_ptr, _stream_ptr(stream))
    if st != RT_OK:
        raise RTError(st, lib().rt_last_error(None).decode())


def rt_probe_bandwidth(device=0, nbytes=32 << 20, passes=20, repeats=5) -> float:
    """Read bandwidth in GB/s of a buffer of `nbytes` (L2 if it fits)."""
    out = ctypes.c_double(0.0)
    st = lib().rt_probe_bandwidth(int(device), int(nbytes), int(passes), int(repeats), ctypes.byref(out))
    if st != RT_OK:
        raise RTError(st, lib().rt_last_error(None).decode())
    return out.value


def rt_dust_temperature(ctx, emission_scale, t_min=1.0, t_max=1e4, absorption_ptr=0, absorption_on_device=0,
                        dst_ptr=0, dst_on_device=0, stream=None) -> int:
    """Equilibrium dust temperatures into dst_ptr; returns the cells held at t_max."""
    n = ctypes.c_int32(0)
    _check(ctx, lib().rt_dust_temperature(ctx, float(emission_scale), float(t_min), float(t_max),
                                          ctypes.c_void_p(int(absorption_ptr) or None), int(absorption_on_device),
                                          ctypes.c_void_p(int(dst_ptr)), int(dst_on_device), ctypes.byref(n),
                                          _stream_ptr(stream)))
    return n.value


def rt_set_dust_emission(ctx, temperature_ptr, on_device, emission_scale, stream=None):
    _check(ctx, lib().rt_set_dust_emission(ctx, ctypes.c_void_p(int(temperature_ptr)), int(on_device),
                                           float(emission_scale), _stream_ptr(stream)))


def rt_read_dust_emission(ctx, dst_ptr, n_elems, on_device, stream=None):
    _check(ctx, lib().rt_read_dust_emission(ctx, ctypes.c_void_p(int(dst_ptr)), int(n_elems), int(on_device),
                                            _stream_ptr(stream)))


def rt_batch_create(ctx, descs) -> int:
    arr = (rt_model_desc * len(descs))(*descs)
    b = ctypes.c_int32()
    _check(ctx, lib().rt_batch_create(ctx, len(descs), arr, ctypes.byref(b)))
    return b.value


def rt_batch_destroy(ctx, batch_id):
    _check(ctx, lib().rt_batch_destroy(ctx, int(batch_id)))


def rt_batch_launch(ctx, batch_id, seed=0, opts=None, stream=None):
    o = opts if opts is not None else rt_default_opts()
    _check(ctx, lib().rt_batch_launch(ctx, int(batch_id), int(seed), ctypes.byref(o), _stream_ptr(stream)))


def rt_batch_reset(ctx, batch_id, stream=None):
    _check(ctx, lib().rt_batch_reset(ctx, int(batch_id), _stream_ptr(stream)))


def rt_batch_read_images(ctx, batch_id, dst_ptr, n_elems, on_device, stream=None):
    _check(ctx, lib().rt_batch_read_images(ctx, int(batch_id), dst_ptr, int(n_elems), int(on_device),
                                           _stream_ptr(stream)))


def rt_batch_read_tallies(ctx, batch_id, dst_ptr, n_elems, on_device, stream=None):
    _check(ctx, lib().rt_batch_read_tallies(ctx, int(batch_id), dst_ptr, int(n_elems), int(on_device),
                                            _stream_ptr(stream)))


def rt_batch_read_stats(ctx, batch_id) -> rt_stats:
    s = rt_stats()
    _check(ctx, lib().rt_batch_read_stats(ctx, int(batch_id), ctypes.byref(s)))
    return s


def rt_batch_tune(ctx, batch_id, seed=0, fraction=0.05, stream=None):
    lanes = ctypes.c_int32()
    run = ctypes.c_uint32()
    _check(ctx, lib().rt_batch_tune(ctx, int(batch_id), int(seed), float(fraction), ctypes.byref(lanes),
                                    ctypes.byref(run), _stream_ptr(stream)))
    return lanes.value, run.value


# ---------------------------------------------------------------- descriptors from workloads
def grid_desc(grid, on_device_arrays=None):
    """rt_grid_desc for a workloads.Grid (host arrays; kept alive by the returned tuple)."""
    d = rt_grid_desc()
    d.bounds[:] = [float(b) for b in np.asarray(grid.bounds, dtype=np.float64)]
    dens = np.ascontiguousarray(grid.density, dtype=np.float32)
    keep = [dens]
    d.density = dens.ctypes.data
    if grid.kind in ("cartesian", "rectilinear"):
        d.kind = RT_GRID_CARTESIAN if grid.kind == "cartesian" else RT_GRID_RECTILINEAR
        nz, ny, nx = dens.shape
        d.nx, d.ny, d.nz = nx, ny, nz
        if grid.kind == "rectilinear":
            for a in range(3):
                e = np.ascontiguousarray(grid.edges[a], dtype=np.float64)
                keep.append(e)
                d.edges[a] = e.ctypes.data
    elif grid.kind == "voronoi":
        d.kind = RT_GRID_VORONOI
        sites = np.ascontiguousarray(grid.sites, dtype=np.float64)
        offsets = np.ascontiguousarray(grid.offsets, dtype=np.int64)
        nbr = np.ascontiguousarray(grid.child, dtype=np.int32)
        keep += [sites, offsets, nbr]
        d.sites, d.offsets, d.child = sites.ctypes.data, offsets.ctypes.data, nbr.ctypes.data
        d.n_nodes = nbr.size
        d.n_leaves = dens.size
    else:
        d.kind = RT_GRID_OCTREE if grid.kind == "octree" else RT_GRID_BINTREE
        child = np.ascontiguousarray(grid.child, dtype=np.int32)
        keep.append(child)
        d.child = child.ctypes.data
        d.n_nodes = child.size
        d.n_leaves = dens.size
        if grid.kind == "bintree":
            axis = np.ascontiguousarray(grid.split_axis, dtype=np.int8)
            keep.append(axis)
            d.split_axis = axis.ctypes.data
    return d, keep


def source_desc(src):
    d = rt_source_desc()
    d.kind = _SOURCE_KIND[src.kind]
    d.center[:] = [float(c) for c in src.center]
    d.scale_r = float(src.scale_r)
    d.scale_z = float(src.scale_z)
    return d


def instrument_desc(q):
    d = rt_instrument_desc()
    d.inclination, d.azimuth, d.position_angle = float(q.inclination), float(q.azimuth), float(q.position_angle)
    d.nx, d.ny = int(q.nx), int(q.ny)
    d.half_x, d.half_y = float(q.half_x), float(q.half_y)
    d.center_x, d.center_y = float(q.center_x), float(q.center_y)
    d.deposit = (RT_DEPOSIT_SED if getattr(q, "sed", False) else
                 RT_DEPOSIT_BILINEAR if q.bilinear else RT_DEPOSIT_NEAREST)
    d.channels = int(q.channels)
    return d


def model_desc(problem, n_packets=None):
    """rt_model_desc for a one-wavelength cartesian Problem with one point
    source and one single-channel frame (host density kept alive by the
    returned tuple)."""
    if problem.grid.kind != "cartesian" or problem.n_lambda != 1 or len(problem.sources) != 1 \
            or problem.sources[0].kind != "point" or len(problem.instruments) != 1 or problem.instruments[0].channels != 1:
        raise ValueError("a batch model has a cartesian grid, one wavelength, one point source and one frame")
    d = rt_model_desc()
    dens = np.ascontiguousarray(problem.grid.density, dtype=np.float32)
    d.nz, d.ny, d.nx = dens.shape
    d.bounds[:] = [float(b) for b in np.asarray(problem.grid.bounds, dtype=np.float64)]
    d.density = dens.ctypes.data
    d.kappa, d.albedo, d.g = float(problem.kappa[0]), float(problem.albedo[0]), float(problem.g[0])
    d.luminosity = float(problem.sources[0].lum[0])
    d.source[:] = [float(c) for c in problem.sources[0].center]
    d.instrument = instrument_desc(problem.instruments[0])
    d.n_packets = int(problem.run.n_per_lambda if n_packets is None else n_packets)
    return d, dens


class Batch:
    """A batch of one-wavelength models (workloads.Problem each) in one
    context: uploaded once, launched any number of times as one persistent
    kernel; images and per-model tallies read back."""

    def __init__(self, problems, device: int = 0, n_packets=None):
        self.problems = list(problems)
        self.device = int(device)
        self.ctx = rt_context_create(self.device)
        try:
            descs, keep = [], []
            for i, p in enumerate(self.problems):
                d, dens = model_desc(p, None if n_packets is None else n_packets[i])
                descs.append(d)
                keep.append(dens)
            self.id = rt_batch_create(self.ctx, descs)
            del keep
        except Exception:
            self.close()
            raise
        self.shapes = [(p.instruments[0].ny, p.instruments[0].nx) for p in self.problems]
        self.n_image = int(sum(a * b for a, b in self.shapes))

    def close(self):
        if getattr(self, "ctx", None) is not None:
            rt_context_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def opts(self, **kw) -> rt_launch_opts:
        o = rt_default_opts()
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown launch option {k}")
            setattr(o, k, v)
        return o

    def launch(self, seed=0, stream=None, **opts):
        rt_batch_launch(self.ctx, self.id, seed, self.opts(**opts), stream)

    def reset(self, stream=None):
        rt_batch_reset(self.ctx, self.id, stream)

    def tune(self, seed=0, fraction=0.05, stream=None):
        return rt_batch_tune(self.ctx, self.id, seed, fraction, stream)

    def images_flat(self, device=True, stream=None):
        if device:
            import torch
            t = torch.empty(self.n_image, dtype=torch.float64, device=f"cuda:{self.device}")
            rt_batch_read_images(self.ctx, self.id, t.data_ptr(), self.n_image, 1, stream)
        else:
            t = np.empty(self.n_image, dtype=np.float64)
            rt_batch_read_images(self.ctx, self.id, t.ctypes.data, self.n_image, 0, stream)
        return t

    def images(self):
        """Per-model images as numpy arrays [ny][nx]."""
        flat = self.images_flat(device=False)
        out, o = [], 0
        for ny, nx in self.shapes:
            out.append(flat[o:o + ny * nx].reshape(ny, nx))
            o += ny * nx
        return out

    def tallies(self):
        """[n_models][4]: emitted, escaped, absorbed, truncated."""
        t = np.empty((len(self.problems), 4), dtype=np.float64)
        rt_batch_read_tallies(self.ctx, self.id, t.ctypes.data, t.size, 0, None)
        return t

    def stats(self) -> dict:
        return rt_batch_read_stats(self.ctx, self.id).as_dict()


class Simulation:
    """A context set up from a :class:`workloads.Problem`: grid, optics,
    sources and instruments uploaded once; packets launched any number of
    times; tallies read into torch tensors or numpy arrays."""

    def __init__(self, problem, device: int = 0, layout: int = 0):
        self.problem = problem
        self.device = int(device)
        self.ctx = rt_context_create(self.device)
        try:
            desc, keep = grid_desc(problem.grid)
            desc.layout = int(layout)
            self.grid_id = rt_create_grid(self.ctx, desc)
            del keep
            rt_set_optics(self.ctx, self.grid_id, problem.kappa, problem.albedo, problem.g, problem.wavelengths)
            rt_add_sources(self.ctx, [source_desc(s) for s in problem.sources], [s.lum for s in problem.sources])
            self.instrument_ids = rt_add_instruments(self.ctx, [instrument_desc(q) for q in problem.instruments])
        except Exception:
            self.close()
            raise
        self.n_lambda = problem.n_lambda
        self.n_cells = problem.grid.n_cells

    def close(self):
        if getattr(self, "ctx", None) is not None:
            rt_context_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def opts(self, **kw) -> rt_launch_opts:
        o = rt_default_opts()
        run = self.problem.run
        o.w_min = run.w_min
        o.max_events = run.max_events
        o.weight_cut = int(run.weight_cut)
        for k, v in kw.items():
            if k in ("records", "trace", "profile"):
                setattr(o, k, v)
            elif not hasattr(o, k):
                raise TypeError(f"unknown launch option {k}")
            else:
                setattr(o, k, v)
        return o

    def launch(self, n_per_lambda=None, first_id=0, seed=None, stream=None, **opts):
        n = self.problem.run.n_per_lambda if n_per_lambda is None else n_per_lambda
        s = self.problem.run.seed if seed is None else seed
        rt_launch_packets(self.ctx, n, first_id, s, self.opts(**opts), stream)

    def reset(self, stream=None):
        rt_reset_tallies(self.ctx, stream)

    def dust_temperature(self, emission_scale, t_min=1.0, t_max=1e4, absorption=None):
        """Equilibrium dust temperatures (float64 numpy array [n_cells]) from
        the context's absorption tallies or a row-major absorption field
        [n_lambda, n_cells]; returns (T, cells held at t_max)."""
        T = np.zeros(self.n_cells, dtype=np.float64)
        keep = None
        ptr = 0
        if absorption is not None:
            keep = np.ascontiguousarray(absorption, dtype=np.float64)
            ptr = keep.ctypes.data
        n = rt_dust_temperature(self.ctx, emission_scale, t_min, t_max, ptr, 0, T.ctypes.data, 0)
        del keep
        return T, n

    def set_dust_emission(self, temperature, emission_scale):
        """Thermal emission of the dust at the temperatures [n_cells]; launches
        with emitter=RT_EMITTER_DUST then emit from the dust."""
        T = np.ascontiguousarray(temperature, dtype=np.float64)
        rt_set_dust_emission(self.ctx, T.ctypes.data, 0, emission_scale)

    def dust_emission(self):
        out = np.zeros((self.n_lambda, self.n_cells), dtype=np.float64)
        rt_read_dust_emission(self.ctx, out.ctypes.data, out.size, 0)
        return out

    def trace(self, packet, lam=0, n_per_lambda=None, seed=None, max_rows=None, **opts):
        """Per-event trace (rt_trace_row) of one packet: a launch of the
        packets [0, n_per_lambda) with the trace of `packet` at wavelength
        `lam` recorded (it adds to the tallies like any launch)."""
        import torch
        n = self.problem.run.n_per_lambda if n_per_lambda is None else n_per_lambda
        cap = int(max_rows or (self.problem.run.max_events + 2))
        buf = torch.zeros(cap * TRACE_DTYPE.itemsize, dtype=torch.uint8, device=f"cuda:{self.device}")
        self.launch(n, 0, seed, trace=buf.data_ptr(), trace_capacity=cap, trace_packet=int(packet),
                    trace_lambda=int(lam), **opts)
        rows = buf.cpu().numpy().view(TRACE_DTYPE)
        st = self.stats()
        n_rows = int(np.count_nonzero(rows["L"] != 0.0))
        del st
        return rows[:n_rows].copy()

    def tune(self, n_per_lambda, seed=0, stream=None, **opts) -> int:
        """Choose the per-event deferral threshold on a sample launch (tallies zeroed after)."""
        return rt_tune(self.ctx, n_per_lambda, seed, self.opts(**opts), stream)

    def tuned(self):
        """(control_lanes, blocks_per_sm) chosen by tune (blocks 0: as many as fit)."""
        return rt_tuned(self.ctx)

    def image_shape(self, q):
        ins = self.problem.instruments[q]
        return (ins.channels, self.n_lambda, ins.ny, ins.nx)

    def images(self, device=True, stream=None):
        """Images per instrument: torch float64 tensors on the device (or numpy on the host)."""
        out = []
        for q in range(len(self.problem.instruments)):
            shape = self.image_shape(q)
            n = int(np.prod(shape))
            if device:
                import torch
                t = torch.empty(shape, dtype=torch.float64, device=f"cuda:{self.device}")
                rt_read_images(self.ctx, q, t.data_ptr(), n, 1, stream)
            else:
                t = np.empty(shape, dtype=np.float64)
                rt_read_images(self.ctx, q, t.ctypes.data, n, 0, stream)
            out.append(t)
        return out

    def absorption(self, device=True, stream=None):
        shape = (self.n_lambda, self.n_cells)
        n = shape[0] * shape[1]
        if device:
            import torch
            t = torch.empty(shape, dtype=torch.float64, device=f"cuda:{self.device}")
            rt_read_absorption(self.ctx, t.data_ptr(), n, 1, stream)
        else:
            t = np.empty(shape, dtype=np.float64)
            rt_read_absorption(self.ctx, t.ctypes.data, n, 0, stream)
        return t

    def stats(self) -> dict:
        return rt_read_stats(self.ctx).as_dict()

    def launch_times(self) -> dict:
        """Device milliseconds of the parts of the last launch with time_parts=1."""
        return rt_read_launch_times(self.ctx)
