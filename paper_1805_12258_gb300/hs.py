"""Thin ctypes binding of libhs (include/hs.h).

The functions named after the C ABI (hs_plan_create, hs_run, ...) only
marshal arguments; every step of harmonic summing runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  If libhs.so is missing
the binding raises: there is no CPU fallback.

Convenience wrappers: ``Plan`` (owns an hs_plan) and ``CandBuffer`` (owns a
device candidate buffer).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# $HS_LIBRARY selects another build of the library (the bounds-checking one,
# in its tests); a path that does not exist fails loudly like a missing build
LIB_PATH = os.environ.get("HS_LIBRARY") or os.path.join(_HERE, "libhs.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "hs.h")

HS_OK, HS_ERR_INVALID, HS_ERR_CUDA, HS_ERR_OOM, HS_ERR_OVERFLOW, HS_ERR_TIMEOUT, \
    HS_ERR_UNSUPPORTED, HS_ERR_BUSY, HS_ERR_BOUNDS = range(9)
HS_F32, HS_BF16, HS_F16 = 0, 1, 2
HS_INDEX_STRETCH, HS_INDEX_HFRAC = 0, 1
HS_ZROUND_SYMMETRIC, HS_ZROUND_FLOOR = 0, 1
HS_KERNEL_AUTO, HS_KERNEL_GENERIC, HS_KERNEL_STAGED = 0, 1, 2
HS_FLAG_LOWP, HS_FLAG_NEAR = 1, 2
HS_KEEP_FIRST, HS_KEEP_LAST, HS_KEEP_LARGEST = 0, 1, 2
KEEP = {"first": HS_KEEP_FIRST, "last": HS_KEEP_LAST, "largest": HS_KEEP_LARGEST}

DTYPES = {"f32": HS_F32, "bf16": HS_BF16, "f16": HS_F16}
INDEX = {"stretch": HS_INDEX_STRETCH, "hfrac": HS_INDEX_HFRAC}
ZROUND = {"symmetric": HS_ZROUND_SYMMETRIC, "floor": HS_ZROUND_FLOOR}
KERNELS = {"auto": HS_KERNEL_AUTO, "generic": HS_KERNEL_GENERIC, "staged": HS_KERNEL_STAGED}

CAND_DTYPE = np.dtype([("bin", "<u4"), ("z", "<i2"), ("k", "u1"), ("flags", "u1"),
                       ("power", "<f4"), ("reserved", "<u4")])
assert CAND_DTYPE.itemsize == 16


class HsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class hs_options(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("index", ctypes.c_int), ("zround", ctypes.c_int),
                ("kernel", ctypes.c_int), ("tile_bins", ctypes.c_int), ("order", ctypes.c_int),
                ("grid_per_sm", ctypes.c_int), ("row_pitch", ctypes.c_int),
                ("stages", ctypes.c_int), ("z_split", ctypes.c_int),
                ("assume_nonneg", ctypes.c_int)]


class hs_cand(ctypes.Structure):
    _fields_ = [("bin", ctypes.c_uint32), ("z", ctypes.c_int16), ("k", ctypes.c_uint8),
                ("flags", ctypes.c_uint8), ("power", ctypes.c_float),
                ("reserved", ctypes.c_uint32)]


class hs_cand_buf(ctypes.Structure):
    _fields_ = [("records", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("capacity", ctypes.c_uint32)]


class hs_beam(ctypes.Structure):
    _fields_ = [("fop", ctypes.c_void_p), ("fop32", ctypes.c_void_p), ("n_bins", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("cands", hs_cand_buf)]


class hs_packed_beam(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("n_bins", ctypes.c_int64), ("cands", hs_cand_buf)]


class hs_server_config(ctypes.Structure):
    _fields_ = [("n_templates", ctypes.c_int), ("H", ctypes.c_int),
                ("thresholds", ctypes.c_void_p), ("n_slots", ctypes.c_int),
                ("slot_bins", ctypes.c_int64), ("cand_capacity", ctypes.c_uint32),
                ("queue_limit", ctypes.c_int), ("max_group", ctypes.c_int),
                ("assume_nonneg", ctypes.c_int)]


class hs_request(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_bins", ctypes.c_int64), ("dtype", ctypes.c_int),
                ("n_signals", ctypes.c_int), ("fop", ctypes.c_void_p), ("fop32", ctypes.c_void_p),
                ("ld", ctypes.c_int64)]


class hs_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int),
                ("n_cands", ctypes.c_uint32), ("group", ctypes.c_int32),
                ("group_size", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class hs_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("groups", ctypes.c_uint64),
                ("points", ctypes.c_uint64), ("dispatch_ns", ctypes.c_uint64),
                ("queued", ctypes.c_int32),
                ("in_flight", ctypes.c_int32), ("free_slots", ctypes.c_int32),
                ("peak_queue", ctypes.c_int32)]


_lib = None


def header_functions() -> list:
    """Names of the functions include/hs.h declares."""
    with open(HEADER) as fh:
        return re.findall(r"^HS_API\s+[\w\s\*]+?\b(hs_\w+)\s*\(", fh.read(), re.M)


def lib():
    """Load libhs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhs.so not found at {LIB_PATH}; run "
                           "`python -m paper_1805_12258_gb300.build` first")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32
    P = ctypes.POINTER
    L.hs_plan_create.argtypes = [P(vp), i32, i64, i32, vp, P(hs_options)]
    L.hs_run.argtypes = [vp, vp, vp, P(hs_cand_buf)]
    L.hs_run_checked.argtypes = [vp, vp, vp, vp, P(hs_cand_buf)]
    L.hs_cand_sync.argtypes = [P(hs_cand_buf), vp, P(u32)]
    L.hs_run_host.argtypes = [vp, vp, vp, P(hs_cand_buf), vp, u32, vp, P(u32)]
    L.hs_run_host_checked.argtypes = [vp, vp, vp, vp, P(hs_cand_buf), vp, u32, vp, P(u32)]
    L.hs_run_host_checked.restype = i32
    L.hs_plan_destroy.argtypes = [vp]
    L.hs_plan_kernel.argtypes = [vp]
    L.hs_plan_tile_bins.argtypes = [vp]
    L.hs_last_launch_count.argtypes = []
    L.hs_plan_set_timing.argtypes = [vp, i32]
    L.hs_plan_kernel_time.argtypes = [vp, P(ctypes.c_double), P(i32)]
    L.hs_pack_paper.argtypes = [P(hs_cand), i32, P(u32), P(ctypes.c_float)]
    L.hs_batch_create.argtypes = [P(vp), i32, i32, vp, P(hs_options), i32]
    L.hs_batch_set_beams.argtypes = [vp, P(hs_beam), i32, vp]
    L.hs_batch_set_packed.argtypes = [vp, vp, vp, i64, P(hs_packed_beam), i32, vp]
    L.hs_batch_set_packed.restype = i32
    L.hs_batch_run.argtypes = [vp, vp]
    L.hs_batch_graph_run.argtypes = [vp, vp]
    L.hs_batch_destroy.argtypes = [vp]
    L.hs_batch_tiles.argtypes = [vp]
    L.hs_batch_tiles.restype = i32
    L.hs_batch_launches.argtypes = [vp]
    L.hs_batch_launches.restype = i32
    L.hs_batch_last_error.argtypes = []
    L.hs_batch_last_error.restype = ctypes.c_char_p
    for name in ("hs_batch_create", "hs_batch_set_beams", "hs_batch_run", "hs_batch_graph_run",
                 "hs_batch_destroy"):
        getattr(L, name).restype = i32
    L.hs_server_create.argtypes = [P(vp), P(hs_server_config)]
    L.hs_server_submit.argtypes = [vp, P(hs_request), P(ctypes.c_uint64)]
    L.hs_server_wait.argtypes = [vp, ctypes.c_uint64, i32, P(hs_result), vp, u32]
    L.hs_server_drain.argtypes = [vp, i32]
    L.hs_server_stats_get.argtypes = [vp, P(hs_server_stats)]
    L.hs_server_destroy.argtypes = [vp]
    L.hs_server_last_error.argtypes = []
    L.hs_server_last_error.restype = ctypes.c_char_p
    L.hs_synth_fop.argtypes = [vp, vp, i32, i32, i64, i64, ctypes.c_uint64, i32, vp]
    for name in ("hs_server_create", "hs_server_submit", "hs_server_wait", "hs_server_drain",
                 "hs_server_stats_get", "hs_server_destroy", "hs_synth_fop"):
        getattr(L, name).restype = i32
    L.hs_postfilter.argtypes = [vp, u32, i32, u32, vp, P(u32)]
    L.hs_postfilter.restype = i32
    L.hs_postfilter_last_error.argtypes = []
    L.hs_postfilter_last_error.restype = ctypes.c_char_p
    L.hs_prefilter_bounds.argtypes = [vp, i32, i32, i32, P(i32), P(ctypes.c_float), P(i32)]
    L.hs_prefilter_bounds.restype = i32
    L.hs_tile_order.argtypes = [i32, i32, vp]
    L.hs_tile_order.restype = i32
    L.hs_selftest_wait_timeout.argtypes = [vp, ctypes.c_uint64, vp]
    L.hs_selftest_wait_timeout.restype = i32
    L.hs_run_range.argtypes = [vp, vp, vp, i64, i64, vp, P(hs_cand_buf), i32]
    L.hs_run_range.restype = i32
    L.hs_run_noalloc.argtypes = [i32, i64, i32, vp, vp, vp, P(hs_cand_buf)]
    L.hs_run_noalloc.restype = i32
    L.hs_noalloc_last_error.argtypes = []
    L.hs_noalloc_last_error.restype = ctypes.c_char_p
    L.hs_status_str.argtypes = [i32]
    L.hs_status_str.restype = ctypes.c_char_p
    L.hs_last_error.argtypes = []
    L.hs_last_error.restype = ctypes.c_char_p
    for name in ("hs_plan_create", "hs_run", "hs_run_checked", "hs_cand_sync", "hs_run_host",
                 "hs_plan_destroy", "hs_pack_paper", "hs_plan_set_timing",
                 "hs_plan_kernel_time"):
        getattr(L, name).restype = i32
    for name in ("hs_plan_kernel", "hs_plan_tile_bins", "hs_last_launch_count"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(status, what, ok=(HS_OK,)):
    if status not in ok:
        raise HsError(status, f"{what}: {lib().hs_last_error().decode()}")
    return status


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


# ---- the C ABI, argument marshalling only ------------------------------------

def hs_plan_create(n_templates, n_bins, H, thresholds, opt: hs_options | None = None):
    """Create a plan; thresholds is a host float32 array [H][n_templates]."""
    ta = np.ascontiguousarray(thresholds, dtype=np.float32)
    if ta.shape != (H, n_templates):
        raise ValueError(f"thresholds must have shape {(H, n_templates)}, got {ta.shape}")
    out = ctypes.c_void_p()
    _check(lib().hs_plan_create(ctypes.byref(out), n_templates, n_bins, H, ta.ctypes.data,
                                ctypes.byref(opt) if opt is not None else None),
           "hs_plan_create")
    return out.value


def hs_run(plan, fop, stream, cands: hs_cand_buf):
    return _check(lib().hs_run(plan, _ptr(fop), _stream_handle(stream), ctypes.byref(cands)),
                  "hs_run")


def hs_run_checked(plan, fop, fop_f32, stream, cands: hs_cand_buf):
    return _check(lib().hs_run_checked(plan, _ptr(fop), _ptr(fop_f32), _stream_handle(stream),
                                       ctypes.byref(cands)), "hs_run_checked")


def hs_cand_sync(cands: hs_cand_buf, stream):
    """Returns (status, n_found); raises on CUDA errors and timeouts."""
    n = ctypes.c_uint32(0)
    st = lib().hs_cand_sync(ctypes.byref(cands), _stream_handle(stream), ctypes.byref(n))
    _check(st, "hs_cand_sync", ok=(HS_OK, HS_ERR_OVERFLOW))
    return st, n.value


def hs_run_host(plan, fop_host, fop_dev, cands: hs_cand_buf, host_records, stream,
                fop32_host=None):
    """Returns (status, n_found); host_records is a CAND_DTYPE numpy array.
    fop32_host: page-locked FP32 copy for the rechecks of a 16-bit plan."""
    n = ctypes.c_uint32(0)
    cap = 0 if host_records is None else len(host_records)
    st = lib().hs_run_host_checked(plan, _ptr(fop_host), _ptr(fop_dev), _ptr(fop32_host),
                                   ctypes.byref(cands), _ptr(host_records) if cap else None,
                                   cap, _stream_handle(stream), ctypes.byref(n))
    _check(st, "hs_run_host_checked", ok=(HS_OK, HS_ERR_OVERFLOW))
    return st, n.value


def hs_run_noalloc(n_templates, n_bins, H, thresholds, fop, stream, cands: hs_cand_buf):
    """hs_run without a plan and without device allocation (see include/hs.h):
    for callers that may not allocate device memory.  H * n_templates must be
    at most 16384; calls share one static threshold table, so calls that
    overlap on the GPU race."""
    ta = np.ascontiguousarray(thresholds, dtype=np.float32)
    if ta.shape != (H, n_templates):
        raise ValueError(f"thresholds must have shape {(H, n_templates)}, got {ta.shape}")
    st = lib().hs_run_noalloc(n_templates, n_bins, H, ta.ctypes.data, _ptr(fop),
                              _stream_handle(stream), ctypes.byref(cands))
    if st != HS_OK:
        raise HsError(st, f"hs_run_noalloc: {lib().hs_noalloc_last_error().decode()}")
    return st


def hs_plan_destroy(plan):
    return _check(lib().hs_plan_destroy(plan), "hs_plan_destroy")


def hs_pack_paper(rec, n_templates):
    """(CL1, CL2) of one record (Section III packing)."""
    c = hs_cand(int(rec["bin"]), int(rec["z"]), int(rec["k"]), int(rec["flags"]),
                float(rec["power"]), 0)
    cl1, cl2 = ctypes.c_uint32(), ctypes.c_float()
    _check(lib().hs_pack_paper(ctypes.byref(c), n_templates, ctypes.byref(cl1),
                               ctypes.byref(cl2)), "hs_pack_paper")
    return cl1.value, cl2.value


def hs_plan_set_timing(plan, enable):
    return _check(lib().hs_plan_set_timing(plan, int(bool(enable))), "hs_plan_set_timing")


def hs_plan_kernel_time(plan):
    """(summed kernel milliseconds, launches) since the last query."""
    ms, n = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(lib().hs_plan_kernel_time(plan, ctypes.byref(ms), ctypes.byref(n)),
           "hs_plan_kernel_time")
    return ms.value, n.value


def hs_prefilter_bounds(thresholds, dtype="f32"):
    """(ends, bounds): the staged kernel's level groups (last level of each)
    and their prefilter bounds for thresholds [H][n_templates]."""
    ta = np.ascontiguousarray(thresholds, dtype=np.float32)
    H, nt = ta.shape
    ends = (ctypes.c_int * 8)()
    bounds = (ctypes.c_float * 8)()
    ng = ctypes.c_int(0)
    _check(lib().hs_prefilter_bounds(ta.ctypes.data, nt, H, DTYPES[dtype], ends, bounds,
                                     ctypes.byref(ng)), "hs_prefilter_bounds")
    g = ng.value
    return (np.array(ends[:g], dtype=np.int32), np.array(bounds[:g], dtype=np.float32))


def hs_tile_order(n_tiles, order=0):
    """The tile indices of a plane in the order a plan visits them."""
    out = np.zeros(max(1, int(n_tiles)), dtype=np.uint32)
    _check(lib().hs_tile_order(int(n_tiles), int(order), out.ctypes.data), "hs_tile_order")
    return out[:int(n_tiles)]


def hs_status_str(s):
    return lib().hs_status_str(s).decode()


def hs_last_launch_count():
    return lib().hs_last_launch_count()


# ---- convenience wrappers ------------------------------------------------------

class CandBuffer:
    """Device candidate buffer: `capacity` 16-byte records + 2 counters."""

    def __init__(self, capacity: int, device="cuda"):
        import torch
        self.capacity = int(capacity)
        self.records = torch.empty(max(1, self.capacity) * 16, dtype=torch.uint8, device=device)
        self.counters = torch.zeros(4, dtype=torch.int32, device=device)
        self.c = hs_cand_buf(self.records.data_ptr(), self.counters.data_ptr(), self.capacity)

    def sync(self, stream=None):
        """(status, n_found) after the stream drains."""
        return hs_cand_sync(self.c, stream)

    def to_numpy(self, n: int) -> np.ndarray:
        n = min(int(n), self.capacity)
        raw = self.records[: n * 16].cpu().numpy()
        return raw.view(CAND_DTYPE).copy()

    def fetch(self, stream=None):
        """Sync and return (records sorted by (k, z, bin), n_found, status)."""
        st, n = self.sync(stream)
        return sort_records(self.to_numpy(n)), n, st


def sort_records(r: np.ndarray) -> np.ndarray:
    if len(r) == 0:
        return r
    return r[np.lexsort((r["bin"], r["z"], r["k"]))]


class Plan:
    """An hs_plan for one plane shape, threshold table and option set."""

    def __init__(self, n_templates, n_bins, H, thresholds, *, dtype="f32", index="stretch",
                 zround="symmetric", kernel="auto", tile_bins=0, order=0, grid_per_sm=0,
                 row_pitch=0, stages=0, z_split=0, assume_nonneg=False):
        opt = hs_options(DTYPES[dtype], INDEX[index], ZROUND[zround], KERNELS[kernel],
                         int(tile_bins), int(order), int(grid_per_sm), int(row_pitch),
                         int(stages), int(z_split), int(bool(assume_nonneg)))
        self.n_templates, self.n_bins, self.H = n_templates, n_bins, H
        self.dtype = dtype
        self.handle = hs_plan_create(n_templates, n_bins, H, thresholds, opt)

    @property
    def kernel(self) -> str:
        return {1: "generic", 2: "staged"}[lib().hs_plan_kernel(self.handle)]

    @property
    def tile_bins(self) -> int:
        return lib().hs_plan_tile_bins(self.handle)

    def run(self, fop, cands: CandBuffer, stream=None, fop_f32=None):
        if fop_f32 is None:
            hs_run(self.handle, fop, stream, cands.c)
        else:
            hs_run_checked(self.handle, fop, fop_f32, stream, cands.c)

    def run_range(self, fop, cands: CandBuffer, f_lo, f_hi, stream=None, fop_f32=None,
                  append=False):
        """Sum output bins [f_lo, f_hi) only (a frequency-band shard)."""
        _check(lib().hs_run_range(self.handle, _ptr(fop), _ptr(fop_f32), int(f_lo), int(f_hi),
                                  _stream_handle(stream), ctypes.byref(cands.c), int(append)),
               "hs_run_range")

    def set_timing(self, enable=True):
        hs_plan_set_timing(self.handle, enable)

    def kernel_time(self):
        """(summed device ms, runs) recorded since the last call while timing
        was on (one event pair per run, around its kernels)."""
        return hs_plan_kernel_time(self.handle)

    def run_host(self, fop_host, fop_dev, cands: CandBuffer, host_records, stream=None,
                 fop32_host=None):
        return hs_run_host(self.handle, fop_host, fop_dev, cands.c, host_records, stream,
                           fop32_host)

    def close(self):
        if getattr(self, "handle", None):
            hs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- batched form --------------------------------------------------------------

def _batch_check(status, what):
    if status != HS_OK:
        raise HsError(status, f"{what}: {lib().hs_batch_last_error().decode()}")
    return status


class Batch:
    """An hs_batch: many planes of one shape (each with its own bin count and
    row pitch) summed by a few launches, each carrying up to K beams'
    descriptors (set_beams), or beams packed side by side in one plane summed
    by one launch (set_packed); graph_run replays a captured CUDA graph of a
    run."""

    def __init__(self, n_templates, H, thresholds, *, dtype="f32", grid_per_sm=0,
                 max_beams=64, order=0, assume_nonneg=False):
        ta = np.ascontiguousarray(thresholds, dtype=np.float32)
        if ta.shape != (H, n_templates):
            raise ValueError(f"thresholds must have shape {(H, n_templates)}, got {ta.shape}")
        opt = hs_options(DTYPES[dtype], 0, 0, 0, 0, int(order), int(grid_per_sm), 0, 0, 0,
                         int(bool(assume_nonneg)))
        out = ctypes.c_void_p()
        _batch_check(lib().hs_batch_create(ctypes.byref(out), n_templates, H, ta.ctypes.data,
                                           ctypes.byref(opt), int(max_beams)), "hs_batch_create")
        self.handle = out.value
        self.n_templates, self.H = n_templates, H
        self._keep = []

    def set_beams(self, beams, stream=None):
        """beams: list of (fop tensor [n_templates][...], n_bins, CandBuffer) or
        (fop, n_bins, CandBuffer, fop32); a beam's row pitch is its tensor's
        row stride (a view into a wider plane keeps that plane's pitch)."""
        arr = (hs_beam * max(1, len(beams)))()
        for i, b in enumerate(beams):
            fop, n_bins, cb = b[0], b[1], b[2]
            fop32 = b[3] if len(b) > 3 else None
            ld = fop.stride(0) if hasattr(fop, "stride") else fop.shape[-1]
            arr[i] = hs_beam(_ptr(fop), _ptr(fop32), int(n_bins), int(ld), cb.c)
        self._keep = list(beams)
        _batch_check(lib().hs_batch_set_beams(self.handle, arr, len(beams),
                                              _stream_handle(stream)), "hs_batch_set_beams")

    def set_packed(self, plane, beams, fop32=None, stream=None):
        """plane: tensor [n_templates][pitch] holding every beam side by side
        along the bins; beams: list of (offset, n_bins, CandBuffer).  One
        summing launch then covers all of them."""
        arr = (hs_packed_beam * max(1, len(beams)))()
        for i, (off, n_bins, cb) in enumerate(beams):
            arr[i] = hs_packed_beam(int(off), int(n_bins), cb.c)
        self._keep = [plane, fop32] + [b[2] for b in beams]
        _batch_check(lib().hs_batch_set_packed(self.handle, _ptr(plane), _ptr(fop32),
                                               int(plane.shape[-1]), arr, len(beams),
                                               _stream_handle(stream)), "hs_batch_set_packed")

    @property
    def tiles(self):
        return lib().hs_batch_tiles(self.handle)

    @property
    def launches(self):
        """Kernel launches one run issues to sum the tiles (reset excluded)."""
        return lib().hs_batch_launches(self.handle)

    def run(self, stream=None):
        _batch_check(lib().hs_batch_run(self.handle, _stream_handle(stream)), "hs_batch_run")

    def graph_run(self, stream=None):
        _batch_check(lib().hs_batch_graph_run(self.handle, _stream_handle(stream)),
                     "hs_batch_graph_run")

    def close(self):
        if getattr(self, "handle", None):
            lib().hs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- serving form ----------------------------------------------------------------

def hs_synth_fop(fop, fop32, dtype, n_templates, n_bins, ld, seed, n_signals, stream=None):
    """Device plane generator (Exponential(1) noise by Philox4x32-10 plus
    harmonic signals) into fop (and fop32 for BF16)."""
    st = lib().hs_synth_fop(_ptr(fop), _ptr(fop32), DTYPES[dtype] if isinstance(dtype, str)
                            else int(dtype), int(n_templates), int(n_bins), int(ld), int(seed),
                            int(n_signals), _stream_handle(stream))
    if st != HS_OK:
        raise HsError(st, f"hs_synth_fop: {lib().hs_server_last_error().decode()}")


class Server:
    """An hs_server: resident plane slots, a dispatcher that admits queued
    requests into free slots and sums each admitted group with the batched
    kernels, and a completion thread that returns candidates to the host."""

    def __init__(self, n_templates, H, thresholds, *, n_slots=16, slot_bins=1 << 22,
                 cand_capacity=4096, queue_limit=1024, max_group=0, assume_nonneg=False):
        ta = np.ascontiguousarray(thresholds, dtype=np.float32)
        if ta.shape != (H, n_templates):
            raise ValueError(f"thresholds must have shape {(H, n_templates)}, got {ta.shape}")
        cfg = hs_server_config(n_templates, H, ta.ctypes.data, int(n_slots), int(slot_bins),
                               int(cand_capacity), int(queue_limit), int(max_group),
                               int(bool(assume_nonneg)))
        out = ctypes.c_void_p()
        st = lib().hs_server_create(ctypes.byref(out), ctypes.byref(cfg))
        if st != HS_OK:
            raise HsError(st, f"hs_server_create: {lib().hs_server_last_error().decode()}")
        self.handle = out.value
        self.n_templates, self.H, self.cand_capacity = n_templates, H, int(cand_capacity)

    def submit(self, seed, n_bins, dtype="f32", n_signals=0, fop=None, fop32=None):
        """Queue a request; returns its ticket, or None when the queue is full.
        fop (and fop32 for BF16): a device plane already resident, summed in
        place instead of generating one from the seed."""
        ld = 0 if fop is None else int(fop.shape[-1])
        req = hs_request(int(seed), int(n_bins), DTYPES[dtype], int(n_signals), _ptr(fop),
                         _ptr(fop32), ld)
        t = ctypes.c_uint64()
        st = lib().hs_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        if st == HS_ERR_BUSY:
            return None
        if st != HS_OK:
            raise HsError(st, f"hs_server_submit: {lib().hs_server_last_error().decode()}")
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """(result dict, records sorted by (k, z, bin)) or None on timeout."""
        res = hs_result()
        recs = np.zeros(self.cand_capacity, dtype=CAND_DTYPE)
        st = lib().hs_server_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(res),
                                  recs.ctypes.data, self.cand_capacity)
        if st == HS_ERR_BUSY:
            return None
        if st != HS_OK:
            raise HsError(st, f"hs_server_wait: {lib().hs_server_last_error().decode()}")
        d = {name: getattr(res, name) for name, _ in hs_result._fields_}
        kept = min(res.n_cands, self.cand_capacity) if res.status in (HS_OK, HS_ERR_OVERFLOW) \
            else 0
        return d, sort_records(recs[:kept])

    def drain(self, timeout_ms=-1):
        return lib().hs_server_drain(self.handle, int(timeout_ms)) == HS_OK

    def stats(self):
        st = hs_server_stats()
        lib().hs_server_stats_get(self.handle, ctypes.byref(st))
        return {name: getattr(st, name) for name, _ in hs_server_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().hs_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def hs_postfilter(records: np.ndarray, policy="last", n_keep=200) -> np.ndarray:
    """The paper's per-level candidate cap (first / last / largest n_keep),
    applied by the library on host records; returns the kept records."""
    rec = np.ascontiguousarray(records, dtype=CAND_DTYPE)
    out = np.zeros(max(1, len(rec)), dtype=CAND_DTYPE)
    n_out = ctypes.c_uint32()
    st = lib().hs_postfilter(rec.ctypes.data if len(rec) else None, len(rec),
                             KEEP[policy] if isinstance(policy, str) else int(policy),
                             int(n_keep), out.ctypes.data, ctypes.byref(n_out))
    if st != HS_OK:
        raise HsError(st, f"hs_postfilter: {lib().hs_postfilter_last_error().decode()}")
    return out[:n_out.value]
