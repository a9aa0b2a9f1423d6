"""FP64 CPU oracle for harmonic summing (arXiv 1805.12258, Eq. 1-2, Algorithms 1-2).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
never does.  The arithmetic lives in ``hs_oracle.c`` (plain C, double
precision); this module only compiles it with gcc and marshals numpy arrays.

Functions
---------
stretch(fop, k)                  Eq. 1, one stretch plane SP_k (gather form)
stretch_adjoint(w, k)            adjoint of Eq. 1 (scatter, from preimages)
planes(fop, H)                   Algorithm 1 order: all HP_k planes
sample(fop, H, z, f)             level values at listed points
detect(fop, H, ta)               Algorithm 2 order: candidates + near list
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libhs_oracle.so")

STRETCH, HFRAC = 0, 1
ZSYM, ZFLOOR = 0, 1
DT_F32, DT_BF16, DT_F16, DT_F64 = 0, 1, 2, 3

CAND_DTYPE = np.dtype([("f", np.int64), ("z", np.int32), ("k", np.int32),
                       ("power", np.float64)])

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hs_oracle.c into libhs_oracle.so (gcc, -O2, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.hso_stretch.argtypes = [vp, i32, i32, i64, i64, i64, i32, vp]
    lib.hso_stretch.restype = i32
    lib.hso_stretch_adjoint.argtypes = [vp, i32, i64, i64, i32, vp]
    lib.hso_stretch_adjoint.restype = i32
    lib.hso_planes.argtypes = [vp, i32, i32, i64, i32, i32, i32, vp]
    lib.hso_planes.restype = i32
    lib.hso_sample.argtypes = [vp, i32, i32, i64, i32, i32, i32, vp, vp, i64, vp]
    lib.hso_sample.restype = i32
    lib.hso_detect.argtypes = [vp, i32, i32, i64, i32, i32, i32, vp, dbl, i64, i64,
                               vp, i64, vp, i64, vp]
    lib.hso_detect.restype = i64
    _lib = lib
    return lib


def _plane_arg(fop, dtype_code=None):
    """Return (contiguous array, dtype code) for a stored FOP.

    float32/float64/float16 numpy arrays map directly; bfloat16 planes are
    passed as uint16 bit patterns with dtype_code=DT_BF16."""
    a = np.ascontiguousarray(fop)
    if dtype_code is None:
        if a.dtype == np.float32:
            dtype_code = DT_F32
        elif a.dtype == np.float64:
            dtype_code = DT_F64
        elif a.dtype == np.float16:
            dtype_code = DT_F16
        else:
            raise TypeError(f"unsupported plane dtype {a.dtype}; pass dtype_code for bf16 bits")
    if a.ndim != 2:
        raise ValueError("FOP must be 2-D [n_templates][n_bins]")
    return a, dtype_code


def _check(rc, what):
    if rc < 0:
        raise ValueError(f"oracle {what}: invalid arguments (rc={rc})")


def stretch(fop, k, *, num=1, zround=ZSYM, dtype_code=None):
    """Eq. 1 with scale num/k: SP(i,j) = FOP(rho(i*num/k), floor(j*num/k))."""
    a, dt = _plane_arg(fop, dtype_code)
    nt, n = a.shape
    out = np.empty((nt, n), np.float64)
    _check(_load().hso_stretch(a.ctypes.data, dt, nt, n, num, k, zround, out.ctypes.data),
           "stretch")
    return out


def stretch_adjoint(w, k, *, zround=ZSYM):
    """Adjoint of Eq. 1 (SP_k^T), written as a scatter from preimages."""
    a = np.ascontiguousarray(w, dtype=np.float64)
    nt, n = a.shape
    out = np.empty((nt, n), np.float64)
    _check(_load().hso_stretch_adjoint(a.ctypes.data, nt, n, k, zround, out.ctypes.data),
           "stretch_adjoint")
    return out


def planes(fop, H, *, index=STRETCH, zround=ZSYM, dtype_code=None):
    """Algorithm 1 order: returns hp[H][n_templates][n_bins] in float64."""
    a, dt = _plane_arg(fop, dtype_code)
    nt, n = a.shape
    out = np.empty((H, nt, n), np.float64)
    _check(_load().hso_planes(a.ctypes.data, dt, nt, n, H, index, zround, out.ctypes.data),
           "planes")
    return out


def sample(fop, H, z, f, *, index=STRETCH, zround=ZSYM, dtype_code=None):
    """Level values at points (z[p], f[p]); returns [npts][H] float64."""
    a, dt = _plane_arg(fop, dtype_code)
    nt, n = a.shape
    z = np.ascontiguousarray(z, dtype=np.int32)
    f = np.ascontiguousarray(f, dtype=np.int64)
    out = np.empty((len(z), H), np.float64)
    _check(_load().hso_sample(a.ctypes.data, dt, nt, n, H, index, zround,
                              z.ctypes.data, f.ctypes.data, len(z), out.ctypes.data),
           "sample")
    return out


def _detect_range(a, dt, H, index, zround, ta, near_rel, f_lo, f_hi, cap, near_cap):
    lib = _load()
    nt, n = a.shape
    while True:
        cands = np.empty(max(cap, 1), CAND_DTYPE)
        near = np.empty(max(near_cap, 1), CAND_DTYPE)
        n_near = ctypes.c_int64(0)
        nc = lib.hso_detect(a.ctypes.data, dt, nt, n, H, index, zround, ta.ctypes.data,
                            near_rel, f_lo, f_hi, cands.ctypes.data, cap,
                            near.ctypes.data, near_cap, ctypes.byref(n_near))
        _check(nc, "detect")
        if nc <= cap and n_near.value <= near_cap:
            return cands[:nc], near[:n_near.value]
        cap, near_cap = max(cap, nc), max(near_cap, n_near.value)


def detect(fop, H, ta, *, index=STRETCH, zround=ZSYM, near_rel=1e-5,
           f_lo=0, f_hi=None, threads=1, dtype_code=None, cap=1 << 16):
    """Algorithm 2 order detection over bins [f_lo, f_hi).

    Returns (candidates, near) as CAND_DTYPE arrays sorted by (k, z, f).
    threads > 1 splits the bin range over Python threads (the C call releases
    the GIL); the arithmetic of every point is unchanged."""
    a, dt = _plane_arg(fop, dtype_code)
    nt, n = a.shape
    f_hi = n if f_hi is None else f_hi
    ta = np.ascontiguousarray(ta, dtype=np.float32)
    if ta.shape != (H, nt):
        raise ValueError(f"thresholds must be [H][n_templates] = {(H, nt)}, got {ta.shape}")
    threads = max(1, min(int(threads), max(1, f_hi - f_lo)))
    edges = np.linspace(f_lo, f_hi, threads + 1).astype(np.int64)
    results = [None] * threads

    def work(t):
        results[t] = _detect_range(a, dt, H, index, zround, ta, near_rel,
                                   int(edges[t]), int(edges[t + 1]), cap, cap)

    if threads == 1:
        work(0)
    else:
        ths = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
    cands = np.concatenate([r[0] for r in results])
    near = np.concatenate([r[1] for r in results])
    return sort_cands(cands), sort_cands(near)


def sort_cands(c):
    """Sort candidate records by (k, z, f)."""
    if len(c) == 0:
        return c
    order = np.lexsort((c["f"], c["z"], c["k"]))
    return c[order]
