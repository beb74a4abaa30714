"""FP64 CPU oracle for ZNCC + DT + WTA (arXiv 2212.00476), as numpy-facing wrappers.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference leg may import this package. It shares no code with the CUDA path
(paper_2212_00476_gb300) and neither imports the other.

The arithmetic lives in zncc_oracle.c (plain C, FP64, pthreads over rows and lines);
this module compiles it with gcc on first use and wraps each entry point:

    window_sums / window_sums_integral   Sec. IV-B-1, Eq. (sum1) and Method 2
    zncc_volume / zncc_at                 Sec. III-A, Eq. (1)
    dt_weights                            Sec. III-B, Eqs. (7)-(11)
    dt_aggregate                          Sec. III-B, Eqs. (3)-(6)
    wta                                   Sec. III-C, Eq. (WTA1)
    run                                   the whole path on one pair
    fastdt_encode / fastdt_decode         Sec. IV-C, the 8-bit code (6-bit value, 2-bit flag)
    fastdt_store / run_fastdt             Sec. IV-C, near-zero-mean 16-bit storage and the code
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zncc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, defines: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile the oracle into a shared library; returns its path."""
    out = out or _LIB_PATH
    if not force and not defines and os.path.exists(out) and \
            os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall",
           *[f"-D{d}" for d in defines], _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i64p = ctypes.POINTER(ctypes.c_int64)
    f64p = ctypes.POINTER(ctypes.c_double)
    i32p = ctypes.POINTER(ctypes.c_int)
    u16p = ctypes.POINTER(ctypes.c_uint16)
    c_int, c_double = ctypes.c_int, ctypes.c_double
    lib.oracle_window_sums.argtypes = [u8p, c_int, c_int, c_int, c_int, c_int, i64p, i64p]
    lib.oracle_window_sums_integral.argtypes = lib.oracle_window_sums.argtypes
    lib.oracle_zncc_at.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, c_int]
    lib.oracle_zncc_at.restype = c_double
    lib.oracle_zncc_volume.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, i32p, c_int,
                                       c_int, f64p]
    lib.oracle_dt_weights.argtypes = [u8p, c_int, c_int, c_double, c_double, c_int,
                                      f64p, f64p, f64p, f64p]
    lib.oracle_dt_aggregate.argtypes = [f64p, c_int, c_int, c_int, f64p, f64p, f64p, f64p,
                                        c_double, c_int, c_int, c_int]
    lib.oracle_wta.argtypes = [f64p, c_int, c_int, c_int, u16p, f64p, f64p]
    lib.oracle_run.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_double, c_double,
                               c_int, c_int, u16p, f64p, f64p]
    lib.oracle_fastdt_encode.argtypes = [ctypes.c_int16]
    lib.oracle_fastdt_encode.restype = ctypes.c_uint8
    lib.oracle_fastdt_decode.argtypes = [ctypes.c_uint8]
    lib.oracle_fastdt_decode.restype = ctypes.c_int16
    lib.oracle_fastdt_store.argtypes = [f64p, f64p, c_int, c_int, c_int, c_int, c_double]
    lib.oracle_dt_aggregate_fastdt.argtypes = [f64p, u8p, c_int, c_int, c_int, c_double, c_double,
                                               c_int, c_int, c_double, c_int]
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library. A path loads a specific build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
               else os.cpu_count() or 1)


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _img(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    assert a.ndim == 2
    return a


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def window_sums(img, r, x_begin=0, x_end=None, lib=None, integral=False):
    """Exact window sums S and Q (int64 [H][x_end-x_begin]) for centres x in [x_begin, x_end)."""
    lib = lib or load()
    img = _img(img)
    H, W = img.shape
    x_end = W if x_end is None else x_end
    S = np.zeros((H, x_end - x_begin), np.int64)
    Q = np.zeros_like(S)
    fn = lib.oracle_window_sums_integral if integral else lib.oracle_window_sums
    _check(fn(_p(img, ctypes.c_uint8), W, H, r, x_begin, x_end, _p(S, ctypes.c_int64),
              _p(Q, ctypes.c_int64)), "window_sums")
    return S, Q


def zncc_at(left, right, r, x, y, d, lib=None):
    lib = lib or load()
    left, right = _img(left), _img(right)
    H, W = left.shape
    return lib.oracle_zncc_at(_p(left, ctypes.c_uint8), _p(right, ctypes.c_uint8), W, H, r,
                              x, y, d)


def zncc_volume(left, right, max_disp, r, planes=None, nthreads=None, lib=None):
    """Eq. (1) cost volume, float64 [H][W][nd] (nd = D, or len(planes))."""
    lib = lib or load()
    left, right = _img(left), _img(right)
    H, W = left.shape
    assert right.shape == left.shape
    nthreads = nthreads or default_threads()
    if planes is None:
        nd, pl = max_disp, None
    else:
        pl = np.ascontiguousarray(planes, dtype=np.int32)
        nd = len(pl)
    C = np.zeros((H, W, nd), np.float64)
    _check(lib.oracle_zncc_volume(_p(left, ctypes.c_uint8), _p(right, ctypes.c_uint8), W, H,
                                  max_disp, r, None if pl is None else _p(pl, ctypes.c_int),
                                  nd, nthreads, _p(C, ctypes.c_double)), "zncc_volume")
    return C


def dt_weights(guide, sigma_s, sigma_r, form=0, lib=None):
    """The four DT weight maps (W_L, W_R, W_U, W_D), float64 [H][W] each."""
    lib = lib or load()
    guide = _img(guide)
    H, W = guide.shape
    w = np.zeros((4, H, W), np.float64)
    _check(lib.oracle_dt_weights(_p(guide, ctypes.c_uint8), W, H, float(sigma_s),
                                 float(sigma_r), form, *[_p(w[i], ctypes.c_double)
                                                         for i in range(4)]), "dt_weights")
    return w


def dt_aggregate(C, weights, sigma_s, iters, scaled=True, nthreads=None, lib=None):
    """Eqs. (3)-(6) repeated `iters` times; returns a new float64 [H][W][nd] array."""
    lib = lib or load()
    C = np.array(C, dtype=np.float64, copy=True, order="C")
    if C.ndim == 2:
        C = C[:, :, None].copy()
    H, W, nd = C.shape
    w = np.ascontiguousarray(weights, dtype=np.float64)
    nthreads = nthreads or default_threads()
    _check(lib.oracle_dt_aggregate(_p(C, ctypes.c_double), W, H, nd,
                                   *[_p(w[i], ctypes.c_double) for i in range(4)],
                                   float(sigma_s), int(iters), int(bool(scaled)), nthreads),
           "dt_aggregate")
    return C


def wta(C, lib=None):
    """Eq. (WTA1): (disparity uint16 [H][W], winning value, gap to the runner-up)."""
    lib = lib or load()
    C = np.ascontiguousarray(C, dtype=np.float64)
    H, W, nd = C.shape
    disp = np.zeros((H, W), np.uint16)
    best = np.zeros((H, W), np.float64)
    gap = np.zeros((H, W), np.float64)
    _check(lib.oracle_wta(_p(C, ctypes.c_double), W, H, nd, _p(disp, ctypes.c_uint16),
                          _p(best, ctypes.c_double), _p(gap, ctypes.c_double)), "wta")
    return disp, best, gap


def ones_response(guide, sigma_s, sigma_r, iters, lib=None):
    """A_hat(x,y): the scaled DT of an all-ones plane, the largest |aggregated cost|
    possible at (x,y) when every input cost lies in [-1, 1]."""
    H, W = np.asarray(guide).shape
    w = dt_weights(guide, sigma_s, sigma_r, lib=lib)
    return dt_aggregate(np.ones((H, W, 1)), w, sigma_s, iters, scaled=True, lib=lib)[:, :, 0]


def run(left, right, max_disp, r, sigma_s=20.0, sigma_r=0.1, iters=3, nthreads=None,
        want_cost=False, lib=None):
    """Whole path: (disparity, gap[, aggregated cost float64 [H][W][D]])."""
    lib = lib or load()
    left, right = _img(left), _img(right)
    H, W = left.shape
    nthreads = nthreads or default_threads()
    disp = np.zeros((H, W), np.uint16)
    gap = np.zeros((H, W), np.float64)
    C = np.zeros((H, W, max_disp), np.float64) if want_cost else None
    _check(lib.oracle_run(_p(left, ctypes.c_uint8), _p(right, ctypes.c_uint8), W, H, max_disp,
                          r, float(sigma_s), float(sigma_r), int(iters), nthreads,
                          _p(disp, ctypes.c_uint16), _p(gap, ctypes.c_double),
                          None if C is None else _p(C, ctypes.c_double)), "run")
    return (disp, gap, C) if want_cost else (disp, gap)


# FastDT storage (Sec. IV-C): d_arb = 0 (the paper's choice) and the 16-bit scale T of this
# build (the per-pixel normalised costs lie in [-2, 2]).
FASTDT_D_ARB = 0
FASTDT_T = 16383.0


def fastdt_encode(value: int, lib=None) -> int:
    """The 8-bit code of a 16-bit two's-complement value."""
    return int((lib or load()).oracle_fastdt_encode(int(value)))


def fastdt_decode(code: int, lib=None) -> int:
    """The 16-bit value an 8-bit code stands for."""
    return int((lib or load()).oracle_fastdt_decode(int(code)))


def fastdt_store(C, ahat, d_arb=FASTDT_D_ARB, T=FASTDT_T, lib=None):
    """One FastDT store of a float64 [H][W][nd] volume (returns a new array)."""
    lib = lib or load()
    C = np.array(C, dtype=np.float64, copy=True, order="C")
    H, W, nd = C.shape
    a = np.ascontiguousarray(ahat, dtype=np.float64)
    _check(lib.oracle_fastdt_store(_p(C, ctypes.c_double), _p(a, ctypes.c_double), W, H, nd, int(d_arb),
                                   float(T)), "fastdt_store")
    return C


def dt_aggregate_fastdt(C, guide, sigma_s, sigma_r, iters, d_arb=FASTDT_D_ARB, T=FASTDT_T, nthreads=None,
                        lib=None):
    """The DT chain with FastDT storage between pass pairs on a float64 [H][W][nd] volume
    (returns a new array): the aggregated volume that WTA reads."""
    lib = lib or load()
    C = np.array(C, dtype=np.float64, copy=True, order="C")
    H, W, nd = C.shape
    g = _img(guide)
    assert g.shape == (H, W)
    _check(lib.oracle_dt_aggregate_fastdt(_p(C, ctypes.c_double), _p(g, ctypes.c_uint8), W, H, nd,
                                          float(sigma_s), float(sigma_r), int(iters), int(d_arb), float(T),
                                          nthreads or default_threads()), "dt_aggregate_fastdt")
    return C


def run_fastdt(left, right, max_disp, r, sigma_s=20.0, sigma_r=0.1, iters=3, d_arb=FASTDT_D_ARB,
               T=FASTDT_T, nthreads=None, lib=None):
    """The whole path with FastDT storage between pass pairs: (disparity, gap)."""
    lib = lib or load()
    left, right = _img(left), _img(right)
    nthreads = nthreads or default_threads()
    C = zncc_volume(left, right, max_disp, r, nthreads=nthreads, lib=lib)
    H, W, _ = C.shape
    _check(lib.oracle_dt_aggregate_fastdt(_p(C, ctypes.c_double), _p(left, ctypes.c_uint8), W, H, max_disp,
                                          float(sigma_s), float(sigma_r), int(iters), int(d_arb), float(T),
                                          nthreads), "dt_aggregate_fastdt")
    disp, _, gap = wta(C, lib=lib)
    return disp, gap
