"""Thin ctypes binding of libzncc.so (include/zncc.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; PyTorch only provides device
memory and streams. There is no CPU fallback: if the library is missing or cannot be
loaded, every call raises.

The methods of ZnccContext carry the names of the C calls they wrap:

    zncc_window_stats, zncc_cost_volume, zncc_cost_volume_scan, zncc_cost_volume_mma,
    dt_aggregate, wta_disparity, zncc_run, zncc_run_host

and the module-level zncc_run_batch, dt_aggregate_noalloc and fastdt_codec wrap the batched
call, the context-free aggregation that allocates nothing and the FastDT code on the device.
serve_create, serve_submit, serve_poll, serve_poll_timed and serve_destroy wrap the serving
calls (a handle in, numpy arrays for the host images), and
ZnccServer bundles them.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libzncc.so")

ZNCC_OK, ZNCC_EINVAL, ZNCC_ENOMEM, ZNCC_ECUDA, ZNCC_EBUSY, ZNCC_ENOTREADY, ZNCC_ETIMEOUT, \
    ZNCC_EUNSUPPORTED = range(8)
ZNCC_F32, ZNCC_F16, ZNCC_I8 = 0, 1, 2
ZNCC_TUNE_ROW_MINB2, ZNCC_TUNE_ROW_SPB, ZNCC_TUNE_H_TQ, ZNCC_TUNE_V_TQ, ZNCC_TUNE_AHAT_SMS = 1, 2, 3, 4, 5
ZNCC_TUNE_PLANE, ZNCC_TUNE_PLANE_CS, ZNCC_TUNE_ROW_LOADS, ZNCC_TUNE_V_LPC = 6, 7, 8, 9
ZNCC_TUNE_LINE_LOADS, ZNCC_TUNE_WAIT_DRILL, ZNCC_TUNE_AHAT_JOIN = 10, 11, 12
STATUS_NAMES = ["ZNCC_OK", "ZNCC_EINVAL", "ZNCC_ENOMEM", "ZNCC_ECUDA", "ZNCC_EBUSY",
                "ZNCC_ENOTREADY", "ZNCC_ETIMEOUT", "ZNCC_EUNSUPPORTED"]

# every entry point declared in include/zncc.h: (name, restype, argtypes)
_vp, _i, _f, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
SIGNATURES = [
    ("zncc_create", _i, [_i, _i, _i, _i, ctypes.POINTER(_vp)]),
    ("zncc_destroy", _i, [_vp]),
    ("zncc_set_stream", _i, [_vp, _vp]),
    ("zncc_volume_bytes", _sz, [_vp, _i]),
    ("zncc_window_stats", _i, [_vp, _vp, _i, _vp, _vp, _vp]),
    ("zncc_cost_volume", _i, [_vp, _vp, _vp, _i, _vp, _i]),
    ("zncc_cost_volume_scan", _i, [_vp, _vp, _vp, _i, _vp, _i]),
    ("zncc_cost_volume_mma", _i, [_vp, _vp, _vp, _i, _vp, _i]),
    ("dt_aggregate", _i, [_vp, _vp, _i, _vp, _i, _f, _f, _i]),
    ("dt_aggregate_noalloc", _i, [_vp, _i, _i, _i, _i, _vp, _i, _f, _f, _i, _vp]),
    ("wta_disparity", _i, [_vp, _vp, _i, _vp]),
    ("fastdt_codec", _i, [_vp, _i, _vp, _vp, _vp]),
    ("zncc_run", _i, [_vp, _vp, _vp, _i, _f, _f, _i, _i, _vp]),
    ("zncc_run_host", _i, [_vp, _vp, _vp, _i, _f, _f, _i, _i, _vp]),
    ("zncc_run_batch", _i, [_vp, _vp, _vp, _vp, _vp, _i, _f, _f, _i, _i]),
    ("serve_create", _i, [_sz, _i, ctypes.POINTER(_vp)]),
    ("serve_submit", _i, [_vp, _vp, _vp, _i, _i, _i, _i, _f, _f, _i, _i,
                          ctypes.POINTER(ctypes.c_uint64)]),
    ("serve_poll", _i, [_vp, ctypes.c_uint64, _vp, _i]),
    ("serve_poll_timed", _i, [_vp, ctypes.c_uint64, _vp, _i, _vp]),
    ("serve_destroy", _i, [_vp]),
    ("serve_last_error", ctypes.c_char_p, [_vp]),
    ("zncc_last_error", ctypes.c_char_p, [_vp]),
    ("zncc_status_string", ctypes.c_char_p, [_i]),
    ("zncc_kernel_launch_count", ctypes.c_uint64, []),
    ("zncc_set_tuning", _i, [_vp, _i, _i]),
    ("zncc_device_faults", _i, [_vp, ctypes.POINTER(ctypes.c_uint32)]),
    ("zncc_profile_enable", _i, [_vp, _i]),
    ("zncc_profile_read", _i, [_vp, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_uint64), _i]),
    ("zncc_profile_nkinds", _i, []),
    ("zncc_profile_kind_name", ctypes.c_char_p, [_i]),
]

_lib = None
_lock = threading.Lock()


class ZnccError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


def lib():
    """The loaded library (built in-tree by build() / __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2212_00476_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(t) -> int:
    """Device pointer of a torch tensor (must be contiguous)."""
    assert t.is_contiguous(), "tensors passed to libzncc must be contiguous"
    return t.data_ptr()


def _img(t) -> int:
    """Device pointer of an image: a 2-D uint8 tensor whose rows are contiguous; its row stride
    (stride(0), at least the width) is passed as the pitch."""
    assert t.dim() == 2 and t.stride(1) == 1 and t.stride(0) >= t.shape[1], \
        "images passed to libzncc must be 2-D with contiguous rows"
    return t.data_ptr()


def _pitch(*imgs) -> int:
    """The common row pitch of images passed together."""
    p = imgs[0].stride(0)
    assert all(t.stride(0) == p for t in imgs), "images passed together must share their row pitch"
    return p


def launch_count() -> int:
    return int(lib().zncc_kernel_launch_count())


def zncc_run_batch(ctxs, lefts, rights, disps, sigma_s, sigma_r, iters, storage=ZNCC_F32):
    """One batched fused run over several pairs (each with its own ZnccContext; the first
    context's stream carries the launches)."""
    n = len(ctxs)
    VP = ctypes.c_void_p * n
    st = lib().zncc_run_batch(VP(*[c._h.value for c in ctxs]), VP(*[_img(t) for t in lefts]),
                              VP(*[_img(t) for t in rights]),
                              (ctypes.c_int * n)(*[_pitch(l, r) for l, r in zip(lefts, rights)]),
                              VP(*[_ptr(t) for t in disps]), n, float(sigma_s), float(sigma_r),
                              int(iters), int(storage))
    if st != ZNCC_OK:
        raise ZnccError(st, lib().zncc_last_error(ctxs[0]._h).decode())


def dt_aggregate_noalloc(guide, cost, sigma_s, sigma_r, iters, dtype=ZNCC_F32, stream=None):
    """DT aggregation of cost ([H][W][D] device tensor) in place, guided by guide ([H][W]
    uint8), without a context and without any allocation: the coefficients go to the
    library's static device scratch (W * H <= 2,097,152). stream: a torch.cuda.Stream or
    None (legacy default stream). Calls whose GPU work overlaps race on the scratch."""
    import torch
    if guide.dim() != 2 or guide.dtype != torch.uint8:
        raise ValueError("guide must be a 2-D uint8 tensor [H][W]")
    if cost.dim() != 3 or tuple(cost.shape[:2]) != tuple(guide.shape):
        raise ValueError(f"cost must be [H][W][D] with [H][W] = {tuple(guide.shape)}, got {tuple(cost.shape)}")
    want = {ZNCC_F32: torch.float32, ZNCC_F16: torch.float16}.get(int(dtype))
    if want is None or cost.dtype != want:
        raise ValueError(f"cost dtype {cost.dtype} does not match the storage flag {dtype}")
    if guide.device != cost.device or guide.device.type != "cuda":
        raise ValueError("guide and cost must be tensors on the same CUDA device")
    H, W = int(guide.shape[0]), int(guide.shape[1])
    D = int(cost.shape[-1])
    s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    st = lib().dt_aggregate_noalloc(_img(guide), guide.stride(0), W, H, D, _ptr(cost), int(dtype),
                                    float(sigma_s), float(sigma_r), int(iters), s)
    if st != ZNCC_OK:
        raise ZnccError(st, lib().zncc_last_error(None).decode())


def fastdt_codec(values, codes=None, decoded=None, stream=None):
    """The FastDT codes (uint8 device tensor) of int16 device values and the values they
    decode to (int16), on the device (Sec. IV-C)."""
    n = int(values.numel())
    s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    st = lib().fastdt_codec(_ptr(values), n, None if codes is None else _ptr(codes),
                            None if decoded is None else _ptr(decoded), s)
    if st != ZNCC_OK:
        raise ZnccError(st, lib().zncc_last_error(None).decode())


def serve_create(volume_budget_bytes: int, max_slots: int):
    """A server handle (ctypes.c_void_p)."""
    h = _vp()
    st = lib().serve_create(int(volume_budget_bytes), int(max_slots), ctypes.byref(h))
    if st != ZNCC_OK:
        raise ZnccError(st, "serve_create")
    return h


def serve_submit(server, left: np.ndarray, right: np.ndarray, max_disp: int, win: int,
                 sigma_s: float, sigma_r: float, iters: int, storage: int = ZNCC_F32) -> int:
    """Queue one pair (uint8 [H][W] host arrays, copied before return); returns its ticket."""
    assert left.dtype == np.uint8 and right.dtype == np.uint8 and left.shape == right.shape
    left = np.ascontiguousarray(left)
    right = np.ascontiguousarray(right)
    t = ctypes.c_uint64()
    st = lib().serve_submit(server, left.ctypes.data, right.ctypes.data, left.shape[1],
                            left.shape[0], int(max_disp), int(win), float(sigma_s),
                            float(sigma_r), int(iters), int(storage), ctypes.byref(t))
    if st != ZNCC_OK:
        raise ZnccError(st, lib().serve_last_error(server).decode() or "serve_submit")
    return int(t.value)


def serve_poll(server, ticket: int, disp: np.ndarray, timeout_us: int = 0) -> int:
    """Status of a request (ZNCC_OK: its map is now in disp, uint16 [H][W]); ZNCC_ENOTREADY
    and ZNCC_ETIMEOUT are returned, not raised, as are the request's own errors."""
    assert disp.dtype == np.uint16 and disp.flags.c_contiguous
    return int(lib().serve_poll(server, ctypes.c_uint64(ticket), disp.ctypes.data, int(timeout_us)))


class ServeTiming(ctypes.Structure):
    """zncc_serve_timing: where a served request's latency went (milliseconds)."""
    _fields_ = [("queue_ms", ctypes.c_double), ("device_wait_ms", ctypes.c_double),
                ("h2d_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("d2h_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("batch_pairs", ctypes.c_int), ("valid", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def serve_poll_timed(server, ticket: int, disp: np.ndarray, timeout_us: int = 0):
    """serve_poll, plus the request's latency breakdown once it has finished: (status, dict or
    None)."""
    assert disp.dtype == np.uint16 and disp.flags.c_contiguous
    t = ServeTiming()
    st = int(lib().serve_poll_timed(server, ctypes.c_uint64(ticket), disp.ctypes.data, int(timeout_us),
                                    ctypes.byref(t)))
    return st, (t.as_dict() if st == ZNCC_OK and t.valid else None)


def serve_destroy(server) -> int:
    return int(lib().serve_destroy(server))


class ZnccServer:
    """A libzncc server: queue pairs from host memory, poll their disparity maps."""

    def __init__(self, volume_budget_bytes: int, max_slots: int = 32):
        self._h = serve_create(volume_budget_bytes, max_slots)

    def submit(self, left, right, max_disp, win, sigma_s, sigma_r, iters, storage=ZNCC_F32):
        return serve_submit(self._h, left, right, max_disp, win, sigma_s, sigma_r, iters, storage)

    def poll(self, ticket, disp, timeout_us=0):
        return serve_poll(self._h, ticket, disp, timeout_us)

    def poll_timed(self, ticket, disp, timeout_us=0):
        return serve_poll_timed(self._h, ticket, disp, timeout_us)

    def last_error(self) -> str:
        return lib().serve_last_error(self._h).decode()

    def close(self) -> int:
        st = ZNCC_OK
        if getattr(self, "_h", None) is not None:
            st = serve_destroy(self._h)
            self._h = None
        return st

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class ZnccContext:
    """A libzncc context for W x H pairs, disparities [0, max_disp), window side `win`."""

    def __init__(self, width: int, height: int, max_disp: int, win: int, stream=None):
        L = lib()
        h = _vp()
        st = L.zncc_create(int(width), int(height), int(max_disp), int(win), ctypes.byref(h))
        if st != ZNCC_OK:
            raise ZnccError(st, L.zncc_last_error(None).decode())
        self._h = h
        self.stream = None
        self.W, self.H, self.D, self.win = int(width), int(height), int(max_disp), int(win)
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime ---------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().zncc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        if st != ZNCC_OK:
            raise ZnccError(st, lib().zncc_last_error(self._h).decode())

    def set_stream(self, stream):
        """Bind a torch.cuda.Stream (or a raw cudaStream_t int, or None)."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(lib().zncc_set_stream(self._h, raw or None))
        self.stream = stream if hasattr(stream, "cuda_stream") else None

    def volume_bytes(self, dtype: int = ZNCC_F32) -> int:
        return int(lib().zncc_volume_bytes(self._h, dtype))

    def set_tuning(self, key: int, value: int):
        self._check(lib().zncc_set_tuning(self._h, int(key), int(value)))

    def device_faults(self) -> int:
        """Faults the context's kernels recorded on the device since the last call (0: none)."""
        v = ctypes.c_uint32(0)
        self._check(lib().zncc_device_faults(self._h, ctypes.byref(v)))
        return int(v.value)

    def profile_enable(self, on: bool = True):
        self._check(lib().zncc_profile_enable(self._h, 1 if on else 0))

    def profile_read(self) -> dict:
        """{kernel kind: (total device ms, launches)} since the previous read."""
        L = lib()
        n = L.zncc_profile_nkinds()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_uint64 * n)()
        self._check(L.zncc_profile_read(self._h, ms, cnt, n))
        return {L.zncc_profile_kind_name(k).decode(): (ms[k], int(cnt[k])) for k in range(n)
                if cnt[k]}

    # -- the C calls --------------------------------------------------------------------
    def zncc_window_stats(self, img, S=None, Q=None, inv_sigma=None):
        self._check(lib().zncc_window_stats(self._h, _img(img), img.stride(0),
                                            _ptr(S) if S is not None else None,
                                            _ptr(Q) if Q is not None else None,
                                            _ptr(inv_sigma) if inv_sigma is not None else None))

    def zncc_cost_volume(self, left, right, cost, dtype: int = ZNCC_F32):
        self._check(lib().zncc_cost_volume(self._h, _img(left), _img(right), _pitch(left, right),
                                           _ptr(cost), dtype))

    def zncc_cost_volume_scan(self, left, right, cost, dtype: int = ZNCC_F32):
        self._check(lib().zncc_cost_volume_scan(self._h, _img(left), _img(right), _pitch(left, right),
                                                _ptr(cost), dtype))

    def zncc_cost_volume_mma(self, left, right, cost, dtype: int = ZNCC_F32):
        self._check(lib().zncc_cost_volume_mma(self._h, _img(left), _img(right), _pitch(left, right),
                                               _ptr(cost), dtype))

    def dt_aggregate(self, guide, cost, sigma_s: float, sigma_r: float, iters: int,
                     dtype: int = ZNCC_F32):
        self._check(lib().dt_aggregate(self._h, _img(guide), guide.stride(0), _ptr(cost), dtype,
                                       float(sigma_s), float(sigma_r), int(iters)))

    def wta_disparity(self, cost, disp, dtype: int = ZNCC_F32):
        self._check(lib().wta_disparity(self._h, _ptr(cost), dtype, _ptr(disp)))

    def zncc_run(self, left, right, disp, sigma_s: float, sigma_r: float, iters: int,
                 storage: int = ZNCC_F32):
        self._check(lib().zncc_run(self._h, _img(left), _img(right), _pitch(left, right),
                                   float(sigma_s), float(sigma_r), int(iters), int(storage),
                                   _ptr(disp)))

    def zncc_run_host(self, left: np.ndarray, right: np.ndarray, disp: np.ndarray,
                      sigma_s: float, sigma_r: float, iters: int, storage: int = ZNCC_F32):
        assert left.dtype == np.uint8 and right.dtype == np.uint8 and disp.dtype == np.uint16
        assert left.flags.c_contiguous and right.flags.c_contiguous and disp.flags.c_contiguous
        self._check(lib().zncc_run_host(self._h, left.ctypes.data, right.ctypes.data,
                                        left.strides[0], float(sigma_s), float(sigma_r),
                                        int(iters), int(storage), disp.ctypes.data))
