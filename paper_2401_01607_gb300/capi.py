"""Python binding of the C ABI in include/taches.h (argument marshalling only).

Every function has the name of its C entry point and does no computing of its
own: it converts arguments (numpy arrays for host buffers, torch CUDA tensors
or raw integers for device buffers), calls libtaches.so and raises TcError on
a non-zero tc_status. Out-parameters become return values.

The library is loaded on first use. If libtaches.so is missing or fails to
load, the call raises at once: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

TC_FP32, TC_BF16, TC_BF16_SPLIT = 0, 1, 2
STATUS = {0: "TC_OK", 1: "TC_EINVAL", 2: "TC_ENOMEM", 3: "TC_ESTATE", 4: "TC_ECUDA", 5: "TC_ETIMEOUT",
          6: "TC_EUNSUPPORTED"}
PRECISIONS = {"fp32": TC_FP32, "bf16": TC_BF16, "bf16split": TC_BF16_SPLIT}


class TcError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        self.status = status
        self.code = STATUS.get(status, str(status))
        super().__init__(f"{fn}: {self.code}: {msg}")


class TcInfo(ctypes.Structure):
    _fields_ = [("channels", ctypes.c_size_t), ("outputs", ctypes.c_size_t), ("L", ctypes.c_size_t),
                ("block", ctypes.c_size_t), ("max_push", ctypes.c_size_t), ("pushed", ctypes.c_uint64),
                ("shared_ir", ctypes.c_int), ("precision", ctypes.c_int), ("state", ctypes.c_int),
                ("max_versions", ctypes.c_int), ("tensor_launches", ctypes.c_uint64),
                ("fp32_fallbacks", ctypes.c_uint64)]


class TcServerStats(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_size_t), ("mem_used", ctypes.c_size_t), ("mem_budget", ctypes.c_size_t),
                ("steps", ctypes.c_uint64), ("blocks", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("busy_s", ctypes.c_double), ("tap_macs", ctypes.c_double),
                ("tensor_launches", ctypes.c_uint64), ("fp32_fallbacks", ctypes.c_uint64),
                ("k1_ms", ctypes.c_double), ("k1_macs", ctypes.c_double), ("pool_admissions", ctypes.c_uint64),
                ("grows", ctypes.c_uint64), ("host_collect_s", ctypes.c_double), ("host_pack_s", ctypes.c_double),
                ("host_deliver_s", ctypes.c_double)]


class TcServerStepRec(ctypes.Structure):
    _fields_ = [("t_begin", ctypes.c_double), ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double),
                ("blocks", ctypes.c_uint32), ("samples", ctypes.c_uint32), ("ctas", ctypes.c_uint32),
                ("variant", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_u64 = ctypes.c_uint64
_int = ctypes.c_int
_SIGS = {
    "tc_open_stream": [_sz, _sz, ctypes.POINTER(_vp)],
    "tc_open_group": [_sz, _sz, _sz, _int, _int, _sz, ctypes.POINTER(_vp)],
    "tc_open_mimo": [_sz, _sz, _sz, _sz, _int, _sz, ctypes.POINTER(_vp)],
    "tc_close": [_vp],
    "tc_reset": [_vp],
    "tc_set_max_versions": [_vp, _int],
    "tc_set_cuda_stream": [_vp, _vp],
    "tc_get_info": [_vp, ctypes.POINTER(TcInfo)],
    "tc_set_ir": [_vp, _vp, _sz],
    "tc_set_ir_at": [_vp, _vp, _sz, _u64],
    "tc_set_crossfade": [_vp, _sz],
    "tc_set_ir_rows": [_vp, _vp, _sz, _u64, _int],
    "tc_push_block": [_vp, _vp, _sz, _vp],
    "tc_push": [_vp, _vp, _sz, _vp, _int],
    "tc_flush": [_vp, _vp, _sz, ctypes.POINTER(_sz)],
    "tc_flush_dev": [_vp, _vp, ctypes.POINTER(_sz)],
    "tc_sync": [_vp],
    "tc_convolve": [_vp, _sz, _vp, _sz, _vp, _vp],
    "tc_convolve_noalloc": [_vp, _sz, _vp, _sz, _vp, _vp],
    "tc_convolve_q15": [_vp, _sz, _vp, _sz, _vp, _vp, _vp],
    "tc_convolve_tc": [_vp, _sz, _vp, _sz, _vp, _int, _vp],
    "tc_selftest_wait": [ctypes.c_ulonglong, _vp],
    "tc_test_inject": [ctypes.c_int, ctypes.c_int],
    "tc_stream_export": [_vp, _vp, _sz, ctypes.POINTER(_sz)],
    "tc_stream_import": [_vp, _vp, _sz],
    "tc_set_tuning": [_vp, _int, ctypes.c_longlong],
    "tc_profile": [_vp, _int],
    "tc_profile_read": [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_u64), ctypes.POINTER(ctypes.c_double)],
    "tc_server_open": [_sz, _sz, ctypes.POINTER(_vp)],
    "tc_server_close": [_vp],
    "tc_server_reserve": [_vp, _sz],
    "tc_server_add": [_vp, _sz, _sz, _vp, _sz, _int, ctypes.POINTER(_u64)],
    "tc_open_stream_ex": [_sz, _sz, _int, _int, _sz, ctypes.POINTER(_vp)],
    "tc_server_add_group": [_vp, _sz, _sz, _sz, _vp, _sz, _int, _int, ctypes.POINTER(_u64)],
    "tc_server_set_ir_at": [_vp, _u64, _vp, _sz, _u64],
    "tc_server_submit": [_vp, _u64, _vp, _sz],
    "tc_server_submit_many": [_vp, _sz, _vp, _vp, _vp, _vp],
    "tc_server_step": [_vp, ctypes.POINTER(_sz)],
    "tc_server_start": [_vp],
    "tc_server_stop": [_vp],
    "tc_server_poll": [_vp, _u64, _vp, _sz, ctypes.POINTER(_sz), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_double)],
    "tc_server_flush": [_vp, _u64, _vp, _sz, ctypes.POINTER(_sz)],
    "tc_server_remove": [_vp, _u64],
    "tc_server_get_stats": [_vp, ctypes.POINTER(TcServerStats)],
    "tc_server_latencies": [_vp, _vp, _vp, _sz, ctypes.POINTER(_sz)],
    "tc_server_latencies_ex": [_vp, _vp, _vp, _vp, _vp, _sz, ctypes.POINTER(_sz)],
    "tc_server_attach_source": [_vp, _u64, _vp, _sz, ctypes.c_double, ctypes.c_double],
    "tc_server_stream_state": [_vp, _u64, ctypes.POINTER(_int)],
    "tc_server_step_log": [_vp, _vp, _sz, ctypes.POINTER(_sz)],
    "tc_server_set_option": [_vp, _int, _int],
}


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Loads libtaches.so (raising if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built: run __graft_entry__.build() (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.tc_last_error.argtypes = []
        lib.tc_last_error.restype = ctypes.c_char_p
        lib.tc_status_str.argtypes = [ctypes.c_int]
        lib.tc_status_str.restype = ctypes.c_char_p
        lib.tc_kernel_launches.argtypes = []
        lib.tc_kernel_launches.restype = ctypes.c_uint64
        lib.tc_server_clock.argtypes = []
        lib.tc_server_clock.restype = ctypes.c_double
        _lib = lib
        return lib


def _call(name: str, *args) -> None:
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        raise TcError(st, name, lib.tc_last_error().decode(errors="replace"))


def _host_f32(a, writable=False):
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags.c_contiguous:
        if writable:
            raise TypeError("host output must be a C-contiguous float32 numpy array")
        a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_vp)


def _dev_ptr(t, dtype: str = "float32") -> int:
    """Device address of a torch CUDA tensor (of `dtype`, contiguous) or a raw integer address."""
    if isinstance(t, int):
        return t
    if getattr(t, "is_cuda", False):
        if not t.is_contiguous():
            raise ValueError("device tensor must be contiguous")
        if str(t.dtype) != "torch." + dtype:
            raise TypeError(f"device tensor must be {dtype}")
        return int(t.data_ptr())
    raise TypeError("expected a torch CUDA tensor or an integer device address")


# ---------------------------------------------------------------------------
# Entry points (same names as include/taches.h)
# ---------------------------------------------------------------------------

def tc_open_stream(L: int, block: int) -> int:
    h = _vp()
    _call("tc_open_stream", L, block, ctypes.byref(h))
    return h.value


def tc_open_stream_ex(L: int, block: int, precision: int = TC_FP32, device: int = -1, max_push: int = 0) -> int:
    h = _vp()
    _call("tc_open_stream_ex", L, block, int(precision), int(device), max_push, ctypes.byref(h))
    return h.value


def tc_open_group(channels: int, L: int, block: int, shared_ir: bool, precision: int = TC_FP32,
                  max_push: int = 0) -> int:
    h = _vp()
    _call("tc_open_group", channels, L, block, int(bool(shared_ir)), int(precision), max_push, ctypes.byref(h))
    return h.value


def tc_open_mimo(nin: int, nout: int, L: int, block: int, precision: int = TC_FP32, max_push: int = 0) -> int:
    h = _vp()
    _call("tc_open_mimo", nin, nout, L, block, int(precision), max_push, ctypes.byref(h))
    return h.value


def tc_close(s: int) -> None:
    _call("tc_close", s)


def tc_reset(s: int) -> None:
    _call("tc_reset", s)


def tc_set_max_versions(s: int, max_versions: int) -> None:
    _call("tc_set_max_versions", s, max_versions)


def tc_set_cuda_stream(s: int, cuda_stream) -> None:
    """cuda_stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    if cuda_stream is None:
        ptr = None
    elif isinstance(cuda_stream, int):
        ptr = cuda_stream
    else:
        ptr = int(cuda_stream.cuda_stream)
    _call("tc_set_cuda_stream", s, ptr)


def tc_get_info(s: int) -> TcInfo:
    info = TcInfo()
    _call("tc_get_info", s, ctypes.byref(info))
    return info


def tc_set_ir(s: int, h) -> None:
    h, p = _host_f32(h)
    _call("tc_set_ir", s, p, h.size)


def tc_set_ir_at(s: int, h, sample: int) -> None:
    h, p = _host_f32(h)
    _call("tc_set_ir_at", s, p, h.size, int(sample))


def tc_set_crossfade(s: int, ramp: int) -> None:
    _call("tc_set_crossfade", s, int(ramp))


def tc_set_ir_rows(s: int, h, n: int, sample: int, on_device: bool = False) -> None:
    """h: [sets][n] float32 (host numpy, or device tensor when on_device)."""
    if on_device:
        _call("tc_set_ir_rows", s, _dev_ptr(h), n, int(sample), 1)
    else:
        h, p = _host_f32(h)
        _call("tc_set_ir_rows", s, p, n, int(sample), 0)


def tc_push_block(s: int, x, y) -> None:
    """x: host [channels][n] float32; y: host [outputs][n] float32, written in place."""
    x, px = _host_f32(x)
    y, py = _host_f32(y, writable=True)
    n = x.shape[-1]
    _call("tc_push_block", s, px, n, py)


TC_PUSH_HOST, TC_PUSH_DEVICE, TC_PUSH_PINNED_ASYNC = 0, 1, 2


def tc_push(s: int, x, n: int, y, on_device: int = TC_PUSH_HOST) -> None:
    """on_device: TC_PUSH_HOST (numpy buffers, synchronous), TC_PUSH_DEVICE (device tensors or addresses,
    enqueued) or TC_PUSH_PINNED_ASYNC (page-locked numpy buffers, enqueued; complete after tc_sync)."""
    mode = int(on_device)
    if mode == TC_PUSH_DEVICE:
        _call("tc_push", s, _dev_ptr(x), n, _dev_ptr(y), 1)
    else:
        x, px = _host_f32(x)
        y, py = _host_f32(y, writable=True)
        _call("tc_push", s, px, n, py, mode)


def tc_flush(s: int, y, cap: int) -> int:
    y, py = _host_f32(y, writable=True)
    n = _sz()
    _call("tc_flush", s, py, cap, ctypes.byref(n))
    return n.value


def tc_flush_dev(s: int, y) -> int:
    n = _sz()
    _call("tc_flush_dev", s, _dev_ptr(y), ctypes.byref(n))
    return n.value


def tc_sync(s: int) -> None:
    _call("tc_sync", s)


def tc_convolve(x, N: int, h, L: int, y, cuda_stream=None) -> None:
    cs = None if cuda_stream is None else (cuda_stream if isinstance(cuda_stream, int) else
                                           int(cuda_stream.cuda_stream))
    _call("tc_convolve", _dev_ptr(x), N, _dev_ptr(h), L, _dev_ptr(y), cs)


(TC_TUNE_K1_CHUNK, TC_TUNE_K2_RANGE, TC_TUNE_K2_PAIR, TC_TUNE_ZERO_SKIP, TC_TUNE_K2_SPLIT, TC_TUNE_K2_FOLD,
 TC_TUNE_K2_ORDER) = range(7)


def tc_set_tuning(s: int, knob: int, value: int) -> None:
    _call("tc_set_tuning", s, int(knob), int(value))


def tc_profile(s: int, enable: bool = True) -> None:
    _call("tc_profile", s, int(bool(enable)))


def tc_profile_read(s: int) -> tuple[float, int, float]:
    """Returns (kernel ms, timed launches, useful multiply-adds) and clears them."""
    ms, n, macs = ctypes.c_double(), _u64(), ctypes.c_double()
    _call("tc_profile_read", s, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(macs))
    return ms.value, int(n.value), macs.value


def tc_convolve_noalloc(x, N: int, h, L: int, y, cuda_stream=None) -> None:
    """As tc_convolve, for callers that cannot allocate: the working memory is a
    fixed 32 MiB device array inside the library (calls must not overlap)."""
    cs = None if cuda_stream is None else (cuda_stream if isinstance(cuda_stream, int) else
                                           int(cuda_stream.cuda_stream))
    _call("tc_convolve_noalloc", _dev_ptr(x), N, _dev_ptr(h), L, _dev_ptr(y), cs)


def tc_convolve_tc(x, N: int, h, L: int, y, precision: int = TC_BF16_SPLIT, cuda_stream=None) -> None:
    """One signal through one IR with the products on the tensor cores (device float32 tensors)."""
    cs = None if cuda_stream is None else (cuda_stream if isinstance(cuda_stream, int) else
                                           int(cuda_stream.cuda_stream))
    _call("tc_convolve_tc", _dev_ptr(x), N, _dev_ptr(h), L, _dev_ptr(y), int(precision), cs)


def tc_convolve_q15(x, N: int, h, L: int, y, acc=None, cuda_stream=None) -> None:
    """Exact Q15 convolution with one requantization per output (Sec. 5.4).
    x (N), h (L), y (N+L-1) are int16 codes on the device; acc, if given, gets the
    exact int64 sums (N+L-1). y may be None when acc is given."""
    cs = None if cuda_stream is None else (cuda_stream if isinstance(cuda_stream, int) else
                                           int(cuda_stream.cuda_stream))
    _call("tc_convolve_q15", _dev_ptr(x, "int16"), N, _dev_ptr(h, "int16"), L,
          None if y is None else _dev_ptr(y, "int16"), None if acc is None else _dev_ptr(acc, "int64"), cs)


def tc_selftest_wait(limit_ns: int, cuda_stream=None) -> None:
    """Runs the bounded-wait check; raises TcError with code TC_ETIMEOUT, its expected outcome."""
    cs = None if cuda_stream is None else (cuda_stream if isinstance(cuda_stream, int) else
                                           int(cuda_stream.cuda_stream))
    _call("tc_selftest_wait", int(limit_ns), cs)


def tc_stream_export(s: int) -> bytes:
    """Checkpoint of the stream (host blob)."""
    n = _sz()
    _call("tc_stream_export", s, None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(max(int(n.value), 1))
    _call("tc_stream_export", s, buf, int(n.value), ctypes.byref(n))
    return buf.raw[:int(n.value)]


def tc_stream_import(s: int, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    _call("tc_stream_import", s, buf, len(blob))


def tc_last_error() -> str:
    return load().tc_last_error().decode(errors="replace")


def tc_status_str(st: int) -> str:
    return load().tc_status_str(st).decode()


TC_INJECT_PUSH_COPY, TC_INJECT_SERVER_STEP = 1, 2


def tc_test_inject(site: int, nth: int) -> None:
    """Test hook: the nth next pass through `site` reports a failure instead of making its call (0 disarms)."""
    _call("tc_test_inject", int(site), int(nth))


def tc_kernel_launches() -> int:
    return int(load().tc_kernel_launches())


# ---------------------------------------------------------------------------
# Serving (tc_server_*): continuous batching of many independent streams
# ---------------------------------------------------------------------------

TC_SERVER_DISCARD_OUTPUT = 1
TC_SERVER_AUTOTUNE, TC_SERVER_GRAPH = 0, 1


def tc_server_set_option(srv: int, option: int, value: int) -> None:
    _call("tc_server_set_option", srv, int(option), int(value))


def tc_server_open(mem_budget_bytes: int, max_step_samples: int = 0) -> int:
    h = _vp()
    _call("tc_server_open", int(mem_budget_bytes), int(max_step_samples), ctypes.byref(h))
    return h.value


def tc_server_close(srv: int) -> None:
    _call("tc_server_close", srv)


def tc_server_reserve(srv: int, nbytes: int) -> None:
    """Maps nbytes of device memory into the server's pool now, so that later admissions do not map
    memory while steps run."""
    _call("tc_server_reserve", srv, int(nbytes))


def tc_server_add(srv: int, L: int, block: int, h, flags: int = 0) -> int:
    h, hp = _host_f32(h)
    sid = _u64()
    _call("tc_server_add", srv, int(L), int(block), hp, h.size, int(flags), ctypes.byref(sid))
    return int(sid.value)


def tc_server_add_group(srv: int, channels: int, L: int, block: int, h, precision: int = 0, flags: int = 0) -> int:
    """A group of `channels` rows sharing IR h; its blocks are [channels][n]."""
    h, hp = _host_f32(h)
    sid = _u64()
    _call("tc_server_add_group", srv, int(channels), int(L), int(block), hp, h.size, int(precision), int(flags),
          ctypes.byref(sid))
    return int(sid.value)


def tc_server_set_ir_at(srv: int, sid: int, h, sample: int) -> None:
    h, hp = _host_f32(h)
    _call("tc_server_set_ir_at", srv, int(sid), hp, h.size, int(sample))


def tc_server_submit(srv: int, sid: int, x) -> None:
    """x: one block, 1-D (a stream) or [channels][n] (a group)."""
    x, xp = _host_f32(x)
    n = x.shape[-1] if x.ndim == 2 else x.size
    _call("tc_server_submit", srv, int(sid), xp, n)


def tc_server_submit_many(srv: int, ids, x_addrs, ns, t_ready=None) -> None:
    """ids: uint64 array; x_addrs: int64 array of host float32 addresses (the
    caller keeps those buffers alive for the call); ns: sample counts;
    t_ready: ready times on tc_server_clock() or None."""
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    xa = np.ascontiguousarray(x_addrs, dtype=np.uint64)
    ns = np.ascontiguousarray(ns, dtype=np.uint64)
    if not (ids.size == xa.size == ns.size):
        raise ValueError("ids, x_addrs and ns must have the same length")
    tr = None if t_ready is None else np.ascontiguousarray(t_ready, dtype=np.float64)
    if tr is not None and tr.size != ids.size:
        raise ValueError("t_ready must have one entry per block")
    _call("tc_server_submit_many", srv, ids.size, ids.ctypes.data_as(_vp), xa.ctypes.data_as(_vp),
          ns.ctypes.data_as(_vp), None if tr is None else tr.ctypes.data_as(_vp))


def tc_server_attach_source(srv: int, sid: int, x, t0: float, fs: float = 48_000.0) -> None:
    """x: C-contiguous float32 numpy array or an integer host address paired
    with n via (addr, n). The caller keeps x alive until the stream is removed."""
    if isinstance(x, tuple):
        addr, n = x
        _call("tc_server_attach_source", srv, int(sid), _vp(int(addr)), int(n), float(t0), float(fs))
        return
    if not isinstance(x, np.ndarray) or x.dtype != np.float32 or not x.flags.c_contiguous:
        raise TypeError("a live source must be a C-contiguous float32 numpy array (it is read in place)")
    n = x.shape[-1] if x.ndim == 2 else x.size  # a group's source is [channels][n]
    _call("tc_server_attach_source", srv, int(sid), x.ctypes.data_as(_vp), n, float(t0), float(fs))


def tc_server_stream_state(srv: int, sid: int) -> int:
    st = _int()
    _call("tc_server_stream_state", srv, int(sid), ctypes.byref(st))
    return int(st.value)


def tc_server_step(srv: int) -> int:
    n = _sz()
    _call("tc_server_step", srv, ctypes.byref(n))
    return int(n.value)


def tc_server_start(srv: int) -> None:
    _call("tc_server_start", srv)


def tc_server_stop(srv: int) -> None:
    _call("tc_server_stop", srv)


def tc_server_poll(srv: int, sid: int, y):
    """Fills y with the stream's oldest finished block; returns (n, t_submit,
    t_done), n = 0 if none is ready."""
    y, yp = _host_f32(y, writable=True)
    n, ts, td = _sz(), ctypes.c_double(), ctypes.c_double()
    _call("tc_server_poll", srv, int(sid), yp, y.size, ctypes.byref(n), ctypes.byref(ts), ctypes.byref(td))
    return int(n.value), ts.value, td.value


def tc_server_flush(srv: int, sid: int, y) -> int:
    y, yp = _host_f32(y, writable=True)
    n = _sz()
    _call("tc_server_flush", srv, int(sid), yp, y.size, ctypes.byref(n))
    return int(n.value)


def tc_server_remove(srv: int, sid: int) -> None:
    _call("tc_server_remove", srv, int(sid))


def tc_server_get_stats(srv: int) -> TcServerStats:
    st = TcServerStats()
    _call("tc_server_get_stats", srv, ctypes.byref(st))
    return st


def tc_server_latencies(srv: int, cap: int = 1 << 20):
    """Returns every recorded (latency seconds, nominal block size) pair as two
    arrays and forgets them."""
    lats, blks = [], []
    while True:
        out = np.empty(int(cap), dtype=np.float64)
        blk = np.empty(int(cap), dtype=np.uint32)
        n = _sz()
        _call("tc_server_latencies", srv, out.ctypes.data_as(_vp), blk.ctypes.data_as(_vp), out.size,
              ctypes.byref(n))
        k = int(n.value)
        lats.append(out[:k])
        blks.append(blk[:k])
        if k < cap:
            break
    return np.concatenate(lats), np.concatenate(blks)


def tc_server_latencies_ex(srv: int, cap: int = 1 << 20):
    """As tc_server_latencies, plus a [n, 3] float32 array of each latency's parts (seconds): ready -> taken
    into a step, taken -> enqueued, enqueued -> on the host; and a uint8 kind per block (0 plain stream,
    1 + precision for a group)."""
    lats, blks, parts, kinds = [], [], [], []
    while True:
        out = np.empty(int(cap), dtype=np.float64)
        blk = np.empty(int(cap), dtype=np.uint32)
        prt = np.empty((int(cap), 3), dtype=np.float32)
        knd = np.empty(int(cap), dtype=np.uint8)
        n = _sz()
        _call("tc_server_latencies_ex", srv, out.ctypes.data_as(_vp), blk.ctypes.data_as(_vp),
              prt.ctypes.data_as(_vp), knd.ctypes.data_as(_vp), out.size, ctypes.byref(n))
        k = int(n.value)
        lats.append(out[:k])
        blks.append(blk[:k])
        parts.append(prt[:k])
        kinds.append(knd[:k])
        if k < cap:
            break
    return np.concatenate(lats), np.concatenate(blks), np.concatenate(parts), np.concatenate(kinds)


def tc_server_step_log(srv: int, cap: int = 1 << 16) -> np.ndarray:
    """Step log as a structured array (t_begin, t_launch, t_done, blocks,
    samples, ctas, variant), oldest first; clears the log."""
    buf = (TcServerStepRec * int(cap))()
    n = _sz()
    _call("tc_server_step_log", srv, ctypes.cast(buf, _vp), int(cap), ctypes.byref(n))
    dt = np.dtype([("t_begin", "f8"), ("t_launch", "f8"), ("t_done", "f8"), ("blocks", "u4"), ("samples", "u4"),
                   ("ctas", "u4"), ("variant", "u4")])
    return np.frombuffer(bytes(buf), dtype=dt, count=int(n.value)).copy()


def tc_server_clock() -> float:
    return float(load().tc_server_clock())
