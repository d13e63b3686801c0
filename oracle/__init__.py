"""FP64 CPU oracle for the taches-algorithm (Millot & Pele, AES 2008).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
CUDA product path never imports it, and this package imports nothing from
the product.

The arithmetic lives in ``taches_oracle.c`` (plain C, binary64, no fast-math,
no FP contraction); this module compiles it with gcc on first use and wraps
it with ctypes. Every function takes float32 inputs (widened exactly) and
returns float64 outputs.

IR versions (time-varying IR, abstract and Sec. 6 of the paper): ``H`` is
``[nver, L]`` float32 and ``vstart`` the first input sample of each version
(``vstart[0] <= 0``, strictly increasing). Sample ``n`` spawns its tache with
``H[v(n)]``, ``v(n) = max{v : vstart[v] <= n}``.

Functions:
  direct(x, H, vstart)            Eq. (4), output by output (Sec. 3.2)
  direct_at(x, H, vstart, m)      Eq. (4) at one output index
  vect(x, H, vstart)              vectorised algorithm (Sec. 4.1)
  buffer(x, H, vstart, Nb)        buffer/ring algorithm (Sec. 4.2), blocks of Nb
  BufferStream(L)                 the buffer algorithm as a push/flush stream
  mimo(X, H, vstart, Nb)          multichannel sums of buffer convolutions
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "taches_oracle.c")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_HERE, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (or one planted-mistake mutant) with gcc."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, f"-DORACLE_MUTANT={mutant}", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64


def _load(mutant: int = 0) -> ctypes.CDLL:
    with _LOCK:
        if mutant in _LIBS:
            return _LIBS[mutant]
        lib = ctypes.CDLL(build(mutant))
        sig = [_f32p, _i64, _f32p, _i64, _i64p, _i64]
        lib.tco_direct_at.argtypes = sig + [_i64]
        lib.tco_direct_at.restype = ctypes.c_double
        lib.tco_direct.argtypes = sig + [_f64p]
        lib.tco_direct.restype = ctypes.c_int
        lib.tco_vect.argtypes = sig + [_f64p]
        lib.tco_vect.restype = ctypes.c_int
        lib.tco_buffer.argtypes = sig + [_i64, _f64p]
        lib.tco_buffer.restype = ctypes.c_int
        lib.tco_buf_open.argtypes = [_i64]
        lib.tco_buf_open.restype = ctypes.c_void_p
        lib.tco_buf_close.argtypes = [ctypes.c_void_p]
        lib.tco_buf_close.restype = None
        lib.tco_buf_push.argtypes = [ctypes.c_void_p, _f32p, _i64, _f32p, _i64p, _i64, _f64p]
        lib.tco_buf_push.restype = ctypes.c_int
        lib.tco_buf_flush.argtypes = [ctypes.c_void_p, _f64p]
        lib.tco_buf_flush.restype = ctypes.c_int
        lib.tco_mimo.argtypes = [_f32p, _i64, _i64, _i64, _f32p, _i64, _i64p, _i64, _i64, _f64p]
        lib.tco_mimo.restype = ctypes.c_int
        lib.tco_direct_at_xf.argtypes = [_f32p, _i64, _f32p, _i64, _i64p, _i64p, _i64, _i64]
        lib.tco_direct_at_xf.restype = ctypes.c_double
        lib.tco_buffer_xf.argtypes = [_f32p, _i64, _f32p, _i64, _i64p, _i64p, _i64, _i64, _f64p]
        lib.tco_buffer_xf.restype = ctypes.c_int
        _i16p = np.ctypeslib.ndpointer(dtype=np.int16, flags="C_CONTIGUOUS")
        _i64o = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        lib.tco_q15_direct.argtypes = [_i16p, _i64, _i16p, _i64, _i64o, _i16p]
        lib.tco_q15_direct.restype = ctypes.c_int
        lib.tco_mutant_id.argtypes = []
        lib.tco_mutant_id.restype = ctypes.c_int
        _LIBS[mutant] = lib
        return lib


def _prep(x, H, vstart):
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    H = np.ascontiguousarray(H, dtype=np.float32)
    if H.ndim == 1:
        H = H.reshape(1, -1)
    if vstart is None:
        vstart = np.zeros(1, dtype=np.int64)
    vstart = np.ascontiguousarray(vstart, dtype=np.int64).reshape(-1)
    if H.shape[0] != vstart.shape[0]:
        raise ValueError("one vstart entry per IR version")
    return x, H, vstart


class Oracle:
    """Bound to one build (mutant 0 is the real oracle)."""

    def __init__(self, mutant: int = 0):
        self.mutant = mutant
        self.lib = _load(mutant)

    def direct_at(self, x, H, vstart, m: int) -> float:
        x, H, vstart = _prep(x, H, vstart)
        return self.lib.tco_direct_at(x, x.size, H.reshape(-1), H.shape[1], vstart, vstart.size, int(m))

    def direct_at_xf(self, x, H, vstart, vramp, m: int) -> float:
        """Eq. (4) with crossfaded IR versions (ramp lengths vramp), one output."""
        x, H, vstart = _prep(x, H, vstart)
        vramp = np.ascontiguousarray(vramp, dtype=np.int64).reshape(-1)
        return self.lib.tco_direct_at_xf(x, x.size, H.reshape(-1), H.shape[1], vstart, vramp, vstart.size, int(m))

    def buffer_xf(self, x, H, vstart, vramp, Nb: int = 8192) -> np.ndarray:
        """The Sec. 4.2 buffer algorithm with crossfaded IR versions: version v
        takes over over vramp[v] samples from vstart[v] on (1 = hard switch)."""
        x, H, vstart = _prep(x, H, vstart)
        vramp = np.ascontiguousarray(vramp, dtype=np.int64).reshape(-1)
        if vramp.size != vstart.size:
            raise ValueError("one ramp per IR version")
        y = np.empty(x.size + H.shape[1] - 1, dtype=np.float64)
        rc = self.lib.tco_buffer_xf(x, x.size, H.reshape(-1), H.shape[1], vstart, vramp, vstart.size, int(Nb), y)
        if rc:
            raise ValueError(f"tco_buffer_xf failed ({rc})")
        return y

    def q15(self, x, h):
        """Exact Q15 convolution (Sec. 5.4, one requantization): returns
        (acc int64 exact sums, y int16 requantized, round half to even)."""
        x = np.ascontiguousarray(x, dtype=np.int16).reshape(-1)
        h = np.ascontiguousarray(h, dtype=np.int16).reshape(-1)
        acc = np.empty(x.size + h.size - 1, dtype=np.int64)
        y = np.empty(x.size + h.size - 1, dtype=np.int16)
        rc = self.lib.tco_q15_direct(x, x.size, h, h.size, acc, y)
        if rc:
            raise ValueError(f"tco_q15_direct failed ({rc})")
        return acc, y

    def direct(self, x, H, vstart=None) -> np.ndarray:
        x, H, vstart = _prep(x, H, vstart)
        y = np.empty(x.size + H.shape[1] - 1, dtype=np.float64)
        rc = self.lib.tco_direct(x, x.size, H.reshape(-1), H.shape[1], vstart, vstart.size, y)
        if rc:
            raise ValueError(f"tco_direct failed ({rc})")
        return y

    def vect(self, x, H, vstart=None) -> np.ndarray:
        x, H, vstart = _prep(x, H, vstart)
        y = np.empty(x.size + H.shape[1] - 1, dtype=np.float64)
        rc = self.lib.tco_vect(x, x.size, H.reshape(-1), H.shape[1], vstart, vstart.size, y)
        if rc:
            raise ValueError(f"tco_vect failed ({rc})")
        return y

    def buffer(self, x, H, vstart=None, Nb: int = 8192) -> np.ndarray:
        x, H, vstart = _prep(x, H, vstart)
        y = np.empty(x.size + H.shape[1] - 1, dtype=np.float64)
        rc = self.lib.tco_buffer(x, x.size, H.reshape(-1), H.shape[1], vstart, vstart.size, int(Nb), y)
        if rc:
            raise ValueError(f"tco_buffer failed ({rc})")
        return y

    def mimo(self, X, H, vstart=None, Nb: int = 8192) -> np.ndarray:
        """X: [nin, N]; H: [nver, nout, nin, L] (or [nout, nin, L]); returns [nout, N+L-1]."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        H = np.ascontiguousarray(H, dtype=np.float32)
        if H.ndim == 3:
            H = H[None]
        nver, nout, nin, L = H.shape
        if X.shape[0] != nin:
            raise ValueError("X rows must equal nin")
        if vstart is None:
            vstart = np.zeros(1, dtype=np.int64)
        vstart = np.ascontiguousarray(vstart, dtype=np.int64)
        N = X.shape[1]
        y = np.empty((nout, N + L - 1), dtype=np.float64)
        rc = self.lib.tco_mimo(X.reshape(-1), nin, nout, N, H.reshape(-1), L, vstart, nver, int(Nb), y.reshape(-1))
        if rc:
            raise ValueError(f"tco_mimo failed ({rc})")
        return y

    def stream(self, L: int) -> "BufferStream":
        return BufferStream(L, self)


class BufferStream:
    """The Sec. 4.2 buffer algorithm as a persistent stream (push blocks, then flush)."""

    def __init__(self, L: int, oracle: Oracle | None = None):
        self.o = oracle or Oracle()
        self.L = int(L)
        self.h = self.o.lib.tco_buf_open(self.L)
        if not self.h:
            raise MemoryError("tco_buf_open failed")

    def push(self, pe, H, vstart=None) -> np.ndarray:
        pe = np.ascontiguousarray(pe, dtype=np.float32).reshape(-1)
        _, H, vstart = _prep(pe[:1] if pe.size else np.zeros(1, np.float32), H, vstart)
        ps = np.empty(pe.size, dtype=np.float64)
        rc = self.o.lib.tco_buf_push(self.h, pe, pe.size, H.reshape(-1), vstart, vstart.size, ps)
        if rc:
            raise ValueError(f"tco_buf_push failed ({rc})")
        return ps

    def flush(self) -> np.ndarray:
        ps = np.empty(self.L - 1, dtype=np.float64)
        self.o.lib.tco_buf_flush(self.h, ps)
        return ps

    def close(self):
        if self.h:
            self.o.lib.tco_buf_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_DEFAULT: Oracle | None = None


def default() -> Oracle:
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle(0)
    return _DEFAULT


def direct(x, H, vstart=None):
    return default().direct(x, H, vstart)


def direct_at(x, H, vstart, m):
    return default().direct_at(x, H, vstart, m)


def vect(x, H, vstart=None):
    return default().vect(x, H, vstart)


def buffer(x, H, vstart=None, Nb: int = 8192):
    return default().buffer(x, H, vstart, Nb)


def buffer_xf(x, H, vstart, vramp, Nb: int = 8192):
    return default().buffer_xf(x, H, vstart, vramp, Nb)


def direct_at_xf(x, H, vstart, vramp, m):
    return default().direct_at_xf(x, H, vstart, vramp, m)


def q15(x, h):
    return default().q15(x, h)


def mimo(X, H, vstart=None, Nb: int = 8192):
    return default().mimo(X, H, vstart, Nb)
