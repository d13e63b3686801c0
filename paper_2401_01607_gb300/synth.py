"""Seeded synthetic workloads for the taches-algorithm convolution.

This module holds input generators only, and none of the convolution
arithmetic. The tests use it to feed the same inputs to the CUDA path and to
the FP64 oracle, and bench.py uses it to build its workloads. It imports
nothing from the CUDA binding or from the oracle.

Stand-ins for the paper's stimuli (Sec. 5.1). The paper's musical stimuli and
its white-noise IRs, made with Audacity, are not available. Inputs are
therefore uniform[-1, 1] float32 "audio" and IRs are exponentially decayed
Gaussian noise h[k] = g_k * exp(-k / tau), with g_k ~ N(0, 1), normalised in
float64 so that sum |h| = 1 and then rounded to float32. The float32 values
are the ground truth that both sides see.

Seeds (numpy PCG64 via default_rng):
  input of stream s in workload c     1000 * c + s
  IR version v of stream s            2_000_000 + 1000 * s + v
  serving trace                       42
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FS = 48_000  # sample rate of every workload (Hz)


def audio(n: int, seed: int) -> np.ndarray:
    """n float32 samples, uniform on [-1, 1]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=int(n)).astype(np.float32)


def audio_block(rows: int, n: int, seed0: int) -> np.ndarray:
    """[rows, n] float32: row s is audio(n, seed0 + s)."""
    out = np.empty((rows, int(n)), dtype=np.float32)
    for s in range(rows):
        out[s] = audio(n, seed0 + s)
    return out


def decayed_ir(L: int, tau: float, seed: int) -> np.ndarray:
    """Exponentially decayed Gaussian noise of length L, sum |h| = 1 (float64 normalisation)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(int(L))
    h = g * np.exp(-np.arange(int(L), dtype=np.float64) / float(tau))
    h /= np.sum(np.abs(h))
    return h.astype(np.float32)


def q15_codes(a: np.ndarray) -> np.ndarray:
    """Q15 codes (int16, value = code / 2^15) of float samples: nearest code, clipped to [-32768, 32767]."""
    return np.clip(np.rint(np.asarray(a, np.float64) * 32768.0), -32768, 32767).astype(np.int16)


def q15_full_range(n: int, seed: int) -> np.ndarray:
    """n int16 codes, uniform over the whole range [-32768, 32767]."""
    return np.random.default_rng(seed).integers(-32768, 32768, int(n)).astype(np.int16)


def ir_seed(stream: int, version: int) -> int:
    return 2_000_000 + 1000 * int(stream) + int(version)


def x_seed(workload: int, stream: int) -> int:
    return 1000 * int(workload) + int(stream)


# ----------------------------------------------------------------------------
# Workload recipes. Sizes are the full ones; the tests shrink them through the
# arguments (fewer streams, shorter signals, shorter IRs) with the same recipe.
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Workload:
    name: str
    x: np.ndarray            # [C, N] float32 (MIMO: [nin, N])
    H: np.ndarray            # [C, nver, L] per stream, or [nver, L] shared, or MIMO [nver, nout, nin, L]
    vstart: np.ndarray       # [nver] int64, first sample of each IR version (same for all streams)
    L: int
    block: int
    shared_ir: bool = False
    mimo: tuple[int, int] | None = None  # (nin, nout)

    @property
    def C(self) -> int:
        return int(self.x.shape[0])

    @property
    def N(self) -> int:
        return int(self.x.shape[1])

    def tap_macs(self) -> int:
        """Useful multiply-adds of the whole job (every tache has L taps, the tail included)."""
        if self.mimo is not None:
            nin, nout = self.mimo
            return nin * nout * self.N * self.L
        return self.C * self.N * self.L


def mono(N: int = 48_000, L: int = 4096, block: int = 64, tau: float = 800.0) -> Workload:
    """Mono plain taches: one stream, one fixed IR (workload 1)."""
    x = audio(N, x_seed(1, 0))[None]
    H = decayed_ir(L, tau, ir_seed(0, 0))[None, None]
    return Workload("mono", x, H, np.zeros(1, np.int64), L, block)


def multi(C: int = 64, N: int = 480_000, L: int = 48_000, block: int = 128,
          swap_every: int = 24_000, tau: float | None = None, stream0: int = 0) -> Workload:
    """Independent streams with their own IRs, each replaced every swap_every samples (workload 2).
    Streams are numbered from stream0 (a shard of a larger set uses its own seeds)."""
    tau = 0.3 * L if tau is None else tau
    nver = max(1, -(-N // swap_every)) if swap_every else 1
    x = audio_block(C, N, x_seed(2, stream0))
    H = np.empty((C, nver, L), dtype=np.float32)
    for s in range(C):
        for v in range(nver):
            H[s, v] = decayed_ir(L, tau, ir_seed(stream0 + s, v))
    vstart = (np.arange(nver, dtype=np.int64) * swap_every) if swap_every else np.zeros(1, np.int64)
    return Workload("multi", x, H, vstart, L, block)


def shared(C: int = 1024, N: int = 240_000, L: int = 96_000, block: int = 256,
           tau: float | None = None) -> Workload:
    """Batch of streams sharing one IR (workload 3)."""
    tau = 0.2 * L if tau is None else tau
    x = audio_block(C, N, x_seed(3, 0))
    H = decayed_ir(L, tau, ir_seed(0, 0))[None]
    return Workload("shared", x, H, np.zeros(1, np.int64), L, block, shared_ir=True)


def mimo(nin: int = 16, nout: int = 16, N: int = 2_880_000, L: int = 192_000, block: int = 512,
         tau: float | None = None) -> Workload:
    """nout outputs, each the sum of nin convolutions (workload 5). IR (o, i) uses stream id o*nin+i."""
    tau = 0.2 * L if tau is None else tau
    x = audio_block(nin, N, x_seed(5, 0))
    H = np.empty((1, nout, nin, L), dtype=np.float32)
    for o in range(nout):
        for i in range(nin):
            H[0, o, i] = decayed_ir(L, tau, ir_seed(o * nin + i, 0))
    return Workload("mimo", x, H, np.zeros(1, np.int64), L, block, mimo=(nin, nout))


# ----------------------------------------------------------------------------
# Serving trace (workload 4): Poisson arrivals of streams of log-uniform
# duration and IR length, block size drawn from {32, 64, 128, 256}; 10 % of
# the streams swap their IR once at a uniform sample.
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class TraceStream:
    sid: int
    arrival_s: float
    n: int           # samples
    L: int
    block: int
    swap_at: int     # -1: no swap
    x_seed: int
    ir_seeds: tuple[int, ...]
    tau: float


def serving_trace(duration_s: float = 60.0, rate_hz: float = 200.0, dur_range=(0.5, 30.0),
                  L_range=(256, 480_000), blocks=(32, 64, 128, 256), swap_frac: float = 0.10,
                  seed: int = 42, max_streams: int | None = None) -> list[TraceStream]:
    rng = np.random.default_rng(seed)
    out: list[TraceStream] = []
    t = 0.0
    sid = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s or (max_streams is not None and sid >= max_streams):
            break
        dur = math.exp(rng.uniform(math.log(dur_range[0]), math.log(dur_range[1])))
        L = int(round(math.exp(rng.uniform(math.log(L_range[0]), math.log(L_range[1])))))
        block = int(blocks[rng.integers(len(blocks))])
        n = int(round(dur * FS))
        swap = rng.uniform() < swap_frac
        swap_at = int(rng.integers(0, n)) if swap else -1
        seeds = (ir_seed(sid, 0), ir_seed(sid, 1)) if swap else (ir_seed(sid, 0),)
        out.append(TraceStream(sid, t, n, L, block, swap_at, x_seed(4, sid), seeds, 0.2 * L))
        sid += 1
    return out
