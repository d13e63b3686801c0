#!/usr/bin/env python3
"""Benchmark of the taches-algorithm convolution on GB300.

Workload (one step): 64 independent streams x 10 s at 48 kHz (480000 float32
samples each, uniform [-1, 1]). Each stream has its own IR of L = 48000 taps
(exp-decayed Gaussian, tau = 14400), and the IR is replaced by a new seeded
one every 24000 samples. Odd swaps fall inside a 128-sample block, and each
swap takes effect at its exact sample. Block size is 128. Every input is
pushed through the C ABI, followed by the L-1 sample flush. Useful work:
64 * 480000 * 48000 tap multiply-adds.

  value    tap-MAC/s with inputs (x and every IR version) resident in device
           memory (device-pointer pushes of P samples per launch)
  e2e      the same step through the C ABI with host buffers (host->device
           copies of x and IRs and device->host copy of y inside the timed region)
  roofline K1 (FP32 gather) useful FLOP/s over its CUDA-event time, against the
           FP32 FMA peak n_SM x 128 FMA/clk x 2 FLOP x 2.07 GHz (n_SM queried on
           the device; the fraction at the sampled median SM clock beside it)
  latency  p50/p99 of one 128-sample block for all 64 streams (host buffers)
           against the real-time deadline 128/48000 s
  cpu_baseline  the FP64 oracle (buffer algorithm) on the host cores, on a
           bounded sample of the same workload

Under torchrun each rank runs its own 64 streams (weak scaling, no collective
on the data path).

Output: each side section (shared IR, MIMO, mono, Q15, one-shot, extensions,
serving) is printed as its own JSON line first; the headline is the LAST line,
one compact JSON object (impl "ours") that carries a few scalars of each side
section. --full-json PATH also writes every section in full to PATH.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2401_01607_gb300 import synth  # noqa: E402  (no CUDA at import)

C_STREAMS = 64
N_SAMPLES = 480_000
L_TAPS = 48_000
BLOCK = 128
SWAP = 24_000
FS = synth.FS
SM_COUNT = 152  # replaced by the device's own count once CUDA is up (set_sm_count)
FMA_PER_CLK = 128
SM_MAX_MHZ = 2070.0
METRIC = "tap-MAC/s and concurrent 48 kHz real-time streams per GB300; p99 block latency"
K2_SRC = os.path.join(ROOT, "paper_2401_01607_gb300", "csrc", "k2_toeplitz_tc.cu")
K3_SRC = os.path.join(ROOT, "paper_2401_01607_gb300", "csrc", "k3_mimo_tc.cu")


def set_sm_count(n: int) -> None:
    """The FP32 and dp2a peaks scale with the SM count the device reports."""
    global SM_COUNT
    if n > 0:
        SM_COUNT = int(n)


def fp32_peak_tflops(mhz: float) -> float:
    return SM_COUNT * FMA_PER_CLK * 2 * mhz * 1e6 / 1e12


DP2A_PER_CLK = 64  # dp2a (and 32-bit IMAD) issue rate per SM per clock


def q15_peak_macs(mhz: float) -> float:
    """Exact Q15 path: one dp2a per tap-MAC, so its ALU peak in tap-MAC/s."""
    return SM_COUNT * DP2A_PER_CLK * mhz * 1e6


def workload_config(P: int) -> dict:
    return {
        "workload": "64 independent streams x 10 s @ 48 kHz, own IRs L=48000 swapped every 24000 samples, block 128",
        "streams": C_STREAMS, "samples_per_stream": N_SAMPLES, "L": L_TAPS, "block": BLOCK,
        "ir_swap_every": SWAP, "push_samples": P,
        "l2": "inputs > L2 (x 123 MB, 1280 IRs 246 MB)",
    }


# ---------------------------------------------------------------------------
# Clocks sampled with nvidia-smi during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "sm_min_mhz": float(min(sm)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores (spawned workers)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    stream, nsamp = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2401_01607_gb300 import synth as sy
    x = sy.audio(nsamp, sy.x_seed(2, stream))
    nver = max(1, math.ceil(nsamp / SWAP))
    H = np.stack([sy.decayed_ir(L_TAPS, 0.3 * L_TAPS, sy.ir_seed(stream, v)) for v in range(nver)])
    vs = np.arange(nver, dtype=np.int64) * SWAP
    o = oracle.Oracle()
    t0 = time.perf_counter()
    o.buffer(x, H, vs, BLOCK)
    return time.perf_counter() - t0


def oracle_baseline(cores: int, nsamp: int) -> dict:
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    jobs = [(s, nsamp) for s in range(cores)]
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        times = pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t0
    slowest = max(times)
    macs = cores * nsamp * L_TAPS
    return {"value": macs / slowest, "unit": "tap-MAC/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} of 64 streams x first {nsamp} samples (IR swaps incl.), FP64 buffer alg., "
                      f"1 stream/core; slowest {slowest:.2f} s, wall {wall:.2f} s",
            "cpu_seconds": float(sum(times)),
            "samples_per_s": cores * nsamp / slowest,
            "realtime_factor_per_core": float(np.median([nsamp / t for t in times])) / FS}


def _oracle_job(args):
    """One bounded oracle job of another workload; returns (seconds, tap-MACs)."""
    kind, a, b = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2401_01607_gb300 import synth as sy
    o = oracle.Oracle()
    if kind == "warm":  # starts the worker and loads the oracle library
        return 0.0, 0
    if kind == "mono":
        w = sy.mono()
        t0 = time.perf_counter()
        o.buffer(w.x[0], w.H[0], w.vstart, w.block)
        return time.perf_counter() - t0, w.N * w.L
    if kind == "shared":  # stream a of the shared-IR workload, first b samples
        L = 96_000
        x = sy.audio(b, sy.x_seed(3, a))
        h = sy.decayed_ir(L, 0.2 * L, sy.ir_seed(0, 0))
        t0 = time.perf_counter()
        o.buffer(x, h[None], np.zeros(1, np.int64), 256)
        return time.perf_counter() - t0, b * L
    if kind == "q15":  # segment a of the Q15 workload's input, b samples, whole IR
        xq = sy.q15_codes(sy.audio(2_880_000, sy.x_seed(7, 0)))[a:a + b]
        hq = sy.q15_codes(sy.decayed_ir(48_000, 4800.0, sy.ir_seed(7, 0)))
        t0 = time.perf_counter()
        o.q15(xq, hq)
        return time.perf_counter() - t0, b * 48_000
    # mimo: pair a = (output, input) of the MIMO workload, first b samples
    L, nin = 192_000, 16
    out_, inp = divmod(a, nin)
    x = sy.audio(b, sy.x_seed(5, 0) + inp)
    h = sy.decayed_ir(L, 0.2 * L, sy.ir_seed(out_ * nin + inp, 0))
    t0 = time.perf_counter()
    o.buffer(x, h[None], np.zeros(1, np.int64), 512)
    return time.perf_counter() - t0, b * L


def oracle_other_workloads(cores: int, only_q15: bool = False) -> dict:
    """The FP64 oracle timed on bounded samples of the mono, shared-IR and MIMO
    workloads, jobs spread over the host cores (spawned before any CUDA call)."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    out = {}
    plans = {"mono": ([("mono", 0, 0)], "the whole mono workload (48000 samples, L=4096), one core"),
             "shared_ir": ([("shared", s_, 24_000) for s_ in range(16)],
                           "16 of the 1024 shared-IR streams, first 24000 samples each (L=96000), one stream per core"),
             "mimo": ([("mimo", a, 4_800) for a in (0 * 16 + i for i in range(16))] +
                      [("mimo", a, 4_800) for a in (15 * 16 + i for i in range(16))],
                      "2 of the 16 MIMO outputs (all 16 inputs each), first 4800 samples (L=192000), "
                      "32 pair jobs over the cores"),
             "q15": ([("q15", 180_000 * k, 24_000) for k in range(16)],
                     "16 segments of 24000 input samples of the Q15 workload (whole 48000-tap IR each), "
                     "one segment per core")}
    if only_q15:
        plans = {"q15": plans["q15"]}
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_job, [("warm", 0, 0)] * cores)
        for name, (jobs, desc) in plans.items():
            t0 = time.perf_counter()
            res = pool.map(_oracle_job, jobs)
            wall = time.perf_counter() - t0
            macs = sum(m for _, m in res)
            cpu_s = float(sum(t for t, _ in res))
            out[name] = {"value": macs / wall, "unit": "tap-MAC/s", "cores": min(cores, len(jobs)), "kind": "oracle",
                         "sample": desc + f"; pool wall {wall:.2f} s", "cpu_seconds": cpu_s,
                         "realtime_factor_per_core": macs / cpu_s / RT_MACS[name],
                         "realtime_unit": RT_UNIT[name]}
    return out


# tap-MAC/s that one real-time unit of each workload needs at 48 kHz, for the oracle's per-core real-time factor
RT_MACS = {"mono": FS * 4096, "shared_ir": FS * 96_000, "mimo": FS * 192_000 * 256, "q15": FS * 48_000}
RT_UNIT = {"mono": "one mono stream (L=4096)", "shared_ir": "one stream of the shared IR (L=96000)",
           "mimo": "the whole 16 x 16 MIMO system (L=192000)", "q15": "one Q15 stream (L=48000)"}


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if "Model name" in ln:
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ---------------------------------------------------------------------------
# Distributed plumbing (torchrun): barrier and max over ranks on the host
# ---------------------------------------------------------------------------
class Dist:
    """Host-side plumbing of a multi-rank run (gloo): a barrier and the max of the
    ranks' times; no collective on the data path. A rank that fails or never
    joins makes the others' next barrier raise (the peer's connection closes,
    or timeout_s passes) instead of hanging."""

    def __init__(self, timeout_s: float = 600.0):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import datetime
            import torch.distributed as dist
            dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=timeout_s))
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# The GPU step
# ---------------------------------------------------------------------------
class Runner:
    def __init__(self, P: int, w, torch):
        from paper_2401_01607_gb300 import capi
        self.capi = capi
        self.torch = torch
        self.P = P
        self.w = w
        self.npush = math.ceil(N_SAMPLES / P)
        # Input laid out push-major: push i is one contiguous [stream][n] slab
        # (n = P except for the last push, which is stored packed as [stream][n]).
        xp = np.zeros((self.npush, C_STREAMS, P), np.float32)
        for i in range(self.npush):
            seg = w.x[:, i * P:(i + 1) * P]
            xp[i].reshape(-1)[:seg.size] = seg.reshape(-1)
        self.x_host_push = xp
        self.H_vmajor = np.ascontiguousarray(np.transpose(w.H, (1, 0, 2)))  # [nver][C][L]
        self.x_d = torch.from_numpy(xp).cuda()
        self.H_d = torch.from_numpy(self.H_vmajor).cuda()
        self.y_d = torch.empty((self.npush, C_STREAMS, P), device="cuda")
        self.tail_d = torch.empty((C_STREAMS, L_TAPS - 1), device="cuda")
        self.ts = torch.cuda.Stream()
        self.s = capi.tc_open_group(C_STREAMS, L_TAPS, BLOCK, False, capi.TC_FP32, P)
        capi.tc_set_cuda_stream(self.s, self.ts)
        self.vstart = [int(v) for v in w.vstart]

    def step_device(self):
        c = self.capi
        c.tc_reset(self.s)
        v = 0
        for i in range(self.npush):
            pos = i * self.P
            n = min(self.P, N_SAMPLES - pos)
            while v < len(self.vstart) and self.vstart[v] < pos + n:
                c.tc_set_ir_rows(self.s, int(self.H_d[v].data_ptr()), L_TAPS, self.vstart[v], on_device=True)
                v += 1
            c.tc_push(self.s, int(self.x_d[i].data_ptr()), n, int(self.y_d[i].data_ptr()), on_device=True)
        c.tc_flush_dev(self.s, int(self.tail_d.data_ptr()))

    def step_host(self, y_host, tail_host, x_host=None, H_host=None):
        """The step through the C ABI with host buffers (x_host, H_host: page-locked
        copies of the push-major input and of the IR versions, else the pageable ones).
        With page-locked buffers the pushes are asynchronous (their copies overlap the
        neighbouring pushes' kernels) and the flush waits for all of them."""
        c = self.capi
        x_host = self.x_host_push if x_host is None else x_host
        H_host = self.H_vmajor if H_host is None else H_host
        c.tc_reset(self.s)
        v = 0
        for i in range(self.npush):
            pos = i * self.P
            n = min(self.P, N_SAMPLES - pos)
            while v < len(self.vstart) and self.vstart[v] < pos + n:
                c.tc_set_ir_rows(self.s, H_host[v], L_TAPS, self.vstart[v])
                v += 1
            xb = x_host[i].reshape(-1)[:C_STREAMS * n]
            yb = y_host[i].reshape(-1)[:C_STREAMS * n]
            c.tc_push(self.s, xb, n, yb, c.TC_PUSH_PINNED_ASYNC if x_host is not self.x_host_push else c.TC_PUSH_HOST)
        c.tc_flush(self.s, tail_host, L_TAPS - 1)

    def close(self):
        self.capi.tc_close(self.s)


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def eq4_at(x: np.ndarray, H: np.ndarray, vstart, m: int) -> float:
    """Eq. (4) at one output m, in float64: the sum over n of x[n] h_{v(n)}[m - n],
    v(n) the last version starting at or before n. A self-check of the timed
    outputs; parity against the oracle is the tests' job."""
    L = H.shape[1]
    lo, hi = max(0, m - L + 1), min(x.size, m + 1)
    if hi <= lo:
        return 0.0
    n = np.arange(lo, hi)
    v = np.searchsorted(np.asarray(vstart, np.int64), n, side="right") - 1
    return float(np.dot(x[lo:hi].astype(np.float64), H[v, m - n].astype(np.float64)))


class PushRun:
    """Device buffers and push loop of one pass over a workload: x [rows, N] laid
    out push-major (push i is one contiguous [row][n] slab), pushes of P samples
    through tc_push with device pointers, then the L-1 flush into tail."""

    def __init__(self, torch, x: np.ndarray, P: int, out_rows: int, L: int):
        rows, N = x.shape
        self.torch, self.P, self.N, self.L, self.out_rows = torch, P, N, L, out_rows
        self.npush = math.ceil(N / P)
        xp = np.zeros((self.npush, rows, P), np.float32)
        for i in range(self.npush):
            seg = x[:, i * P:(i + 1) * P]
            xp[i].reshape(-1)[:seg.size] = seg.reshape(-1)
        self.x_d = torch.from_numpy(xp).cuda()
        self.y_d = torch.empty((self.npush, out_rows, P), device="cuda")
        self.tail_d = torch.empty((out_rows, L - 1), device="cuda")
        self.ts = torch.cuda.Stream()

    def run(self, capi, s, h_ptr: int, n_samples: int | None = None) -> None:
        n_samples = self.N if n_samples is None else n_samples
        capi.tc_reset(s)
        capi.tc_set_ir_rows(s, h_ptr, self.L, 0, on_device=True)
        pos = 0
        for i in range(self.npush):
            if pos >= n_samples:
                break
            n = min(self.P, n_samples - pos)
            capi.tc_push(s, int(self.x_d[i].data_ptr()), n, int(self.y_d[i].data_ptr()), on_device=True)
            pos += n
        capi.tc_flush_dev(s, int(self.tail_d.data_ptr()))

    def outputs(self, picks) -> np.ndarray:
        """Outputs (row, m) of the last full pass, m in [0, N + L - 1)."""
        y = self.y_d.cpu().numpy()
        tail = self.tail_d.cpu().numpy()
        got = []
        for r, m in picks:
            if m < self.N:
                i, j = divmod(m, self.P)
                n = min(self.P, self.N - i * self.P)
                got.append(y[i].reshape(-1)[r * n + j])
            else:
                got.append(tail[r, m - self.N])
        return np.array(got, np.float64)

    def close(self):
        del self.x_d, self.y_d, self.tail_d
        self.torch.cuda.empty_cache()


def _err(got: np.ndarray, ref: np.ndarray) -> dict:
    return {"sampled_outputs": int(got.size), "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_abs": float(np.max(np.abs(got - ref))), "against": "Eq. (4) at each output, float64"}


def shared_picks(C: int, N: int, L: int):
    rng = np.random.default_rng(7)
    return [(int(rng.integers(C)), int(rng.integers(N + L - 1))) for _ in range(24)]


def mimo_picks(nout: int, N: int, L: int):
    rng = np.random.default_rng(9)
    return [(int(rng.integers(nout)), int(rng.integers(N + L - 1))) for _ in range(32)]


def bench_shared(torch, steps: int, warmup: int, P: int = 8192, C: int = 1024, N: int = 240_000,
                 precisions=("bf16split", "bf16", "fp32")) -> dict:
    """Shared-IR workload: 1024 streams x 5 s at 48 kHz, one IR L = 96000 (tau 19200), block 256.
    Each precision is one full pass per step (pushes of P samples, device pointers, then the flush).
    C and N shrink it for profiling captures."""
    from paper_2401_01607_gb300 import capi
    L, B = 96_000, 256
    w = synth.shared(C=C, N=N, L=L, block=B)
    run = PushRun(torch, w.x, P, C, L)
    h_d = torch.from_numpy(np.ascontiguousarray(w.H[0][None])).cuda()
    macs = C * N * L
    peaks = load_peaks()
    bf16_peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    out = {"workload": "%d streams x %d samples (%.1f s @ 48 kHz), one shared IR L=96000 tau=19200, "
                       "block 256, pushes of %d" % (C, N, N / FS, P), "tap_macs": macs}
    ts = run.ts
    picks = shared_picks(C, N, L)
    refs = np.array([eq4_at(w.x[c], w.H, w.vstart, m) for c, m in picks])
    for name, prec in (("bf16split", capi.TC_BF16_SPLIT), ("bf16", capi.TC_BF16), ("fp32", capi.TC_FP32)):
        if name not in precisions:
            continue
        s = capi.tc_open_group(C, L, B, True, prec, P)
        capi.tc_set_cuda_stream(s, ts)

        def step():
            run.run(capi, s, int(h_d.data_ptr()))

        nst = 1 if name == "fp32" else steps
        for _ in range(max(1, warmup if name != "fp32" else 1)):
            step()
        torch.cuda.synchronize()
        capi.tc_profile(s, True)
        clk = ClockSampler(torch.cuda.current_device())
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ts)
        for _ in range(nst):
            step()
        e1.record(ts)
        e1.synchronize()
        clk_r = clk.stop()
        k_ms, k_n, k_macs = capi.tc_profile_read(s)
        capi.tc_profile(s, False)
        info = capi.tc_get_info(s)
        capi.tc_close(s)
        ms = e0.elapsed_time(e1) / nst
        r = {"ms_per_step": ms, "value": macs / (ms / 1e3), "unit": "tap-MAC/s",
             "kernel_ms_per_step": k_ms / nst, "launches_per_step": k_n / nst,
             "check": _err(run.outputs(picks), refs), "clocks": clk_r,
             "tensor_launches": int(info.tensor_launches), "fp32_fallbacks": int(info.fp32_fallbacks)}
        if name != "fp32":
            nprod = 3 if name == "bf16split" else 1
            tflops = 2.0 * nprod * k_macs / (k_ms / 1e3) / 1e12 if k_ms > 0 else 0.0
            r["roofline"] = {"bound": "tensor", "achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                             "frac": tflops / bf16_peak,
                             "traffic": traffic_from_profile(K2_SRC, "k2_toeplitz_traffic.txt",
                                                             f"{name}-C{C}-P{P}") if C == 1024 else None,
                             "traffic_unit": "DRAM bytes per push (the push's K2 launch, one ncu capture)",
                             "kernel": ("k2_toeplitz_c2p" if name == "bf16" else "k2_toeplitz_c2s") +
                                       " (tcgen05 cta_group::2 kind::f16, persistent, K parts folded in the kernel)",
                             "peak_basis": "measured cuBLAS bf16, sustained (MEASURED_PEAKS.json)",
                             "flops_counted": f"2 x {nprod} products x useful tap-MACs"}
        else:
            tflops = 2.0 * k_macs / (k_ms / 1e3) / 1e12 if k_ms > 0 else 0.0
            r["roofline"] = {"bound": "alu", "achieved": tflops, "peak": fp32_peak_tflops(SM_MAX_MHZ),
                             "unit": "TFLOP/s", "frac": tflops / fp32_peak_tflops(SM_MAX_MHZ),
                             "kernel": "k1_gather (FP32 FMA)"}
        out[name] = r
    del h_d
    run.close()
    return out


def bench_mimo(torch, P: int = 8192, precisions=("bf16split", "bf16", "fp32"), L: int = 192_000,
               seconds: float = 60.0) -> dict:
    """MIMO workload: 16 inputs x 60 s at 48 kHz, 16 x 16 IRs of L = 192000
    (tau 38400), block 512; each output is the sum of 16 convolutions. One
    step = the whole signal pushed (device pointers, P samples per push) and
    the L-1 flush: FP32 on K1, BF16 split and BF16 on the tensor cores (K3).
    Sampled outputs are checked against the oracle's direct sums (one per
    input, added in FP64). L and seconds shrink it for profiling captures."""
    from paper_2401_01607_gb300 import capi
    w = synth.mimo(N=int(seconds * FS), L=L)
    nin, nout = w.mimo
    N, L, B = w.x.shape[1], w.L, w.block
    run = PushRun(torch, w.x, P, nout, L)
    h_d = torch.from_numpy(np.ascontiguousarray(w.H[0])).cuda()  # [nout][nin][L]
    ts = run.ts
    macs = nout * nin * N * L
    picks = mimo_picks(nout, N, L)
    refs = np.array([sum(eq4_at(w.x[i_], w.H[0, o, i_][None], w.vstart, m) for i_ in range(nin))
                     for o, m in picks])
    peaks = load_peaks()
    bf16_peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    out = {"workload": "MIMO 16 x 16, %g s @ 48 kHz (%d samples per input), L=%d tau=%g, block 512, pushes of %d"
                       % (seconds, N, L, 0.2 * L, P), "tap_macs": macs}
    for name in precisions:
        prec = {"fp32": capi.TC_FP32, "bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT}[name]
        s = capi.tc_open_mimo(nin, nout, L, B, prec, P)
        try:
            capi.tc_set_cuda_stream(s, ts)
            run.run(capi, s, int(h_d.data_ptr()), 4 * P)  # warm-up: a short segment
            ts.synchronize()
            capi.tc_profile(s, True)
            clk = ClockSampler(torch.cuda.current_device())
            clk.start()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ts)
            run.run(capi, s, int(h_d.data_ptr()))
            e1.record(ts)
            e1.synchronize()
            clk_r = clk.stop()
            k_ms, k_n, k_macs = capi.tc_profile_read(s)
            capi.tc_profile(s, False)
            info = capi.tc_get_info(s)
        finally:
            capi.tc_close(s)
        ms = e0.elapsed_time(e1)
        r = {"ms_per_step": ms, "value": macs / (ms / 1e3), "unit": "tap-MAC/s",
             "realtime_factor": (N / FS) / (ms / 1e3), "kernel_ms_per_step": k_ms, "launches": k_n,
             "check": _err(run.outputs(picks), refs), "clocks": clk_r,
             "tensor_launches": int(info.tensor_launches), "fp32_fallbacks": int(info.fp32_fallbacks)}
        if name == "fp32":
            tflops = 2.0 * k_macs / (k_ms / 1e3) / 1e12 if k_ms > 0 else 0.0
            peak = fp32_peak_tflops(SM_MAX_MHZ)
            r["roofline"] = {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                             "frac": tflops / peak, "kernel": "k1_gather (FP32 FMA), 16 inputs per output item"}
        else:
            nprod = 3 if name == "bf16split" else 1
            tflops = 2.0 * nprod * k_macs / (k_ms / 1e3) / 1e12 if k_ms > 0 else 0.0
            r["roofline"] = {"bound": "tensor", "achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                             "frac": tflops / bf16_peak,
                             "traffic": traffic_from_profile(K3_SRC, "k3_mimo_traffic.txt",
                                                             f"{name}-L{L}-P{P}") if seconds == 60.0 else None,
                             "traffic_unit": "DRAM bytes per push (K3 + k3_rev + k3_reduce, one ncu capture)",
                             "kernel": "k3_mimo (tcgen05 kind::f16) + k3_rev + k3_reduce",
                             "peak_basis": "measured cuBLAS bf16, sustained (MEASURED_PEAKS.json)",
                             "flops_counted": f"2 x {nprod} products x useful tap-MACs"}
        out[name] = r
    del h_d
    run.close()
    return out


def bench_mono(capi) -> dict:
    """Mono workload: 48000 samples, L = 4096 (tau 800), block 64. Streamed block
    by block through tc_push_block (host buffers): per-block latency against
    the 64/48000 s deadline; and the whole signal as one tc_convolve call."""
    import torch
    w = synth.mono()
    x = np.ascontiguousarray(w.x[0])
    h = np.ascontiguousarray(w.H[0][0])
    N, L, B = x.size, w.L, w.block
    s = capi.tc_open_stream(L, B)
    lat = []
    try:
        capi.tc_set_ir(s, h)
        yb = np.empty(B, np.float32)
        for rep in range(2):  # the first pass warms up
            capi.tc_reset(s)
            capi.tc_set_ir(s, h)
            lat = []
            t_all = time.perf_counter()
            for pos in range(0, N, B):
                t = time.perf_counter()
                capi.tc_push_block(s, x[pos:pos + B], yb)
                lat.append(time.perf_counter() - t)
            tail = np.empty(L - 1, np.float32)
            capi.tc_flush(s, tail, L - 1)
            t_all = time.perf_counter() - t_all
    finally:
        capi.tc_close(s)
    lat = np.array(lat) * 1e3
    x_d = torch.from_numpy(x).cuda()
    h_d = torch.from_numpy(h).cuda()
    y_d = torch.empty(N + L - 1, device="cuda")
    capi.tc_convolve(x_d, N, h_d, L, y_d)
    torch.cuda.synchronize()
    reps = 20
    t = time.perf_counter()
    for _ in range(reps):
        capi.tc_convolve(x_d, N, h_d, L, y_d)
    torch.cuda.synchronize()
    t_conv = (time.perf_counter() - t) / reps
    return {"workload": "mono: 48000 samples, L=4096 tau=800, block 64",
            "blocks": int(lat.size), "deadline_ms": B / FS * 1e3, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "misses": int(np.sum(lat > B / FS * 1e3)),
            "streamed_realtime_factor": (N / FS) / t_all,
            "one_shot_ms": t_conv * 1e3, "one_shot_tap_macs_per_s": N * L / t_conv,
            "mode": "tc_push_block per 64-sample block (host buffers, synchronous), then tc_flush; one-shot "
                    "tc_convolve on device buffers"}


def bench_ext(torch, capi, steps: int = 3) -> dict:
    """The gather's extensions on the 64-stream recipe (own IRs L = 48000, a new IR every 24000 samples,
    pushes of 8192 on device pointers): zero gating on an input that is silent half of the time (0.5 s of
    sound, 0.5 s of zeros), with and without gating, outputs compared bit for bit; and crossfaded IR switches
    (480-sample ramps) against hard ones, on the plain input."""
    w = synth.multi(C=C_STREAMS, N=N_SAMPLES, L=L_TAPS, block=BLOCK, swap_every=SWAP)
    gate = np.ones(N_SAMPLES, np.float32)
    for k in range(0, N_SAMPLES, FS):
        gate[k + FS // 2:k + FS] = 0.0
    out = {"workload": "64 streams x 10 s, own IRs L=48000 swapped every 24000 samples, pushes of 8192"}
    H_d = torch.from_numpy(np.ascontiguousarray(np.transpose(w.H, (1, 0, 2)))).cuda()  # [nver][C][L]
    vstart = [int(v) for v in w.vstart]

    def timed_pass(x, zero_skip: int, ramp: int):
        run = PushRun(torch, x, 8192, C_STREAMS, L_TAPS)
        s = capi.tc_open_group(C_STREAMS, L_TAPS, BLOCK, False, capi.TC_FP32, 8192)
        try:
            capi.tc_set_cuda_stream(s, run.ts)
            capi.tc_set_tuning(s, capi.TC_TUNE_ZERO_SKIP, zero_skip)

            def one():
                capi.tc_reset(s)
                capi.tc_set_crossfade(s, 1)
                v = 0
                for i in range(run.npush):
                    pos = i * 8192
                    n = min(8192, N_SAMPLES - pos)
                    while v < len(vstart) and vstart[v] < pos + n:
                        capi.tc_set_crossfade(s, ramp if v > 0 else 1)
                        capi.tc_set_ir_rows(s, int(H_d[v].data_ptr()), L_TAPS, vstart[v], on_device=True)
                        v += 1
                    capi.tc_push(s, int(run.x_d[i].data_ptr()), n, int(run.y_d[i].data_ptr()), on_device=True)
                capi.tc_flush_dev(s, int(run.tail_d.data_ptr()))

            one()
            run.ts.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(run.ts)
            for _ in range(steps):
                one()
            e1.record(run.ts)
            e1.synchronize()
            y = torch.cat([run.y_d.reshape(-1), run.tail_d.reshape(-1)]).cpu()
            return e0.elapsed_time(e1) / steps, y
        finally:
            capi.tc_close(s)
            run.close()

    xg = w.x * gate[None, :]
    ms_off, y_off = timed_pass(xg, 0, 1)
    ms_on, y_on = timed_pass(xg, 1, 1)
    out["zero_gating"] = {"input": "0.5 s of sound then 0.5 s of zeros, repeated", "ms_without": ms_off,
                          "ms_with": ms_on, "speedup": ms_off / ms_on,
                          "bit_identical": bool(torch.equal(y_off, y_on))}
    ms_hard, _ = timed_pass(w.x, 0, 1)
    ms_xf, y_xf = timed_pass(w.x, 0, 480)
    out["crossfade"] = {"ramp_samples": 480, "ms_hard_switches": ms_hard, "ms_crossfaded": ms_xf,
                        "overhead": ms_xf / ms_hard - 1.0}
    torch.cuda.empty_cache()
    return out


Q15_N, Q15_L = 2_880_000, 48_000


def q15_inputs():
    """Q15 workload: 60 s of 48 kHz audio and a 1 s decayed IR (tau 0.1 s, sum |h| = 1), as Q15 codes."""
    xq = synth.q15_codes(synth.audio(Q15_N, synth.x_seed(7, 0)))
    hq = synth.q15_codes(synth.decayed_ir(Q15_L, 4800.0, synth.ir_seed(7, 0)))
    return xq, hq


def bench_q15(torch, capi, reps: int = 6) -> dict:
    """Exact Q15 fixed point (K4 + one requantization, Sec. 5.4) on device buffers,
    each inner-loop form; L2 flushed before each timed call; then the same call
    with host buffers (copies inside the timed region)."""
    xq, hq = q15_inputs()
    N, L = Q15_N, Q15_L
    ny = N + L - 1
    st = torch.cuda.current_stream()
    x_d, h_d = torch.from_numpy(xq).cuda(), torch.from_numpy(hq).cuda()
    y_d = torch.empty(ny, dtype=torch.int16, device="cuda")
    acc_d = torch.empty(ny, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"workload": f"Q15 codes, N={N} (60 s at 48 kHz), L={L} (1 s IR, tau 0.1 s)",
           "macs_per_call": N * L, "l2": "256 MB buffer written before each timed call"}
    saved = os.environ.get("TC_Q15_INNER")
    ys = {}
    try:
        for inner in ("dp2a", "imad"):
            os.environ["TC_Q15_INNER"] = inner
            for _ in range(2):
                capi.tc_convolve_q15(x_d, N, h_d, L, y_d, acc_d, st)
            l0 = capi.tc_kernel_launches()
            tot = 0.0
            for _ in range(reps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                capi.tc_convolve_q15(x_d, N, h_d, L, y_d, acc_d, st)
                e1.record(st)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            ms = tot / reps
            out[inner] = {"ms_per_call": ms, "tap_macs_per_s": N * L / (ms / 1e3),
                          "gpu_launches_per_call": (capi.tc_kernel_launches() - l0) / reps}
            ys[inner] = (y_d.cpu().numpy(), acc_d.cpu().numpy())
    finally:
        if saved is None:
            os.environ.pop("TC_Q15_INNER", None)
        else:
            os.environ["TC_Q15_INNER"] = saved
    # K4 runs one dp2a per tap-MAC (two per pair of taps: high and low byte of h).
    peak = q15_peak_macs(SM_MAX_MHZ) / 1e12
    achieved = out["dp2a"]["tap_macs_per_s"] / 1e12
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T dp2a/s",
                       "frac": achieved / peak, "traffic": None,
                       "kernel": "k4_q15 (dp2a form) + k4_requant, whole call timed (memset, K4, requant)",
                       "peak_basis": f"{SM_COUNT} SM x 64 dp2a/clk x 2070 MHz (max SM clock); 64/clk/SM measured by an "
                                     "issue-rate loop, the same rate as 32-bit IMAD",
                       "work_counted": "one dp2a per useful tap-MAC (N x L per call)"}
    out["forms_agree_bitwise"] = bool(np.array_equal(ys["dp2a"][0], ys["imad"][0]) and
                                      np.array_equal(ys["dp2a"][1], ys["imad"][1]))
    # e2e: pinned host codes in, int16 outputs out, copies inside the timed region.
    x_h = torch.from_numpy(xq).pin_memory()
    h_h = torch.from_numpy(hq).pin_memory()
    y_h = torch.empty(ny, dtype=torch.int16).pin_memory()
    t_e2e = []
    for rep in range(4):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x_d.copy_(x_h, non_blocking=True)
        h_d.copy_(h_h, non_blocking=True)
        capi.tc_convolve_q15(x_d, N, h_d, L, y_d, None, st)
        y_h.copy_(y_d, non_blocking=True)
        st.synchronize()
        if rep:
            t_e2e.append(time.perf_counter() - t0)
    dt = float(np.mean(t_e2e))
    out["e2e"] = {"value": N * L / dt, "unit": "tap-MAC/s", "h2d_bytes_per_step": 2 * (N + L),
                  "d2h_bytes_per_step": 2 * ny, "ms_per_step": dt * 1e3,
                  "path": "pinned host codes -> tc_convolve_q15 (no acc) -> pinned host outputs"}
    # The host-buffer call must give the device call's outputs bit for bit (parity with the
    # oracle is the tests' job: tests/test_gpu_q15.py checks this workload's launch).
    out["e2e_matches_device"] = bool(np.array_equal(y_h.numpy(), ys["dp2a"][0]))
    del flush
    torch.cuda.empty_cache()
    return out


def bench_offline(torch, capi, reps: int = 3) -> dict:
    """One-shot tc_convolve on device buffers: a short sound through a long IR (the roles are swapped,
    Sec. 3.2, and timed both ways) and a long signal through a 1 s IR; each also through
    tc_convolve_noalloc and through tc_convolve_tc (tensor cores, BF16 split and BF16). Beside it, as
    context only, an FFT convolution of the same operands with torch.fft (cuFFT, FP32), the paper's
    comparison method."""
    out = {}
    cases = {"short_sound_long_ir": (4_800, 480_000), "long_signal_1s_ir": (2_880_000, 48_000)}
    saved = os.environ.get("TC_NO_ROLE_SWAP")
    st = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    try:
        for name, (N, L) in cases.items():
            x = torch.from_numpy(synth.audio(N, synth.x_seed(8, 0))).cuda()
            h = torch.from_numpy(synth.decayed_ir(L, 0.2 * L, synth.ir_seed(8, 0))).cuda()
            y = torch.empty(N + L - 1, device="cuda")
            os.environ.pop("TC_NO_ROLE_SWAP", None)
            ms = timed(lambda: capi.tc_convolve(x, N, h, L, y))
            r = {"N": N, "L": L, "tc_convolve_ms": ms, "tap_macs_per_s": N * L / (ms / 1e3)}
            # The same convolution without per-call allocation (fixed working array in the library).
            ms_na = timed(lambda: capi.tc_convolve_noalloc(x, N, h, L, y))
            r["noalloc_ms"] = ms_na
            r["noalloc_tap_macs_per_s"] = N * L / (ms_na / 1e3)
            if N < L:
                os.environ["TC_NO_ROLE_SWAP"] = "1"
                y2 = torch.empty_like(y)
                ms2 = timed(lambda: capi.tc_convolve(x, N, h, L, y2))
                os.environ.pop("TC_NO_ROLE_SWAP", None)
                r["caller_roles_ms"] = ms2
                r["role_swap_speedup"] = ms2 / ms
                r["orientations_rel_l2"] = float(torch.linalg.norm(y - y2) / torch.linalg.norm(y2))
            # The same convolution with the products on the tensor cores (256-sample output rows as K2's
            # channels), against the FP32 result.
            # Whole synchronous calls back to back: fractions of the burst peak (a call times alone) and,
            # beside it, of the sustained one.
            peaks = load_peaks()
            bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
            bf16_sus = float(peaks.get("bf16_tflops_sustained", 1700.0))
            for pname, pcode, nprod in (("bf16split", capi.TC_BF16_SPLIT, 3), ("bf16", capi.TC_BF16, 1)):
                yt = torch.empty_like(y)
                ms_t = timed(lambda: capi.tc_convolve_tc(x, N, h, L, yt, pcode))
                tfl = 2.0 * nprod * N * L / (ms_t / 1e3) / 1e12
                r["tensor_" + pname] = {"ms": ms_t, "tap_macs_per_s": N * L / (ms_t / 1e3),
                                        "rel_l2_vs_fp32": float(torch.linalg.norm(yt - y) / torch.linalg.norm(y)),
                                        "tflops_counted": tfl, "frac_of_bf16_peak": tfl / bf16_peak,
                                        "frac_of_bf16_sustained": tfl / bf16_sus}
            nfft = 1 << int(math.ceil(math.log2(N + L - 1)))

            def fft_conv():
                return torch.fft.irfft(torch.fft.rfft(x, nfft) * torch.fft.rfft(h, nfft), nfft)[:N + L - 1]

            r["fft_context_ms"] = timed(fft_conv)
            yf = fft_conv()
            r["fft_vs_taches_rel_l2"] = float(torch.linalg.norm(yf - y) / torch.linalg.norm(y))
            out[name] = r
    finally:
        if saved is None:
            os.environ.pop("TC_NO_ROLE_SWAP", None)
        else:
            os.environ["TC_NO_ROLE_SWAP"] = saved
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# Serving: continuous batching (tc_server_*) under real-time pacing
# ---------------------------------------------------------------------------

def _ir_maker(seed: int = 123, nmax: int = 480_000):
    """IRs of the serving recipe (exp-decayed Gaussian, sum |h| = 1) cut from one
    seeded Gaussian pool: stream seed s starts at offset s mod 4096."""
    g = np.random.default_rng(seed).standard_normal(nmax + 4096)

    def make(L: int, tau: float, s: int) -> np.ndarray:
        off = int(s) % 4096
        h = g[off:off + L] * np.exp(-np.arange(L) / max(float(tau), 1.0))
        return (h / np.abs(h).sum()).astype(np.float32)
    return make


def _lat_summary(lat: np.ndarray, blk: np.ndarray) -> dict:
    if lat.size == 0:
        return {"blocks": 0}
    dl = blk.astype(np.float64) / FS
    out = {"blocks": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3),
           "deadline_miss_frac": float(np.mean(lat > dl)), "by_block": {}}
    for b in sorted(set(blk.tolist())):
        m = blk == b
        out["by_block"][str(b)] = {"blocks": int(m.sum()), "deadline_ms": b / FS * 1e3,
                                   "p50_ms": float(np.percentile(lat[m], 50) * 1e3),
                                   "p99_ms": float(np.percentile(lat[m], 99) * 1e3),
                                   "miss_frac": float(np.mean(lat[m] > b / FS))}
    return out


def _k1_roofline(st0, st1) -> dict:
    """The serving steps' K1 work-list launches between two stats snapshots: useful FLOP over their
    CUDA-event time, against the FP32 FMA peak."""
    ms = st1.k1_ms - st0.k1_ms
    macs = st1.k1_macs - st0.k1_macs
    tfl = 2.0 * macs / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    return {"launch_ms": ms, "tflops": tfl, "frac_of_fp32_peak": tfl / fp32_peak_tflops(SM_MAX_MHZ)}


def bench_capacity(torch, capi, H64: np.ndarray, pool: np.ndarray, paced_s: float = 2.0) -> dict:
    """Concurrent real-time streams of the 64-stream recipe (L = 48000, block 128,
    own IRs) that one GB300 serves, batched (tc_server) and with one plain
    launch per stream and block.
      per-stream: M streams are served if one synchronous push per stream
        (the cycle) takes at most half the block period (a block that arrives
        just after its turn waits one cycle, then is served in the next).
      batched: M streams are served if, with every stream reading a live
        48 kHz source at a random phase and the worker thread running steps,
        the p99 block latency (from the block's ready time to its result on
        the host) is within the block deadline and at most 0.1 % of blocks
        miss it. A sweep of synchronous one-block-per-stream steps gives the
        starting point; paced runs then step M up (or down) by 25 %."""
    L, B = H64.shape[1], BLOCK
    period = B / FS
    out = {"workload": f"streams with own IRs L={L} (tau 14400), block {B} at 48 kHz (deadline %.3f ms)"
                       % (period * 1e3)}
    # Plain per-stream launches: one tc_push_block per stream and block.
    nps = 64
    ss = [capi.tc_open_stream(L, B) for _ in range(nps)]
    try:
        for i, s in enumerate(ss):
            capi.tc_set_ir(s, H64[i % 64])
        xb = np.ascontiguousarray(pool[:B])
        yb = np.empty(B, np.float32)
        for _ in range(3):
            for s in ss:
                capi.tc_push_block(s, xb, yb)
        t = time.perf_counter()
        rounds = 10
        for _ in range(rounds):
            for s in ss:
                capi.tc_push_block(s, xb, yb)
        t_ps = (time.perf_counter() - t) / (rounds * nps)
        # Best case for per-stream launches: device buffers, one CUDA stream,
        # one synchronisation per round.
        ts = torch.cuda.Stream()
        xd = torch.from_numpy(xb).cuda()
        yd = torch.empty(B, device="cuda")
        for s in ss:
            capi.tc_set_cuda_stream(s, ts)
        for s in ss:
            capi.tc_push(s, int(xd.data_ptr()), B, int(yd.data_ptr()), on_device=True)
        ts.synchronize()
        t = time.perf_counter()
        for _ in range(rounds):
            for s in ss:
                capi.tc_push(s, int(xd.data_ptr()), B, int(yd.data_ptr()), on_device=True)
            ts.synchronize()
        t_async = (time.perf_counter() - t) / (rounds * nps)
    finally:
        for s in ss:
            capi.tc_close(s)
    out["per_stream"] = {"ms_per_block_push": t_ps * 1e3, "streams": int(period / 2 / t_ps),
                         "mode": "tc_push_block per stream and block, host buffers (synchronous)"}
    out["per_stream_async"] = {"ms_per_block_push": t_async * 1e3, "streams": int(period / 2 / t_async),
                               "mode": "tc_push per stream and block, device buffers, one CUDA stream"}

    srv = capi.tc_server_open(200 << 30, 1 << 22)
    ids: list[int] = []
    try:
        capi.tc_server_reserve(srv, 24 << 30)  # about 8000 such streams: no pool growth during the paced runs
        def set_count(M, fresh=False):
            if fresh:
                for sid in ids:
                    capi.tc_server_remove(srv, sid)
                ids.clear()
            while len(ids) < M:
                ids.append(capi.tc_server_add(srv, L, B, H64[len(ids) % 64], capi.TC_SERVER_DISCARD_OUTPUT))
            while len(ids) > M:
                capi.tc_server_remove(srv, ids.pop())

        # Sweep: synchronous steps over one block of each of M streams.
        def cycle(M, reps=6):
            set_count(M)
            a = np.asarray(ids[:M], np.uint64)
            addr = np.full(M, pool.ctypes.data, np.uint64)
            ns = np.full(M, B, np.uint64)
            ts_ = []
            for r in range(2 + reps):
                t = time.perf_counter()
                capi.tc_server_submit_many(srv, a, addr, ns)
                while capi.tc_server_step(srv):  # a step holds what the gather's buffers hold
                    pass
                ts_.append(time.perf_counter() - t)
            capi.tc_server_latencies(srv)
            return float(np.mean(ts_[2:]))

        sweep = {}
        for M in (256, 512, 1024, 2048, 3072, 4096, 6144, 8192):
            sweep[M] = cycle(M)
            if sweep[M] > period:
                break
        ok = [m for m, t in sweep.items() if t <= period / 2]
        m0 = max(ok) if ok else 256

        # Paced runs: live sources, worker thread.
        def paced(M, seed=11):
            set_count(M, fresh=True)
            capi.tc_server_latencies(srv)  # empty the log (the worker is stopped)
            b_start = capi.tc_server_get_stats(srv).blocks
            rng = np.random.default_rng(seed)
            warm = 1.2  # seconds of audio before recording starts: past L = 1 s, every history full
            n_src = int((warm + paced_s) * FS)
            t_start = capi.tc_server_clock() + 0.05
            capi.tc_server_start(srv)
            for sid in ids:
                off = int(rng.integers(0, pool.size - n_src))
                capi.tc_server_attach_source(srv, sid, (pool.ctypes.data + 4 * off, n_src),
                                             t_start + rng.uniform(0, period))
            while capi.tc_server_clock() < t_start + warm:
                time.sleep(0.01)
            # Warm-up blocks are not counted: the log is read once at the end and the records of the blocks
            # completed before st0 (completion order) dropped, so that nothing reads it while the worker runs.
            st0 = capi.tc_server_get_stats(srv)
            n_warm = st0.blocks - b_start
            t_rec = capi.tc_server_clock()
            t_end = t_start + warm + paced_s + period + 2.0
            while capi.tc_server_clock() < t_end:
                time.sleep(0.02)
                if capi.tc_server_clock() > t_start + warm + paced_s + period and \
                        all(capi.tc_server_stream_state(srv, sid) == 2 for sid in ids):
                    break
            capi.tc_server_stop(srv)
            st1 = capi.tc_server_get_stats(srv)
            lat, blk = capi.tc_server_latencies(srv)
            lat, blk = lat[n_warm:], blk[n_warm:]
            steps = st1.steps - st0.steps
            wall = max(capi.tc_server_clock() - t_rec, 1e-9)
            r = dict(_lat_summary(lat, blk), streams=M, seconds_of_audio=paced_s, warmup_s=warm,
                     steps=int(steps), blocks_per_step=(st1.blocks - st0.blocks) / max(steps, 1),
                     pool_admissions=int(st1.pool_admissions), step_buffer_grows=int(st1.grows - st0.grows),
                     host_us_per_block={k: 1e6 * (getattr(st1, "host_" + k + "_s") - getattr(st0, "host_" + k + "_s")) /
                                        max(st1.blocks - st0.blocks, 1) for k in ("collect", "pack", "deliver")},
                     served_tap_macs_per_s=(st1.tap_macs - st0.tap_macs) / wall,
                     k1=_k1_roofline(st0, st1))
            r["pass"] = bool(r.get("blocks", 0) > 0 and r["p99_ms"] <= period * 1e3
                             and r["deadline_miss_frac"] <= 1e-3)
            paced.last = r
            return r

        def rung(M):
            """A paced run; a failing one is run once more and the count passes only if the repeat does (a single
            stall of the host or driver in a 2 s run can fail a count the server sustains). Both are reported."""
            r = paced(M)
            if not r["pass"]:
                first = {k: r[k] for k in ("p50_ms", "p99_ms", "max_ms", "deadline_miss_frac") if k in r}
                r = dict(paced(M, seed=12), first_attempt=first)
                paced.last = r
            return r

        runs = {}
        best = None
        fail = None
        M = m0
        step = 1.25 if rung(M)["pass"] else 0.8  # direction from the first run
        runs[str(M)] = paced.last
        if runs[str(M)]["pass"]:
            best = M
        else:
            fail = M
        for _ in range(5):
            M = max(128, int(M * step) // 128 * 128)
            if str(M) in runs:
                break
            r = rung(M)
            runs[str(M)] = r
            if r["pass"]:
                best = max(best or 0, M)
                if step < 1:
                    break  # first pass going down
            else:
                fail = M if fail is None else min(fail, M)
                if step > 1:
                    break  # first failure going up
        # Two bisection steps between the largest passing and the smallest failing count.
        for _ in range(2):
            if best is None or fail is None or fail - best <= 128:
                break
            M = (best + fail) // 2 // 128 * 128
            if M <= best or str(M) in runs:
                break
            r = rung(M)
            runs[str(M)] = r
            if r["pass"]:
                best = M
            else:
                fail = M
        out["batched"] = {"streams": best or 0,
                          "criterion": "paced (1.2 s warm-up, 2 s recorded): p99 <= deadline and <= 0.1 % misses; "
                                       "a failing count is run once more",
                          "sync_cycle_ms": {str(k): v * 1e3 for k, v in sorted(sweep.items())},
                          "mode": "tc_server worker thread, live 48 kHz sources, random phases"}
        out["batched_paced"] = {k: {kk: vv for kk, vv in v.items() if kk != "by_block"} for k, v in runs.items()}
    finally:
        capi.tc_server_close(srv)
    out["ratio_batched_vs_per_stream"] = out["batched"]["streams"] / max(out["per_stream"]["streams"], 1)
    out["ratio_batched_vs_per_stream_async"] = out["batched"]["streams"] / max(out["per_stream_async"]["streams"], 1)
    return out


def bench_groups(capi, paced_s: float = 1.5, C: int = 128, L: int = 96_000, B: int = 256,
                 precisions=("bf16split", "fp32"),
                 ladder=(4, 8, 16, 24, 32, 40, 48, 64, 80, 96, 112, 128, 144, 160, 192, 256)) -> dict:
    """Serving of shared-IR groups (tc_server_add_group): G groups of C channels, each group one IR of
    L taps (tau 0.2 L) and a live [C][n] 48 kHz source at a random phase, block B. For each precision
    the group count G rises until the p99 block latency exceeds the deadline B/fs or more than 0.1 %
    of blocks miss it; the largest passing G is the capacity. A failed rung is run once more on a fresh
    server (both attempts reported)."""
    period = B / FS
    warm = 0.3
    n_src = int((warm + paced_s + 0.2) * FS)
    src = np.ascontiguousarray(synth.audio_block(C, n_src, synth.x_seed(9, 0)))
    irs = [synth.decayed_ir(L, 0.2 * L, synth.ir_seed(9, g)) for g in range(max(ladder))]
    out = {"workload": f"groups of {C} channels sharing one IR L={L} (tau {0.2 * L:g}), block {B} at 48 kHz "
                       f"(deadline {period * 1e3:.3f} ms); live sources, worker thread",
           "tap_macs_per_group_realtime": C * FS * L}
    for name in precisions:
        code = {"fp32": capi.TC_FP32, "bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT}[name]
        runs, best = {}, 0
        def rung(G):
            """One paced run of G groups on a fresh server; None if G groups are not admitted."""
            srv = capi.tc_server_open(240 << 30, 1 << 22)
            try:
                try:
                    ids = [capi.tc_server_add_group(srv, C, L, B, irs[g], code, capi.TC_SERVER_DISCARD_OUTPUT)
                           for g in range(G)]
                except capi.TcError as e:  # no room for G groups: the ladder ends here
                    return {"groups": G, "pass": False, "admission": str(e)[:200]}
                rng = np.random.default_rng(G)
                t_start = capi.tc_server_clock() + 0.05
                capi.tc_server_start(srv)
                for sid in ids:
                    capi.tc_server_attach_source(srv, sid, src, t_start + rng.uniform(0, period))
                while capi.tc_server_clock() < t_start + warm:
                    time.sleep(0.01)
                st0 = capi.tc_server_get_stats(srv)  # its first st0.blocks latency records are the warm-up's
                t_rec = capi.tc_server_clock()
                t_end = t_start + n_src / FS + period + 3.0
                while capi.tc_server_clock() < t_end:
                    time.sleep(0.02)
                    if all(capi.tc_server_stream_state(srv, sid) == 2 for sid in ids):
                        break
                capi.tc_server_stop(srv)
                st1 = capi.tc_server_get_stats(srv)
                lat, blk = capi.tc_server_latencies(srv)
                lat, blk = lat[st0.blocks:], blk[st0.blocks:]
                wall = max(capi.tc_server_clock() - t_rec, 1e-9)
                steps = st1.steps - st0.steps
                r = dict(_lat_summary(lat, blk), groups=G, channels=G * C, steps=int(steps),
                         served_tap_macs_per_s=(st1.tap_macs - st0.tap_macs) / wall,
                         tensor_launches=int(st1.tensor_launches), fp32_fallbacks=int(st1.fp32_fallbacks))
                r.pop("by_block", None)
                r["pass"] = bool(r.get("blocks", 0) > 0 and r["p99_ms"] <= period * 1e3
                                 and r["deadline_miss_frac"] <= 1e-3)
                return r
            finally:
                capi.tc_server_close(srv)

        for G in ladder:
            r = rung(G)
            if not r["pass"] and "admission" not in r:
                # One repeat on a fresh server: a single host stall of tens of ms in a 1.5 s run fails a rung
                # that the GPU sustains. Both attempts are reported; the rung passes only if the repeat does.
                first = {k: r[k] for k in ("p50_ms", "p99_ms", "max_ms", "deadline_miss_frac") if k in r}
                r = rung(G)
                r["first_attempt"] = first
            runs[str(G)] = r
            if not r["pass"]:
                break
            best = G
        out[name] = {"groups": best, "channels": best * C, "runs": runs}
    return out


RESERVE_TRACE = 12 << 30  # device bytes reserved for the trace server's streams before the replay


TRACE_GROUPS = 8          # BF16-split shared-IR groups in the trace: 16-channel sources through one IR
TRACE_GROUP_C = 16
TRACE_GROUP_SECONDS = 12.0
TRACE_GROUP_BLOCK = 256


def trace_groups(seconds: float):
    """The trace's multichannel part: group g (16 channels sharing one IR of L log-uniform in [4800, 96000],
    tau 0.2 L, block 256) plays a 12 s source from 4 + (seconds - 16) g / 8 s into the trace."""
    rng = np.random.default_rng(4343)
    out = []
    for g in range(TRACE_GROUPS):
        L = int(np.exp(rng.uniform(np.log(4800), np.log(96_000))))
        start = 4.0 + max(seconds - 16.0, 0.0) * g / TRACE_GROUPS
        n = int(min(TRACE_GROUP_SECONDS, max(seconds - start, 1.0)) * FS)
        x = synth.audio_block(TRACE_GROUP_C, n, synth.x_seed(11, g))
        h = synth.decayed_ir(L, 0.2 * L, synth.ir_seed(11, g))
        out.append((start, L, x, h))
    return out


def bench_trace(capi, pool: np.ndarray, seconds: float, budget_gb: float = 96.0) -> dict:
    """Serving trace replayed in real time: Poisson arrivals (200 streams/s),
    durations 0.5-30 s, IR lengths 256-480000, blocks {32..256}, 10 % with a
    mid-stream IR swap. A stream is admitted at its arrival (memory budget;
    it waits and retries when the budget is full), reads a live 48 kHz source
    from then on and is removed once drained. Beside them, 8 shared-IR groups
    of 16 channels in BF16 split (multichannel sources through one room
    response), admitted before the replay, each playing a 12 s live source from
    its start time; their outputs are kept and checked against Eq. 4. The
    worker thread runs the steps; this thread admits, removes and polls."""
    tr = synth.serving_trace(duration_s=seconds)
    make = _ir_maker()
    irs = {t.sid: [make(t.L, t.tau, sd) for sd in t.ir_seeds] for t in tr}
    grp = trace_groups(seconds)
    srv = capi.tc_server_open(int(budget_gb * (1 << 30)), 1 << 22)
    waits, max_active, live = 0, 0, {}
    gids, gouts, gfill = [], [], []
    try:
        # Groups are admitted here, not at their start: opening a group allocates device memory, which stalls
        # running steps.
        for start, L, x, h in grp:
            gids.append(capi.tc_server_add_group(srv, TRACE_GROUP_C, L, TRACE_GROUP_BLOCK, h, capi.TC_BF16_SPLIT))
            gouts.append(np.zeros((TRACE_GROUP_C, x.shape[1]), np.float32))  # written in place as blocks arrive
            gfill.append(0)
        gbuf = np.empty(TRACE_GROUP_C * TRACE_GROUP_BLOCK, np.float32)

        def poll_groups():
            for gi, gid in enumerate(gids):
                while True:
                    n, _, _ = capi.tc_server_poll(srv, gid, gbuf)
                    if n == 0:
                        break
                    c = n // TRACE_GROUP_C
                    gouts[gi][:, gfill[gi]:gfill[gi] + c] = gbuf[:n].reshape(TRACE_GROUP_C, c)
                    gfill[gi] += c

        # The trace's streams hold about 6-8 GB at their peak: reserved before the replay, so that admissions
        # carve their state from it (growing the pool while steps run stalled them for 1-65 ms).
        capi.tc_server_reserve(srv, RESERVE_TRACE)
        capi.tc_server_start(srv)
        t_start = capi.tc_server_clock() + 0.02
        t_end = t_start + seconds
        for (start, L, x, h), gid in zip(grp, gids):
            capi.tc_server_attach_source(srv, gid, x, t_start + start)
        pending = list(tr)
        slow = []  # steps of over 2 ms, from the step log drained every 0.5 s (it keeps the last 65536 steps)
        logs = []
        t_drain = t_start + 0.5

        lat_parts = []  # the latency log, read every 0.5 s (an O(1) swap in the server): the worker's log stays
        # small and reuses the memory it freed instead of touching new pages for the whole trace

        def drain_log():
            lat_parts.append(capi.tc_server_latencies_ex(srv))
            lg = capi.tc_server_step_log(srv, 1 << 15)
            logs.append(lg)
            if len(lg):
                k = (lg["t_done"] - lg["t_begin"]) > 2e-3
                prev = np.concatenate([[lg["t_done"][0]], lg["t_done"][:-1]])
                for i in np.nonzero(k)[0]:
                    slow.append((float(lg["t_begin"][i] - t_start), float(lg["t_launch"][i] - lg["t_begin"][i]) * 1e3,
                                 float(lg["t_done"][i] - lg["t_launch"][i]) * 1e3,
                                 float(max(lg["t_begin"][i] - prev[i], 0.0)) * 1e3, int(lg["blocks"][i])))
            return lg

        while True:
            now = capi.tc_server_clock()
            if now >= t_end:
                break
            if now >= t_drain:
                drain_log()
                t_drain = now + 0.5
            poll_groups()
            while pending and t_start + pending[0].arrival_s <= now:
                t = pending[0]
                try:
                    sid = capi.tc_server_add(srv, t.L, t.block, irs[t.sid][0], capi.TC_SERVER_DISCARD_OUTPUT)
                except capi.TcError as e:
                    if e.code != "TC_ENOMEM":
                        raise
                    waits += 1
                    break
                if t.swap_at >= 0:
                    capi.tc_server_set_ir_at(srv, sid, irs[t.sid][1], t.swap_at)
                off = (t.sid * 7919) % (pool.size - t.n) if t.n < pool.size else 0
                n = min(t.n, pool.size)
                t0 = capi.tc_server_clock()
                capi.tc_server_attach_source(srv, sid, (pool.ctypes.data + 4 * off, n), t0)
                live[sid] = t0 + n / FS
                pending.pop(0)
            max_active = max(max_active, len(live))
            for sid in [k for k, te in live.items() if te <= now]:
                if capi.tc_server_stream_state(srv, sid) == 2:
                    capi.tc_server_remove(srv, sid)
                    del live[sid]
            time.sleep(0.001)
        capi.tc_server_stop(srv)
        poll_groups()
        st = capi.tc_server_get_stats(srv)
        k1 = _k1_roofline(capi.TcServerStats(), st)
        drain_log()
        lat, blk, parts, kind = (np.concatenate([lp[i] for lp in lat_parts]) for i in range(4))
        steplog = np.concatenate(logs)
    finally:
        capi.tc_server_close(srv)
    arrived = sum(1 for t in tr if t.arrival_s < seconds)
    # Diagnostics: step durations (the last steps of the log) and how the
    # 32-sample blocks' misses spread over the run (completion order, 20 bins).
    diag = {"reserved_gb": RESERVE_TRACE / (1 << 30), "pool_admissions": int(st.pool_admissions),
            "step_buffer_grows": int(st.grows),
            # the 12 longest steps over 2 ms: (s into the trace, collect+pack ms, enqueue->done ms,
            # idle ms before the step, blocks)
            "slow_steps": sorted(slow, key=lambda r: -(r[1] + r[2]))[:12], "slow_step_count": len(slow)}
    if len(steplog):
        dur = (steplog["t_done"] - steplog["t_begin"]) * 1e3
        gpu = (steplog["t_done"] - steplog["t_launch"]) * 1e3
        host = (steplog["t_launch"] - steplog["t_begin"]) * 1e3
        k = int(np.argmax(dur))
        diag["step_ms"] = {"steps": int(dur.size), "p50": float(np.percentile(dur, 50)),
                           "p99": float(np.percentile(dur, 99)), "max": float(dur.max()),
                           "launch_to_done_p99": float(np.percentile(gpu, 99)),
                           "longest": {"collect_pack_ms": float(host[k]), "launch_to_done_ms": float(gpu[k]),
                                       "s_before_last_step": float(steplog["t_done"][-1] - steplog["t_begin"][k]),
                                       "blocks": int(steplog["blocks"][k]), "samples": int(steplog["samples"][k])},
                           "over_0.3ms": int(np.sum(dur > 0.3))}
    # Where the latency goes: per block, ready -> taken into a step (wait), taken -> enqueued (host),
    # enqueued -> on the host (gpu); p99 of each part, and their means over the blocks that missed.
    if parts.size:
        names = ("wait", "host", "gpu")
        late = lat > blk.astype(np.float64) / FS
        diag["parts_ms"] = {"p99": {n: float(np.percentile(parts[:, i], 99) * 1e3) for i, n in enumerate(names)},
                            "missed_mean": {n: float(parts[late, i].mean() * 1e3) if late.any() else None
                                            for i, n in enumerate(names)},
                            "missed": int(late.sum())}
    m32 = (blk == 32) & (kind == 0)
    if m32.any():
        miss = lat[m32] > 32 / FS
        diag["miss32_by_twentieth"] = [float(x.mean()) for x in np.array_split(miss, 20)]
    # The groups: latency (BF16 split, block 256) and accuracy of 512 contiguous outputs of channels 0 and 15 of
    # each group, at the middle of what it delivered, against Eq. (4) in float64.
    groups = {"groups": TRACE_GROUPS, "channels": TRACE_GROUP_C, "precision": "bf16split",
              "block": TRACE_GROUP_BLOCK, "L": [int(g[1]) for g in grp], "source_s": TRACE_GROUP_SECONDS,
              "latency": _lat_summary(lat[kind == 1 + capi.TC_BF16_SPLIT], blk[kind == 1 + capi.TC_BF16_SPLIT])}
    groups["latency"].pop("by_block", None)
    got, ref = [], []
    for (start, L, x, h), outs, nf in zip(grp, gouts, gfill):
        if nf == 0:
            continue
        y = outs[:, :nf]
        m0 = max(0, y.shape[1] // 2 - 256)
        for c in (0, TRACE_GROUP_C - 1):
            for m in range(m0, min(m0 + 512, y.shape[1])):
                got.append(float(y[c, m]))
                ref.append(eq4_at(x[c], h[None], [0], m))
    if got:
        groups["check"] = _err(np.array(got), np.array(ref))
        groups["check"]["contiguous"] = "512 outputs x channels 0 and 15 x each group"
    groups["delivered_outputs"] = int(sum(gfill))
    own = kind == 0
    return dict(_lat_summary(lat[own], blk[own]), seconds=seconds, streams_arrived=arrived, max_active=max_active,
                groups_bf16split=groups,
                served_tap_macs_per_s=st.tap_macs / seconds, steps=int(st.steps),
                blocks_per_step=st.blocks / max(st.steps, 1), busy_frac=st.busy_s / seconds,
                admission_waits=waits, mem_budget_gb=budget_gb, diagnostics=diag, k1=k1,
                precision="fp32 for the streams with their own IR (a real-time block fills at most 1/64 of a "
                          "tensor-core tile); bf16split for the shared-IR groups (groups_bf16split)",
                inputs="live 48 kHz sources cut from a seeded audio pool; IRs cut from a seeded Gaussian pool")


def bench_serving(torch, capi, H64: np.ndarray, trace_s: float) -> dict:
    pool = synth.audio(32 * FS, 4242)
    out = {"capacity": bench_capacity(torch, capi, H64, pool)}
    out["groups"] = bench_groups(capi)
    if trace_s > 0:
        out["trace"] = bench_trace(capi, pool, trace_s)
    return out


def main_picks(n_check: int = 64):
    rng = np.random.default_rng(123)
    return [(int(rng.integers(C_STREAMS)), int(rng.integers(N_SAMPLES + L_TAPS - 1))) for _ in range(n_check)]


def runner_outputs(runner, picks) -> np.ndarray:
    """Outputs (stream, m) of the runner's last device step."""
    y = runner.y_d.cpu().numpy()
    tail = runner.tail_d.cpu().numpy()
    got = []
    for c, m in picks:
        if m < N_SAMPLES:
            i, j = divmod(m, runner.P)
            n = min(runner.P, N_SAMPLES - i * runner.P)
            got.append(y[i].reshape(-1)[c * n + j])
        else:
            got.append(tail[c, m - N_SAMPLES])
    return np.array(got, np.float64)


def check_sampled(runner, n_check=64) -> dict:
    """Sampled outputs of the last device step against Eq. (4) at each output."""
    picks = main_picks(n_check)
    w = runner.w
    ref = np.array([eq4_at(w.x[c], w.H[c], w.vstart, m) for c, m in picks])
    return _err(runner_outputs(runner, picks), ref)


def traffic_from_profile(kernel_src: str, table: str = "k1_gather_traffic.txt", tag: str = "") -> float | None:
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture) from a committed
    profile table under profiles/, used only while the kernel's source still has the hash it had at capture
    time (else None: the counters are stale). Lines: traffic_bytes_per_launch <bytes> <sha256[:16]> [tag]."""
    import hashlib
    path = os.path.join(ROOT, "profiles", table)
    if not os.path.exists(path):
        return None
    digest = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    for ln in open(path):
        parts = ln.split()
        if (len(parts) >= 3 and parts[0] == "traffic_bytes_per_launch" and parts[2] == digest and
                (parts[3] if len(parts) > 3 else "") == tag):
            return float(parts[1])
    return None


def _sig(v, n: int = 4):
    """Rounds floats to n significant digits (recursively) to keep the headline short."""
    if isinstance(v, float):
        return float(f"{v:.{n}g}") if math.isfinite(v) else None
    if isinstance(v, dict):
        return {k: _sig(x, n) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [_sig(x, n) for x in v]
    return v


def _get(d, *path):
    for k in path:
        if not isinstance(d, dict) or k not in d:
            return None
        d = d[k]
    return d


def _tc_summary(sec: dict | None) -> dict | None:
    """Per precision: T tap-MAC/s, roofline fraction and relative L2 of the sampled check."""
    if not isinstance(sec, dict):
        return None
    if "error" in sec:
        return {"error": sec["error"][:120]}
    out = {}
    for name in ("bf16split", "bf16", "fp32"):
        r = sec.get(name)
        if isinstance(r, dict):
            out[name] = {"T": r["value"] / 1e12, "frac": _get(r, "roofline", "frac"),
                         "rel_l2": _get(r, "check", "rel_l2")}
    return out


HEADLINE_MAX = 2900  # bytes: the driver keeps only the tail of the output (about 3 KB)


def headline(line: dict, sections: dict) -> dict:
    """The last output line: the contract's keys with short values, plus a few scalars of each side section
    (the side lines printed before it hold everything)."""
    h = dict(line)
    rf = dict(line["roofline"])
    rf.pop("peak_basis", None)
    rf["peak_basis"] = f"{SM_COUNT} SM x 128 FMA/clk x 2 x 2070 MHz"
    h["roofline"] = rf
    cpu = line.get("cpu_baseline")
    if cpu:
        h["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample") if k in cpu}
        h["cpu_baseline"]["sample"] = str(cpu.get("sample", ""))[:110]
    e2e = line.get("e2e")
    if e2e:
        h["e2e"] = {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "ms_per_step")}
    if line.get("clocks"):
        h["clocks"] = {k: line["clocks"][k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    if line.get("check"):
        h["check"] = {k: line["check"][k] for k in ("sampled_outputs", "rel_l2", "max_abs")}
    side = {}
    side["shared_ir"] = _tc_summary(sections.get("shared_ir"))
    side["mimo"] = _tc_summary(sections.get("mimo"))
    sv = sections.get("serving")
    if isinstance(sv, dict):
        cap = sv.get("capacity") or {}
        grp = sv.get("groups") or {}
        tr = sv.get("trace") or {}
        side["serving"] = {
            "streams_batched": _get(cap, "batched", "streams"), "streams_per_stream": _get(cap, "per_stream", "streams"),
            "streams_per_stream_async": _get(cap, "per_stream_async", "streams"),
            "group_channels": {k: _get(grp, k, "channels") for k in ("bf16split", "fp32") if k in grp},
            "trace": {"s": tr.get("seconds"), "max_active": tr.get("max_active"), "p50_ms": tr.get("p50_ms"),
                      "p99_ms": {b: v.get("p99_ms") for b, v in (tr.get("by_block") or {}).items()},
                      "miss": {b: v.get("miss_frac") for b, v in (tr.get("by_block") or {}).items()},
                      "bf16split_groups": {"p99_ms": _get(tr, "groups_bf16split", "latency", "p99_ms"),
                                           "miss": _get(tr, "groups_bf16split", "latency", "deadline_miss_frac"),
                                           "rel_l2": _get(tr, "groups_bf16split", "check", "rel_l2")}}
            if tr else None}
        if "error" in sv:
            side["serving"] = {"error": str(sv["error"])[:120]}
    q = sections.get("q15")
    if isinstance(q, dict) and "dp2a" in q:
        side["q15"] = {"T": q["dp2a"]["tap_macs_per_s"] / 1e12, "frac": _get(q, "roofline", "frac"),
                       "bit_exact_forms": q.get("forms_agree_bitwise"), "e2e_T": _get(q, "e2e", "value") / 1e12}
    mono = sections.get("mono")
    if isinstance(mono, dict) and "p99_ms" in mono:
        side["mono"] = {"p99_ms": mono["p99_ms"], "deadline_ms": mono["deadline_ms"],
                        "one_shot_ms": mono.get("one_shot_ms"),
                        "tc_bf16split_frac": _get(mono, "offline", "long_signal_1s_ir", "tensor_bf16split",
                                                  "frac_of_bf16_peak"),
                        "tc_bf16_frac": _get(mono, "offline", "long_signal_1s_ir", "tensor_bf16", "frac_of_bf16_peak"),
                        "tc_bf16_frac_sustained": _get(mono, "offline", "long_signal_1s_ir", "tensor_bf16",
                                                       "frac_of_bf16_sustained")}
    ext = sections.get("ext")
    if isinstance(ext, dict) and "zero_gating" in ext:
        side["ext"] = {"gating_speedup": ext["zero_gating"]["speedup"],
                       "gating_bit_identical": ext["zero_gating"]["bit_identical"],
                       "xfade_overhead": _get(ext, "crossfade", "overhead")}
    lat = sections.get("latency")
    if isinstance(lat, dict):
        side["block_latency"] = {"p99_ms": lat["p99_ms"], "deadline_ms": lat["deadline_ms"]}
    h = _sig(h)
    h["side"] = _sig({k: v for k, v in side.items() if v is not None}, 3)
    # Drop the least important side entries until the line fits.
    for k in ("ext", "mono", "block_latency", "q15", "mimo", "shared_ir", "serving"):
        if len(json.dumps(h)) <= HEADLINE_MAX:
            break
        h["side"].pop(k, None)
    if len(json.dumps(h)) > HEADLINE_MAX:
        h.pop("side", None)
    return h


def run_reference(args, dist: Dist) -> None:
    if dist.rank != 0:
        return
    cores = os.cpu_count() or 1
    nsamp = args.ref_samples
    times = []
    for i in range(args.warmup + args.steps):
        r = oracle_baseline(cores, nsamp)
        if i >= args.warmup:
            times.append(r)
    value = float(np.median([t["value"] for t in times]))
    ms = float(np.median([cores * nsamp * L_TAPS / t["value"] for t in times])) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "tap-MAC/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.push),
            "cpu_baseline": {"value": value, "unit": "tap-MAC/s", "cores": cores, "kind": "oracle",
                             "sample": times[-1]["sample"], "cpu_model": cpu_model(),
                             "samples_per_s": float(np.median([t["samples_per_s"] for t in times])),
                             "realtime_factor_per_core":
                                 float(np.median([t["realtime_factor_per_core"] for t in times]))},
            "e2e": {"value": value, "unit": "tap-MAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--push", type=int, default=0, help="samples per push (0: autotune)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-shared", action="store_true", help="skip the shared-IR tensor-core section")
    ap.add_argument("--only-shared", action="store_true", help="run only the shared-IR section")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving section")
    ap.add_argument("--only-serving", action="store_true", help="run only the serving section")
    ap.add_argument("--trace-seconds", type=float, default=60.0)
    ap.add_argument("--only-trace", action="store_true", help="run only the serving trace")
    ap.add_argument("--no-mimo", action="store_true", help="skip the MIMO section")
    ap.add_argument("--no-q15", action="store_true", help="skip the exact Q15 section")
    ap.add_argument("--only-q15", action="store_true", help="run only the exact Q15 section")
    ap.add_argument("--only-offline", action="store_true", help="run only the one-shot (role swap) section")
    ap.add_argument("--only-ext", action="store_true", help="run only the zero-gating / crossfade section")
    ap.add_argument("--only-groups", action="store_true", help="run only the shared-IR group serving section")
    ap.add_argument("--groups-prec", default="bf16split,fp32", help="group serving section: precisions")
    ap.add_argument("--only-mimo", action="store_true", help="run only the MIMO section")
    ap.add_argument("--mimo-prec", default="bf16split,bf16,fp32", help="MIMO section: precisions")
    ap.add_argument("--mimo-L", type=int, default=192_000, help="MIMO section: IR length")
    ap.add_argument("--mimo-seconds", type=float, default=60.0, help="MIMO section: seconds of input")
    ap.add_argument("--shared-C", type=int, default=1024, help="shared-IR section: streams")
    ap.add_argument("--shared-N", type=int, default=240_000, help="shared-IR section: samples per stream")
    ap.add_argument("--shared-prec", default="bf16split,bf16,fp32", help="shared-IR section: precisions")
    ap.add_argument("--cpu-samples", type=int, default=30_000)
    ap.add_argument("--ref-samples", type=int, default=6_000)
    ap.add_argument("--full-json", default="", help="also write every section in full to this file")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)
        dist.close()
        return

    # CPU baseline first: the spawned oracle workers start before any CUDA call.
    cpu = None
    cpu_other = {}
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu:
        cpu = oracle_baseline(os.cpu_count() or 1, args.cpu_samples)
        cpu["cpu_model"] = cpu_model()
        if not (args.only_shared or args.only_serving):
            cpu_other = oracle_other_workloads(os.cpu_count() or 1, only_q15=args.only_q15)

    import torch
    import paper_2401_01607_gb300 as pkg
    from paper_2401_01607_gb300 import capi
    pkg.build()
    torch.cuda.set_device(dist.local)
    dev = torch.cuda.current_device()
    set_sm_count(torch.cuda.get_device_properties(dev).multi_processor_count)

    if args.only_shared:
        print(json.dumps({"shared_ir": bench_shared(torch, max(1, args.steps), max(1, args.warmup), C=args.shared_C,
                                                    N=args.shared_N, precisions=args.shared_prec.split(","))}),
              flush=True)
        dist.close()
        return
    if args.only_mimo:
        mimo = bench_mimo(torch, precisions=args.mimo_prec.split(","), L=args.mimo_L, seconds=args.mimo_seconds)
        mono = bench_mono(capi)
        if cpu_other:
            mimo["cpu_baseline"], mono["cpu_baseline"] = cpu_other["mimo"], cpu_other["mono"]
        print(json.dumps({"mimo": mimo, "mono": mono}), flush=True)
        dist.close()
        return
    if args.only_trace:
        pool = synth.audio(32 * FS, 4242)
        print(json.dumps({"trace": bench_trace(capi, pool, args.trace_seconds)}), flush=True)
        dist.close()
        return
    if args.only_groups:
        print(json.dumps({"groups": bench_groups(capi, precisions=args.groups_prec.split(","))}), flush=True)
        dist.close()
        return
    if args.only_offline:
        print(json.dumps({"offline": bench_offline(torch, capi)}), flush=True)
        dist.close()
        return
    if args.only_ext:
        print(json.dumps({"ext": bench_ext(torch, capi)}), flush=True)
        dist.close()
        return
    if args.only_q15:
        q15 = bench_q15(torch, capi)
        if cpu_other:
            q15["cpu_baseline"] = cpu_other["q15"]
        print(json.dumps({"q15": q15}), flush=True)
        dist.close()
        return
    if args.only_serving:
        H64 = np.stack([synth.decayed_ir(L_TAPS, 14_400.0, synth.ir_seed(c, 0)) for c in range(64)])
        print(json.dumps({"serving": bench_serving(torch, capi, H64, args.trace_seconds)}), flush=True)
        dist.close()
        return

    w = synth.multi(C=C_STREAMS, N=N_SAMPLES, L=L_TAPS, block=BLOCK, swap_every=SWAP,
                    stream0=dist.rank * C_STREAMS)

    # Blocks per launch: pick the fastest push size on a short segment.
    P = args.push
    tune = {}
    if P == 0:
        for cand in (1024, 2048, 4096, 8192):
            r = Runner(cand, w, torch)
            c = r.capi
            c.tc_reset(r.s)
            c.tc_set_ir_rows(r.s, int(r.H_d[0].data_ptr()), L_TAPS, 0, on_device=True)
            pushes = max(2, 16384 // cand)
            for rep in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(r.ts)
                for i in range(pushes):
                    c.tc_push(r.s, int(r.x_d[i].data_ptr()), cand, int(r.y_d[i].data_ptr()), on_device=True)
                e1.record(r.ts)
                e1.synchronize()
            tune[cand] = e0.elapsed_time(e1) / (pushes * cand)
            r.close()
            del r
            torch.cuda.empty_cache()
        P = min(tune, key=tune.get)

    runner = Runner(P, w, torch)
    for _ in range(args.warmup):
        runner.step_device()
    torch.cuda.synchronize()

    launches0 = capi.tc_kernel_launches()
    capi.tc_profile(runner.s, True)
    clocks = ClockSampler(dev)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(runner.ts)
    for _ in range(args.steps):
        runner.step_device()
    e_end.record(runner.ts)
    e_end.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    dist.barrier()
    launches = capi.tc_kernel_launches() - launches0
    k_ms, k_launches, k_macs = capi.tc_profile_read(runner.s)
    capi.tc_profile(runner.s, False)
    t_ms = e_start.elapsed_time(e_end)
    t_ms_max = dist.max(t_ms)
    macs_step = C_STREAMS * N_SAMPLES * L_TAPS
    value = macs_step * dist.world * args.steps / (t_ms_max / 1e3)
    ms_per_step = t_ms_max / args.steps

    check = None if args.no_check else check_sampled(runner)

    # Roofline of K1: useful FLOPs per launch over its average event time.
    k1_flops_per_launch = 2.0 * k_macs / max(k_launches, 1)
    k1_avg_s = (k_ms / max(k_launches, 1)) / 1e3
    achieved = k1_flops_per_launch / k1_avg_s / 1e12 if k1_avg_s > 0 else 0.0
    peak = fp32_peak_tflops(SM_MAX_MHZ)
    traffic = traffic_from_profile(os.path.join(ROOT, "paper_2401_01607_gb300", "csrc", "k1_gather.cu"))
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "k1_gather (FP32 FMA gather)",
                "peak_basis": f"{SM_COUNT} SM (queried) x 128 FP32 FMA/clk x 2 FLOP x 2070 MHz (max SM clock)",
                "k1_launches": k_launches, "k1_avg_ms": k1_avg_s * 1e3,
                "k1_share_of_step": (k_ms / args.steps) / ms_per_step if ms_per_step > 0 else None}
    if clk:
        roofline["frac_at_measured_clock"] = achieved / fp32_peak_tflops(clk["sm_mhz"])

    e2e = None
    if not args.no_e2e:
        # Page-locked host buffers (the copy engines move them without staging).
        pins = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                for a in (runner.x_host_push, runner.H_vmajor)]
        x_pin, H_pin = (t.numpy() for t in pins)
        y_t = torch.empty((runner.npush, C_STREAMS, P), dtype=torch.float32, pin_memory=True)
        tail_t = torch.empty((C_STREAMS, L_TAPS - 1), dtype=torch.float32, pin_memory=True)
        y_host, tail_host = y_t.numpy(), tail_t.numpy()
        runner.step_host(y_host, tail_host, x_pin, H_pin)  # warm
        reps = max(1, args.steps)  # the same step count as the device-resident value
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            runner.step_host(y_host, tail_host, x_pin, H_pin)
        dt = dist.max(time.perf_counter() - t0) / reps
        nver = len(runner.vstart)
        h2d = C_STREAMS * N_SAMPLES * 4 + nver * C_STREAMS * L_TAPS * 4
        d2h = C_STREAMS * (N_SAMPLES + L_TAPS - 1) * 4
        e2e = {"value": macs_step * dist.world / dt, "unit": "tap-MAC/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3,
               "path": "tc_set_ir_rows / tc_push (asynchronous, page-locked) / tc_flush with page-locked host buffers"}

    latency = None
    if not args.no_latency:
        # Real-time block latency: one 128-sample block per stream per call, host buffers.
        s2 = capi.tc_open_group(C_STREAMS, L_TAPS, BLOCK, False, capi.TC_FP32, BLOCK)
        try:
            capi.tc_set_ir_rows(s2, runner.H_vmajor[0], L_TAPS, 0)
            xb = np.ascontiguousarray(runner.w.x[:, :BLOCK])
            yb = np.empty((C_STREAMS, BLOCK), np.float32)
            # Fill the history to a full window first.
            for _ in range(L_TAPS // BLOCK + 2):
                capi.tc_push_block(s2, xb, yb)
            lat = []
            for _ in range(400):
                t0 = time.perf_counter()
                capi.tc_push_block(s2, xb, yb)
                lat.append(time.perf_counter() - t0)
        finally:
            capi.tc_close(s2)
        lat = np.array(lat) * 1e3
        deadline = BLOCK / FS * 1e3
        latency = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "max_ms": float(lat.max()), "deadline_ms": deadline,
                   "misses": int(np.sum(lat > deadline)), "blocks": int(lat.size),
                   "mode": "64 streams, one 128-sample block per tc_push_block call, host buffers"}

    runner.close()
    del runner
    torch.cuda.empty_cache()
    def guarded(fn):
        """Runs a side section; its failure is reported in its own entry and does not lose the main line."""
        try:
            return fn()
        except Exception as e:  # noqa: BLE001
            return {"error": f"{type(e).__name__}: {e}"[:500]}

    shared = None
    if not args.no_shared and dist.world == 1:
        shared = guarded(lambda: bench_shared(torch, steps=2, warmup=1))
        if cpu_other:
            shared["cpu_baseline"] = cpu_other["shared_ir"]
    mimo = mono = None
    if not args.no_mimo and dist.world == 1:
        mimo = guarded(lambda: bench_mimo(torch))
        mono = guarded(lambda: bench_mono(capi))
        mono["offline"] = guarded(lambda: bench_offline(torch, capi))
        if cpu_other:
            mimo["cpu_baseline"], mono["cpu_baseline"] = cpu_other["mimo"], cpu_other["mono"]
    ext = None
    if not args.no_mimo and dist.world == 1:
        ext = guarded(lambda: bench_ext(torch, capi))
    q15 = None
    if not args.no_q15 and dist.world == 1:
        q15 = guarded(lambda: bench_q15(torch, capi))
        if cpu_other:
            q15["cpu_baseline"] = cpu_other["q15"]
    serving = None
    if not args.no_serving and dist.world == 1:
        serving = guarded(lambda: bench_serving(torch, capi, np.ascontiguousarray(w.H[:, 0]), args.trace_seconds))
    if dist.rank == 0:
        per_stream_rt = FS * L_TAPS  # tap-MAC/s one real-time stream needs
        sections = {"shared_ir": shared, "mimo": mimo, "mono": mono, "q15": q15, "ext": ext, "serving": serving,
                    "latency": latency, "autotune_push_ms_per_sample": {str(k): v for k, v in tune.items()} or None}
        # Side sections first, one JSON line each (in full); the headline is the last line.
        for name, sec in sections.items():
            if sec is not None:
                print(json.dumps({"section": name, name: sec}), flush=True)
        line = {"impl": "ours", "metric": METRIC, "value": value, "unit": "tap-MAC/s", "n_gpus": dist.world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": workload_config(P),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": int(launches), "check": check,
                "realtime_streams_48k": value / per_stream_rt}
        if args.full_json:
            with open(args.full_json, "w") as f:
                json.dump(dict(line, **sections), f)
        print(json.dumps(headline(line, sections)), flush=True)
    dist.close()


if __name__ == "__main__":
    main()
