"""The timed workloads at full size, in the launch configuration the benchmark
times (its own push loops: bench.Runner and bench.PushRun, pushes of 8192
samples on device pointers, then the flush), against the FP64 oracle's direct
sum at each output (Eq. 4): random sampled outputs, and every output of
contiguous windows of 1024 outputs placed where a fault would hide (a push and
tile edge, a history compaction, the odd mid-block IR swaps and the outputs
where a swap leaves the IR's reach, the N-1/N flush seam, the last output
N+L-2), at least 10^4 contiguous outputs per workload and precision. Each
window is held to the relative-L2 tolerance on its own; its max-abs error is
printed beside it.

  multi   64 streams x 480000 samples, own IRs L = 48000 swapped every 24000
          samples (20 versions), block 128: K1
  shared  1024 streams x 240000 samples, one IR L = 96000, block 256: K2
          (BF16 split, BF16) and K1 (FP32)
  mimo    16 x 16, 60 s per input, L = 192000, block 512: K3 (BF16 split, BF16)
          and K1 (FP32)
  serving the Poisson serving trace replayed in real time through the worker
          (3 s of it, outputs kept): K1 work lists
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import bench
import oracle
from gpu_helpers import TOL, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu

P = 8192
W = 1024  # outputs per contiguous window


def _refs_job(args):
    """Oracle direct sums (Eq. 4) of outputs ms of one output row: sum over inputs i of x_i * h_i."""
    xs, Hs, vstart, ms = args
    import oracle as o
    return np.array([sum(o.direct_at(x, H, vstart, int(m)) for x, H in zip(xs, Hs)) for m in ms])


def window_refs(jobs):
    """jobs: (xs, Hs, vstart, ms) per output row; the oracle over spawned host processes (no fork after CUDA)."""
    split = []
    for j, (xs, Hs, vstart, ms) in enumerate(jobs):
        for part in np.array_split(np.asarray(ms), max(1, len(ms) // 256)):
            split.append((j, (xs, Hs, vstart, part)))
    with mp.get_context("spawn").Pool(min(len(split), os.cpu_count() or 1)) as pool:
        res = pool.map(_refs_job, [a for _, a in split])
    out = [[] for _ in jobs]
    for (j, _), r in zip(split, res):
        out[j].append(r)
    return [np.concatenate(o) for o in out]


def compaction_starts(L: int, max_push: int, N: int, P_: int) -> list[int]:
    """Push start positions at which a stream's history compacts (the host rule of the C ABI's ring:
    keep = L + 7040 + 16 rounded up to 8, cap = 2 keep + max_push + 672 rounded up to 64, base starts
    at -keep; a push of n at pos compacts when pos + n + 136 > base + cap, base -> floor8(pos - keep))."""
    keep = -(-(L + 7040 + 16) // 8) * 8
    cap = -(-(2 * keep + max_push + 672) // 64) * 64
    base, out = -keep, []
    for pos in range(0, N, P_):
        n = min(P_, N - pos)
        if pos + n + 136 > base + cap:
            base = (pos - keep) // 8 * 8
            out.append(pos)
    return out


def check_windows(name, got_rows, refs, starts, tol):
    """Per-window relative L2 (and max-abs, printed) of contiguous outputs."""
    worst = 0.0
    for (row, m0), g, r in zip(starts, got_rows, refs):
        err = rel_l2(g, r)
        mab = float(np.max(np.abs(np.asarray(g, np.float64) - r)))
        print(f"{name}: row {row} outputs [{m0}, {m0 + len(g)}): rel_l2={err:.3g} max_abs={mab:.3g}")
        assert err <= tol, (name, row, m0, err, mab)
        worst = max(worst, err)
    return worst


@pytest.fixture(scope="module")
def torch():
    import paper_2401_01607_gb300 as pkg
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()
    return t


def push_rows(y_d, tail_d, P_: int, N: int, rows) -> dict:
    """Whole output rows (input part, then the L-1 flush tail) from push-major device outputs."""
    y = y_d.cpu().numpy()
    tail = tail_d.cpu().numpy()
    out = {}
    for r in rows:
        parts = []
        for i in range(y.shape[0]):
            n = min(P_, N - i * P_)
            parts.append(y[i].reshape(-1)[r * n:(r + 1) * n])
        parts.append(tail[r])
        out[r] = np.concatenate(parts)
    return out


def test_multi_full_size(torch):
    w = synth.multi(C=bench.C_STREAMS, N=bench.N_SAMPLES, L=bench.L_TAPS, block=bench.BLOCK,
                    swap_every=bench.SWAP)
    N, L = bench.N_SAMPLES, bench.L_TAPS
    r = bench.Runner(P, w, torch)
    try:
        r.step_device()
        torch.cuda.synchronize()
        picks = bench.main_picks(96)
        got = bench.runner_outputs(r, picks)
        rows = push_rows(r.y_d, r.tail_d, P, N, (0, 63))
    finally:
        r.close()
    ref = np.array([oracle.direct_at(w.x[c], w.H[c], w.vstart, m) for c, m in picks])
    err = rel_l2(got, ref)
    print(f"multi: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL["fp32"]
    # Windows: the odd swap at 24000 (offset 64 of block 187); 72000, another odd swap, with 71999 = 24000 +
    # L - 1 where the first swap's old version leaves the IR's reach; the first history compaction (a push
    # edge and 128-output tile edges); the N-1/N flush seam; the last output N + L - 2.
    comp = compaction_starts(L, P, N, P)
    assert comp, "the run compacts its history"
    m0s = [24000 - W // 2, 72000 - W // 2, comp[0] - W // 2, N - W // 2, N + L - 1 - W]
    starts = [(c, m0) for c in (0, 63) for m0 in m0s]
    refs = window_refs([([w.x[c]], [w.H[c]], w.vstart, np.arange(m0, m0 + W)) for c, m0 in starts])
    check_windows("multi", [rows[c][m0:m0 + W] for c, m0 in starts], refs, starts, TOL["fp32"])


SHARED_ROWS = (0, 127, 128, 1023)  # 127/128: two channel tiles of K2


@pytest.fixture(scope="module")
def shared_workload():
    w = synth.shared(C=1024, N=240_000, L=96_000, block=256)
    N, L = w.x.shape[1], w.L
    comp = compaction_starts(L, P, N, P)
    assert comp
    m0s = [3 * P - W // 2, comp[0] - W // 2, L - W // 2, N - W // 2, N + L - 1 - W]
    starts = [(c, m0) for c in SHARED_ROWS for m0 in m0s]
    refs = window_refs([([w.x[c]], [w.H], w.vstart, np.arange(m0, m0 + W)) for c, m0 in starts])
    return w, starts, refs


@pytest.mark.parametrize("prec", ["bf16split", "bf16", "fp32"])
def test_shared_full_size(torch, shared_workload, prec):
    w, starts, wrefs = shared_workload
    C, N, L, B = w.x.shape[0], w.x.shape[1], w.L, w.block
    run = bench.PushRun(torch, w.x, P, C, L)
    h_d = torch.from_numpy(np.ascontiguousarray(w.H[0][None])).cuda()
    code = {"fp32": capi.TC_FP32, "bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT}[prec]
    s = capi.tc_open_group(C, L, B, True, code, P)
    try:
        capi.tc_set_cuda_stream(s, run.ts)
        run.run(capi, s, int(h_d.data_ptr()))
        run.ts.synchronize()
        info = capi.tc_get_info(s)
        rng = np.random.default_rng(70)
        picks = [(int(rng.integers(C)), int(rng.integers(N + L - 1))) for _ in range(64)]
        got = run.outputs(picks)
        rows = push_rows(run.y_d, run.tail_d, P, N, SHARED_ROWS)
    finally:
        capi.tc_close(s)
        run.close()
    if prec != "fp32":
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    ref = np.array([oracle.direct_at(w.x[c], w.H, w.vstart, m) for c, m in picks])
    err = rel_l2(got, ref)
    print(f"shared {prec}: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL[prec]
    check_windows(f"shared {prec}", [rows[c][m0:m0 + W] for c, m0 in starts], wrefs, starts, TOL[prec])


@pytest.fixture(scope="module")
def mimo_workload():
    w = synth.mimo(N=2_880_000, L=192_000)
    nin, nout = w.mimo
    rng = np.random.default_rng(90)
    picks = [(int(rng.integers(nout)), int(rng.integers(w.x.shape[1] + w.L - 1))) for _ in range(64)]
    refs = np.array([sum(oracle.direct_at(w.x[i], w.H[0, o, i][None], w.vstart, m) for i in range(nin))
                     for o, m in picks])
    N, L = w.x.shape[1], w.L
    comp = compaction_starts(L, P, N, P)
    assert comp
    m0s = [L - 1 - W // 2, comp[0] - W // 2, 100 * P - W // 2, N - W // 2, N + L - 1 - W]
    starts = [(o, m0) for o in (0, 15) for m0 in m0s]
    wrefs = window_refs([(list(w.x), [w.H[0, o, i][None] for i in range(nin)], w.vstart, np.arange(m0, m0 + W))
                         for o, m0 in starts])
    return w, picks, refs, starts, wrefs


@pytest.mark.parametrize("prec", ["bf16split", "bf16", "fp32"])
def test_mimo_full_size(torch, mimo_workload, prec):
    w, picks, refs, starts, wrefs = mimo_workload
    nin, nout = w.mimo
    N = w.x.shape[1]
    L, B = w.L, w.block
    run = bench.PushRun(torch, w.x, P, nout, L)
    h_d = torch.from_numpy(np.ascontiguousarray(w.H[0])).cuda()
    code = {"fp32": capi.TC_FP32, "bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT}[prec]
    s = capi.tc_open_mimo(nin, nout, L, B, code, P)
    try:
        capi.tc_set_cuda_stream(s, run.ts)
        run.run(capi, s, int(h_d.data_ptr()))
        run.ts.synchronize()
        info = capi.tc_get_info(s)
        got = run.outputs(picks)
        rows = push_rows(run.y_d, run.tail_d, P, N, (0, 15))
    finally:
        capi.tc_close(s)
        run.close()
    if prec != "fp32":
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    err = rel_l2(got, refs)
    print(f"mimo {prec}: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL[prec]
    check_windows(f"mimo {prec}", [rows[o][m0:m0 + W] for o, m0 in starts], wrefs, starts, TOL[prec])


def test_serving_trace_sampled(torch):
    """The serving trace as the benchmark replays it (Poisson arrivals, IRs up to 480000 taps, blocks of
    32-256, 10 % with an IR swap, live 48 kHz sources, worker thread), 3 s, outputs kept: 96 sampled outputs
    of the delivered blocks against the oracle's direct sum (Eq. 4, per-sample versions)."""
    import time
    FS = synth.FS
    seconds = 3.0
    tr = synth.serving_trace(duration_s=seconds)
    make = bench._ir_maker()
    pool = synth.audio(32 * FS, 4242)
    srv = capi.tc_server_open(96 << 30, 1 << 22)
    streams = {}
    outs = {}
    try:
        capi.tc_server_start(srv)
        t_start = capi.tc_server_clock() + 0.02
        pending = list(tr)
        ybuf = np.empty(256, np.float32)

        def drain():
            for sid in streams:
                while True:
                    n, _, _ = capi.tc_server_poll(srv, sid, ybuf)
                    if n == 0:
                        break
                    outs[sid].append(ybuf[:n].copy())

        while capi.tc_server_clock() < t_start + seconds:
            now = capi.tc_server_clock()
            while pending and t_start + pending[0].arrival_s <= now:
                t = pending.pop(0)
                H = np.stack([make(t.L, t.tau, sd) for sd in t.ir_seeds])
                sid = capi.tc_server_add(srv, t.L, t.block, H[0])
                if t.swap_at >= 0:
                    capi.tc_server_set_ir_at(srv, sid, H[1], t.swap_at)
                off = (t.sid * 7919) % (pool.size - t.n) if t.n < pool.size else 0
                n = min(t.n, pool.size)
                capi.tc_server_attach_source(srv, sid, (pool.ctypes.data + 4 * off, n), capi.tc_server_clock())
                vstart = [0] if t.swap_at < 0 else [0, t.swap_at]
                streams[sid] = (pool[off:off + n], H, np.asarray(vstart, np.int64))
                outs[sid] = []
            drain()
            time.sleep(0.002)
        capi.tc_server_stop(srv)
        drain()
    finally:
        capi.tc_server_close(srv)
    ys = {sid: np.concatenate(v) for sid, v in outs.items() if v}
    assert len(ys) >= 100  # streams with delivered output
    rng = np.random.default_rng(97)
    sids = sorted(ys)
    got, ref = [], []
    for _ in range(96):
        sid = sids[int(rng.integers(len(sids)))]
        y = ys[sid]
        m = int(rng.integers(y.size))
        x, H, vstart = streams[sid]
        got.append(float(y[m]))
        ref.append(oracle.direct_at(x, H, vstart, m))
    err = rel_l2(np.array(got), np.array(ref))
    print(f"serving trace: {len(ys)} streams delivered, 96 sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL["fp32"]
    # Contiguous windows of W delivered outputs (many blocks of each stream): around the IR swap of streams
    # that swap (the switch sample inside the window), else the last W delivered outputs; 10 windows.
    starts = []
    for sid in sids:
        x, H, vstart = streams[sid]
        n = ys[sid].size
        if len(vstart) > 1 and W // 2 <= vstart[1] <= n - W // 2:
            starts.append((sid, int(vstart[1]) - W // 2))
    for sid in sids:
        if len(starts) >= 10:
            break
        if ys[sid].size >= W and all(sid != s_ for s_, _ in starts):
            starts.append((sid, ys[sid].size - W))
    starts = starts[:10]
    assert len(starts) == 10
    wrefs = window_refs([([streams[sid][0]], [streams[sid][1]], streams[sid][2], np.arange(m0, m0 + W))
                         for sid, m0 in starts])
    check_windows("serving trace", [ys[sid][m0:m0 + W] for sid, m0 in starts], wrefs, starts, TOL["fp32"])
