"""The timed workloads at full size, in the launch configuration the benchmark
times (its own push loops: bench.Runner and bench.PushRun, pushes of 8192
samples on device pointers, then the flush), sampled outputs against the FP64
oracle one by one (Eq. 4 at each output).

  multi   64 streams x 480000 samples, own IRs L = 48000 swapped every 24000
          samples (20 versions), block 128: K1
  shared  1024 streams x 240000 samples, one IR L = 96000, block 256: K2
          (BF16 split, BF16) and K1 (FP32)
  mimo    16 x 16, 60 s per input, L = 192000, block 512: K3 (BF16 split, BF16)
          and K1 (FP32)
  serving the Poisson serving trace replayed in real time through the worker
          (3 s of it, outputs kept): K1 work lists
"""
import numpy as np
import pytest

import bench
import oracle
from gpu_helpers import TOL, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu

P = 8192


@pytest.fixture(scope="module")
def torch():
    import paper_2401_01607_gb300 as pkg
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()
    return t


def test_multi_full_size(torch):
    w = synth.multi(C=bench.C_STREAMS, N=bench.N_SAMPLES, L=bench.L_TAPS, block=bench.BLOCK,
                    swap_every=bench.SWAP)
    r = bench.Runner(P, w, torch)
    try:
        r.step_device()
        torch.cuda.synchronize()
        picks = bench.main_picks(96)
        got = bench.runner_outputs(r, picks)
    finally:
        r.close()
    ref = np.array([oracle.direct_at(w.x[c], w.H[c], w.vstart, m) for c, m in picks])
    err = rel_l2(got, ref)
    print(f"multi: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL["fp32"]


@pytest.fixture(scope="module")
def shared_workload():
    return synth.shared(C=1024, N=240_000, L=96_000, block=256)


@pytest.mark.parametrize("prec", ["bf16split", "bf16", "fp32"])
def test_shared_full_size(torch, shared_workload, prec):
    w = shared_workload
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
    finally:
        capi.tc_close(s)
        run.close()
    if prec != "fp32":
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    ref = np.array([oracle.direct_at(w.x[c], w.H, w.vstart, m) for c, m in picks])
    err = rel_l2(got, ref)
    print(f"shared {prec}: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL[prec]


@pytest.fixture(scope="module")
def mimo_workload():
    w = synth.mimo(N=2_880_000, L=192_000)
    nin, nout = w.mimo
    rng = np.random.default_rng(90)
    picks = [(int(rng.integers(nout)), int(rng.integers(w.x.shape[1] + w.L - 1))) for _ in range(64)]
    refs = np.array([sum(oracle.direct_at(w.x[i], w.H[0, o, i][None], w.vstart, m) for i in range(nin))
                     for o, m in picks])
    return w, picks, refs


@pytest.mark.parametrize("prec", ["bf16split", "bf16", "fp32"])
def test_mimo_full_size(torch, mimo_workload, prec):
    w, picks, refs = mimo_workload
    nin, nout = w.mimo
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
    finally:
        capi.tc_close(s)
        run.close()
    if prec != "fp32":
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    err = rel_l2(got, refs)
    print(f"mimo {prec}: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL[prec]


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
