"""Continuous batching (tc_server_*) through the C ABI.

Each stream of a mixed batch must give the same output as when it runs alone,
and both must match the FP64 oracle's buffer algorithm (Sec. 4.2, per-sample
IR versions) within the FP32 tolerance (relative L2 <= 1e-6).
"""
import time

import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2401_01607_gb300 as pkg
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()


def _small_trace(k=7, seed=5):
    """Serving-trace recipe shrunk so the oracle finishes in seconds: short
    streams, IRs up to 20000 taps, half of them with a mid-stream IR swap."""
    tr = synth.serving_trace(duration_s=10.0, rate_hz=50.0, dur_range=(0.01, 0.12), L_range=(1, 20_000),
                             swap_frac=0.5, seed=seed, max_streams=k)
    out = []
    for t in tr:
        x = synth.audio(t.n, t.x_seed)
        H = np.stack([synth.decayed_ir(t.L, max(1.0, t.tau), s) for s in t.ir_seeds])
        vstart = [0] if t.swap_at < 0 else [0, t.swap_at]
        out.append((t, x, H, vstart))
    return out


def _oracle(t, x, H, vstart):
    return oracle.buffer(x, H, np.asarray(vstart, np.int64), t.block)


def _run(streams, order_seed=None, options=(), reserve=0):
    """Runs the streams through one server with manual steps. order_seed None:
    one stream at a time (alone); else interleaved at random (mix).
    options: (option, value) pairs. reserve: bytes mapped into the server's
    pool before the first admission. Returns {index: y[N + L - 1]}."""
    srv = capi.tc_server_open(8 << 30, 1 << 20)
    try:
        if reserve:
            capi.tc_server_reserve(srv, reserve)
        for opt, val in options:
            capi.tc_server_set_option(srv, opt, val)
        ids = [capi.tc_server_add(srv, t.L, t.block, H[0]) for (t, x, H, vs) in streams]
        nblk = [-(-t.n // t.block) for (t, x, H, vs) in streams]
        sent = [0] * len(streams)
        outs = [[] for _ in streams]

        def submit(i):
            t, x, H, vs = streams[i]
            b = sent[i]
            lo, hi = b * t.block, min(t.n, (b + 1) * t.block)
            if len(vs) > 1 and lo <= vs[1] < hi:
                capi.tc_server_set_ir_at(srv, ids[i], H[1], vs[1])
            capi.tc_server_submit(srv, ids[i], x[lo:hi])
            sent[i] += 1

        def drain(i):
            t = streams[i][0]
            y = np.empty(t.block, np.float32)
            while True:
                n, _, _ = capi.tc_server_poll(srv, ids[i], y)
                if n == 0:
                    break
                outs[i].append(y[:n].copy())

        if order_seed is None:
            for i in range(len(streams)):
                while sent[i] < nblk[i]:
                    submit(i)
                    capi.tc_server_step(srv)
                drain(i)
        else:
            rng = np.random.default_rng(order_seed)
            while any(sent[i] < nblk[i] for i in range(len(streams))):
                for i in range(len(streams)):
                    # 0, 1 or 2 blocks queued per stream per round: steps mix
                    # streams in changing combinations and queues build up.
                    for _ in range(int(rng.integers(0, 3))):
                        if sent[i] < nblk[i]:
                            submit(i)
                if rng.uniform() < 0.7:
                    capi.tc_server_step(srv)
                for i in range(len(streams)):
                    drain(i)
            while capi.tc_server_step(srv):
                pass
            for i in range(len(streams)):
                drain(i)
        res = {}
        for i, (t, x, H, vs) in enumerate(streams):
            tail = np.empty(max(t.L - 1, 1), np.float32)
            n = capi.tc_server_flush(srv, ids[i], tail)
            assert n == t.L - 1
            res[i] = np.concatenate(outs[i] + [tail[:n]])
            assert res[i].size == t.n + t.L - 1
            capi.tc_server_remove(srv, ids[i])
        st = capi.tc_server_get_stats(srv)
        assert st.streams == 0 and st.mem_used == 0
    finally:
        capi.tc_server_close(srv)
    return res


def test_alone_equals_mix_equals_oracle():
    streams = _small_trace()
    alone = _run(streams)
    mix = _run(streams, order_seed=1)
    for i, s in enumerate(streams):
        t = s[0]
        ref = _oracle(*s)
        e_alone, e_mix, e_am = rel_l2(alone[i], ref), rel_l2(mix[i], ref), rel_l2(mix[i], alone[i])
        print(f"stream {i}: L={t.L} block={t.block} n={t.n} swap={t.swap_at} "
              f"alone={e_alone:.2e} mix={e_mix:.2e} mix-vs-alone={e_am:.2e}")
        assert e_alone <= TOL["fp32"], (i, e_alone)
        assert e_mix <= TOL["fp32"], (i, e_mix)
        assert e_am <= TOL["fp32"], (i, e_am)


@pytest.mark.parametrize("reserve", [4 << 20, 256 << 20])
def test_reserved_memory_mix_equals_oracle(reserve):
    """With a reservation (tc_server_reserve), admissions carve their state from it: 4 MiB holds only some
    of the streams (the others fall back to the pool), 256 MiB all of them. The mix still matches the
    oracle, and the budget accounting returns to zero after the removals."""
    streams = _small_trace(k=5, seed=11)
    mix = _run(streams, order_seed=3, reserve=reserve)
    for i, s in enumerate(streams):
        assert rel_l2(mix[i], _oracle(*s)) <= TOL["fp32"], i


def test_reserved_memory_is_reused_after_removal():
    """Streams admitted one after another into a reservation that holds about two of them: each removal's
    range comes back once its steps have completed, and every stream still matches the oracle."""
    streams = _small_trace(k=6, seed=13)
    srv = capi.tc_server_open(1 << 30, 1 << 20)
    try:
        capi.tc_server_reserve(srv, 4 << 20)
        with pytest.raises(capi.TcError) as ei:
            capi.tc_server_reserve(srv, 4 << 20)
        assert ei.value.code == "TC_ESTATE"
        for t, x, H, vs in streams:
            sid = capi.tc_server_add(srv, t.L, t.block, H[0])
            outs = []
            y = np.empty(t.block, np.float32)
            for b in range(-(-t.n // t.block)):
                lo, hi = b * t.block, min(t.n, (b + 1) * t.block)
                if len(vs) > 1 and lo <= vs[1] < hi:
                    capi.tc_server_set_ir_at(srv, sid, H[1], vs[1])
                capi.tc_server_submit(srv, sid, x[lo:hi])
                capi.tc_server_step(srv)
                n, _, _ = capi.tc_server_poll(srv, sid, y)
                outs.append(y[:n].copy())
            tail = np.empty(max(t.L - 1, 1), np.float32)
            n = capi.tc_server_flush(srv, sid, tail)
            got = np.concatenate(outs + [tail[:n]])
            assert rel_l2(got, _oracle(t, x, H, vs)) <= TOL["fp32"]
            capi.tc_server_remove(srv, sid)
        assert capi.tc_server_get_stats(srv).mem_used == 0
    finally:
        capi.tc_server_close(srv)


def test_worker_thread_continuous_batching():
    """Blocks submitted while the worker runs steps join later steps; every
    result still matches the oracle and every block's latency is recorded."""
    streams = _small_trace(k=5, seed=9)
    srv = capi.tc_server_open(4 << 30, 1 << 20)
    try:
        ids = [capi.tc_server_add(srv, t.L, t.block, H[0]) for (t, x, H, vs) in streams]
        capi.tc_server_start(srv)
        with pytest.raises(capi.TcError) as ei:
            capi.tc_server_step(srv)
        assert ei.value.code == "TC_ESTATE"
        outs = [[] for _ in streams]
        sent = [0] * len(streams)
        total = 0
        nblk = [-(-t.n // t.block) for (t, x, H, vs) in streams]
        rng = np.random.default_rng(3)
        while any(sent[i] < nblk[i] for i in range(len(streams))):
            for i, (t, x, H, vs) in enumerate(streams):
                if sent[i] >= nblk[i] or rng.uniform() < 0.3:
                    continue
                lo, hi = sent[i] * t.block, min(t.n, (sent[i] + 1) * t.block)
                if len(vs) > 1 and lo <= vs[1] < hi:
                    capi.tc_server_set_ir_at(srv, ids[i], H[1], vs[1])
                capi.tc_server_submit(srv, ids[i], x[lo:hi])
                sent[i] += 1
                total += 1
            time.sleep(0.0005)
            for i, (t, x, H, vs) in enumerate(streams):
                y = np.empty(t.block, np.float32)
                n, ts, td = capi.tc_server_poll(srv, ids[i], y)
                if n:
                    assert td >= ts
                    outs[i].append(y[:n].copy())
        deadline = time.monotonic() + 30
        while sum(map(len, outs)) < total and time.monotonic() < deadline:
            for i, (t, x, H, vs) in enumerate(streams):
                y = np.empty(t.block, np.float32)
                n, _, _ = capi.tc_server_poll(srv, ids[i], y)
                if n:
                    outs[i].append(y[:n].copy())
        capi.tc_server_stop(srv)
        assert sum(map(len, outs)) == total
        lat, blk, parts, kind = capi.tc_server_latencies_ex(srv)
        assert lat.size == total and np.all(lat >= 0)
        assert np.all(kind == 0)  # plain streams only
        assert set(blk.tolist()) <= {t.block for (t, x, H, vs) in streams}
        # The three parts (ready -> taken, taken -> enqueued, enqueued -> on the host) add up to each latency
        # (float32 parts of float64 latencies), and only the first can be negative: never.
        assert parts.shape == (total, 3) and np.all(parts >= 0)
        assert np.allclose(parts.astype(np.float64).sum(axis=1), lat, rtol=1e-5, atol=1e-6)
        st = capi.tc_server_get_stats(srv)
        assert st.blocks == total and st.steps <= total
        for i, s in enumerate(streams):
            t = s[0]
            tail = np.empty(max(t.L - 1, 1), np.float32)
            n = capi.tc_server_flush(srv, ids[i], tail)
            y = np.concatenate(outs[i] + [tail[:n]])
            assert rel_l2(y, _oracle(*s)) <= TOL["fp32"]
    finally:
        capi.tc_server_close(srv)


def test_admission_by_memory_budget():
    h = synth.decayed_ir(10_000, 2000.0, 1)
    srv = capi.tc_server_open(1 << 40, 1 << 16)
    try:
        a = capi.tc_server_add(srv, 10_000, 128, h)
        per = capi.tc_server_get_stats(srv).mem_used
        capi.tc_server_remove(srv, a)
    finally:
        capi.tc_server_close(srv)
    srv = capi.tc_server_open(2 * per + per // 2, 1 << 16)
    try:
        a = capi.tc_server_add(srv, 10_000, 128, h)
        capi.tc_server_add(srv, 10_000, 128, h)
        with pytest.raises(capi.TcError) as ei:
            capi.tc_server_add(srv, 10_000, 128, h)
        assert ei.value.code == "TC_ENOMEM"
        st = capi.tc_server_get_stats(srv)
        assert st.rejected == 1 and st.streams == 2 and st.mem_used == 2 * per
        capi.tc_server_remove(srv, a)
        capi.tc_server_add(srv, 10_000, 128, h)
        assert capi.tc_server_get_stats(srv).streams == 2
    finally:
        capi.tc_server_close(srv)


def test_one_batched_launch_per_step():
    """A step over many streams is one scatter kernel plus one K1 work-list launch."""
    srv = capi.tc_server_open(8 << 30, 1 << 20)
    try:
        ids = [capi.tc_server_add(srv, 300 + 977 * i, 64 + 32 * (i % 3), synth.decayed_ir(300 + 977 * i, 200.0, i))
               for i in range(40)]
        x = synth.audio(128, 1)
        capi.tc_server_submit_many(srv, ids, [x.ctypes.data] * len(ids), [64] * len(ids))
        before = capi.tc_kernel_launches()
        assert capi.tc_server_step(srv) == len(ids)
        assert capi.tc_kernel_launches() - before == 2
    finally:
        capi.tc_server_close(srv)


def test_server_errors():
    h = synth.decayed_ir(500, 100.0, 2)
    srv = capi.tc_server_open(1 << 30, 1 << 16)
    try:
        sid = capi.tc_server_add(srv, 500, 64, h)
        for bad in [lambda: capi.tc_server_add(srv, 500, 64, np.zeros(501, np.float32)),
                    lambda: capi.tc_server_add(srv, 500, 1 << 17, h),
                    lambda: capi.tc_server_submit(srv, sid + 99, np.zeros(8, np.float32)),
                    lambda: capi.tc_server_submit(srv, sid, np.zeros(65, np.float32))]:
            with pytest.raises(capi.TcError) as ei:
                bad()
            assert ei.value.code == "TC_EINVAL"
        capi.tc_server_submit(srv, sid, np.ones(64, np.float32))
        with pytest.raises(capi.TcError) as ei:
            capi.tc_server_set_ir_at(srv, sid, h, 10)  # sample already submitted
        assert ei.value.code == "TC_EINVAL"
        capi.tc_server_submit(srv, sid, np.ones(10, np.float32))  # short: the last block
        with pytest.raises(capi.TcError) as ei:
            capi.tc_server_submit(srv, sid, np.ones(10, np.float32))
        assert ei.value.code == "TC_ESTATE"
        tail = np.empty(499, np.float32)
        assert capi.tc_server_flush(srv, sid, tail) == 499
        y = np.empty(64, np.float32)
        n1, _, _ = capi.tc_server_poll(srv, sid, y)
        first = y[:n1].copy()
        n2, _, _ = capi.tc_server_poll(srv, sid, y)
        assert (n1, n2) == (64, 10)
        ref = oracle.buffer(np.ones(74, np.float32), h[None], np.zeros(1, np.int64), 64)
        got = np.concatenate([first, y[:10], tail])
        assert rel_l2(got, ref) <= TOL["fp32"]
    finally:
        capi.tc_server_close(srv)


def test_live_source_streams():
    """Streams fed from live sources (tc_server_attach_source): paced at
    48 kHz, one whose blocks are all due at once, and one that had blocks
    submitted before its source; all match the oracle, each source block's
    latency is recorded from its ready time, and the state goes 0 -> 2."""
    streams = _small_trace(k=3, seed=21)
    srv = capi.tc_server_open(4 << 30, 1 << 20)
    try:
        ids = [capi.tc_server_add(srv, t.L, t.block, H[0]) for (t, x, H, vs) in streams]
        for i, (t, x, H, vs) in enumerate(streams):
            if len(vs) > 1:
                capi.tc_server_set_ir_at(srv, ids[i], H[1], vs[1])
        assert capi.tc_server_stream_state(srv, ids[0]) == 0
        # Stream 2: its first two blocks are submitted, the source continues.
        t2, x2 = streams[2][0], streams[2][1]
        head = 2 * t2.block
        for b in range(2):
            capi.tc_server_submit(srv, ids[2], x2[b * t2.block:(b + 1) * t2.block])
        capi.tc_server_start(srv)
        now = capi.tc_server_clock()
        srcs = [np.ascontiguousarray(streams[0][1]), np.ascontiguousarray(streams[1][1]),
                np.ascontiguousarray(x2[head:])]
        # Wait until the two submitted blocks of stream 2 have run.
        deadline = time.monotonic() + 10
        while capi.tc_server_get_stats(srv).blocks < 2 and time.monotonic() < deadline:
            time.sleep(0.001)
        capi.tc_server_attach_source(srv, ids[0], srcs[0], now + 0.01)          # paced at 48 kHz
        capi.tc_server_attach_source(srv, ids[1], srcs[1], now - 100.0)         # all due at once
        capi.tc_server_attach_source(srv, ids[2], srcs[2], now, fs=480_000.0)  # 10x real time
        with pytest.raises(capi.TcError) as ei:
            capi.tc_server_submit(srv, ids[0], srcs[0][:8])
        assert ei.value.code == "TC_ESTATE"
        deadline = time.monotonic() + 30
        while time.monotonic() < deadline and any(capi.tc_server_stream_state(srv, i) != 2 for i in ids):
            time.sleep(0.005)
        assert all(capi.tc_server_stream_state(srv, i) == 2 for i in ids)
        capi.tc_server_stop(srv)
        lat, blk = capi.tc_server_latencies(srv)
        nblocks = sum(-(-t.n // t.block) for (t, x, H, vs) in streams)
        assert lat.size == nblocks and np.all(lat >= 0)
        for i, s in enumerate(streams):
            t = s[0]
            outs = []
            y = np.empty(t.block, np.float32)
            while True:
                n, ts, td = capi.tc_server_poll(srv, ids[i], y)
                if n == 0:
                    break
                assert td >= ts
                outs.append(y[:n].copy())
            tail = np.empty(max(t.L - 1, 1), np.float32)
            n = capi.tc_server_flush(srv, ids[i], tail)
            got = np.concatenate(outs + [tail[:n]])
            assert rel_l2(got, _oracle(*s)) <= TOL["fp32"], i
    finally:
        capi.tc_server_close(srv)


@pytest.mark.parametrize("graph,autotune", [(1, 1), (1, 0), (0, 0)])
def test_graph_replay_and_autotune_modes(graph, autotune):
    """The step replayed as a CUDA graph, with and without the chunk autotuner
    (which tries every chunk variant on the first steps of a class): the mix
    still matches the oracle and the same streams run alone."""
    streams = _small_trace(k=6, seed=31)
    opts = [(capi.TC_SERVER_GRAPH, graph), (capi.TC_SERVER_AUTOTUNE, autotune)]
    mix = _run(streams, order_seed=2, options=opts)
    for i, s in enumerate(streams):
        assert rel_l2(mix[i], _oracle(*s)) <= TOL["fp32"], i


# ---------------------------------------------------------------------------
# Groups: C channels sharing one IR (tc_server_add_group), K2 in the BF16 modes
# ---------------------------------------------------------------------------

def _group_ref(X, H, vstart, block):
    return np.stack([oracle.buffer(X[c], H, np.asarray(vstart, np.int64), block) for c in range(X.shape[0])])


def _poll_group(srv, gid, C, block, outs):
    y = np.empty(C * block, np.float32)
    while True:
        n, _, _ = capi.tc_server_poll(srv, gid, y)
        if n == 0:
            return
        outs.append(y[:n].reshape(C, n // C).copy())


@pytest.mark.parametrize("prec", ["bf16split", "bf16", "fp32"])
def test_group_in_a_mix_matches_oracle(prec):
    """A 200-channel group (two 128-channel tiles, the second ragged) with an IR switch inside a block,
    served in changing mixes with two plain streams, and alone; every channel against the oracle, and the
    group's output in the mix against its output alone."""
    C, N, L, B = 200, 5_000, 3_000, 128
    X = synth.audio_block(C, N, 600)
    H = np.stack([synth.decayed_ir(L, 0.2 * L, 700 + v) for v in range(2)])
    vstart = [0, 2_600]
    ref = _group_ref(X, H, vstart, B)
    y_mix, st = _group_run(prec, X, H, vstart, L, B, _small_trace(k=2, seed=9))
    y_alone, _ = _group_run(prec, X, H, vstart, L, B, [])
    err, err_alone, err_am = rel_l2(y_mix, ref), rel_l2(y_alone, ref), rel_l2(y_mix, y_alone)
    print(f"group {prec}: mix {err:.3g}, alone {err_alone:.3g}, mix vs alone {err_am:.3g}, "
          f"tensor launches {st.tensor_launches}, fallbacks {st.fp32_fallbacks}")
    assert err <= TOL[prec] and err_alone <= TOL[prec] and err_am <= TOL[prec]
    if prec != "fp32":
        assert st.tensor_launches > 0 and st.fp32_fallbacks > 0  # the switch's windows ran on the gather
    else:
        assert st.tensor_launches == 0


def _group_run(prec, X, H, vstart, L, B, plain):
    """Serves the group (and the plain streams, in changing mixes) through manual steps; returns the group's
    [C, N + L - 1] output and the server's stats."""
    code = {"fp32": capi.TC_FP32, "bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT}[prec]
    C, N = X.shape
    np_ = len(plain)
    srv = capi.tc_server_open(8 << 30, 1 << 20)
    try:
        gid = capi.tc_server_add_group(srv, C, L, B, H[0], code)
        pids = [capi.tc_server_add(srv, t.L, t.block, Hp[0]) for (t, x, Hp, vs) in plain]
        nblk_g = -(-N // B)
        sent_g, sent_p = 0, [0] * np_
        outs_g, outs_p = [], [[] for _ in range(np_)]
        rng = np.random.default_rng(3)
        while sent_g < nblk_g or any(sent_p[i] < -(-plain[i][0].n // plain[i][0].block) for i in range(np_)):
            for _ in range(int(rng.integers(0, 3))):
                if sent_g < nblk_g:
                    lo, hi = sent_g * B, min(N, (sent_g + 1) * B)
                    if lo <= vstart[1] < hi:
                        capi.tc_server_set_ir_at(srv, gid, H[1], vstart[1])
                    capi.tc_server_submit(srv, gid, np.ascontiguousarray(X[:, lo:hi]))
                    sent_g += 1
            for i, (t, x, Hp, vs) in enumerate(plain):
                if sent_p[i] * t.block < t.n and rng.uniform() < 0.7:
                    lo, hi = sent_p[i] * t.block, min(t.n, (sent_p[i] + 1) * t.block)
                    if len(vs) > 1 and lo <= vs[1] < hi:
                        capi.tc_server_set_ir_at(srv, pids[i], Hp[1], vs[1])
                    capi.tc_server_submit(srv, pids[i], x[lo:hi])
                    sent_p[i] += 1
            if rng.uniform() < 0.6:
                capi.tc_server_step(srv)
            _poll_group(srv, gid, C, B, outs_g)
            for i, (t, *_r) in enumerate(plain):
                y = np.empty(t.block, np.float32)
                while True:
                    n, _, _ = capi.tc_server_poll(srv, pids[i], y)
                    if n == 0:
                        break
                    outs_p[i].append(y[:n].copy())
        while capi.tc_server_step(srv):
            pass
        _poll_group(srv, gid, C, B, outs_g)
        for i, (t, *_r) in enumerate(plain):
            y = np.empty(t.block, np.float32)
            while True:
                n, _, _ = capi.tc_server_poll(srv, pids[i], y)
                if n == 0:
                    break
                outs_p[i].append(y[:n].copy())
        tail = np.empty(C * (L - 1), np.float32)
        assert capi.tc_server_flush(srv, gid, tail) == C * (L - 1)
        yg = np.concatenate(outs_g + [tail.reshape(C, L - 1)], axis=1)
        st = capi.tc_server_get_stats(srv)
        for i, (t, x, Hp, vs) in enumerate(plain):
            tl = np.empty(max(t.L - 1, 1), np.float32)
            n = capi.tc_server_flush(srv, pids[i], tl)
            yp = np.concatenate(outs_p[i] + [tl[:n]])
            assert rel_l2(yp, _oracle(t, x, Hp, vs)) <= TOL["fp32"]
            capi.tc_server_remove(srv, pids[i])
        capi.tc_server_remove(srv, gid)
        assert capi.tc_server_get_stats(srv).mem_used == 0
    finally:
        capi.tc_server_close(srv)
    assert yg.shape == (C, N + L - 1)
    return yg, st


@pytest.mark.parametrize("prec", ["bf16split", "fp32"])
def test_group_live_source_worker(prec):
    """A 128-channel group read from a live [C][N] source by the worker thread, beside a plain stream."""
    code = {"fp32": capi.TC_FP32, "bf16split": capi.TC_BF16_SPLIT}[prec]
    C, N, L, B = 128, 12_000, 4_000, 256
    X = np.ascontiguousarray(synth.audio_block(C, N, 800))
    h = synth.decayed_ir(L, 0.2 * L, 801)
    srv = capi.tc_server_open(8 << 30, 1 << 20)
    try:
        gid = capi.tc_server_add_group(srv, C, L, B, h, code)
        capi.tc_server_start(srv)
        capi.tc_server_attach_source(srv, gid, X, capi.tc_server_clock() + 0.01, 480_000.0)
        outs = []
        deadline = time.time() + 60
        while capi.tc_server_stream_state(srv, gid) != 2 and time.time() < deadline:
            _poll_group(srv, gid, C, B, outs)
            time.sleep(0.002)
        capi.tc_server_stop(srv)
        _poll_group(srv, gid, C, B, outs)
        tail = np.empty(C * (L - 1), np.float32)
        capi.tc_server_flush(srv, gid, tail)
        y = np.concatenate(outs + [tail.reshape(C, L - 1)], axis=1)
        capi.tc_server_remove(srv, gid)
    finally:
        capi.tc_server_close(srv)
    ref = _group_ref(X, h[None], [0], B)
    assert y.shape == ref.shape
    assert rel_l2(y, ref) <= TOL[prec]


def test_group_errors():
    srv = capi.tc_server_open(1 << 30, 1 << 16)
    try:
        h = np.ones(10, np.float32)
        with pytest.raises(capi.TcError):
            capi.tc_server_add_group(srv, 4, 100, 64, h, 7)  # unknown precision
        with pytest.raises(capi.TcError):
            capi.tc_server_add_group(srv, 1024, 100, 128, h, capi.TC_FP32)  # 1024 x 128 > one step
        with pytest.raises(capi.TcError):
            capi.tc_server_add_group(srv, 0, 100, 64, h, capi.TC_FP32)
    finally:
        capi.tc_server_close(srv)
