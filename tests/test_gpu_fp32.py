"""FP32 gather (K1) through the C ABI against the FP64 oracle, element by element.

Tolerance: relative L2 <= 1e-6 (FP32 path); max-abs is reported beside it.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, max_abs, rel_l2, stream_host
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


def _ref(x, H, vstart, block):
    return oracle.buffer(x, H, np.asarray(vstart, np.int64), block)


def test_mono_workload_full_size():
    """Mono workload (48000 samples, L=4096, block 64), block by block, every output checked."""
    w = synth.mono()
    y = stream_host(w.x, w.H[0], w.vstart, w.L, w.block)
    ref = _ref(w.x[0], w.H[0], w.vstart, w.block)
    assert y.shape == (1, 48000 + 4096 - 1)
    err = rel_l2(y[0], ref)
    print(f"mono rel_l2={err:.3g} max_abs={max_abs(y[0], ref):.3g}")
    assert err <= TOL["fp32"]


def test_unit_impulse_is_exact():
    L, B = 5000, 64
    h = synth.decayed_ir(L, 1000.0, 7)
    for n0 in (0, 37, 700):
        x = np.zeros(1000, np.float32)
        x[n0] = 1.0
        y = stream_host(x, h[None], [0], L, B)[0]
        ref = np.zeros(1000 + L - 1, np.float32)
        ref[n0:n0 + L] = h
        assert np.array_equal(y, ref), n0


@pytest.mark.parametrize("N,L,B", [(1000, 1, 64), (777, 3, 5), (100, 257, 64), (333, 4096, 37), (64, 64, 64),
                                   (5000, 700, 256), (129, 9000, 128), (2000, 31, 2000)])
def test_ragged_shapes(N, L, B):
    rng = np.random.default_rng(N * 7 + L)
    x = rng.uniform(-1, 1, N).astype(np.float32)
    h = synth.decayed_ir(L, max(1.0, 0.3 * L), N + L)
    y = stream_host(x, h[None], [0], L, B)[0]
    ref = _ref(x, h[None], [0], B)
    assert y.shape == ref.shape
    assert rel_l2(y, ref) <= TOL["fp32"], rel_l2(y, ref)


@pytest.mark.parametrize("switches", [[0, 96], [0, 100], [0, 1, 2, 3], [0, 500, 501, 1500, 2900]])
def test_ir_switch_per_sample(switches):
    """IR replaced at exact samples, inside blocks and on block edges (abstract, Sec. 6)."""
    N, L, B = 3000, 1500, 64
    x = synth.audio(N, 11)
    H = np.stack([synth.decayed_ir(L, 400.0, 100 + v) for v in range(len(switches))])
    y = stream_host(x, H, switches, L, B)[0]
    ref = _ref(x, H, switches, B)
    assert rel_l2(y, ref) <= TOL["fp32"], rel_l2(y, ref)


def test_multi_stream_group_with_swaps():
    """Workload-2 recipe, shrunk: 8 streams, own IRs, swap every 3000 samples (odd swaps mid-block)."""
    w = synth.multi(C=8, N=20_000, L=6_000, block=128, swap_every=3_000)
    y = stream_host(w.x, w.H, w.vstart, w.L, w.block, max_push=1024)
    for c in range(w.C):
        ref = _ref(w.x[c], w.H[c], w.vstart, w.block)
        assert rel_l2(y[c], ref) <= TOL["fp32"], (c, rel_l2(y[c], ref))


def test_multi_block_push_matches_block_by_block():
    """Nb and the push size change only timing (Sec. 5.2, Table 2)."""
    N, L, B = 6000, 2500, 64
    x = synth.audio(N, 5)
    H = np.stack([synth.decayed_ir(L, 600.0, 40 + v) for v in range(2)])
    vs = [0, 2222]
    a = stream_host(x, H, vs, L, B)[0]
    b = stream_host(x, H, vs, L, B, max_push=1024)[0]
    c = stream_host(x, H, vs, L, B, pushes=[64, 128, 1024, 64, 640], max_push=1024)[0]
    ref = _ref(x, H, vs, B)
    for y in (a, b, c):
        assert rel_l2(y, ref) <= TOL["fp32"]
    assert rel_l2(a, b) <= 2 * TOL["fp32"]


def test_long_ir_variant():
    """L = 480000 taps (longest serving IR): sampled outputs against Eq. (4) one by one."""
    N, L, B = 4096, 480_000, 256
    x = synth.audio(N, 9)
    h = synth.decayed_ir(L, 0.2 * L, 10)
    y = stream_host(x, h[None], [0], L, B, max_push=4096)[0]
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.integers(0, N + L - 1, 64), [0, N - 1, N, N + L - 2]])
    got = y[idx].astype(np.float64)
    ref = np.array([oracle.direct_at(x, h[None], [0], int(m)) for m in idx])
    assert rel_l2(got, ref) <= TOL["fp32"]


def test_device_pointer_path_matches_host_path():
    torch = pytest.importorskip("torch")
    N, L, B, C = 4096, 3000, 128, 4
    x = synth.audio_block(C, N, 77)
    H = np.stack([synth.decayed_ir(L, 900.0, 300 + c) for c in range(C)])
    host = stream_host(x, H[:, None], [0], L, B, max_push=512)
    s = capi.tc_open_group(C, L, B, False, capi.TC_FP32, 512)
    try:
        capi.tc_set_ir_rows(s, torch.from_numpy(H).cuda(), L, 0, on_device=True)
        xd = torch.from_numpy(x).cuda()
        outs = []
        for pos in range(0, N, 512):
            xb = xd[:, pos:pos + 512].contiguous()
            yb = torch.empty_like(xb)
            capi.tc_push(s, xb, 512, yb, on_device=True)
            outs.append(yb)
        tail = torch.empty((C, L - 1), device="cuda")
        capi.tc_flush_dev(s, tail)
        capi.tc_sync(s)
        dev = torch.cat(outs + [tail], dim=1).cpu().numpy()
    finally:
        capi.tc_close(s)
    assert dev.shape == host.shape
    assert rel_l2(dev, host) <= 1e-7


def test_pinned_host_buffers_match_pageable():
    """Page-locked host buffers take the direct-copy path (no staging through the stream's own pinned
    buffers): IR rows, pushes and the flush give the same bits as pageable buffers."""
    torch = pytest.importorskip("torch")
    N, L, B, C = 4096, 3000, 128, 4
    x = synth.audio_block(C, N, 78)
    H = np.stack([[synth.decayed_ir(L, 900.0, 400 + 10 * v + c) for c in range(C)] for v in range(2)])
    vstart = [0, 1500]

    def run(pin):
        def host(a):
            a = np.ascontiguousarray(a, np.float32)
            return torch.from_numpy(a).pin_memory().numpy() if pin else a

        s = capi.tc_open_group(C, L, B, False, capi.TC_FP32, 512)
        try:
            capi.tc_set_ir_rows(s, host(H[0]), L, 0)
            outs = []
            for pos in range(0, N, 512):
                if pos <= vstart[1] < pos + 512:
                    capi.tc_set_ir_rows(s, host(H[1]), L, vstart[1])
                yb = host(np.empty((C, 512), np.float32))
                capi.tc_push(s, host(x[:, pos:pos + 512]), 512, yb)
                outs.append(yb.copy())
            tail = host(np.empty((C, L - 1), np.float32))
            capi.tc_flush(s, tail, L - 1)
            outs.append(tail.copy())
        finally:
            capi.tc_close(s)
        return np.concatenate(outs, axis=1)

    a, b = run(True), run(False)
    assert np.array_equal(a, b)
    ref = np.stack([oracle.buffer(x[c], H[:, c], np.asarray(vstart, np.int64), B) for c in range(C)])
    assert rel_l2(a, ref) <= TOL["fp32"]


def test_async_pinned_pushes_match_synchronous():
    """TC_PUSH_PINNED_ASYNC: pushes enqueue their copies on a second stream through two staging slots; with
    IR switches uploaded from page-locked rows in between, the outputs (complete after the flush) equal the
    synchronous pushes' bit for bit. Pageable buffers are refused."""
    torch = pytest.importorskip("torch")
    N, L, B, C, P = 6000, 3000, 128, 4, 512
    x = synth.audio_block(C, N, 79)
    H = np.stack([[synth.decayed_ir(L, 900.0, 500 + 10 * v + c) for c in range(C)] for v in range(3)])
    vstart = [0, 1500, 3300]

    def pin(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory().numpy()

    def run(mode):
        s = capi.tc_open_group(C, L, B, False, capi.TC_FP32, P)
        outs = []
        try:
            capi.tc_set_ir_rows(s, pin(H[0]), L, 0)
            v = 1
            for pos in range(0, N, P):
                n = min(P, N - pos)
                while v < len(vstart) and vstart[v] < pos + n:
                    capi.tc_set_ir_rows(s, pin(H[v]), L, vstart[v])
                    v += 1
                yb = pin(np.zeros((C, n), np.float32))
                capi.tc_push(s, pin(x[:, pos:pos + n]), n, yb, mode)
                outs.append(yb)
            tail = pin(np.empty((C, L - 1), np.float32))
            capi.tc_flush(s, tail, L - 1)
            outs.append(tail)
        finally:
            capi.tc_close(s)
        return np.concatenate(outs, axis=1)

    a, b = run(capi.TC_PUSH_PINNED_ASYNC), run(capi.TC_PUSH_HOST)
    assert np.array_equal(a, b)
    ref = np.stack([oracle.buffer(x[c], H[:, c], np.asarray(vstart, np.int64), B) for c in range(C)])
    assert rel_l2(a, ref) <= TOL["fp32"]
    s = capi.tc_open_group(C, L, B, False, capi.TC_FP32, P)
    try:
        capi.tc_set_ir_rows(s, H[0], L, 0)
        with pytest.raises(capi.TcError) as e:
            capi.tc_push(s, np.zeros((C, P), np.float32), P, np.zeros((C, P), np.float32), capi.TC_PUSH_PINNED_ASYNC)
        assert e.value.code == "TC_EINVAL"
    finally:
        capi.tc_close(s)


def test_convolve_one_shot():
    torch = pytest.importorskip("torch")
    N, L = 10_000, 2_048
    x = synth.audio(N, 1)
    h = synth.decayed_ir(L, 500.0, 2)
    y = torch.empty(N + L - 1, device="cuda")
    capi.tc_convolve(torch.from_numpy(x).cuda(), N, torch.from_numpy(h).cuda(), L, y)
    ref = oracle.buffer(x, h[None], None, 4096)
    assert rel_l2(y.cpu().numpy(), ref) <= TOL["fp32"]


@pytest.mark.parametrize("swap", ["1", "0"])
def test_convolve_role_swap(monkeypatch, swap):
    """A short sound through a long IR (N < L): tc_convolve swaps the roles (Sec. 3.2, x * h = h * x) unless
    TC_NO_ROLE_SWAP=1; both orientations match the oracle."""
    torch = pytest.importorskip("torch")
    monkeypatch.setenv("TC_NO_ROLE_SWAP", "0" if swap == "1" else "1")
    N, L = 1_500, 40_000
    x = synth.audio(N, 11)
    h = synth.decayed_ir(L, 0.2 * L, 12)
    y = torch.full((N + L - 1,), float("nan"), device="cuda")
    capi.tc_convolve(torch.from_numpy(x).cuda(), N, torch.from_numpy(h).cuda(), L, y)
    ref = oracle.buffer(x, h[None], None, 4096)
    assert rel_l2(y.cpu().numpy(), ref) <= TOL["fp32"]


def test_mimo_fp32():
    nin, nout, N, L, B = 3, 2, 3000, 1000, 128
    X = synth.audio_block(nin, N, 50)
    H = np.stack([[synth.decayed_ir(L, 250.0, 60 + o * nin + i) for i in range(nin)] for o in range(nout)])
    s = capi.tc_open_mimo(nin, nout, L, B, capi.TC_FP32, 512)
    try:
        capi.tc_set_ir_rows(s, np.ascontiguousarray(H), L, 0)
        outs = []
        for pos in range(0, N, 512):
            n = min(512, N - pos)
            y = np.empty((nout, n), np.float32)
            capi.tc_push(s, np.ascontiguousarray(X[:, pos:pos + n]), n, y)
            outs.append(y)
        tail = np.empty((nout, L - 1), np.float32)
        capi.tc_flush(s, tail, L - 1)
        y = np.concatenate(outs + [tail], axis=1)
    finally:
        capi.tc_close(s)
    ref = oracle.mimo(X, H, None, B)
    assert rel_l2(y, ref) <= TOL["fp32"], rel_l2(y, ref)


def test_errors_are_status_codes():
    L, B = 100, 16
    s = capi.tc_open_stream(L, B)
    try:
        x = np.zeros(B, np.float32)
        y = np.empty(B, np.float32)
        with pytest.raises(capi.TcError) as e:
            capi.tc_push_block(s, x, y)           # no IR yet
        assert e.value.code == "TC_ESTATE"
        h = np.ones(L, np.float32)
        with pytest.raises(capi.TcError) as e:
            capi.tc_set_ir(s, np.ones(L + 1, np.float32))  # longer than L
        assert e.value.code == "TC_EINVAL"
        capi.tc_set_ir(s, h)
        with pytest.raises(capi.TcError) as e:
            capi.tc_push_block(s, np.zeros(B + 1, np.float32), np.empty(B + 1, np.float32))
        assert e.value.code == "TC_EINVAL"
        capi.tc_push_block(s, x, y)
        with pytest.raises(capi.TcError) as e:
            capi.tc_set_ir_at(s, h, 3)                # in the past
        assert e.value.code == "TC_EINVAL"
        for k in range(1, 4):
            capi.tc_set_ir_at(s, h, B + k)
        with pytest.raises(capi.TcError) as e:
            capi.tc_set_ir_at(s, h, B + 9)            # 4 live versions already
        assert e.value.code == "TC_ENOMEM"
        capi.tc_push_block(s, x[:5], y[:5])          # short block ends the stream
        with pytest.raises(capi.TcError) as e:
            capi.tc_push_block(s, x, y)
        assert e.value.code == "TC_ESTATE"
        tail = np.empty(L - 1, np.float32)
        capi.tc_flush(s, tail, L - 1)
        with pytest.raises(capi.TcError) as e:
            capi.tc_flush(s, tail, L - 1)
        assert e.value.code == "TC_ESTATE"
        capi.tc_reset(s)
        capi.tc_set_ir(s, h)
        capi.tc_push_block(s, np.ones(B, np.float32), y)
        assert np.array_equal(y, np.arange(1, B + 1, dtype=np.float32))
    finally:
        capi.tc_close(s)


def _ref_xf(x, H, vstart, ramps, B):
    return oracle.buffer_xf(x, H, np.asarray(vstart, np.int64), np.asarray(ramps, np.int64), B)


@pytest.mark.parametrize("vstart,ramps", [([0, 500, 2000], [1, 300, 1]), ([0, 777], [1, 1500]),
                                          ([0, 100, 101], [1, 1, 1]), ([0, 64, 3000], [1, 2000, 900])])
def test_crossfade_group(vstart, ramps):
    """Continuous time-varying IR (Sec. 6): each switch is a crossfade over
    `ramp` samples; 4 channels with their own IRs, ragged pushes."""
    C, N, L, B = 4, 4500, 1500, 64
    x = synth.audio_block(C, N, 91)
    H = np.stack([np.stack([synth.decayed_ir(L, 300.0, 9000 + 10 * c + v) for v in range(len(vstart))])
                  for c in range(C)])
    y = stream_host(x, H, vstart, L, B, pushes=[64, 448, 64, 1024, 192], max_push=1024, ramps=ramps)
    for c in range(C):
        ref = _ref_xf(x[c], H[c], vstart, ramps, B)
        err = rel_l2(y[c], ref)
        assert err <= TOL["fp32"], (c, err)


def test_crossfade_ramp_one_is_the_hard_switch():
    """Ramps of one sample give the same result as the hard switches."""
    N, L, B = 3000, 1200, 128
    x = synth.audio(N, 92)
    H = np.stack([synth.decayed_ir(L, 300.0, 9100 + v) for v in range(3)])
    vs = [0, 700, 1400]
    y1 = stream_host(x, H, vs, L, B, ramps=[1, 1, 1])
    y0 = stream_host(x, H, vs, L, B)
    assert np.array_equal(y1, y0)


def test_crossfade_on_the_tensor_path_falls_back_exactly():
    """A BF16-split shared-IR group with a crossfade: windows that read the
    ramp run on the FP32 gather, the rest on the tensor cores."""
    C, N, L, B = 130, 8000, 1000, 128
    X = synth.audio_block(C, N, 93)
    H = np.stack([synth.decayed_ir(L, 200.0, 9200 + v) for v in range(2)])
    vs, rp = [0, 3000], [1, 700]
    s = capi.tc_open_group(C, L, B, True, capi.TC_BF16_SPLIT, 512)
    try:
        outs, pos, v = [], 0, 0
        while pos < N:
            n = min(512, N - pos)
            while v < len(vs) and vs[v] < pos + n:
                capi.tc_set_crossfade(s, rp[v] if v else 1)
                capi.tc_set_ir_rows(s, H[v][None], L, max(vs[v], pos))
                v += 1
            y = np.empty((C, n), np.float32)
            capi.tc_push(s, np.ascontiguousarray(X[:, pos:pos + n]), n, y)
            outs.append(y)
            pos += n
        tail = np.empty((C, L - 1), np.float32)
        capi.tc_flush(s, tail, L - 1)
        info = capi.tc_get_info(s)
    finally:
        capi.tc_close(s)
    y = np.concatenate(outs + [tail], axis=1)
    assert info.tensor_launches > 0 and info.fp32_fallbacks > 0
    for c in (0, 64, 129):
        err = rel_l2(y[c], _ref_xf(X[c], H, vs, rp, B))
        assert err <= TOL["bf16split"], (c, err)


def test_crossfade_errors():
    L, B = 200, 32
    s = capi.tc_open_stream(L, B)
    try:
        h = synth.decayed_ir(L, 50.0, 1)
        with pytest.raises(capi.TcError) as e:
            capi.tc_set_crossfade(s, 0)
        assert e.value.code == "TC_EINVAL"
        capi.tc_set_ir(s, h)
        capi.tc_set_crossfade(s, 100)
        capi.tc_set_ir_at(s, h, 50)
        with pytest.raises(capi.TcError) as e:
            capi.tc_set_ir_at(s, h, 120)  # the crossfade to 50 runs until sample 149
        assert e.value.code == "TC_EINVAL"
        capi.tc_set_ir_at(s, h, 149)
    finally:
        capi.tc_close(s)


def test_zero_gating_is_exact():
    """Zero gating (the zero-skip of Sec. 3.2 / 4.2 at block level, threshold
    0): input with long silent stretches gives bit-identical output with the
    gating on and off, for every chunk variant, and matches the oracle."""
    C, N, L, B = 3, 40_000, 9000, 128
    x = synth.audio_block(C, N, 95)
    x[:, 2000:21000] = 0.0   # silence longer than L: whole windows are zero
    x[1, 30000:31000] = 0.0
    H = np.stack([np.stack([synth.decayed_ir(L, 1500.0, 9300 + 10 * c + v) for v in range(2)])
                  for c in range(C)])
    vs = [0, 25000]
    outs = {}
    for variant in (0, 1, 2):
        for gate in (0, 1):
            s = capi.tc_open_group(C, L, B, False, capi.TC_FP32, 8192)
            try:
                capi.tc_set_tuning(s, capi.TC_TUNE_K1_CHUNK, variant)
                capi.tc_set_tuning(s, capi.TC_TUNE_ZERO_SKIP, gate)
                res, pos, v = [], 0, 0
                while pos < N:
                    n = min(8192, N - pos)
                    while v < len(vs) and vs[v] < pos + n:
                        capi.tc_set_ir_rows(s, np.ascontiguousarray(H[:, v]), L, max(vs[v], pos))
                        v += 1
                    y = np.empty((C, n), np.float32)
                    capi.tc_push(s, np.ascontiguousarray(x[:, pos:pos + n]), n, y)
                    res.append(y)
                    pos += n
                tail = np.empty((C, L - 1), np.float32)
                capi.tc_flush(s, tail, L - 1)
            finally:
                capi.tc_close(s)
            outs[(variant, gate)] = np.concatenate(res + [tail], axis=1)
        assert np.array_equal(outs[(variant, 0)], outs[(variant, 1)]), variant
    for c in range(C):
        ref = _ref(x[c], H[c], vs, B)
        assert rel_l2(outs[(2, 1)][c], ref) <= TOL["fp32"], c
