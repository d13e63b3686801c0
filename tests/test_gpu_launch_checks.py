"""The host's launch check (TC_CHECK_LAUNCH=1: every K1 launch of a stream checks, before it runs, that its staged
windows are 16-byte aligned and inside the history rows, its tap chunks inside the IR slot, its versions' slots
and its scratch within bounds) accepts every launch of streams that cover the layouts: ragged blocks and IR
lengths, every chunk variant, history compactions, per-sample switches and crossfades, multi-block pushes, the
flush, MIMO, and the FP32 fallback windows of a BF16 group; the results still match the oracle.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, rel_l2, stream_host
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _checked(monkeypatch):
    import paper_2401_01607_gb300 as pkg
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()
    monkeypatch.setenv("TC_CHECK_LAUNCH", "1")


@pytest.mark.parametrize("N,L,B,variant", [(3000, 1, 64, -1), (5000, 700, 37, 0), (20000, 9000, 128, 1),
                                           (30000, 7041, 256, 2), (129, 20000, 128, -1)])
def test_streams_pass_the_launch_check(N, L, B, variant):
    x = synth.audio(N, 700 + L)
    H = np.stack([synth.decayed_ir(L, max(1.0, 0.2 * L), 710 + v) for v in range(3)])
    vstart = [0, N // 3, N // 3 + 1]
    s = capi.tc_open_group(1, L, B, True, capi.TC_FP32, 8 * B)
    outs = []
    try:
        capi.tc_set_tuning(s, capi.TC_TUNE_K1_CHUNK, variant)
        pos, v, k = 0, 0, 0
        while pos < N:
            n = min((1 + k % 8) * B, N - pos)   # one to eight blocks per push
            k += 1
            while v < len(vstart) and vstart[v] < pos + n:
                capi.tc_set_ir_rows(s, H[v][None], L, max(vstart[v], pos))
                v += 1
            y = np.empty((1, n), np.float32)
            capi.tc_push(s, x[None, pos:pos + n].copy(), n, y)
            outs.append(y[0])
            pos += n
        tail = np.empty((1, max(L - 1, 1)), np.float32)
        if L > 1:
            capi.tc_flush(s, tail, L - 1)
            outs.append(tail[0])
    finally:
        capi.tc_close(s)
    ref = oracle.buffer(x, H, np.asarray(vstart, np.int64), B)
    assert rel_l2(np.concatenate(outs), ref) <= TOL["fp32"]


def test_groups_mimo_and_fallbacks_pass_the_launch_check():
    # Per-channel IRs with crossfades.
    C, N, L, B = 3, 6000, 1500, 64
    x = synth.audio_block(C, N, 720)
    H = np.stack([np.stack([synth.decayed_ir(L, 300.0, 730 + 10 * c + v) for v in range(2)]) for c in range(C)])
    y = stream_host(x, H, [0, 2500], L, B, pushes=[64, 640, 1024], max_push=1024, shared_ir=False, ramps=[1, 400])
    for c in range(C):
        ref = oracle.buffer_xf(x[c], H[c], np.array([0, 2500], np.int64), np.array([1, 400], np.int64), B)
        assert rel_l2(y[c], ref) <= TOL["fp32"]
    # A BF16-split group whose windows across a switch run on K1.
    C, N, L, B = 130, 4000, 800, 128
    X = synth.audio_block(C, N, 740)
    Hs = np.stack([synth.decayed_ir(L, 160.0, 750 + v) for v in range(2)])
    y = stream_host(X, Hs, [0, 1700], L, B, max_push=512, precision=capi.TC_BF16_SPLIT)
    ref = oracle.buffer(X[129], Hs, np.array([0, 1700], np.int64), B)
    assert rel_l2(y[129], ref) <= TOL["bf16split"]
    # MIMO on K1.
    nin, nout, N, L, B = 2, 3, 3000, 600, 64
    Xm = synth.audio_block(nin, N, 760)
    Hm = np.stack([[synth.decayed_ir(L, 120.0, 770 + 2 * o + i) for i in range(nin)] for o in range(nout)])
    s = capi.tc_open_mimo(nin, nout, L, B, capi.TC_FP32, 512)
    outs = []
    try:
        capi.tc_set_ir_rows(s, Hm.reshape(nout * nin, L), L, 0)
        for pos in range(0, N, 512):
            n = min(512, N - pos)
            ym = np.empty((nout, n), np.float32)
            capi.tc_push(s, np.ascontiguousarray(Xm[:, pos:pos + n]), n, ym)
            outs.append(ym)
        tail = np.empty((nout, L - 1), np.float32)
        capi.tc_flush(s, tail, L - 1)
    finally:
        capi.tc_close(s)
    assert rel_l2(np.concatenate(outs + [tail], axis=1), oracle.mimo(Xm, Hm, None, B)) <= TOL["fp32"]
