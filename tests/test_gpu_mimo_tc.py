"""MIMO on the tensor cores (K3): BF16 and BF16 hi/lo split against the FP64 oracle.

Each output is the sum over the inputs of one convolution per pair (Eq. 4 per
pair). Tolerances (relative L2): BF16 hi/lo split <= 1e-5, plain BF16 <= 3e-3.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu

PREC = {"bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT, "fp32": capi.TC_FP32}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2401_01607_gb300 as pkg
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()


def run_mimo(X, H, vstart, L, B, prec, max_push, tuning=()):
    """X [nin, N]; H [nver, nout, nin, L]; returns (y [nout, N + L - 1], info).
    tuning: (knob, value) pairs set before the first push."""
    nin, N = X.shape
    nout = H.shape[1]
    s = capi.tc_open_mimo(nin, nout, L, B, PREC[prec], max_push)
    try:
        for knob, value in tuning:
            capi.tc_set_tuning(s, knob, value)
        outs, pos, v = [], 0, 0
        while pos < N:
            n = min(max_push, N - pos)
            while v < len(vstart) and vstart[v] < pos + n:
                capi.tc_set_ir_rows(s, np.ascontiguousarray(H[v]), L, max(int(vstart[v]), pos))
                v += 1
            y = np.empty((nout, n), np.float32)
            capi.tc_push(s, np.ascontiguousarray(X[:, pos:pos + n]), n, y)
            outs.append(y)
            pos += n
        tail = np.empty((nout, L - 1), np.float32)
        capi.tc_flush(s, tail, L - 1)
        info = capi.tc_get_info(s)
    finally:
        capi.tc_close(s)
    return np.concatenate(outs + [tail], axis=1), info


def irs(nver, nout, nin, L, seed):
    return np.stack([[[synth.decayed_ir(L, 0.2 * L, seed + 1000 * v + o * nin + i) for i in range(nin)]
                      for o in range(nout)] for v in range(nver)])


@pytest.mark.parametrize("prec", ["bf16split", "bf16"])
def test_mimo_small(prec):
    """3 inputs x 2 outputs, ragged pushes (1280 = a tile and a quarter) and tail."""
    nin, nout, N, L, B = 3, 2, 5000, 3000, 256
    X = synth.audio_block(nin, N, 7000)
    H = irs(1, nout, nin, L, 70)
    y, info = run_mimo(X, H, [0], L, B, prec, 1280)
    assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    ref = oracle.mimo(X, H, None, B)
    err = rel_l2(y, ref)
    print(f"{prec}: rel_l2 {err:.3g}")
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", ["bf16split", "bf16"])
def test_mimo_16x16_split_k(prec):
    """16 x 16 with L = 20000: K = 16 inputs x 20000 taps split over CTAs."""
    nin, nout, N, L, B = 16, 16, 2200, 20_000, 512
    X = synth.audio_block(nin, N, 7100)
    H = irs(1, nout, nin, L, 71)
    y, info = run_mimo(X, H, [0], L, B, prec, 2048)
    assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    for o in (0, 7, 15):
        ref = sum(oracle.buffer(X[i], H[0, o, i][None], np.zeros(1, np.int64), B) for i in range(nin))
        err = rel_l2(y[o], ref)
        print(f"{prec} output {o}: rel_l2 {err:.3g}")
        assert err <= TOL[prec], (o, err)


@pytest.mark.parametrize("prec,rng", [("bf16split", 5), ("bf16split", 12), ("bf16", 3), ("bf16", 20)])
def test_mimo_runs_of_any_length(prec, rng):
    """TMEM runs of a set length (TC_TUNE_K2_RANGE, rounded up to whole pipeline stages of 8 K blocks in BF16
    and 4 in the split): every run boundary falls on a stage boundary and the drains match the runs."""
    nin, nout, N, L, B = 4, 5, 2200, 9000, 512
    X = synth.audio_block(nin, N, 7300 + rng)
    H = irs(1, nout, nin, L, 73)
    y, info = run_mimo(X, H, [0], L, B, prec, 2048, tuning=[(capi.TC_TUNE_K2_RANGE, rng)])
    assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    ref = oracle.mimo(X, H, None, B)
    assert rel_l2(y, ref) <= TOL[prec], rel_l2(y, ref)


def test_mimo_ir_switch_falls_back():
    """An IR switch mid-stream: launches whose window straddles it run on the FP32 gather."""
    nin, nout, N, L, B = 2, 3, 6000, 800, 256
    X = synth.audio_block(nin, N, 7200)
    H = irs(2, nout, nin, L, 72)
    y, info = run_mimo(X, H, [0, 3000], L, B, "bf16split", 1024)
    assert info.tensor_launches > 0 and info.fp32_fallbacks > 0
    ref = oracle.mimo(X, H, np.array([0, 3000], np.int64), B)
    assert rel_l2(y, ref) <= TOL["bf16split"], rel_l2(y, ref)
