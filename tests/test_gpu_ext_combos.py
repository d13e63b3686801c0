"""The gather's extensions together and on the other stream kinds, against the oracle's crossfade form (Sec. 6:
an IR that changes progressively):
  * crossfaded switches on a MIMO stream, in FP32 (K1) and in BF16 split (K3, with the windows that read a ramp
    on the FP32 gather);
  * zero gating (exact, threshold 0) on a group whose switches crossfade: bit-identical with and without.
"""
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


def _stream(s, X, rows_of_version, vstart, ramps, L, push, nout):
    """Pushes X [rows][N] in pushes of `push`, registering version v (its IR rows) at vstart[v] with a
    crossfade of ramps[v] samples; returns [nout][N + L - 1]."""
    N = X.shape[1]
    outs, pos, v = [], 0, 0
    while pos < N:
        n = min(push, N - pos)
        while v < len(vstart) and vstart[v] < pos + n:
            capi.tc_set_crossfade(s, ramps[v] if v else 1)
            capi.tc_set_ir_rows(s, np.ascontiguousarray(rows_of_version(v), np.float32), L, max(vstart[v], pos))
            v += 1
        y = np.empty((nout, n), np.float32)
        capi.tc_push(s, np.ascontiguousarray(X[:, pos:pos + n]), n, y)
        outs.append(y)
        pos += n
    tail = np.empty((nout, L - 1), np.float32)
    capi.tc_flush(s, tail, L - 1)
    return np.concatenate(outs + [tail], axis=1)


@pytest.mark.parametrize("prec", ["fp32", "bf16split"])
def test_crossfade_on_a_mimo_stream(prec):
    nin, nout, N, L, B, push = 3, 2, 5000, 900, 64, 512
    vstart, ramps = [0, 2100], [1, 700]
    X = synth.audio_block(nin, N, 96)
    H = np.stack([np.stack([np.stack([synth.decayed_ir(L, 180.0, 9400 + 100 * v + 10 * o + i) for i in range(nin)])
                            for o in range(nout)]) for v in range(len(vstart))])     # [v][o][i][L]
    code = {"fp32": capi.TC_FP32, "bf16split": capi.TC_BF16_SPLIT}[prec]
    s = capi.tc_open_mimo(nin, nout, L, B, code, push)
    try:
        y = _stream(s, X, lambda v: H[v].reshape(nout * nin, L), vstart, ramps, L, push, nout)
        info = capi.tc_get_info(s)
    finally:
        capi.tc_close(s)
    if prec != "fp32":
        assert info.tensor_launches > 0 and info.fp32_fallbacks > 0
    vs, rp = np.asarray(vstart, np.int64), np.asarray(ramps, np.int64)
    for o in range(nout):
        ref = sum(oracle.buffer_xf(X[i], H[:, o, i], vs, rp, B) for i in range(nin))
        err = rel_l2(y[o], ref)
        assert err <= TOL[prec], (o, err)


def test_zero_gating_with_crossfades_is_exact():
    C, N, L, B, push = 3, 30000, 5000, 128, 4096
    vstart, ramps = [0, 9000, 20000], [1, 800, 300]
    X = synth.audio_block(C, N, 97)
    X[:, 2000:14000] = 0.0           # silence longer than L, across the first crossfade
    X[2, 21000:26000] = 0.0
    H = np.stack([np.stack([synth.decayed_ir(L, 1000.0, 9500 + 10 * c + v) for v in range(len(vstart))])
                  for c in range(C)])                                                   # [c][v][L]
    outs = {}
    for gate in (0, 1):
        s = capi.tc_open_group(C, L, B, False, capi.TC_FP32, push)
        try:
            capi.tc_set_tuning(s, capi.TC_TUNE_ZERO_SKIP, gate)
            outs[gate] = _stream(s, X, lambda v: H[:, v], vstart, ramps, L, push, C)
        finally:
            capi.tc_close(s)
    assert np.array_equal(outs[0], outs[1])
    vs, rp = np.asarray(vstart, np.int64), np.asarray(ramps, np.int64)
    for c in range(C):
        err = rel_l2(outs[1][c], oracle.buffer_xf(X[c], H[c], vs, rp, B))
        assert err <= TOL["fp32"], (c, err)
