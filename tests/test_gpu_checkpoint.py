"""Checkpoint / resume (tc_stream_export / tc_stream_import): a run split at a push boundary, exported,
and resumed in a new stream gives the same bits as the unsplit run; on the gather (K1, with IR switches and a
crossfade), the shared-IR tensor path (K2), a mono stream on K2's row view and the MIMO tensor path (K3). The
unsplit run is also checked against the oracle.
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


def _run(open_fn, X, irs, L, P, split_at=None):
    """Pushes X [rows, N] in pieces of P; irs: [(sample, rows array, ramp)] registered before the push that
    holds their sample. split_at: number of pushes after which the stream is exported, closed, and resumed
    in a fresh stream. Returns y [out_rows, N + L - 1]."""
    rows, N = X.shape
    s = open_fn()
    outs, k = [], 0
    try:
        for i, pos in enumerate(range(0, N, P)):
            if split_at is not None and i == split_at:
                blob = capi.tc_stream_export(s)
                capi.tc_close(s)
                s = open_fn()
                capi.tc_stream_import(s, blob)
            n = min(P, N - pos)
            while k < len(irs) and irs[k][0] < pos + n:
                sample, Hk, ramp = irs[k]
                capi.tc_set_crossfade(s, ramp)
                capi.tc_set_ir_rows(s, np.ascontiguousarray(Hk), L, sample)
                k += 1
            y = np.empty((capi.tc_get_info(s).outputs, n), np.float32)
            capi.tc_push(s, np.ascontiguousarray(X[:, pos:pos + n]), n, y)
            outs.append(y)
        tail = np.empty((capi.tc_get_info(s).outputs, L - 1), np.float32)
        capi.tc_flush(s, tail, L - 1)
    finally:
        capi.tc_close(s)
    return np.concatenate(outs + [tail], axis=1)


def test_gather_with_switches_and_crossfade_resumes_bit_exact():
    C, N, L, B, P = 4, 6000, 3000, 128, 512
    X = synth.audio_block(C, N, 500)
    H = [np.stack([synth.decayed_ir(L, 900.0, 510 + 10 * v + c) for c in range(C)]) for v in range(3)]
    irs = [(0, H[0], 1), (1000, H[1], 1), (2600, H[2], 200)]

    def opener():
        return capi.tc_open_group(C, L, B, False, capi.TC_FP32, P)

    whole = _run(opener, X, irs, L, P)
    for split in (1, 3, 5, 11):
        resumed = _run(opener, X, irs, L, P, split_at=split)
        assert np.array_equal(whole, resumed), split
    # The unsplit run against the oracle's crossfade form.
    Hv = np.stack(H)  # [nver, C, L]
    vstart = np.array([0, 1000, 2600], np.int64)
    ramps = np.array([1, 1, 200], np.int64)
    for c in (0, 3):
        ref = oracle.buffer_xf(X[c], Hv[:, c], vstart, ramps, B)
        assert rel_l2(whole[c], ref) <= TOL["fp32"]


@pytest.mark.parametrize("prec", ["bf16split", "bf16"])
def test_shared_ir_tensor_path_resumes_bit_exact(prec):
    code = {"bf16split": capi.TC_BF16_SPLIT, "bf16": capi.TC_BF16}[prec]
    C, N, L, B, P = 130, 5000, 3000, 256, 1024
    X = synth.audio_block(C, N, 520)
    h = synth.decayed_ir(L, 600.0, 521)[None]
    irs = [(0, h, 1)]

    def opener():
        return capi.tc_open_group(C, L, B, True, code, P)

    whole = _run(opener, X, irs, L, P)
    resumed = _run(opener, X, irs, L, P, split_at=2)
    assert np.array_equal(whole, resumed)
    assert rel_l2(whole[129], oracle.buffer(X[129], h, None, B)) <= TOL[prec]


def test_mimo_tensor_path_resumes_bit_exact():
    nin, nout, N, L, B, P = 2, 3, 6000, 2000, 512, 1024
    X = synth.audio_block(nin, N, 530)
    H = np.stack([[synth.decayed_ir(L, 400.0, 540 + 2 * o + i) for i in range(nin)] for o in range(nout)])
    irs = [(0, H, 1)]

    def opener():
        return capi.tc_open_mimo(nin, nout, L, B, capi.TC_BF16_SPLIT, P)

    whole = _run(opener, X, irs, L, P)
    resumed = _run(opener, X, irs, L, P, split_at=3)
    assert np.array_equal(whole, resumed)
    assert rel_l2(whole, oracle.mimo(X, H[None], None, B)) <= TOL["bf16split"]


def test_mono_row_view_resumes_bit_exact():
    """A mono BF16-split stream on device 0 (K2 on 256-sample rows), with an IR switch whose windows run on
    the FP32 gather."""
    N, L, B, P = 20000, 3000, 256, 2048
    X = synth.audio_block(1, N, 550)
    H = [synth.decayed_ir(L, 600.0, 551 + v)[None] for v in range(2)]
    irs = [(0, H[0], 1), (9000, H[1], 1)]

    def opener():
        return capi.tc_open_stream_ex(L, B, capi.TC_BF16_SPLIT, 0, P)

    whole = _run(opener, X, irs, L, P)
    for split in (2, 5):
        assert np.array_equal(whole, _run(opener, X, irs, L, P, split_at=split)), split
    ref = oracle.buffer(X[0], np.concatenate(H), np.array([0, 9000], np.int64), B)
    assert rel_l2(whole[0], ref) <= TOL["bf16split"]


def test_import_rejects_other_shapes_and_foreign_blobs():
    s = capi.tc_open_group(2, 500, 64, False, capi.TC_FP32, 128)
    t = capi.tc_open_group(2, 600, 64, False, capi.TC_FP32, 128)
    try:
        capi.tc_set_ir_rows(s, np.ones((2, 500), np.float32), 500, 0)
        capi.tc_push(s, np.ones((2, 128), np.float32), 128, np.empty((2, 128), np.float32))
        blob = capi.tc_stream_export(s)
        with pytest.raises(capi.TcError) as e:
            capi.tc_stream_import(t, blob)  # another L
        assert e.value.code == "TC_EINVAL"
        bad = bytearray(blob)
        bad[0] ^= 0xFF
        with pytest.raises(capi.TcError) as e:
            capi.tc_stream_import(s, bytes(bad))
        assert e.value.code == "TC_EINVAL"
        with pytest.raises(capi.TcError):
            capi.tc_stream_import(s, blob[:len(blob) // 2])  # truncated
    finally:
        capi.tc_close(s)
        capi.tc_close(t)
