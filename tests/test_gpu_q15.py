"""Exact Q15 fixed-point convolution (K4, Sec. 5.4) through the C ABI against
the integer oracle: bit-exact int64 sums and int16 outputs, both inner-loop forms.
"""
import numpy as np
import pytest

import oracle
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu

INNER = ["dp2a", "imad"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2401_01607_gb300 as pkg
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()


@pytest.fixture(params=INNER)
def inner(request, monkeypatch):
    monkeypatch.setenv("TC_Q15_INNER", request.param)
    return request.param


def _gpu(xq, hq, want_y=True, want_acc=True):
    import torch
    N, L = xq.size, hq.size
    x = torch.from_numpy(xq).cuda()
    h = torch.from_numpy(hq).cuda()
    y = torch.full((N + L - 1,), 12345, dtype=torch.int16, device="cuda") if want_y else None
    acc = torch.full((N + L - 1,), -7, dtype=torch.int64, device="cuda") if want_acc else None
    capi.tc_convolve_q15(x, N, h, L, y, acc)
    return (None if acc is None else acc.cpu().numpy()), (None if y is None else y.cpu().numpy())


# Sizes span one tile (1024 outputs x 2048 taps), several tiles, and ragged tails on both axes.
SHAPES = [(1, 1), (5, 3), (1000, 1), (1, 3000), (3000, 2049), (4097, 4100), (20_000, 6_001), (1024, 2048)]


@pytest.mark.parametrize("N,L", SHAPES)
def test_full_range_bit_exact(inner, N, L):
    xq = synth.q15_full_range(N, 100 + N)
    hq = synth.q15_full_range(L, 200 + L)
    acc, y = _gpu(xq, hq)
    racc, ry = oracle.q15(xq, hq)
    np.testing.assert_array_equal(acc, racc)
    np.testing.assert_array_equal(y, ry)


def test_audio_codes_bit_exact(inner):
    """Q15 codes of the synthetic audio and a decayed IR (sum |h| = 1): the no-saturation regime."""
    N, L = 30_000, 4_800
    xq = synth.q15_codes(synth.audio(N, 7))
    hq = synth.q15_codes(synth.decayed_ir(L, 800.0, 8))
    acc, y = _gpu(xq, hq)
    racc, ry = oracle.q15(xq, hq)
    np.testing.assert_array_equal(acc, racc)
    np.testing.assert_array_equal(y, ry)


def test_halves_and_saturation(inner):
    """Sums that are exact odd multiples of 2^14 (round half to even) and full-scale sums (saturation)."""
    xq = np.array([1, 0, 0, 3, -1], np.int16)
    hq = np.array([16384, -16384, 16384, -32768, 16384, 49152 - 65536], np.int16)
    acc, y = _gpu(xq, hq)
    racc, ry = oracle.q15(xq, hq)
    np.testing.assert_array_equal(acc, racc)
    np.testing.assert_array_equal(y, ry)
    xq = np.full(5000, -32768, np.int16)
    hq = np.concatenate([np.full(3000, -32768, np.int16), np.full(3000, 32767, np.int16)])
    acc, y = _gpu(xq, hq)
    racc, ry = oracle.q15(xq, hq)
    np.testing.assert_array_equal(acc, racc)
    np.testing.assert_array_equal(y, ry)
    assert y.max() == 32767 and y.min() == -32768


def test_role_swap_is_bit_identical(monkeypatch):
    """N < L: the roles are swapped (Sec. 3.2) unless TC_NO_ROLE_SWAP=1; integer sums make both
    orientations bit-identical to the oracle."""
    xq = synth.q15_full_range(700, 31)
    hq = synth.q15_full_range(9_000, 32)
    racc, ry = oracle.q15(xq, hq)
    for flag in ("0", "1"):
        monkeypatch.setenv("TC_NO_ROLE_SWAP", flag)
        acc, y = _gpu(xq, hq)
        np.testing.assert_array_equal(acc, racc)
        np.testing.assert_array_equal(y, ry)


def test_acc_only_and_y_only():
    xq = synth.q15_full_range(2500, 1)
    hq = synth.q15_full_range(700, 2)
    racc, ry = oracle.q15(xq, hq)
    acc, y = _gpu(xq, hq, want_y=False)
    assert y is None
    np.testing.assert_array_equal(acc, racc)
    acc, y = _gpu(xq, hq, want_acc=False)
    assert acc is None
    np.testing.assert_array_equal(y, ry)


def test_errors():
    import torch
    x = torch.zeros(16, dtype=torch.int16, device="cuda")
    y = torch.zeros(16, dtype=torch.int16, device="cuda")
    with pytest.raises(capi.TcError):
        capi.tc_convolve_q15(x, 0, x, 1, y)
    with pytest.raises(capi.TcError):
        capi.tc_convolve_q15(x, 1, x, 0, y)
    with pytest.raises(capi.TcError):
        capi.tc_convolve_q15(x, 1, x, (1 << 19) + 1, y)
    with pytest.raises(capi.TcError):
        capi.tc_convolve_q15(x, 1, x, 1, None, None)


FULL_N, FULL_L = 2_880_000, 48_000
FULL_SPANS = [(0, 1500), (1_234_567, 1500), (FULL_N + FULL_L - 1 - 1500, 1500)]


@pytest.fixture(scope="module")
def full_size():
    """The timed workload (60 s of 48 kHz audio as Q15 codes, a 1 s decayed IR) and, per checked
    span of outputs, the oracle's result on the input window that reaches it."""
    xq = synth.q15_codes(synth.audio(FULL_N, synth.x_seed(7, 0)))
    hq = synth.q15_codes(synth.decayed_ir(FULL_L, 4800.0, synth.ir_seed(7, 0)))
    refs = []
    for s, span in FULL_SPANS:
        lo = max(0, s - FULL_L + 1)
        racc, ry = oracle.q15(xq[lo:min(FULL_N, s + span)], hq)
        refs.append((racc[s - lo:s - lo + span], ry[s - lo:s - lo + span]))
    return xq, hq, refs


def test_full_size_sampled(inner, full_size):
    """Spans at the start, the middle and the flushed tail of the full-size launch."""
    xq, hq, refs = full_size
    acc, y = _gpu(xq, hq)
    for (s, span), (racc, ry) in zip(FULL_SPANS, refs):
        np.testing.assert_array_equal(acc[s:s + span], racc)
        np.testing.assert_array_equal(y[s:s + span], ry)
