"""Shared-IR groups on the tensor cores (K2): BF16 and BF16 hi/lo split against the FP64 oracle.

Tolerances (relative L2): BF16 hi/lo split <= 1e-5, plain BF16 <= 3e-3.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, max_abs, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu

PREC = {"bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2401_01607_gb300 as pkg
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()


def run_group(X, H, vstart, L, block, prec, max_push, tuning=()):
    """Streams X [C, N] through a shared-IR group; returns (y [C, N+L-1], info).
    tuning: (knob, value) pairs set before the first push."""
    C, N = X.shape
    s = capi.tc_open_group(C, L, block, True, PREC[prec], max_push)
    try:
        for knob, value in tuning:
            capi.tc_set_tuning(s, knob, value)
        outs, pos, v = [], 0, 0
        while pos < N:
            n = min(max_push, N - pos)
            while v < len(vstart) and vstart[v] < pos + n:
                capi.tc_set_ir_rows(s, H[v][None], H.shape[1], max(int(vstart[v]), pos))
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
    return np.concatenate(outs + [tail], axis=1), info


def check(y, X, H, vstart, block, prec, rows=None):
    rows = range(X.shape[0]) if rows is None else rows
    errs = []
    for c in rows:
        ref = oracle.buffer(X[c], H, np.asarray(vstart, np.int64), block)
        errs.append(rel_l2(y[c], ref))
    worst = max(errs)
    print(f"{prec}: worst rel_l2 {worst:.3g}")
    assert worst <= TOL[prec], worst


@pytest.mark.parametrize("prec", ["bf16split", "bf16"])
def test_shared_ir_small(prec):
    """200 channels (two channel tiles, ragged), ragged pushes and tail."""
    C, N, L, B = 200, 5000, 3000, 256
    X = synth.audio_block(C, N, 3000)
    H = synth.decayed_ir(L, 0.2 * L, 77)[None]
    y, info = run_group(X, H, [0], L, B, prec, 1024)
    assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    check(y, X, H, [0], B, prec, rows=[0, 1, 127, 128, 150, 199])


@pytest.mark.parametrize("prec", ["bf16split", "bf16"])
def test_shared_ir_long_split_k(prec):
    """L = 20000: K split over several CTAs, then the pairwise K-range reduction."""
    C, N, L, B = 256, 3000, 20_000, 256
    X = synth.audio_block(C, N, 4000)
    H = synth.decayed_ir(L, 0.2 * L, 78)[None]
    y, info = run_group(X, H, [0], L, B, prec, 3072)
    assert info.tensor_launches > 0
    check(y, X, H, [0], B, prec, rows=[0, 97, 255])


def test_shared_ir_switch_falls_back_exactly():
    """An IR switch mid-stream: windows that straddle it run on the FP32 gather, the rest on K2."""
    C, N, L, B = 130, 6000, 1000, 128
    X = synth.audio_block(C, N, 5000)
    H = np.stack([synth.decayed_ir(L, 200.0, 90 + v) for v in range(2)])
    vs = [0, 2500]
    y, info = run_group(X, H, vs, L, B, "bf16split", 512)
    assert info.tensor_launches > 0 and info.fp32_fallbacks > 0
    check(y, X, H, vs, B, "bf16split", rows=[0, 64, 129])


@pytest.mark.parametrize("pair", [2, 3, 1, 0])
@pytest.mark.parametrize("L", [3000, 20_000])
def test_bf16_two_tiles_per_cta(pair, L):
    """Plain BF16 on persistent CTA pairs (tcgen05 cta_group::2, default), on
    CTA pairs launched per unit, with two channel tiles per CTA, and with one:
    300 channels = three tiles, so the second pair is half outside the group;
    the K range splits over CTAs at L = 20000."""
    C, N, B = 300, 2600, 256
    X = synth.audio_block(C, N, 6000 + L)
    H = synth.decayed_ir(L, 0.2 * L, 79)[None]
    y, info = run_group(X, H, [0], L, B, "bf16", 1280, tuning=[(capi.TC_TUNE_K2_PAIR, pair)])
    assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    check(y, X, H, [0], B, "bf16", rows=[0, 127, 128, 255, 256, 299])


@pytest.mark.parametrize("nsplit", [2, 3, 5, 8, 13, 16, 17])
@pytest.mark.parametrize("prec,pair", [("bf16", 2), ("bf16", 0), ("bf16split", 2)])
def test_k_parts_folded_in_kernel_equal_k2_reduce(prec, pair, nsplit):
    """The tensor-core kernels add a tile's K parts themselves (the warp that
    takes a slice's last ticket folds it, by the same pairwise tree as
    k2_reduce): on the persistent CTA pairs (plain BF16) and on the one-tile
    kernel (plain BF16 with TC_TUNE_K2_PAIR 0; the BF16 split). With the fold
    switched off, k2_reduce adds the same parts. Both give the same bits, in
    pushes (aligned rows) and in the flush (rows of odd pitch L - 1), and match
    the oracle. 17 parts are beyond the in-kernel fold and go to k2_reduce
    either way."""
    C, N, L, B = 300, 2600, 20_000, 256
    X = synth.audio_block(C, N, 8000 + nsplit)
    H = synth.decayed_ir(L, 0.2 * L, 81)[None]
    ys = {}
    for fold in (1, 0):
        ys[fold], info = run_group(X, H, [0], L, B, prec, 1280,
                                   tuning=[(capi.TC_TUNE_K2_PAIR, pair), (capi.TC_TUNE_K2_SPLIT, nsplit),
                                           (capi.TC_TUNE_K2_FOLD, fold)])
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    assert np.array_equal(ys[1], ys[0]), np.argwhere(ys[1] != ys[0])[:5]
    check(ys[1], X, H, [0], B, prec, rows=[0, 31, 32, 127, 128, 255, 256, 299])


@pytest.mark.parametrize("nsplit,rng", [(1, 16), (3, 16), (4, 5), (17, 16)])
def test_split_on_cta_pairs_equals_single_tiles(nsplit, rng):
    """The BF16 split on persistent CTA pairs (each SM staging half of the
    operands, runs of `range` K blocks drained into FP32 registers) computes
    exactly what the one-tile kernel computes with the same K parts and runs:
    same bits, in pushes and in the flush (odd pitch); and both match the
    oracle. 300 channels: the second pair is half outside the group. An odd
    range leaves a short last run in every part."""
    C, N, L, B = 300, 2600, 20_000, 256
    X = synth.audio_block(C, N, 9000 + nsplit)
    H = synth.decayed_ir(L, 0.2 * L, 83)[None]
    ys = {}
    for pair in (2, 0):
        ys[pair], info = run_group(X, H, [0], L, B, "bf16split", 1280,
                                   tuning=[(capi.TC_TUNE_K2_PAIR, pair), (capi.TC_TUNE_K2_SPLIT, nsplit),
                                           (capi.TC_TUNE_K2_RANGE, rng)])
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    assert np.array_equal(ys[2], ys[0]), np.argwhere(ys[2] != ys[0])[:5]
    check(ys[2], X, H, [0], B, "bf16split", rows=[0, 31, 127, 128, 255, 256, 299])


@pytest.mark.parametrize("nsplit", [-1, 3, 17])
@pytest.mark.parametrize("prec", ["bf16", "bf16split"])
def test_one_channel_tile_pairs_output_tiles(prec, nsplit):
    """A group of at most 128 channels runs on the persistent CTA pairs with the two CTAs on two adjacent output
    tiles of the same channels (each multiplies its own X window by the shared IR tile). With the same K parts it
    gives the same bits as one tile per CTA (TC_TUNE_K2_PAIR 0), in pushes of 5 output tiles (the last pair has one)
    and in a flush of odd pitch; with the planned K parts (-1) the two forms plan for different unit counts, so
    there only the oracle decides."""
    C, N, L, B = 100, 2600, 20_000, 256
    X = synth.audio_block(C, N, 9700 + max(nsplit, 0))
    H = synth.decayed_ir(L, 0.2 * L, 85)[None]
    ys = {}
    for pair in (2, 0):
        ys[pair], info = run_group(X, H, [0], L, B, prec, 1280,
                                   tuning=[(capi.TC_TUNE_K2_PAIR, pair), (capi.TC_TUNE_K2_SPLIT, nsplit)])
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    if nsplit > 0:
        assert np.array_equal(ys[2], ys[0]), np.argwhere(ys[2] != ys[0])[:5]
    check(ys[2], X, H, [0], B, prec, rows=[0, 31, 32, 63, 99])
    check(ys[0], X, H, [0], B, prec, rows=[0, 99])


@pytest.mark.parametrize("prec", ["bf16", "bf16split"])
def test_unit_order_of_cta_pairs_does_not_change_bits(prec):
    """The persistent CTA pairs take their units in one of three orders; each
    unit computes the same sums whichever pair takes it, and the K parts are
    folded by the same tree, so all three give the same bits."""
    C, N, L, B = 520, 2600, 20_000, 256
    X = synth.audio_block(C, N, 9500)
    H = synth.decayed_ir(L, 0.2 * L, 84)[None]
    ys = [run_group(X, H, [0], L, B, prec, 1280, tuning=[(capi.TC_TUNE_K2_ORDER, o)])[0] for o in (0, 1, 2)]
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])
    check(ys[0], X, H, [0], B, prec, rows=[0, 255, 256, 511, 512, 519])


@pytest.mark.parametrize("prec", ["bf16split", "bf16"])
def test_short_ir_one_k_part_odd_pitch(prec):
    """A short IR (L = 700: fewer than 32 K blocks, so one K part and the epilogue writes y itself) with
    pushes and a flush whose output rows have odd pitch (476 and 699 floats): rows start unaligned."""
    C, N, L, B = 130, 1500, 700, 256
    X = synth.audio_block(C, N, 3100)
    H = synth.decayed_ir(L, 140.0, 78)[None]
    y, info = run_group(X, H, [0], L, B, prec, 1024)
    assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    check(y, X, H, [0], B, prec, rows=[0, 1, 2, 3, 65, 127, 128, 129])


@pytest.mark.parametrize("prec", ["bf16split", "bf16"])
@pytest.mark.parametrize("N,L", [(100_000, 3_000), (2_000, 70_000), (1, 1), (300, 257), (40_000, 40_000)])
def test_single_signal_on_the_tensor_cores(prec, N, L):
    """tc_convolve_tc: one signal, the output cut into 256-sample rows that run as K2's channels (overlapping
    windows of one input); role swap when N < L; ragged rows and tiles."""
    torch = pytest.importorskip("torch")
    x = synth.audio(N, 900 + N)
    h = synth.decayed_ir(L, max(1.0, 0.2 * L), 901 + L)
    y = torch.full((N + L - 1,), float("nan"), device="cuda")
    capi.tc_convolve_tc(torch.from_numpy(x).cuda(), N, torch.from_numpy(h).cuda(), L, y, PREC[prec])
    ref = oracle.buffer(x, h[None], None, 4096) if N >= L else oracle.buffer(h, x[None], None, 4096)
    got = y.cpu().numpy()
    assert np.all(np.isfinite(got))
    err = rel_l2(got, ref)
    print(f"{prec} N={N} L={L}: rel_l2={err:.3g}")
    assert err <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16split", "bf16"])
@pytest.mark.parametrize("P", [4096, 256, 128])
def test_mono_stream_on_the_tensor_cores(prec, P):
    """tc_open_stream_ex in the BF16 modes: pushes of >= 256 samples run K2 on the push's 256-sample rows
    (overlapping windows of the one history), shorter ones as a one-channel tile; an IR switch inside the run
    (windows that straddle it fall back to K1), a short last push and the flush."""
    L, N = 3000, 20_000
    x = synth.audio(N, 950 + P)
    H = np.stack([synth.decayed_ir(L, 600.0, 951 + v) for v in range(2)])
    vstart = [0, 9000]
    s = capi.tc_open_stream_ex(L, min(P, 256), PREC[prec], -1, P)
    outs = []
    try:
        capi.tc_set_ir(s, H[0])
        capi.tc_set_ir_at(s, H[1], vstart[1])
        for pos in range(0, N, P):
            n = min(P, N - pos)
            y = np.empty((1, n), np.float32)
            capi.tc_push(s, np.ascontiguousarray(x[None, pos:pos + n]), n, y)
            outs.append(y)
        tail = np.empty((1, L - 1), np.float32)
        capi.tc_flush(s, tail, L - 1)
        info = capi.tc_get_info(s)
    finally:
        capi.tc_close(s)
    y = np.concatenate(outs + [tail], axis=1)[0]
    ref = oracle.buffer(x, H, np.asarray(vstart, np.int64), min(P, 256))
    err = rel_l2(y, ref)
    print(f"mono {prec} P={P}: rel_l2={err:.3g}, tensor launches {info.tensor_launches}, fallbacks {info.fp32_fallbacks}")
    assert info.tensor_launches > 0
    assert err <= TOL[prec]


def test_tuning_knobs_reject_values_out_of_range():
    """Every tuning knob of the tensor path takes -1 (default) or its documented range; anything else is
    TC_EINVAL and leaves the stream usable."""
    s = capi.tc_open_group(4, 1000, 256, True, capi.TC_BF16, 1024)
    try:
        for knob, good, bad in [(capi.TC_TUNE_K2_RANGE, (-1, 1, 4096), (0, 4097)),
                                (capi.TC_TUNE_K2_PAIR, (-1, 0, 1, 2, 3), (4, -2)),
                                (capi.TC_TUNE_K2_SPLIT, (-1, 1, 64), (0, 65)),
                                (capi.TC_TUNE_K2_FOLD, (-1, 0, 1), (2, -2)),
                                (capi.TC_TUNE_K2_ORDER, (-1, 0, 1, 2), (3, -2)),
                                (99, (), (0,))]:
            for v in good:
                capi.tc_set_tuning(s, knob, v)
            for v in bad:
                with pytest.raises(capi.TcError) as e:
                    capi.tc_set_tuning(s, knob, v)
                assert e.value.code == "TC_EINVAL", (knob, v)
        h = synth.decayed_ir(1000, 200.0, 78)
        capi.tc_set_ir_rows(s, h[None], 1000, 0)
        X = synth.audio_block(4, 600, 77)
        y = np.empty((4, 600), np.float32)
        capi.tc_push(s, np.ascontiguousarray(X), 600, y)  # still usable
        ref = oracle.buffer(X[1], h[None], np.zeros(1, np.int64), 256)[:600]
        assert rel_l2(y[1], ref) <= TOL["bf16"]
    finally:
        capi.tc_close(s)
