"""Guard canaries around caller-owned device buffers: every device-pointer entry point writes only inside the
output it was given.

Each output sits between two margins of 4096 elements filled with a marker (a NaN payload for float32, fixed
codes for int16 and int64) that is checked after the call; the inputs are checked unchanged, and the results
against the oracle. The cases take ragged sizes: outputs that end inside a tile, a flush whose rows have the odd
pitch L - 1, a K2 launch with one K part, the tensor-core row view of one signal, MIMO with fewer than 16 outputs.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu

PAD = 4096
MARK = {"float32": 0x7FC0DEAD, "int16": -12345, "int64": 0x5A5A5A5A5A5A5A5A}


@pytest.fixture(scope="module")
def torch():
    import paper_2401_01607_gb300 as pkg
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()
    return t


class Guarded:
    """A device buffer of n elements between two marked margins."""

    def __init__(self, torch, n, dtype="float32"):
        self.torch, self.n, self.dtype = torch, n, dtype
        tdt = {"float32": torch.float32, "int16": torch.int16, "int64": torch.int64}[dtype]
        self.buf = torch.empty(n + 2 * PAD, dtype=tdt, device="cuda")
        self._bits().fill_(MARK[dtype])

    def _bits(self):
        return self.buf.view(self.torch.int32) if self.dtype == "float32" else self.buf

    def body(self):
        return self.buf[PAD:PAD + self.n]

    def check(self, what):
        self.torch.cuda.synchronize()
        bits = self._bits()
        for name, part in (("before", bits[:PAD]), ("after", bits[PAD + self.n:])):
            bad = int((part != MARK[self.dtype]).sum())
            assert bad == 0, f"{what}: {bad} elements written {name} the output"


def test_one_shot_calls_write_only_their_output(torch):
    for i, (N, L) in enumerate([(1000, 700), (300, 5000), (4099, 129)]):
        x = synth.audio(N, 900 + i)
        h = synth.decayed_ir(L, 0.2 * L, 910 + i)
        ref = oracle.direct(x, h[None])
        xd, hd = torch.from_numpy(x).cuda(), torch.from_numpy(h).cuda()
        for name, call, tol in (("tc_convolve", lambda y: capi.tc_convolve(xd, N, hd, L, y), TOL["fp32"]),
                                ("tc_convolve_noalloc", lambda y: capi.tc_convolve_noalloc(xd, N, hd, L, y),
                                 TOL["fp32"]),
                                ("tc_convolve_tc", lambda y: capi.tc_convolve_tc(xd, N, hd, L, y, capi.TC_BF16_SPLIT),
                                 TOL["bf16split"])):
            y = Guarded(torch, N + L - 1)
            call(y.body())
            y.check(f"{name} N={N} L={L}")
            assert rel_l2(y.body().cpu().numpy(), ref) <= tol, (name, N, L)
        assert np.array_equal(xd.cpu().numpy(), x) and np.array_equal(hd.cpu().numpy(), h)


def test_q15_writes_only_y_and_acc(torch):
    for i, (N, L) in enumerate([(1000, 700), (200, 3000), (2049, 2047)]):
        xq = synth.q15_full_range(N, 920 + i)
        hq = synth.q15_full_range(L, 930 + i)
        racc, ry = oracle.q15(xq, hq)
        xd, hd = torch.from_numpy(xq).cuda(), torch.from_numpy(hq).cuda()
        y = Guarded(torch, N + L - 1, "int16")
        acc = Guarded(torch, N + L - 1, "int64")
        capi.tc_convolve_q15(xd, N, hd, L, y.body(), acc.body())
        y.check(f"q15 y N={N} L={L}")
        acc.check(f"q15 acc N={N} L={L}")
        np.testing.assert_array_equal(acc.body().cpu().numpy(), racc)
        np.testing.assert_array_equal(y.body().cpu().numpy(), ry)
        assert np.array_equal(xd.cpu().numpy(), xq) and np.array_equal(hd.cpu().numpy(), hq)


def _open(kind):
    """(stream, channels, outputs, L, block, max_push, IR rows [sets][L], tolerance)."""
    if kind == "own_ir_fp32":
        C, L, B, mp = 5, 1000, 128, 1024
        H = np.stack([synth.decayed_ir(L, 0.2 * L, 940 + c) for c in range(C)])
        return capi.tc_open_group(C, L, B, False, capi.TC_FP32, mp), C, C, L, B, mp, H, TOL["fp32"]
    if kind == "shared_bf16split":
        C, L, B, mp = 130, 700, 64, 960
        H = synth.decayed_ir(L, 0.2 * L, 950)[None]
        return capi.tc_open_group(C, L, B, True, capi.TC_BF16_SPLIT, mp), C, C, L, B, mp, H, TOL["bf16split"]
    if kind == "mono_rows_bf16split":
        L, B, mp = 700, 256, 2048
        H = synth.decayed_ir(L, 0.2 * L, 960)[None]
        return capi.tc_open_stream_ex(L, B, capi.TC_BF16_SPLIT, -1, mp), 1, 1, L, B, mp, H, TOL["bf16split"]
    nin, nout, L, B, mp = 3, 2, 300, 64, 960
    H = np.stack([synth.decayed_ir(L, 0.2 * L, 970 + k) for k in range(nout * nin)])
    return capi.tc_open_mimo(nin, nout, L, B, capi.TC_BF16_SPLIT, mp), nin, nout, L, B, mp, H, TOL["bf16split"]


@pytest.mark.parametrize("kind", ["own_ir_fp32", "shared_bf16split", "mono_rows_bf16split", "mimo_bf16split"])
def test_device_pushes_and_flush_write_only_their_rows(torch, kind):
    s, C, nout, L, B, mp, H, tol = _open(kind)
    pushes = [mp, mp, B + 37]                        # two full pushes, then a ragged last one
    N = sum(pushes)
    X = np.stack([synth.audio(N, 980 + c) for c in range(C)])
    outs = []
    try:
        capi.tc_set_ir_rows(s, np.ascontiguousarray(H, np.float32), L, 0)
        pos = 0
        for n in pushes:
            xd = torch.from_numpy(np.ascontiguousarray(X[:, pos:pos + n])).cuda()
            x_before = xd.clone()
            y = Guarded(torch, nout * n)
            capi.tc_push(s, xd, n, y.body(), capi.TC_PUSH_DEVICE)
            capi.tc_sync(s)
            y.check(f"{kind} push of {n}")
            assert torch.equal(xd, x_before)
            outs.append(y.body().cpu().numpy().reshape(nout, n))
            pos += n
        tail = Guarded(torch, nout * (L - 1))
        capi.tc_flush_dev(s, tail.body())
        capi.tc_sync(s)
        tail.check(f"{kind} flush")
        outs.append(tail.body().cpu().numpy().reshape(nout, L - 1))
    finally:
        capi.tc_close(s)
    got = np.concatenate(outs, axis=1)
    if kind == "mimo_bf16split":
        ref = oracle.mimo(X, H.reshape(nout, C, L))
    elif kind == "own_ir_fp32":
        ref = np.stack([oracle.buffer(X[c], H[c][None], None, B) for c in range(C)])
    else:
        ref = np.stack([oracle.buffer(X[c], H, None, B) for c in range(C)])
    assert got.shape == ref.shape
    assert rel_l2(got, ref) <= tol, kind
