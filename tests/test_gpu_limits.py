"""Maximum sizes against the oracle: the longest IR of the exact Q15 path (2^19 taps, caller's roles), a stream
whose IR (3 million taps) needs the largest tap chunks, and a served stream at the server's longest IR; one past
each limit is refused with TC_EINVAL.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu

SERVER_MAX_L = 4095 * 32 * 20 - 8  # K1's pairwise chunk stack x the smallest tap chunk


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2401_01607_gb300 as pkg
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()


def test_q15_longest_ir_bit_exact(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setenv("TC_NO_ROLE_SWAP", "1")
    N, L = 200, 1 << 19
    xq = synth.q15_full_range(N, 61)
    hq = synth.q15_full_range(L, 62)
    y = torch.empty(N + L - 1, dtype=torch.int16, device="cuda")
    acc = torch.empty(N + L - 1, dtype=torch.int64, device="cuda")
    capi.tc_convolve_q15(torch.from_numpy(xq).cuda(), N, torch.from_numpy(hq).cuda(), L, y, acc)
    racc, ry = oracle.q15(xq, hq)
    np.testing.assert_array_equal(acc.cpu().numpy(), racc)
    np.testing.assert_array_equal(y.cpu().numpy(), ry)
    with pytest.raises(capi.TcError) as e:
        capi.tc_convolve_q15(torch.from_numpy(xq).cuda(), N, torch.from_numpy(hq).cuda(), L + 1, y, acc)
    assert e.value.code == "TC_EINVAL"


def test_stream_with_a_3_million_tap_ir():
    N, L, B = 512, 3_000_000, 256
    x = synth.audio(N, 63)
    h = synth.decayed_ir(L, 0.2 * L, 64)
    s = capi.tc_open_stream(L, B)
    outs = []
    try:
        capi.tc_set_ir(s, h)
        for pos in range(0, N, B):
            y = np.empty(B, np.float32)
            capi.tc_push_block(s, x[pos:pos + B], y)
            outs.append(y)
        tail = np.empty(L - 1, np.float32)
        capi.tc_flush(s, tail, L - 1)
    finally:
        capi.tc_close(s)
    got = np.concatenate(outs + [tail])
    ref = oracle.buffer(x, h[None], None, B)
    assert got.shape == ref.shape
    assert rel_l2(got, ref) <= TOL["fp32"]


def test_server_stream_at_the_longest_ir():
    L, B, N = SERVER_MAX_L, 128, 512
    x = synth.audio(N, 65)
    h = synth.decayed_ir(L, 0.2 * L, 66)
    srv = capi.tc_server_open(16 << 30, 1 << 20)
    try:
        with pytest.raises(capi.TcError) as e:
            capi.tc_server_add(srv, L + 1, B, h[:1000])
        assert e.value.code == "TC_EINVAL"
        sid = capi.tc_server_add(srv, L, B, h)
        outs = []
        y = np.empty(B, np.float32)
        for pos in range(0, N, B):
            capi.tc_server_submit(srv, sid, x[pos:pos + B])
            capi.tc_server_step(srv)
            n, _, _ = capi.tc_server_poll(srv, sid, y)
            assert n == B
            outs.append(y.copy())
        capi.tc_server_remove(srv, sid)
    finally:
        capi.tc_server_close(srv)
    got = np.concatenate(outs)
    ref = oracle.buffer(x, h[None], None, B)[:N]
    assert rel_l2(got, ref) <= TOL["fp32"]
