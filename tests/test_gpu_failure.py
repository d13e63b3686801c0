"""Failure detection without a GPU fault: a device-side wait that nothing satisfies runs out, the kernel
reports into its error word and returns, the call returns TC_ETIMEOUT, and the context stays usable. Failures
injected on the host (tc_test_inject: a push's input copy, a server step's launch) return TC_ECUDA, leave a
stream usable, stop the server's worker with the error, and leave no block counted as in flight.
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


def test_bounded_wait_runs_out_and_the_context_survives():
    torch = pytest.importorskip("torch")
    t0 = time.perf_counter()
    with pytest.raises(capi.TcError) as e:
        capi.tc_selftest_wait(20_000_000)  # 20 ms
    dt = time.perf_counter() - t0
    assert e.value.code == "TC_ETIMEOUT"
    assert 0.015 <= dt < 2.0, dt
    # The context still works: a convolution right after matches the oracle.
    N, L = 3000, 700
    x = synth.audio(N, 5)
    h = synth.decayed_ir(L, 140.0, 6)
    y = torch.empty(N + L - 1, device="cuda")
    capi.tc_convolve(torch.from_numpy(x).cuda(), N, torch.from_numpy(h).cuda(), L, y)
    assert rel_l2(y.cpu().numpy(), oracle.buffer(x, h[None], None, 512)) <= TOL["fp32"]


def test_selftest_rejects_bad_limits():
    for bad in (0, 10_000_000_001):
        with pytest.raises(capi.TcError) as e:
            capi.tc_selftest_wait(bad)
        assert e.value.code == "TC_EINVAL"


def test_injected_copy_failure_leaves_the_stream_usable():
    L, B = 1000, 128
    x = synth.audio(10 * B, 501)
    h = synth.decayed_ir(L, 200.0, 502)
    s = capi.tc_open_stream(L, B)
    outs, failures = [], 0
    try:
        capi.tc_set_ir(s, h)
        capi.tc_test_inject(capi.TC_INJECT_PUSH_COPY, 3)
        pos = 0
        while pos < x.size:
            y = np.empty(B, np.float32)
            try:
                capi.tc_push_block(s, x[pos:pos + B], y)
            except capi.TcError as e:
                assert e.code == "TC_ECUDA" and "injected" in str(e)
                failures += 1
                continue  # the same block again
            outs.append(y)
            pos += B
        tail = np.empty(L - 1, np.float32)
        capi.tc_flush(s, tail, L - 1)
    finally:
        capi.tc_test_inject(capi.TC_INJECT_PUSH_COPY, 0)
        capi.tc_close(s)
    assert failures == 1
    got = np.concatenate(outs + [tail])
    assert rel_l2(got, oracle.buffer(x, h[None], None, B)) <= TOL["fp32"]


def test_injected_step_failure_drops_its_blocks_and_stops_the_worker():
    L, B = 2000, 128
    x = synth.audio(40 * B, 610)
    srv = capi.tc_server_open(4 << 30, 1 << 20)
    try:
        # Steps on the calling thread: the second one fails.
        ids = [capi.tc_server_add(srv, L, B, synth.decayed_ir(L, 400.0, 600 + i)) for i in range(6)]
        capi.tc_test_inject(capi.TC_INJECT_SERVER_STEP, 2)
        for sid in ids:
            capi.tc_server_submit(srv, sid, x[:B])
        assert capi.tc_server_step(srv) == len(ids)
        for sid in ids:
            capi.tc_server_submit(srv, sid, x[B:2 * B])
        with pytest.raises(capi.TcError) as e:
            capi.tc_server_step(srv)
        assert e.value.code == "TC_ECUDA" and "injected" in str(e.value)
        for sid in ids:  # nothing of the failed step is left in flight
            capi.tc_server_remove(srv, sid)

        # The server still serves: a new stream matches the oracle.
        h = synth.decayed_ir(L, 400.0, 620)
        sid = capi.tc_server_add(srv, L, B, h)
        y, outs = np.empty(B, np.float32), []
        for k in range(4):
            capi.tc_server_submit(srv, sid, x[k * B:(k + 1) * B])
            capi.tc_server_step(srv)
            n, _, _ = capi.tc_server_poll(srv, sid, y)
            assert n == B
            outs.append(y.copy())
        capi.tc_server_remove(srv, sid)
        ref = oracle.buffer(x[:4 * B], h[None], None, B)[:4 * B]
        assert rel_l2(np.concatenate(outs), ref) <= TOL["fp32"]

        # The worker thread: its third step fails, the worker stops, stop reports the failure.
        ids = [capi.tc_server_add(srv, L, B, synth.decayed_ir(L, 400.0, 630 + i)) for i in range(4)]
        capi.tc_test_inject(capi.TC_INJECT_SERVER_STEP, 3)
        capi.tc_server_start(srv)
        for k in range(20):
            for sid in ids:
                capi.tc_server_submit(srv, sid, x[k * B:(k + 1) * B])
            time.sleep(0.003)
        time.sleep(0.2)
        with pytest.raises(capi.TcError) as e:
            capi.tc_server_stop(srv)
        assert e.value.code == "TC_ECUDA" and "injected" in str(e.value)
        while capi.tc_server_step(srv) > 0:  # what was still queued runs on the calling thread
            pass
        for sid in ids:
            capi.tc_server_remove(srv, sid)
    finally:
        capi.tc_test_inject(capi.TC_INJECT_SERVER_STEP, 0)
        capi.tc_server_close(srv)
