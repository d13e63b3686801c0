"""Failure detection without a GPU fault: a device-side wait that nothing satisfies runs out, the kernel
reports into its error word and returns, the call returns TC_ETIMEOUT, and the context stays usable.
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
