"""tc_convolve_noalloc, the allocation-free one-shot convolution, against tc_convolve.

Some callers cannot allocate device memory where they call. A real-time
audio callback is one: cudaMalloc can block for an unbounded time there. A
host program whose own allocator owns the GPU's memory is another.
tc_convolve_noalloc keeps its working memory in a fixed device array inside
the library instead of allocating. This test calls it twice in a row through
the C ABI and checks each result against the allocating entry point,
tc_convolve, within the FP32 tolerance used by every FP32 parity test
(relative L2 <= 1e-6). The second call is smaller, and it also checks that
the first call's leftovers in the shared array do not leak into it.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_helpers import TOL, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_01607_gb300 as pkg
    pkg.build()
    capi.load()
    for N, L, seed in [(60_000, 9_000, 1), (5_000, 20_000, 2)]:
        x = torch.from_numpy(synth.audio(N, seed)).cuda()
        h = torch.from_numpy(synth.decayed_ir(L, 0.3 * L, seed + 100)).cuda()
        y_ref = torch.empty(N + L - 1, device="cuda")
        y_na = torch.full((N + L - 1,), float("nan"), device="cuda")
        capi.tc_convolve(x, N, h, L, y_ref)
        capi.tc_convolve_noalloc(x, N, h, L, y_na)
        a = y_na.cpu().numpy()
        b = y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        err = rel_l2(a, b)
        assert err <= TOL["fp32"], (N, L, err)


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N, L = 12_000_000, 1000
    x = torch.zeros(16, device="cuda")  # never read: the size check comes first
    with pytest.raises(capi.TcError) as e:
        capi.tc_convolve_noalloc(x, N, x, L, x)
    assert e.value.code == "TC_EINVAL"
    assert "MiB" in str(e.value)


def test_noalloc_role_swap_fits_a_long_ir():
    """N = 3000 through L = 2 million taps needs about 26 million floats of working set in the caller's
    roles, beyond the 32 MiB array; with the roles swapped (Sec. 3.2) it needs about 2.05 million. The
    result matches tc_convolve run in the caller's roles (TC_NO_ROLE_SWAP=1)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    N, L = 3_000, 2_000_000
    x = torch.from_numpy(synth.audio(N, 5)).cuda()
    h = torch.from_numpy(synth.decayed_ir(L, 0.2 * L, 6)).cuda()
    y_na = torch.full((N + L - 1,), float("nan"), device="cuda")
    y_ref = torch.empty(N + L - 1, device="cuda")
    capi.tc_convolve_noalloc(x, N, h, L, y_na)
    os.environ["TC_NO_ROLE_SWAP"] = "1"
    try:
        capi.tc_convolve(x, N, h, L, y_ref)
    finally:
        del os.environ["TC_NO_ROLE_SWAP"]
    a = y_na.cpu().numpy()
    assert np.all(np.isfinite(a))
    assert rel_l2(a, y_ref.cpu().numpy()) <= TOL["fp32"]
