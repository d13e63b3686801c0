"""tc_convolve_noalloc, the allocation-free one-shot convolution, against the FP64 oracle and tc_convolve.

Some callers cannot allocate device memory where they call. A real-time
audio callback is one: cudaMalloc can block for an unbounded time there. A
host program whose own allocator owns the GPU's memory is another.
tc_convolve_noalloc keeps its working memory in a fixed device array inside
the library instead of allocating. This test calls it twice in a row through
the C ABI and checks each result element by element against the FP64 oracle
(the buffer taches-algorithm of Sec. 4.2) within the FP32 tolerance used by
every FP32 parity test (relative L2 <= 1e-6), and against the allocating
entry point, tc_convolve. The second call is smaller, and it also checks
that the first call's leftovers in the shared array do not leak into it.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_helpers import TOL, max_abs, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_01607_gb300 as pkg
    pkg.build()
    capi.load()
    return torch


def test_noalloc_matches_the_oracle_twice(oracle, monkeypatch):
    torch = _cuda()
    monkeypatch.delenv("TC_NO_ROLE_SWAP", raising=False)
    for N, L, seed in [(60_000, 9_000, 1), (5_000, 20_000, 2)]:
        xh = synth.audio(N, seed)
        hh = synth.decayed_ir(L, 0.3 * L, seed + 100)
        x = torch.from_numpy(xh).cuda()
        h = torch.from_numpy(hh).cuda()
        y_ref = torch.empty(N + L - 1, device="cuda")
        y_na = torch.full((N + L - 1,), float("nan"), device="cuda")
        capi.tc_convolve(x, N, h, L, y_ref)
        capi.tc_convolve_noalloc(x, N, h, L, y_na)
        a = y_na.cpu().numpy()
        assert np.all(np.isfinite(a))
        ref = oracle.buffer(xh, hh[None], np.zeros(1, np.int64), 4096)
        assert ref.shape == a.shape
        err = rel_l2(a, ref)
        assert err <= TOL["fp32"], (N, L, err, max_abs(a, ref))
        assert rel_l2(a, y_ref.cpu().numpy()) <= TOL["fp32"], (N, L)


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = _cuda()
    x = torch.zeros(16, device="cuda")  # never read: the size checks come first
    for N, L in [(12_000_000, 1000), (2**64 - 1, 1000), (1000, 2**64 - 1), (2**63, 2**63)]:
        with pytest.raises(capi.TcError) as e:
            capi.tc_convolve_noalloc(x, N, x, L, x)
        assert e.value.code == "TC_EINVAL", (N, L)
        assert "MiB" in str(e.value)


def test_noalloc_role_swap_fits_a_long_ir(oracle, monkeypatch):
    """N = 3000 through L = 2 million taps needs about 26 million floats of working set in the caller's
    roles, beyond the 32 MiB array; with the roles swapped (Sec. 3.2) it needs about 2.05 million. The
    result matches the oracle's direct sum (Eq. 4) on contiguous windows of 1024 outputs (start, the
    N-1/N seam, the middle, the last output) and tc_convolve run in the caller's roles (TC_NO_ROLE_SWAP=1)."""
    torch = _cuda()
    N, L = 3_000, 2_000_000
    xh = synth.audio(N, 5)
    hh = synth.decayed_ir(L, 0.2 * L, 6)
    x = torch.from_numpy(xh).cuda()
    h = torch.from_numpy(hh).cuda()
    y_na = torch.full((N + L - 1,), float("nan"), device="cuda")
    y_ref = torch.empty(N + L - 1, device="cuda")
    monkeypatch.delenv("TC_NO_ROLE_SWAP", raising=False)
    capi.tc_convolve_noalloc(x, N, h, L, y_na)
    monkeypatch.setenv("TC_NO_ROLE_SWAP", "1")
    capi.tc_convolve(x, N, h, L, y_ref)
    monkeypatch.delenv("TC_NO_ROLE_SWAP", raising=False)
    a = y_na.cpu().numpy()
    assert np.all(np.isfinite(a))
    assert rel_l2(a, y_ref.cpu().numpy()) <= TOL["fp32"]
    ny = N + L - 1
    H = hh[None]
    vs = np.zeros(1, np.int64)
    for m0 in (0, N - 512, ny // 2, ny - 1024):
        ms = np.arange(m0, m0 + 1024)
        ref = np.array([oracle.direct_at(xh, H, vs, int(m)) for m in ms])
        assert rel_l2(a[ms], ref) <= TOL["fp32"], m0
