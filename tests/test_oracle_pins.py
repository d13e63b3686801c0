"""The FP64 oracle against the facts that pin it (CPU only)."""
import numpy as np
import pytest

import oracle_pins as P


@pytest.mark.parametrize("name", list(P.ALL))
def test_pin(oracle, name):
    msg = P.ALL[name](oracle)
    assert msg is None, msg


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_planted_mistake_is_caught(mutant):
    """Each mutant build plants one plausible mistake; some pin must fail."""
    import oracle as O
    o = O.Oracle(mutant)
    assert o.lib.tco_mutant_id() == mutant
    res = P.run_all(o)
    failed = [k for k, v in res.items() if v is not None]
    assert failed, f"mutant {mutant} passed every pin"


def test_scipy_fftconvolve_full_mono(oracle):
    """Mono workload size (48000 x 4096): buffer oracle vs an FP64 FFT convolution."""
    scipy_signal = pytest.importorskip("scipy.signal")
    from paper_2401_01607_gb300 import synth
    w = synth.mono()
    y = oracle.buffer(w.x[0], w.H[0], None, 64)
    ref = scipy_signal.fftconvolve(w.x[0].astype(np.float64), w.H[0, 0].astype(np.float64))
    assert y.shape == (48000 + 4096 - 1,)
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel < 1e-13, rel


def test_direct_at_spot_checks_multi_shape(oracle):
    """Spot checks at a large IR (workload 2 shape, shortened input): direct_at vs numpy on masked pieces."""
    from paper_2401_01607_gb300 import synth
    w = synth.multi(C=1, N=60_000, L=48_000, swap_every=24_000)
    x, H, vs = w.x[0], w.H[0], w.vstart
    v_of_n = np.searchsorted(vs, np.arange(w.N), side="right") - 1
    rng = np.random.default_rng(11)
    for m in rng.integers(0, w.N + w.L - 1, 6):
        ref = 0.0
        for v in range(H.shape[0]):
            lo, hi = max(0, m - w.L + 1), min(m, w.N - 1)
            n = np.arange(lo, hi + 1)
            sel = v_of_n[n] == v
            ref += float(np.dot(x[n[sel]].astype(np.float64), H[v, m - n[sel]].astype(np.float64)))
        got = oracle.direct_at(x, H, vs, int(m))
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (m, got, ref)
