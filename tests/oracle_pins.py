"""Checks that pin the FP64 oracle to facts other than itself.

Each check returns None when it holds and a message when it fails. The
pytest tests in test_oracle_pins.py run them against the real oracle; the
mutant test runs them against builds with one planted mistake and requires
that at least one check fails for each.

What each check rests on:
  worked_example   hand-added taches of a 6x3 example (Sec. 3.2, Fig. 4-5 shape)
  impulse          x = delta reproduces h exactly (the tache of a unit impulse)
  numpy_convolve   fixed IR reduces to the textbook convolution (numpy)
  ir_switch        one or more IR switches reduce to a sum of plain convolutions
                   of the masked input (abstract, Sec. 6)
  commutativity    x * h = h * x (Sec. 3.2, Fig. 6)
  linearity        y(a x1 + b x2) = a y(x1) + b y(x2)
  sum_invariant    sum y = sum_n x[n] * sum h_{v(n)}
  closed_form      sinusoid through an exponential IR: a geometric sum
  length           output length N + L - 1 (Sec. 4.1 temporal overflow)
  block_invariance Nb changes nothing but timing (Sec. 5.2, Table 2)
  forms_agree      direct, vectorised and buffer forms give the same values
  mimo             multichannel sum equals the sum of per-pair convolutions
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(a - b) / den)


def read_golden(name="worked_6x3.txt"):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = np.array([float(v) for v in rest])
    return vals


def _forms(o, x, H, vstart, Nb=3):
    return {
        "direct": o.direct(x, H, vstart),
        "vect": o.vect(x, H, vstart),
        "buffer": o.buffer(x, H, vstart, Nb),
    }


def check_worked_example(o):
    g = read_golden()
    x = g["x"].astype(np.float32)
    h = g["h"].astype(np.float32)
    h2 = g["h2"].astype(np.float32)
    s = int(g["switch_at"][0])
    for name, y in _forms(o, x, h, None).items():
        if y.shape != g["y"].shape or not np.array_equal(y, g["y"]):
            return f"{name}: {y} != {g['y']}"
    H = np.stack([h, h2])
    vs = np.array([0, s], np.int64)
    for Nb in (1, 2, 4, 6):
        for name, y in _forms(o, x, H, vs, Nb).items():
            if not np.array_equal(y, g["y_switch"]):
                return f"switch {name} Nb={Nb}: {y} != {g['y_switch']}"
    return None


def check_impulse(o):
    r = _rng(1)
    for N, L, n0 in [(50, 13, 0), (50, 13, 49), (20, 37, 5), (7, 7, 3)]:
        h = r.standard_normal(L).astype(np.float32)
        x = np.zeros(N, np.float32)
        x[n0] = 1.0
        ref = np.zeros(N + L - 1)
        ref[n0:n0 + L] = h
        for name, y in _forms(o, x, h, None, Nb=4).items():
            if not np.array_equal(y, ref):
                return f"{name} N={N} L={L} n0={n0}"
    return None


def check_numpy_convolve(o):
    r = _rng(2)
    for N, L, Nb in [(100, 17, 8), (33, 64, 5), (64, 64, 64), (257, 31, 100), (5, 1, 2), (1, 9, 1)]:
        x = r.uniform(-1, 1, N).astype(np.float32)
        h = r.standard_normal(L).astype(np.float32)
        ref = np.convolve(x.astype(np.float64), h.astype(np.float64))
        for name, y in _forms(o, x, h, None, Nb=Nb).items():
            if y.shape != ref.shape:
                return f"{name}: length {y.shape} != {ref.shape}"
            err = np.max(np.abs(y - ref)) / max(np.max(np.abs(ref)), 1e-300)
            if err > 1e-13:
                return f"{name} N={N} L={L}: rel {err:.3g}"
    return None


def check_ir_switch(o):
    r = _rng(3)
    for N, L, starts, Nb in [(200, 30, [0, 57], 16), (200, 30, [0, 64], 16), (300, 50, [0, 40, 41, 170], 7),
                              (90, 120, [-5, 10, 60], 9)]:
        x = r.uniform(-1, 1, N).astype(np.float32)
        nv = len(starts)
        H = r.standard_normal((nv, L)).astype(np.float32)
        vs = np.array(starts, np.int64)
        n = np.arange(N)
        v_of_n = np.searchsorted(vs, n, side="right") - 1
        ref = np.zeros(N + L - 1)
        for v in range(nv):
            xm = np.where(v_of_n == v, x.astype(np.float64), 0.0)
            ref += np.convolve(xm, H[v].astype(np.float64))
        for name, y in _forms(o, x, H, vs, Nb=Nb).items():
            err = np.max(np.abs(y - ref)) / max(np.max(np.abs(ref)), 1e-300)
            if err > 1e-13:
                return f"{name} starts={starts}: rel {err:.3g}"
    return None


def check_commutativity(o):
    r = _rng(4)
    x = r.uniform(-1, 1, 45).astype(np.float32)
    h = r.standard_normal(19).astype(np.float32)
    for Nb in (4, 45):
        a = o.buffer(x, h, None, Nb)
        b = o.buffer(h, x, None, Nb)
        if a.shape != b.shape or _rel(a, b) > 1e-14:
            return f"buffer Nb={Nb}: x*h != h*x"
    if _rel(o.direct(x, h), o.direct(h, x)) > 1e-14:
        return "direct: x*h != h*x"
    return None


def check_linearity(o):
    r = _rng(5)
    x1 = r.integers(-100, 101, 80).astype(np.float32)
    x2 = r.integers(-100, 101, 80).astype(np.float32)
    x3 = (2.0 * x1 - 3.0 * x2).astype(np.float32)  # exact in float32
    H = r.standard_normal((2, 21)).astype(np.float32)
    vs = np.array([0, 33], np.int64)
    for name in ("direct", "vect", "buffer"):
        f = getattr(o, name)
        args = (vs, 6) if name == "buffer" else (vs,)
        y1, y2, y3 = f(x1, H, *args), f(x2, H, *args), f(x3, H, *args)
        if _rel(y3, 2.0 * y1 - 3.0 * y2) > 1e-14:
            return f"{name}: not linear"
    return None


def check_sum_invariant(o):
    r = _rng(6)
    x = r.uniform(-1, 1, 150).astype(np.float32)
    H = r.standard_normal((3, 40)).astype(np.float32)
    vs = np.array([0, 50, 97], np.int64)
    v_of_n = np.searchsorted(vs, np.arange(150), side="right") - 1
    ref = float(np.sum(x.astype(np.float64) * H.astype(np.float64).sum(axis=1)[v_of_n]))
    scale = float(np.sum(np.abs(x)) * np.max(np.sum(np.abs(H.astype(np.float64)), axis=1)))
    for name, y in _forms(o, x, H, vs, Nb=11).items():
        if abs(float(np.sum(y)) - ref) > 1e-12 * scale:
            return f"{name}: sum {np.sum(y)} != {ref}"
    return None


def check_closed_form(o):
    # x[n] = sin(w n), n < N; h[k] = a^k, k < L. Then
    # y[m] = Im( e^{i w m} sum_{k=k0}^{k1} (a e^{-i w})^k ),  k0 = max(0, m-N+1), k1 = min(m, L-1),
    # a geometric sum. Inputs are float32-rounded, so the tolerance is the
    # rounding of x and h: |dy| <= (2^-24 + 2^-24 + 2^-48) sum |x||h| per sample.
    N, L, w, a = 300, 120, 0.37, 0.985
    n = np.arange(N)
    x = np.sin(w * n).astype(np.float32)
    h = (a ** np.arange(L)).astype(np.float32)
    m = np.arange(N + L - 1)
    k0 = np.maximum(0, m - N + 1)
    k1 = np.minimum(m, L - 1)
    q = a * np.exp(-1j * w)
    geo = (q ** k0 - q ** (k1 + 1)) / (1 - q)
    ref = np.imag(np.exp(1j * w * m) * geo)
    bound = (2.0 ** -23 + 2.0 ** -48) * np.convolve(np.abs(np.sin(w * n)), a ** np.arange(L)) + 1e-12
    for name, y in _forms(o, x, h, None, Nb=32).items():
        bad = np.abs(y - ref) > bound
        if np.any(bad):
            i = int(np.argmax(bad))
            return f"{name}: m={i} y={y[i]} closed={ref[i]}"
    return None


def check_length(o):
    r = _rng(7)
    for N, L in [(1, 1), (1, 5), (5, 1), (10, 3), (3, 10)]:
        x = r.uniform(-1, 1, N).astype(np.float32)
        h = r.standard_normal(L).astype(np.float32)
        for name, y in _forms(o, x, h, None, Nb=2).items():
            if y.shape != (N + L - 1,):
                return f"{name} N={N} L={L}: len {y.shape}"
        s = o.stream(L)
        got = np.concatenate([s.push(x, h), s.flush()])
        s.close()
        if got.shape != (N + L - 1,):
            return f"stream N={N} L={L}: len {got.shape}"
    return None


def check_block_invariance(o):
    r = _rng(8)
    N, L = 123, 29
    x = r.uniform(-1, 1, N).astype(np.float32)
    H = r.standard_normal((2, L)).astype(np.float32)
    vs = np.array([0, 61], np.int64)
    ref = o.buffer(x, H, vs, 1)
    for Nb in (2, 3, 7, 28, 29, 30, 64, 123, 500):
        y = o.buffer(x, H, vs, Nb)
        if not np.array_equal(y, ref):
            return f"Nb={Nb} differs"
    # Streamed in uneven pieces, then flushed.
    s = o.stream(L)
    parts, pos = [], 0
    for step in (5, 1, 17, 40, 60):
        parts.append(s.push(x[pos:pos + step], H, vs))
        pos += step
    parts.append(s.flush())
    s.close()
    if not np.array_equal(np.concatenate(parts), ref):
        return "streamed pieces differ"
    return None


def check_forms_agree(o):
    r = _rng(9)
    x = r.uniform(-1, 1, 77).astype(np.float32)
    H = r.standard_normal((2, 33)).astype(np.float32)
    vs = np.array([0, 40], np.int64)
    f = _forms(o, x, H, vs, Nb=10)
    if not (np.array_equal(f["direct"], f["vect"]) and np.array_equal(f["vect"], f["buffer"])):
        return "direct / vect / buffer differ"
    for m in (0, 10, 76, 77 + 31):
        if o.direct_at(x, H, vs, m) != f["direct"][m]:
            return f"direct_at({m}) differs"
    return None


def check_mimo(o):
    r = _rng(10)
    nin, nout, N, L = 3, 2, 40, 11
    X = r.uniform(-1, 1, (nin, N)).astype(np.float32)
    H = r.standard_normal((2, nout, nin, L)).astype(np.float32)
    vs = np.array([0, 17], np.int64)
    y = o.mimo(X, H, vs, Nb=6)
    v_of_n = np.searchsorted(vs, np.arange(N), side="right") - 1
    for oo in range(nout):
        ref = np.zeros(N + L - 1)
        for i in range(nin):
            for v in range(2):
                xm = np.where(v_of_n == v, X[i].astype(np.float64), 0.0)
                ref += np.convolve(xm, H[v, oo, i].astype(np.float64))
        if np.max(np.abs(y[oo] - ref)) > 1e-13 * max(1.0, np.max(np.abs(ref))):
            return f"output {oo} differs"
    return None


def _xf_weights(vstart, vramp, n):
    """Per-sample weights of the crossfaded versions: alpha_v(n) =
    clamp((n - vstart[v] + 1) / vramp[v], 0, 1), alpha_0 = 1, and
    w_v = alpha_v - alpha_{v+1} (the definition; checked for sanity here)."""
    nv = len(vstart)
    alpha = np.ones((nv + 1, n.size))
    for v in range(1, nv):
        alpha[v] = np.clip((n - vstart[v] + 1) / vramp[v], 0.0, 1.0)
    alpha[nv] = 0.0
    return alpha[:-1] - alpha[1:]


def check_crossfade_hard(o):
    """Ramps of one sample are the hard switches: same outputs, bit for bit."""
    r = _rng(21)
    for N, L, starts, Nb in [(200, 30, [0, 57], 16), (300, 50, [0, 40, 41, 170], 7), (90, 120, [-5, 10, 60], 9)]:
        x = r.uniform(-1, 1, N).astype(np.float32)
        H = r.standard_normal((len(starts), L)).astype(np.float32)
        vs = np.array(starts, np.int64)
        y = o.buffer_xf(x, H, vs, np.ones(len(starts), np.int64), Nb)
        ref = o.buffer(x, H, vs, Nb)
        if not np.array_equal(y, ref):
            return f"starts={starts}: max diff {np.max(np.abs(y - ref)):.3g}"
    return None


def check_crossfade_superposition(o):
    """A crossfade is the sum of plain convolutions of weighted inputs:
    y = sum_v conv(x * w_v, H[v]) (for two versions: conv(x (1 - alpha), h_a)
    + conv(x alpha, h_b)); the weights lie in [0, 1] and add up to 1."""
    r = _rng(22)
    for N, L, starts, ramps, Nb in [(400, 60, [0, 100], [1, 50], 16), (500, 40, [0, 30, 300], [1, 200, 7], 13),
                                    (300, 90, [-10, 5, 120], [1, 1, 100], 64), (256, 33, [0, 0 + 1], [1, 256], 32)]:
        x = r.uniform(-1, 1, N).astype(np.float32)
        H = r.standard_normal((len(starts), L)).astype(np.float32)
        vs, vr = np.array(starts, np.int64), np.array(ramps, np.int64)
        n = np.arange(N)
        w = _xf_weights(vs, vr, n)
        if np.any(w < -1e-15) or np.any(w > 1 + 1e-15) or np.max(np.abs(w.sum(axis=0) - 1.0)) > 1e-15:
            return f"weights out of range for starts={starts} ramps={ramps}"
        ref = np.zeros(N + L - 1)
        for v in range(len(starts)):
            ref += np.convolve(x.astype(np.float64) * w[v], H[v].astype(np.float64))
        y = o.buffer_xf(x, H, vs, vr, Nb)
        err = np.max(np.abs(y - ref)) / max(np.max(np.abs(ref)), 1e-300)
        if err > 1e-13:
            return f"starts={starts} ramps={ramps}: rel {err:.3g}"
        # The direct form, at a few outputs.
        for m in (0, starts[-1] + 3 if starts[-1] >= 0 else 5, N // 2, N + L - 2):
            d = o.direct_at_xf(x, H, vs, vr, m)
            if abs(d - y[m]) > 1e-12 * max(1.0, abs(y[m])):
                return f"direct_at_xf m={m}: {d} vs {y[m]}"
        # Sum invariant: sum y = sum_n x[n] * sum_v w_v(n) sum_k H[v][k].
        hs = H.astype(np.float64).sum(axis=1)
        tot = float(np.sum(x.astype(np.float64) * (w * hs[:, None]).sum(axis=0)))
        if abs(y.sum() - tot) > 1e-9 * max(1.0, np.abs(y).sum()):
            return f"sum invariant: {y.sum()} vs {tot}"
    return None


def check_q15_exact(o):
    """Exact fixed point (Sec. 5.4): on Q15 data the FP64 buffer oracle is
    itself exact (every product has <= 32 significant bits and every partial
    sum is a multiple of 2^-30 below 2^19), so the integer sums must equal
    2^30 times it, exactly; the single requantization is round half to even
    (numpy.rint) of sum / 2^15, saturated to int16. Includes exact halves and
    saturating sums."""
    r = _rng(30)
    for N, L in [(300, 40), (50, 200), (1, 1), (777, 513)]:
        xq = r.integers(-32768, 32768, N).astype(np.int16)
        hq = r.integers(-32768, 32768, L).astype(np.int16)
        acc, y = o.q15(xq, hq)
        f = o.buffer(xq.astype(np.float32) / 32768.0, (hq.astype(np.float32) / 32768.0)[None], None, 37)
        if not np.array_equal(acc.astype(np.float64), f * 2.0 ** 30):
            return f"N={N} L={L}: integer sums differ from the exact FP64 form"
        ref = np.clip(np.rint(acc / 32768.0), -32768, 32767).astype(np.int16)
        if not np.array_equal(y, ref):
            return f"N={N} L={L}: requantization differs"
    # Exact halves: x = 1 (Q15 raw 1), taps of odd multiples of 2^14 -> sums k * 2^14.
    xq = np.array([1, 0, 0], np.int16)
    hq = np.array([16384, -16384, 16384 * 3 // 3, -32768], np.int16)
    acc, y = o.q15(xq, hq)
    ref = np.clip(np.rint(acc / 32768.0), -32768, 32767).astype(np.int16)
    if not np.array_equal(y, ref):
        return f"halves: {y} vs {ref}"
    # Saturation: full-scale input against a full-scale IR.
    acc, y = o.q15(np.full(8, -32768, np.int16), np.full(8, -32768, np.int16))
    if y.max() != 32767:
        return "no positive saturation"
    return None


ALL = {
    "worked_example": check_worked_example,
    "impulse": check_impulse,
    "numpy_convolve": check_numpy_convolve,
    "ir_switch": check_ir_switch,
    "commutativity": check_commutativity,
    "linearity": check_linearity,
    "sum_invariant": check_sum_invariant,
    "closed_form": check_closed_form,
    "length": check_length,
    "block_invariance": check_block_invariance,
    "forms_agree": check_forms_agree,
    "mimo": check_mimo,
    "crossfade_hard": check_crossfade_hard,
    "crossfade_superposition": check_crossfade_superposition,
    "q15_exact": check_q15_exact,
}


def run_all(o):
    out = {}
    for name, fn in ALL.items():
        try:
            out[name] = fn(o)
        except Exception as e:  # a crash of the oracle under test counts as a failure
            out[name] = f"raised {type(e).__name__}: {e}"
    return out
