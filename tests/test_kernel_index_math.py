"""CPU checks of the kernels' index arithmetic, restated from the CUDA sources (no GPU).

The GPU parity tests check the kernels' results; these check, on every index a small launch can produce, the
reasoning that the kernels' bounds and decompositions rest on. Each test restates the formulas of one kernel
(the file named in its docstring) and must change with it:

  * K1 (`csrc/k1_gather.cu`): the closed-form range of passes a thread runs for one IR version equals the
    per-pass test; every shared-memory read of a pass stays inside the staged window and IR chunk, and inside
    the TMA part (A or B) that the pass waits for; staged windows and IR chunks start on 16-byte boundaries
    and stay inside the history row and the IR slot kept by the host (`csrc/capi.cu`); and the whole
    decomposition (tiles, tap chunks, version masking, passes, the sliding 20-register window) adds up to
    Eq. 4 with per-sample IR versions.
  * K2 (`csrc/k2_toeplitz_tc.cu`, `csrc/oneshot.cu`): the Toeplitz product on an 8-sample grid (shift delta),
    and the row view of one signal (rows of 256 outputs as channels), equal the convolution.
  * K2 persistent CTA pairs: K blocks of 32 and 64 samples tile every tap once and k2_tprep's threads write
    every tile element once; the units of every order, with pairs of channel tiles or (one channel tile) of
    output tiles, cover every (tile, output tile, K part) once inside the allocated partials and tickets; the
    in-kernel fold adds K parts bit for bit as k2_reduce does; a row view's flat output limit writes every
    output once.
  * K3 (`csrc/k3_mimo_tc.cu`): the phase reshaping of a MIMO output tile (row r, phase p, output o; A a strided
    view of the reversed input, B the phase-shifted IRs) equals the sum of convolutions.
"""
import numpy as np

# K1 constants (tc_internal.h, k1_gather.cu)
MO = 128          # outputs per tile
SEG = 20          # taps per thread per pass
VARIANTS = (1, 4, 11)
KC_MAX = 32 * SEG * 11
INF = 1 << 62


def fdiv(x, d):
    return x // d  # floor division, as the kernel's floor_div


def k1_shift_e(t0, base):
    d = (t0 + 1 - base) % 4
    return (4 - d) & 3


def k1_parts(P):
    """Passes fed by TMA part A, its IR taps and the first staged sample it covers."""
    KC = 32 * SEG * P
    PA = (P + 2) // 3 if P >= 4 else P
    HA = 32 * SEG * PA
    return PA, HA, KC - HA


def k1_pass_range(P, s, out_hi, kc0, a, b, L):
    """Closed form of the passes thread (s, out_hi) runs for a version owning samples [a, b)."""
    seg_hi = min(fdiv(out_hi - kc0 - a, SEG), fdiv(L - 1 - kc0, SEG))
    seg_lo = -(1 << 40) if b >= INF else fdiv(out_hi - kc0 - (15 + SEG - 1) - b, SEG) + 1
    p_lo = max(0, min(P, -fdiv(s - seg_lo, 32)))
    p_hi = max(-1, min(P - 1, fdiv(seg_hi - s, 32)))
    return p_lo, p_hi


def k1_pass_needed(P, p, s, out_hi, kc0, a, b, L):
    """Per-pass test: the 35 samples the pass reads meet [a, b) and its first tap is inside the IR."""
    seg = 32 * p + s
    newest = out_hi - (kc0 + SEG * seg)      # sample read by the pass's first tap for the last output
    oldest = newest - 15 - (SEG - 1)         # sample read by its last tap for the first output
    return newest >= a and oldest < b and kc0 + SEG * seg <= L - 1


def test_k1_pass_range_closed_form_equals_the_per_pass_test():
    rng = np.random.default_rng(11)
    for _ in range(40000):
        P = int(rng.choice(VARIANTS))
        KC = 32 * SEG * P
        s, g = int(rng.integers(32)), int(rng.integers(8))
        L = int(rng.choice([1, 2, 19, 20, 21, 640, 641, 2560, 7040, 7041, 48000, int(rng.integers(1, 200000))]))
        e = int(rng.integers(4))
        nchunk = (L + e + KC - 1) // KC
        kc0 = int(rng.integers(nchunk)) * KC - e
        t0 = int(rng.integers(-1000, 10**7))
        out_hi = t0 + 16 * g + 15
        n_lo = t0 - kc0 - KC + 1
        n_end = n_lo + KC + MO
        mode = int(rng.integers(4))
        a = -10**9 if mode in (0, 2) else int(rng.integers(n_lo - 50, n_end + 50))
        if mode in (0, 1):
            b = INF
        else:
            b = int(rng.integers(max(a + 1, n_lo - 50), n_end + 100))
        lo, hi = k1_pass_range(P, s, out_hi, kc0, a, b, L)
        want = [p for p in range(P) if k1_pass_needed(P, p, s, out_hi, kc0, a, b, L)]
        assert list(range(lo, hi + 1)) == want, (P, s, out_hi, kc0, a, b, L)


def test_k1_shared_reads_stay_inside_the_stage_and_their_part():
    for P in VARIANTS:
        KC = 32 * SEG * P
        XS = KC + MO
        PA, HA, XA = k1_parts(P)
        assert XA % 4 == 0 and HA % 4 == 0
        for p in range(P):
            for s in range(32):
                seg = 32 * p + s
                h_lo, h_hi = SEG * seg, SEG * seg + SEG           # hp[0, 20)
                assert h_lo % 4 == 0 and 0 <= h_lo and h_hi <= KC
                for g in range(8):
                    ia = 16 * g - SEG * seg + KC - 4
                    x_lo, x_hi = ia - 16, ia + 20                 # xp[-16, 20): window and 4 refills
                    assert ia % 4 == 0 and x_lo >= 0 and x_hi <= XS, (P, p, s, g)
                    if p < PA:
                        assert x_lo >= XA and h_hi <= HA          # part A only
                    else:
                        assert x_hi <= XA + MO                    # zero gating tests xs[0, XA + 128)
        # The tight corners: the newest read of the stage and its first element are both used.
        assert 16 * 7 + KC - 4 + 20 == XS and 16 * 0 - SEG * (32 * P - 1) + KC - 4 - 16 == 0


def test_k1_shared_memory_fits_four_ctas_per_sm():
    for P in VARIANTS:
        KC = 32 * SEG * P
        stage = (KC + MO) + KC
        tail = 8 * MO + 12 * MO       # reduction area + pairwise stack, overlaying the stage
        dyn = 4 * max(stage, tail)
        static = 2 * 8 + 4 + 4 + 8 + 256  # mbarriers, flags, the list item copy (upper bound)
        assert 4 * (dyn + static + 1024) <= 228 * 1024, P   # 1 KB per CTA reserved by the system


def test_k1_windows_are_aligned_and_inside_the_history_and_ir_slot():
    """Host layout (`csrc/capi.cu`): keep = L + KC_MAX + 16 samples behind the next push, compaction to
    floor8(pos - keep) when a push and one tile of overrun would pass the row's end; IR copy e shifted by e
    taps in a slot of Lpad = L + 4 + KC_MAX (rounded to 4) floats."""
    rng = np.random.default_rng(12)
    for _ in range(300):
        L = int(rng.choice([1, 5, 700, 7040, 7041, 48000, int(rng.integers(1, 300000))]))
        max_push = int(rng.choice([64, 128, 1000, 8192]))
        keep = -(-(L + KC_MAX + 16) // 8) * 8
        cap = -(-(2 * keep + max_push + 512 + 160) // 64) * 64
        Lpad = -(-(L + 4 + KC_MAX) // 4) * 4
        base, pos = -keep, 0
        for _ in range(int(rng.integers(1, 30))):
            n = int(rng.integers(1, max_push + 1))
            if not (pos + n + MO + 8 <= base + cap):
                nb = (pos - keep) // 8 * 8
                assert nb - base >= pos - nb and (pos - nb) + n + MO + 8 <= cap
                base = nb
            assert base % 8 == 0 and pos - base >= keep
            t0, e = pos, k1_shift_e(pos, base)
            for P in VARIANTS:
                KC = 32 * SEG * P
                nchunk = (L + e + KC - 1) // KC
                assert nchunk * KC <= Lpad                       # IR chunk reads inside the slot copy
                for tile in range(-(-n // MO)):
                    for chunk in range(nchunk):
                        kc0 = chunk * KC - e
                        n_lo = t0 + MO * tile - kc0 - KC + 1
                        assert (n_lo - base) % 4 == 0            # 16-byte aligned TMA source
                        assert n_lo >= base and n_lo + KC + MO <= base + cap, (L, n, P, tile, chunk)
            pos += n


def k1_emulate_launch(x, H, vstart, L, t0, nout, P, e):
    """K1's decomposition of one launch, in float64: y[t0 + i] for i < nout. Returns the sum over the passes
    of the closed-form ranges and the sum over every pass (the skipped passes must add exact zeros)."""
    KC = 32 * SEG * P
    XS = KC + MO
    nchunk = (L + e + KC - 1) // KC
    ntile = -(-nout // MO)
    N = x.size
    g = np.arange(8)[:, None]
    seg = (32 * np.arange(P)[None, :] + np.arange(32)[:, None]).reshape(-1)   # (s, p) pairs
    s_of, p_of = seg % 32, seg // 32
    r = np.arange(16)
    j = np.arange(SEG)
    ia = 16 * g - SEG * seg[None, :] + KC - 4                                 # [g][seg]
    # tap j of output r reads the window's xp[3 + r - j], xp = xs + ia
    xidx = ia[:, :, None, None] + 3 + r[None, None, :, None] - j[None, None, None, :]
    hidx = SEG * seg[:, None] + j[None, :]
    y = np.zeros(ntile * MO)
    y_all = np.zeros(ntile * MO)
    for tile in range(ntile):
        tt0 = t0 + MO * tile
        for chunk in range(nchunk):
            kc0 = chunk * KC - e
            n_lo = tt0 - kc0 - KC + 1
            for v in range(len(vstart)):
                a = vstart[v]
                b = vstart[v + 1] if v + 1 < len(vstart) else INF
                if b <= n_lo or a >= n_lo + XS:
                    continue
                n = n_lo + np.arange(XS)
                ok = (n >= 0) & (n < N) & (n >= a) & (n < b)
                xs = np.where(ok, x[np.clip(n, 0, max(N - 1, 0))], 0.0)
                taps = kc0 + np.arange(KC)                  # copy e of the IR slot: tap kc0 + i at index i
                hs = np.where((taps >= 0) & (taps < L), H[v][np.clip(taps, 0, L - 1)], 0.0)
                contrib = np.einsum("gsrj,sj->gsr", xs[xidx], hs[hidx])   # [g][seg][r]
                run = np.zeros((8, seg.size), bool)
                for gg in range(8):
                    out_hi = tt0 + 16 * gg + 15
                    for ss in range(32):
                        lo, hi = k1_pass_range(P, ss, out_hi, kc0, a, b, L)
                        run[gg] |= (s_of == ss) & (p_of >= lo) & (p_of <= hi)
                rows = tile * MO + 16 * np.arange(8)[:, None] + r[None, :]
                y[rows] += np.einsum("gsr,gs->gr", contrib, run)
                y_all[rows] += contrib.sum(axis=1)
    return y[:nout], y_all[:nout]


def eq4_reference(x, H, vstart, L):
    """Eq. 4 with per-sample versions: the superposition of each version's taches (np.convolve)."""
    y = np.zeros(x.size + L - 1)
    for v in range(len(vstart)):
        a = vstart[v]
        b = vstart[v + 1] if v + 1 < len(vstart) else x.size
        xv = np.zeros_like(x)
        xv[a:b] = x[a:b]
        y += np.convolve(xv, H[v])
    return y


def test_k1_decomposition_adds_up_to_eq4():
    rng = np.random.default_rng(13)
    cases = [  # N, L, P, versions, pushes
        (200, 1, 1, [0], [64, 64, 72]),
        (900, 700, 1, [0, 333, 334], [128, 300, 472]),
        (1500, 3000, 4, [0, 1000], [256, 1000, 244]),
        (300, 7100, 11, [0, 150], [300]),
    ]
    for N, L, P, vstart, pushes in cases:
        x = rng.uniform(-1, 1, N)
        H = rng.standard_normal((len(vstart), L))
        ref = eq4_reference(x, H, vstart, L)
        pushes = pushes + [L - 1]                              # the flush: L - 1 more outputs
        keep = -(-(L + KC_MAX + 16) // 8) * 8
        base, t0 = -keep, 0          # a multiple of 8, like every base after a compaction
        got, got_all = [], []
        for n in pushes:
            e = k1_shift_e(t0, base)
            yy, yy_all = k1_emulate_launch(x, H, vstart, L, t0, n, P, e)
            got.append(yy)
            got_all.append(yy_all)
            t0 += n
        got, got_all = np.concatenate(got), np.concatenate(got_all)
        assert got.size == N + L - 1
        scale = np.abs(ref).max()
        # the passes outside the closed-form range add exact zeros
        assert np.array_equal(got, got_all), (N, L, P)
        assert np.abs(got - ref).max() <= 1e-12 * scale, (N, L, P)


def test_k2_toeplitz_product_on_the_8_sample_grid():
    """Y[c][t0 + i] = sum_j X[c][w0 + j] T[i][j], T[i][j] = h[L - 1 + delta + i - j], w0 = t0 - L + 1 - delta,
    with w0 on the 8-sample grid (k2_toeplitz, k2_tprep)."""
    rng = np.random.default_rng(14)
    C, N, L, nout = 3, 900, 257, 256
    X = rng.uniform(-1, 1, (C, N))
    h = rng.standard_normal(L)
    ref = np.stack([np.convolve(X[c], h) for c in range(C)])
    for t0 in (0, 5, 8, 300, 643):
        delta = (t0 - L + 1) % 8
        w0 = t0 - L + 1 - delta
        assert w0 % 8 == 0
        K = -(-(nout + L - 1 + delta) // 32) * 32            # whole K blocks of 32 samples
        i = np.arange(nout)[:, None]
        jj = np.arange(K)[None, :]
        k = L - 1 + delta + i - jj
        T = np.where((k >= 0) & (k < L), h[np.clip(k, 0, L - 1)], 0.0)
        n = w0 + np.arange(K)
        Xw = np.where((n >= 0) & (n < N), X[:, np.clip(n, 0, N - 1)], 0.0)
        Y = Xw @ T.T
        m = t0 + np.arange(nout)
        ok = m < N + L - 1
        assert np.abs(Y[:, ok] - ref[:, m[ok]]).max() <= 1e-12 * np.abs(ref).max()


def test_k2_row_view_of_one_signal():
    """tc_convolve_tc: rows of 256 outputs are K2 channels; row r reads xs from 256 r on, xs = x delayed by
    L - 1 (zeros around it); y[256 r + i] = sum_j T[i][j] xs[256 r + j], T[i][j] = h[L - 1 + i - j]."""
    rng = np.random.default_rng(15)
    for N, L in [(1000, 1), (1000, 300), (700, 2000), (5000, 4097)]:
        x = rng.uniform(-1, 1, N)
        h = rng.standard_normal(L)
        ref = np.convolve(x, h)
        M = N + L - 1
        R = -(-M // 256)
        nkb = -(-(L - 1 + 256) // 32)
        xs = np.zeros(256 * R + 32 * nkb)
        xs[L - 1:L - 1 + N] = x
        i = np.arange(256)[:, None]
        jj = np.arange(32 * nkb)[None, :]
        k = L - 1 + i - jj
        T = np.where((k >= 0) & (k < L), h[np.clip(k, 0, L - 1)], 0.0)
        rows = np.stack([xs[256 * r:256 * r + 32 * nkb] for r in range(R)])  # overlapping view, stride 256
        y = (rows @ T.T).reshape(-1)[:M]
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max(), (N, L)


def test_k3_phase_reshaping_of_a_mimo_tile():
    """K3: for a tile of 1024 output times ending at Tb, t = Tb - 8 r - p, D[r][16 p + o] =
    sum_i sum_k' A_i[r][k'] B_i[k'][16 p + o], A_i[r][k'] = xr_i[s0 + 8 r + k'] with xr_i[j] = x_i[R - j] and
    s0 = R - Tb, B_i[k'][16 p + o] = h_{o,i}[k' - p]; K blocks of 32, nkbp = ceil((L + 7) / 2048) * 64."""
    rng = np.random.default_rng(16)
    nin, nout, L, N = 3, 5, 300, 2500
    X = rng.uniform(-1, 1, (nin, N))
    H = rng.standard_normal((nout, nin, L))
    ref = np.zeros((nout, N + L - 1))
    for o in range(nout):
        for i in range(nin):
            ref[o] += np.convolve(X[i], H[o, i])
    nkbp = -(-(L + 7) // 2048) * 64
    K = 32 * nkbp
    Bm = np.zeros((nin, K, 128))
    for col in range(128):
        p, o = col >> 4, col & 15
        if o < nout:
            k = np.arange(K) - p
            ok = (k >= 0) & (k < L)
            Bm[:, ok, col] = H[o][:, k[ok]]
    R = N + L + 2048
    j = np.arange(R + K + 1024)
    n = R - j
    xr = np.where((n >= 0) & (n < N), X[:, np.clip(n, 0, N - 1)], 0.0)
    r = np.arange(128)[:, None]
    kk = np.arange(K)[None, :]
    for Tb in (1023, 1500, 2900, N + L - 2):
        s0 = R - Tb
        D = sum(xr[i][s0 + 8 * r + kk] @ Bm[i] for i in range(nin))
        for col in range(128):
            p, o = col >> 4, col & 15
            if o >= nout:
                continue
            t = Tb - 8 * np.arange(128) - p
            ok = (t >= 0) & (t < N + L - 1)
            assert np.abs(D[ok, col] - ref[o, t[ok]]).max() <= 1e-11 * np.abs(ref).max(), (Tb, col)


# K2 persistent CTA pairs (k2_toeplitz_tc.cu: k2_unit, k2_cta, k2_fold_*; capi.cu: launch_k2)
K2_M, K2_N = 128, 256


def k2_nkb(L, delta, kbs):
    return (L - 1 + delta + K2_N + kbs - 1) // kbs


def test_k2_toeplitz_tiles_in_k_blocks_of_32_and_64():
    """k2_tprep: T[kb][i][j] = h[L - 1 + delta + i - kbs kb - j] in K blocks of kbs = 32 (split) or 64 (plain);
    nkb = k2_nkb(L, delta, kbs) blocks cover every tap of every output of the tile, and one thread's group of eight
    j (q -> jg = q mod kbs/8, row r = q div kbs/8) writes each element of the tiles exactly once."""
    rng = np.random.default_rng(17)
    for kbs in (32, 64):
        sh = 3 if kbs == 64 else 2
        for L, delta in [(1, 0), (257, 3), (1000, 7), (4097, 5)]:
            h = rng.standard_normal(L)
            nkb = k2_nkb(L, delta, kbs)
            kb = np.arange(nkb)[:, None, None]
            i = np.arange(K2_N)[None, :, None]
            j = np.arange(kbs)[None, None, :]
            k = L - 1 + delta + i - kbs * kb - j
            T = np.where((k >= 0) & (k < L), h[np.clip(k, 0, L - 1)], 0.0)
            # every tap of every output row appears once, in its K block
            for row in (0, 1, K2_N - 1):
                taps = k[:, row, :].reshape(-1)
                taps = taps[(taps >= 0) & (taps < L)]
                assert np.array_equal(np.sort(taps), np.arange(L)), (kbs, L, delta, row)
            # the thread decomposition of k2_tprep_group writes each element once
            total = (nkb * K2_N) << sh
            q = np.arange(total)
            jg = q & ((1 << sh) - 1)
            r = q >> sh
            o = (r * kbs + 8 * jg)[:, None] + np.arange(8)[None, :]
            assert np.array_equal(np.sort(o.reshape(-1)), np.arange(nkb * K2_N * kbs))
            flat = T.reshape(-1)
            assert flat.shape[0] == nkb * K2_N * kbs


def k2_units(ntile_c, ntile_o, nsplit, order, pair_o):
    """(unit, rank) -> (tc1, ot, part) as k2_unit and k2_cta compute them."""
    nto = (ntile_o + 1) // 2 if pair_o else ntile_o
    out = []
    for u0 in range(ntile_c * nto * nsplit):
        u = u0
        if order == 1:
            tile_o = u % nto; u //= nto; part = u % nsplit; tile_c = u // nsplit
        elif order == 2:
            tile_o = u % nto; u //= nto; tile_c = u % ntile_c; part = u // ntile_c
        else:
            part = u % nsplit; u //= nsplit; tile_o = u % nto; tile_c = u // nto
        for rank in (0, 1):
            tc1 = tile_c if pair_o else tile_c * 2 + rank
            ot = tile_o * 2 + rank if pair_o else tile_o
            out.append((tc1, ot, part))
    return out


def test_k2_pair_units_cover_every_tile_and_part_once():
    """The persistent CTA pairs: over all units and both CTAs, every (128-channel tile, output tile, K part) is
    computed once by a CTA whose output tile exists (live), in every unit order, with pairs of channel tiles or,
    for a group of one channel tile, pairs of output tiles (the odd last one's partner is not live); the partial
    and ticket indices of the live CTAs stay inside what launch_k2 allocates
    (2 ceil(tiles / 2) x ntile_o x nsplit tiles of 128 x 256 floats, 8 tickets per tile)."""
    for C in (1, 100, 128, 129, 300, 1024):
        ntile_c1 = -(-C // K2_M)
        for ntile_o in (1, 2, 5, 32):
            for nsplit in (1, 3, 4, 17):
                pair_o = ntile_c1 == 1 and ntile_o >= 2
                ntile_c = ntile_c1 if pair_o else (ntile_c1 + 1) // 2
                alloc_tiles = 2 * ((ntile_c1 + 1) // 2) * ntile_o
                for order in (0, 1, 2):
                    cover = {}
                    for tc1, ot, part in k2_units(ntile_c, ntile_o, nsplit, order, pair_o):
                        if ot >= ntile_o:
                            assert pair_o and ntile_o % 2 == 1 and ot == ntile_o  # only the odd tile's partner
                            continue
                        if tc1 * K2_M >= C:
                            continue  # rows past the group: computed, never stored
                        key = (tc1, ot, part)
                        cover[key] = cover.get(key, 0) + 1
                        tile = tc1 * ntile_o + ot
                        assert (tile * nsplit + part) < alloc_tiles * nsplit
                        assert tile * 8 + 7 < alloc_tiles * 8
                    want = {(t, o, p) for t in range(ntile_c1) for o in range(ntile_o) for p in range(nsplit)}
                    assert set(cover) == want and all(v == 1 for v in cover.values()), (C, ntile_o, nsplit, order)


def fold_carry(v):
    """k2_fold_rows: adjacent pairs level by level, an odd last element carried up (float32)."""
    v = list(v)
    while len(v) > 1:
        n = len(v)
        nxt = [np.float32(v[2 * s] + v[2 * s + 1]) for s in range(n // 2)]
        if n & 1:
            nxt.append(v[n - 1])
        v = nxt
    return v[0]


def fold_padded(v):
    """k2_reduce: zero-padded to 64 leaves, adjacent pairs level by level (float32)."""
    w = [np.float32(x) for x in v] + [np.float32(0.0)] * (64 - len(v))
    while len(w) > 1:
        w = [np.float32(w[2 * s] + w[2 * s + 1]) for s in range(len(w) // 2)]
    return w[0]


def test_k2_fold_tree_equals_the_zero_padded_reduce_tree():
    """The in-kernel fold of 2..16 K parts adds them as k2_reduce does, bit for bit in float32: carrying an odd
    element up unchanged is the zero-padded tree, since x + 0 = x (only the sign of a zero may differ)."""
    rng = np.random.default_rng(18)
    for n in range(1, 17):
        for _ in range(200):
            v = (rng.standard_normal(n) * 10.0 ** rng.integers(-3, 4, n)).astype(np.float32)
            a, b = fold_carry(v), fold_padded(v)
            assert a == b and np.float32(a).tobytes() in (np.float32(b).tobytes(), np.float32(-b).tobytes()), (n, v)


def test_k2_row_view_writes_each_output_once_up_to_y_total():
    """k2_ylim with a flat destination (row pitch 256): over the rows and column halves of every tile, the kept
    writes cover [0, y_total) exactly once (the last row cut at the end of y)."""
    for y_total in (256, 257, 1000, 32768, 40001):
        rows = -(-y_total // 256)
        hits = np.zeros(rows * 256, np.int64)
        for c in range(rows):
            for half in (0, 1):
                col = half * 128
                lim = min(256 - col, y_total - c * 256 - col)  # nout = 256 per row, tile_o = 0
                if lim > 0:
                    start = c * 256 + col
                    hits[start:start + min(lim, 128)] += 1
        assert np.array_equal(hits[:y_total], np.ones(y_total, np.int64)) and not hits[y_total:].any(), y_total
