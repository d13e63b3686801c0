/*
 * taches_oracle.c -- plain, slow, FP64 CPU oracle for the taches-algorithm
 * (L. Millot and G. Pele, "An alternative approach for the convolution in
 * time-domain: the taches-algorithms", AES 125th Convention, paper 7412, 2008).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the CPU-baseline
 * leg of the benchmark are the only code allowed to load this library. The
 * CUDA product path never calls it, and the two share no code.
 *
 * Arithmetic: IEEE binary64, round to nearest. The binary32 inputs are widened
 * exactly. Build with -O2, without -ffast-math, with -ffp-contract=off, so
 * that every product and every sum is rounded once, in the order written here.
 *
 * Time-varying IR ("taches semantics"). The abstract and Sec. 6 say the IR may
 * be replaced while the computation runs, "even sample-by-sample": the new IR
 * applies to the next input samples, and taches already spawned keep the IR
 * they were spawned with. The oracle represents this with IR versions:
 *   H[v*L + k]  tap k of version v, 0 <= k < L (shorter IRs zero-padded)
 *   vstart[v]   first input sample that uses version v; vstart[0] <= 0 and
 *               vstart is strictly increasing.
 * Input sample n spawns the tache x[n] * H[v(n)][.], where
 * v(n) = max{ v : vstart[v] <= n }. So the output is
 *   y[m] = sum_{n} x[n] * H[v(n)][m - n],   0 <= m < N + L - 1,      (Eq. 4)
 * with the sum over 0 <= n < N and 0 <= m - n < L.
 *
 * Three independent forms are provided, each following one passage:
 *   tco_direct / tco_direct_at : Eq. (4) summed output by output (Sec. 3.2).
 *   tco_vect                   : the vectorised algorithm of Sec. 4.1.
 *   tco_buf_*                  : the buffer (ring) algorithm of Sec. 4.2,
 *                                with the readings listed at tco_buf_push.
 * Plus tco_mimo, a sum over input channels of buffer-algorithm outputs,
 * tco_direct_at_xf / tco_buffer_xf, the crossfaded (continuous) form of the
 * time-varying IR, and tco_q15_direct, the exact fixed-point form.
 *
 * Parity pins (tests): unit impulse, linearity, commutativity (Sec. 3.2,
 * Fig. 6), output length N+L-1 (Sec. 4.1), sum invariant, a geometric-sum
 * closed form, numpy/scipy convolution for the fixed-IR special case, the
 * IR-switch reduction to two plain convolutions, block-size invariance
 * (Table 2's Nb only changes timing), and a hand-worked 6x3 example in the
 * shape of Fig. 4-5.
 *
 * ORACLE_MUTANT (compile-time, tests only): plants one known mistake so that
 * the test suite can show that its pins catch it. 0 = no mutant.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* v(n): the version active for input sample n (last v with vstart[v] <= n). */
static int64_t version_of(const int64_t *vstart, int64_t nver, int64_t n)
{
    int64_t v = 0;
    while (v + 1 < nver && vstart[v + 1] <= n)
        ++v;
    return v;
}

static int check_versions(const int64_t *vstart, int64_t nver)
{
    if (nver < 1 || vstart[0] > 0)
        return -1;
    for (int64_t v = 1; v < nver; ++v)
        if (vstart[v] <= vstart[v - 1])
            return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. (4), Sec. 3.2: one output sample as a sum over the input samples
 * whose taches reach it.                                               */
/* ------------------------------------------------------------------ */
double tco_direct_at(const float *x, int64_t N, const float *H, int64_t L,
                     const int64_t *vstart, int64_t nver, int64_t m)
{
    double acc = 0.0;
    int64_t n_lo = m - (L - 1);
    if (n_lo < 0)
        n_lo = 0;
    int64_t n_hi = m;
    if (n_hi > N - 1)
        n_hi = N - 1;
    for (int64_t n = n_lo; n <= n_hi; ++n) {
#if ORACLE_MUTANT == 2
        int64_t v = version_of(vstart, nver, m);     /* IR picked at output time */
#else
        int64_t v = version_of(vstart, nver, n);     /* IR of the spawning sample */
#endif
        acc += (double)x[n] * (double)H[v * L + (m - n)];
    }
    return acc;
}

int tco_direct(const float *x, int64_t N, const float *H, int64_t L,
               const int64_t *vstart, int64_t nver, double *y)
{
    if (N < 1 || L < 1 || check_versions(vstart, nver))
        return -1;
    for (int64_t m = 0; m < N + L - 1; ++m)
        y[m] = tco_direct_at(x, N, H, L, vstart, nver, m);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1, vectorised algorithm: a residue vector r of length Nh gets
 * the new tache e(n)*h added, r(1) is the next output, r is shifted left
 * with a zero appended; after the last input the residue minus its last
 * (zero) element is the temporal overflow.                             */
/* ------------------------------------------------------------------ */
int tco_vect(const float *x, int64_t N, const float *H, int64_t L,
             const int64_t *vstart, int64_t nver, double *y)
{
    if (N < 1 || L < 1 || check_versions(vstart, nver))
        return -1;
    double *r = (double *)calloc((size_t)L, sizeof(double));
    if (!r)
        return -2;
    int64_t out = 0;
    for (int64_t n = 0; n < N; ++n) {
        const float *h = H + version_of(vstart, nver, n) * L;
        double e = (double)x[n];
        for (int64_t k = 0; k < L; ++k)
            r[k] += e * (double)h[k];
        y[out++] = r[0];
        memmove(r, r + 1, (size_t)(L - 1) * sizeof(double));
#if ORACLE_MUTANT != 6
        r[L - 1] = 0.0;                                  /* shift left, append a zero */
#endif
    }
    for (int64_t k = 0; k < L - 1; ++k)
        y[out++] = r[k];
    free(r);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.2, buffer algorithm, as a persistent stream state.            */
/* ------------------------------------------------------------------ */
typedef struct tco_buf {
    int64_t L;        /* ring length = IR length (Nh)                  */
    double *r;        /* circular residue, r[0..L-1]                   */
    int64_t rho;      /* 0-based r_index: slot of the next output      */
    int64_t n_in;     /* input samples consumed so far                 */
} tco_buf;

tco_buf *tco_buf_open(int64_t L)
{
    if (L < 1)
        return NULL;
    tco_buf *s = (tco_buf *)calloc(1, sizeof(tco_buf));
    if (!s)
        return NULL;
    s->r = (double *)calloc((size_t)L, sizeof(double));   /* r(1..Nh) <- 0 */
    if (!s->r) {
        free(s);
        return NULL;
    }
    s->L = L;
    s->rho = 0;                                          /* r_index <- 1 (1-based) */
    s->n_in = 0;
    return s;
}

void tco_buf_close(tco_buf *s)
{
    if (s) {
        free(s->r);
        free(s);
    }
}

/* One sample step: add the tache e0*h into the ring, emit, clear, advance. */
static double buf_step(tco_buf *s, double e0, const float *h)
{
    const int64_t L = s->L;
    double *restrict r = s->r;
    const int64_t rho = s->rho;
#if ORACLE_MUTANT == 1
    /* Offsets exactly as printed in Sec. 4.2: the first tap lands one slot
     * after r_index and the last tap lands on r_index itself.            */
    for (int64_t i = rho + 1; i < L; ++i)
        r[i] += e0 * (double)h[i - rho - 1];
    for (int64_t i = 0; i <= rho; ++i)
        r[i] += e0 * (double)h[L - 1 - rho + i];
#else
    /* Reading 1: tap j (0-based) lands on slot (rho + j) mod L, so tap 0
     * is in the slot emitted now. Written as the paper's two wrapped
     * loops over contiguous ranges.                                      */
    int64_t taps = L;
#if ORACLE_MUTANT == 3
    taps = L - 1;                                        /* last tap dropped */
#endif
    int64_t first = L - rho;                             /* taps before the wrap */
    if (first > taps)
        first = taps;
    for (int64_t j = 0; j < first; ++j)
        r[rho + j] += e0 * (double)h[j];
    for (int64_t j = first; j < taps; ++j)
        r[rho + j - L] += e0 * (double)h[j];
#endif
    double out = r[rho];                                 /* sp(n) <- r(r_index) */
#if ORACLE_MUTANT != 5
    r[rho] = 0.0;                                        /* r(r_index) <- 0 */
#endif
    s->rho = (rho + 1 < L) ? rho + 1 : 0;                /* advance with wrap (reading 2) */
    return out;
}

/* Push one input block pe[0..nb-1] and receive ps[0..nb-1].
 * Readings of the printed pseudo-code (Sec. 4.2):
 *  1. tap offsets: tap j goes to slot (r_index + j) mod Nh (see buf_step);
 *  2. the index wraps to the first slot;
 *  3. the "while" over blocks is the caller's loop; one call = one block;
 *  4. r and r_index are initialised once per stream (tco_buf_open) and
 *     persist across blocks;
 *  5. sp and ps name the same output block;
 *  6. a block may be shorter than Nb (the last one);
 * and the IR of sample n is H[v(n)] (per-sample versions, Sec. 6).      */
int tco_buf_push(tco_buf *s, const float *pe, int64_t nb,
                 const float *H, const int64_t *vstart, int64_t nver, double *ps)
{
    if (!s || nb < 0 || check_versions(vstart, nver))
        return -1;
    for (int64_t n = 0; n < nb; ++n) {
        const int64_t nabs = s->n_in + n;
        const float *h = H + version_of(vstart, nver, nabs) * s->L;
        ps[n] = buf_step(s, (double)pe[n], h);
    }
    s->n_in += nb;
    return 0;
}

/* Temporal overflow (Sec. 4.1, applied to the buffer form, reading 7): the
 * L-1 samples still in the ring, in emission order. Equivalent to pushing
 * L-1 zeros. Leaves the ring cleared.                                     */
int tco_buf_flush(tco_buf *s, double *ps)
{
    if (!s)
        return -1;
    int64_t tail = s->L - 1;
#if ORACLE_MUTANT == 4
    tail = s->L - 2;                                    /* last overflow sample lost */
#endif
    for (int64_t n = 0; n < tail; ++n) {
        ps[n] = s->r[s->rho];
        s->r[s->rho] = 0.0;
        s->rho = (s->rho + 1 < s->L) ? s->rho + 1 : 0;
    }
    return 0;
}

/* Whole signal through the buffer algorithm in blocks of Nb, then flush.
 * y receives N + L - 1 samples.                                         */
int tco_buffer(const float *x, int64_t N, const float *H, int64_t L,
               const int64_t *vstart, int64_t nver, int64_t Nb, double *y)
{
    if (N < 1 || L < 1 || Nb < 1 || check_versions(vstart, nver))
        return -1;
    tco_buf *s = tco_buf_open(L);
    if (!s)
        return -2;
    for (int64_t b = 0; b < N; b += Nb) {
        int64_t nb = (N - b < Nb) ? N - b : Nb;          /* Nb <- min(Nb, size(pe)) */
        tco_buf_push(s, x + b, nb, H, vstart, nver, y + b);
    }
    tco_buf_flush(s, y + N);
    tco_buf_close(s);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Multichannel use (Sec. 5.1 and 6 mention multichannel stimuli):
 * nout outputs, each the sum over nin inputs of the buffer-algorithm
 * convolution of input i with IR (o, i).
 *   x:  [nin][N]          H: [nver][nout][nin][L]       y: [nout][N+L-1]
 * The per-pair outputs are summed in FP64 in input order.              */
/* ------------------------------------------------------------------ */
int tco_mimo(const float *x, int64_t nin, int64_t nout, int64_t N,
             const float *H, int64_t L, const int64_t *vstart, int64_t nver,
             int64_t Nb, double *y)
{
    if (nin < 1 || nout < 1 || N < 1 || L < 1 || Nb < 1 || check_versions(vstart, nver))
        return -1;
    const int64_t ny = N + L - 1;
    double *tmp = (double *)malloc((size_t)ny * sizeof(double));
    float *Hp = (float *)malloc((size_t)(nver * L) * sizeof(float));
    if (!tmp || !Hp) {
        free(tmp);
        free(Hp);
        return -2;
    }
    for (int64_t o = 0; o < nout; ++o) {
        double *yo = y + o * ny;
        for (int64_t m = 0; m < ny; ++m)
            yo[m] = 0.0;
        for (int64_t i = 0; i < nin; ++i) {
            for (int64_t v = 0; v < nver; ++v)
#if ORACLE_MUTANT == 7
                memcpy(Hp + v * L, H + ((v * nout + i % nout) * nin + o % nin) * L, (size_t)L * sizeof(float));
#else
                memcpy(Hp + v * L, H + ((v * nout + o) * nin + i) * L, (size_t)L * sizeof(float));
#endif
            tco_buffer(x + i * N, N, Hp, L, vstart, nver, Nb, tmp);
            for (int64_t m = 0; m < ny; ++m)
                yo[m] += tmp[m];
        }
    }
    free(tmp);
    free(Hp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Continuous time-varying IR (Sec. 6: the IR may also change
 * progressively, e.g. a decay changed little by little). A switch becomes a
 * crossfade: version v takes over from version v-1 over vramp[v] >= 1 input
 * samples from vstart[v] on,
 *   alpha_v(n) = clamp((n - vstart[v] + 1) / vramp[v], 0, 1),  alpha_0 = 1,
 * and input sample n spawns its tache with the mixed IR
 *   h_n = sum_v (alpha_v(n) - alpha_{v+1}(n)) H[v]     (alpha_nver = 0).
 * vramp[v] = 1 is the hard switch of the forms above. A crossfade starts only
 * once the previous one has ended: vstart[v+1] >= vstart[v] + vramp[v] - 1,
 * so every weight lies in [0, 1] and the weights of a sample add up to 1.
 * The taches semantics are unchanged: the IR of a tache is fixed when its
 * sample arrives.                                                        */
/* ------------------------------------------------------------------ */
static int check_ramps(const int64_t *vstart, const int64_t *vramp, int64_t nver)
{
    if (check_versions(vstart, nver))
        return -1;
    for (int64_t v = 0; v < nver; ++v) {
        if (vramp[v] < 1)
            return -1;
        if (v + 1 < nver && vstart[v + 1] < vstart[v] + vramp[v] - 1)
            return -1;
    }
    return 0;
}

static double alpha_of(const int64_t *vstart, const int64_t *vramp, int64_t nver, int64_t v, int64_t n)
{
    if (v == 0)
        return 1.0;
    if (v >= nver)
        return 0.0;
#if ORACLE_MUTANT == 8
    double a = (double)(n - vstart[v]) / (double)vramp[v];  /* ramp one sample late */
#else
    double a = (double)(n - vstart[v] + 1) / (double)vramp[v];
#endif
    return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
}

/* Tap k of the mixed IR of input sample n. */
static double mixed_tap(const float *H, int64_t L, const int64_t *vstart, const int64_t *vramp, int64_t nver,
                        int64_t n, int64_t k)
{
    double h = 0.0;
    for (int64_t v = 0; v < nver; ++v) {
        const double w = alpha_of(vstart, vramp, nver, v, n) - alpha_of(vstart, vramp, nver, v + 1, n);
        if (w != 0.0)
            h += w * (double)H[v * L + k];
    }
    return h;
}

/* Eq. (4) with mixed IRs, one output sample. */
double tco_direct_at_xf(const float *x, int64_t N, const float *H, int64_t L, const int64_t *vstart,
                        const int64_t *vramp, int64_t nver, int64_t m)
{
    double acc = 0.0;
    int64_t n_lo = m - (L - 1);
    if (n_lo < 0)
        n_lo = 0;
    int64_t n_hi = m;
    if (n_hi > N - 1)
        n_hi = N - 1;
    for (int64_t n = n_lo; n <= n_hi; ++n)
        acc += (double)x[n] * mixed_tap(H, L, vstart, vramp, nver, n, m - n);
    return acc;
}

/* The buffer algorithm (Sec. 4.2, readings as tco_buf_push) with mixed IRs,
 * in blocks of Nb, then the flush: y receives N + L - 1 samples.          */
int tco_buffer_xf(const float *x, int64_t N, const float *H, int64_t L, const int64_t *vstart,
                  const int64_t *vramp, int64_t nver, int64_t Nb, double *y)
{
    if (N < 1 || L < 1 || Nb < 1 || check_ramps(vstart, vramp, nver))
        return -1;
    tco_buf *s = tco_buf_open(L);
    double *h = (double *)malloc((size_t)L * sizeof(double));
    if (!s || !h) {
        tco_buf_close(s);
        free(h);
        return -2;
    }
    for (int64_t b = 0; b < N; b += Nb) {
        const int64_t nb = (N - b < Nb) ? N - b : Nb;
        for (int64_t n = b; n < b + nb; ++n) {
            for (int64_t k = 0; k < L; ++k)
                h[k] = mixed_tap(H, L, vstart, vramp, nver, n, k);
            /* The tache x[n] * h_n into the ring: tap j on slot (rho + j) mod L. */
            const double e0 = (double)x[n];
            double *r = s->r;
            const int64_t rho = s->rho;
            for (int64_t j = 0; j < L; ++j) {
                int64_t slot = rho + j;
                if (slot >= L)
                    slot -= L;
                r[slot] += e0 * h[j];
            }
            y[n] = r[rho];
            r[rho] = 0.0;
            s->rho = (rho + 1 < L) ? rho + 1 : 0;
        }
        s->n_in += nb;
    }
    tco_buf_flush(s, y + N);
    tco_buf_close(s);
    free(h);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Exact fixed point with one requantization (Sec. 5.4, "ideal
 * requantization": an accumulator of unlimited range, a single
 * requantization at the end of each output sample). Input and taps are Q15
 * (int16); each product is exact in 32 bits; the sum of an output's products
 * is kept exactly in 64 bits (|sum| < 2^49 for L <= 2^19), then requantized
 * once to Q15: round half to even of sum / 2^15, saturated to int16.
 *   acc[m] = sum_n x[n] * h[m - n]   (exact),   y[m] = sat16(rne(acc[m] / 2^15)).
 * acc or y may be NULL.                                                  */
/* ------------------------------------------------------------------ */
static int16_t requant_q15(int64_t a)
{
#if ORACLE_MUTANT == 9
    int64_t q = (a + (1 << 14)) >> 15;                     /* rounds halves up, not to even */
#else
    int64_t q = a >> 15;                                   /* floor(a / 2^15) */
    const int64_t rem = a - q * 32768;                     /* in [0, 2^15) */
    if (rem > 16384 || (rem == 16384 && (q & 1)))
        ++q;
#endif
    if (q > 32767)
        q = 32767;
    if (q < -32768)
        q = -32768;
    return (int16_t)q;
}

int tco_q15_direct(const int16_t *x, int64_t N, const int16_t *h, int64_t L, int64_t *acc, int16_t *y)
{
    if (N < 1 || L < 1 || L > (int64_t)1 << 19)
        return -1;
    for (int64_t m = 0; m < N + L - 1; ++m) {
        int64_t n_lo = m - (L - 1);
        if (n_lo < 0)
            n_lo = 0;
        const int64_t n_hi = (m < N - 1) ? m : N - 1;
        int64_t a = 0;
        for (int64_t n = n_lo; n <= n_hi; ++n)
            a += (int64_t)((int32_t)x[n] * (int32_t)h[m - n]);
        if (acc)
            acc[m] = a;
        if (y)
            y[m] = requant_q15(a);
    }
    return 0;
}

int tco_mutant_id(void) { return ORACLE_MUTANT; }
