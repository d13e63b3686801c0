// tc_internal.h -- host/device structures shared by the kernels and the C ABI
// implementation. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "taches.h"

namespace tc {

// NVTX range over a host-side phase (push, IR upload, flush, server step):
// profilers that attach to the process show where host time goes; without
// one attached a range costs a few nanoseconds. NVTX 3 is header-only.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// ---------------------------------------------------------------------------
// K1: FP32 output-side gather (per-stream IRs, or any IR layout).
//
// The launch computes, for every item c (a channel, or a MIMO output) and every
// output sample t0 <= m < t0 + nout,
//     y_c[m] = sum_{i < nin} sum_{k < L} h_{c,i,v(m-k)}[k] * x_{c,i}[m-k],
// where x_{c,i} is a row of the input history and v(n) the IR version of
// input sample n (Eq. 4 with per-sample versions).
//
// Work split: output tiles of K1_MO = 128 samples x tap chunk-tasks of KC
// taps (nin * nchunk per tile); one CTA per (item, tile, chunk-task). A CTA sums
// its chunk in FP32 registers. Sub-segments are combined by a pairwise tree,
// and the chunk sums of a tile by a pairwise tree run by the tile's last CTA.
// ---------------------------------------------------------------------------
constexpr int K1_MO = 128;           // outputs per tile
constexpr int K1_THREADS = 256;      // 8 output groups of 16 x 32 tap sub-segments
constexpr int K1_SEG = 20;           // taps per thread per pass
constexpr int K1_PBIG = 11;                   // passes of the largest chunk (4 CTAs of it fit an SM)
constexpr int K1_KC_MAX = 32 * K1_SEG * K1_PBIG;  // largest tap chunk of any variant
constexpr int K1_MAX_CHUNK_TASKS = 4095;     // chunk-tasks per tile (12-level pairwise stack)

struct K1Params {
    // Input history: sample n of history row r is hist[r * pitch + (n - base)].
    // The host keeps base % 4 == 0, pitch % 4 == 0 and zeros before sample 0.
    const float *hist;
    long long pitch;
    long long base;
    long long x_item_rows;   // history row of (item c, input i) = c * x_item_rows + i * x_in_rows
    long long x_in_rows;

    // IR slots. Tap k of slot s, item c, input i is stored four times, shifted
    // by e = 0..3 taps: ir[s*slot + c*item + i*in + e*phase + k + e]. The
    // shifted copies let every tap chunk start on a 16-byte boundary.
    const float *ir;
    long long ir_slot, ir_item, ir_in, ir_phase;
    int L;

    // IR versions of item c: entries [c * vt_item, c * vt_item + nver[c]).
    // vstart ascending; the version with the largest vstart <= n owns n. With
    // ramps, version v takes over from v - 1 over vramp[v] samples from
    // vstart[v] on: sample n's tache uses sum_v (alpha_v(n) - alpha_{v+1}(n)) h_v,
    // alpha_v(n) = clamp((n - vstart[v] + 1) / vramp[v], 0, 1), alpha_0 = 1.
    const long long *vstart;
    const int *vslot;
    const int *nver;
    const int *vramp;        // crossfade ramp of each version (samples, >= 1), or null: hard switches
    int vt_item;             // 0: one table shared by all items

    int nitems;
    int nin;
    long long t0;            // first output sample of the launch
    int nout;                // outputs per item
    int ntile;               // ceil(nout / K1_MO)
    int e;                   // tap shift so that chunk starts are 16-byte aligned
    int nchunk;              // tap chunks per input (filled by k1_launch)

    float *y;                // output of item c, sample t0 + j: y[c * y_pitch + j]
    long long y_pitch;

    float *partial;          // [nitems][ntile][nin*nchunk][K1_MO] chunk sums
    unsigned *counter;       // [nitems][ntile], zero between launches
    int *err;                // device error word
    int zero_skip;           // 1: skip passes whose staged input is all zero (exact)
    int has_end;             // 1: input samples n >= x_end are zero (the flush after the last input): chunks
    long long x_end;         //    and passes that read only such samples are skipped (exact)
};

// Variants: passes of K1_SEG taps per thread per chunk (KC = 32 * 20 * P).
enum K1Variant { K1_P1 = 0, K1_P4 = 1, K1_P11 = 2, K1_NVARIANTS = 3 };
int k1_chunk_taps(int variant);

struct K1Plan {
    int variant;
    int nchunk;
    long long ctas;
};

// Chunk alignment shift for a launch starting at output t0 with history base.
inline int k1_shift_e(long long t0, long long base)
{
    long long d = ((t0 + 1 - base) % 4 + 4) % 4;
    return (int)((4 - d) & 3);
}

// Plans a launch: the largest chunk that still gives the GPU a few waves of
// CTAs. forced_variant >= 0 picks one.
cudaError_t k1_plan(long long L, int e, int nin, int nitems, int ntile, int forced_variant, K1Plan *plan);

// Chunk-sum scratch (floats) a launch over `tiles` tiles may need with any variant.
long long k1_partial_floats_max(long long L, int nin, long long tiles);

// Work-list launch (continuous batching): item i (fully filled K1Params,
// nchunk included, its own partial/counter scratch) owns CTAs
// [cta_begin[i], cta_begin[i+1]); all items use one chunk variant.
cudaError_t k1_launch_list(const K1Params *d_items, const long long *d_cta_begin, int nitems, long long total_ctas,
                           int variant, cudaStream_t st);

// The work-list kernel of a variant (for CUDA-graph kernel nodes): its
// arguments are (K1Params unused, const K1Params *items, const long long
// *cta_begin, int nitems), 256 threads, *smem bytes of dynamic shared memory.
const void *k1_list_kernel(int variant, size_t *smem);

// Launches K1 for plan on st (fills p.nchunk).
cudaError_t k1_launch(K1Params &p, const K1Plan &plan, cudaStream_t st);

// ---------------------------------------------------------------------------
// IR preparation: writes the four shifted copies of each IR row into a slot.
//   dst[r * row_stride + e * phase + j] = (0 <= j - e < n) ? src[r * src_pitch + j - e] : 0
// for j in [0, Lpad). Rows r in [0, rows).
// ---------------------------------------------------------------------------
cudaError_t ir_prep_launch(const float *src, long long src_pitch, long long n, int rows,
                           float *dst, long long row_stride, long long phase, long long Lpad,
                           cudaStream_t st);

// ---------------------------------------------------------------------------
// K2: shared-IR contraction on the tensor cores (k2_toeplitz_tc.cu).
//   Y[c][t0+i] = sum_j X[c][w0+j] T[i][j],  T[i][j] = h[L - 1 + delta + i - j],
//   w0 = t0 - L + 1 - delta on an 8-sample grid of the history.
// Tiles: 128 channels x 256 outputs x K blocks of 32 samples.
// ---------------------------------------------------------------------------
struct K2Params {
    int C;                   // channels (rows of the history)
    int nout;                // outputs per channel in this launch
    int ntile_c, ntile_o;    // ceil(C / 128), ceil(nout / 256)
    long long x_col0;        // history column of w0 for output tile 0 (multiple of 8)
    int nkb;                 // K blocks per output tile
    int nsplit, kb_per;      // K parts per tile (one CTA each) and blocks per part
    int range;               // K blocks per serial TMEM run before the drain to FP32 registers
    int pair_o;              // persistent CTA pairs of a group of one channel tile: the two CTAs take two
                             // adjacent output tiles of the same channels (ntile_c counts channel tiles)
    int order;               // persistent CTA pairs: order of the units (0 K part fastest, then output
                             // tile; 1 output tile fastest, then K part; 2 output tile, channel tile, K part)
    float *y;                // y[c * y_pitch + j], j < nout
    long long y_pitch;
    long long y_total;       // > 0: y is flat and writes at c * y_pitch + j >= y_total are dropped
    float *partial;          // [ntile_c][ntile_o][nsplit][128][256] (nsplit > 1)
    unsigned *ticket;        // persistent CTA pairs: [2 ntile_c][ntile_o][8] K-part tickets per warp slice,
                             // zero between launches; null = parts added by k2_reduce
    int *err;
};
int k2_tile_m();
int k2_tile_n();
int k2_kblock(int nprod);  // samples per K block: 64 for plain BF16 (nprod 1), 32 for the split (3)
long long k2_nkb(long long L, int delta, int kbs);
size_t k2_smem_bytes(int nprod);
// Toeplitz tiles of IR h (fp32, L taps) for shift delta: hi/lo bf16 [nkb][256][kbs].
cudaError_t k2_tprep_launch(const float *h, int L, int delta, int nkb, int kbs, void *thi, void *tlo,
                            cudaStream_t st);
// One-shot preparation in one launch: xhi/xlo[d] = bf16 split of x[d - off] on
// [off, off + N), 0 elsewhere in [0, npad) (xlo may be null); the Toeplitz
// tiles of h at shift 0 (as k2_tprep_launch); zero[0, nzero) = 0.
cudaError_t k2_oneshot_prep_launch(const float *x, long long N, long long off, long long npad, void *xhi, void *xlo,
                                   const float *h, int L, int nkb, int kbs, void *thi, void *tlo, unsigned *zero,
                                   long long nzero, cudaStream_t st);
// bf16 hi/lo split of history columns [col0, col0 + n) of `rows` rows.
cudaError_t k2_split_launch(const float *hist, long long pitch, int rows, long long col0, long long n, void *hhi,
                            void *hlo, cudaStream_t st);
// nprod = 1 (BF16) or 3 (BF16 hi/lo split), K blocks of kbs = k2_kblock(nprod)
// samples. Maps: X over the bf16 history [rows][pitch], box kbs x 128; T over
// [nkb * 256][kbs], box kbs x 256 (encode_bf16_2d picks the swizzle).
cudaError_t k2_launch(const CUtensorMap &mx_hi, const CUtensorMap &mx_lo, const CUtensorMap &mt_hi,
                      const CUtensorMap &mt_lo, const K2Params &p, int nprod, cudaStream_t st);
// Plain BF16 with two 128-channel tiles per CTA sharing each T stage. p.ntile_c
// counts tile pairs (ceil(C / 256)); one TMEM run per unit (range >= kb_per).
cudaError_t k2_launch_pair(const CUtensorMap &mx_hi, const CUtensorMap &mt_hi, const K2Params &p, cudaStream_t st);
// Plain BF16 on CTA pairs (clusters of two, tcgen05 cta_group::2): a unit of
// 256 channels x 256 outputs per pair, p.ntile_c counting tile pairs as for
// k2_launch_pair; one TMEM run per unit. mt2_hi: T over [nkb * 256][64] with
// a box of 64 x 128 (each CTA loads its 128-output half).
cudaError_t k2_launch_c2(const CUtensorMap &mx_hi, const CUtensorMap &mt2_hi, const K2Params &p, cudaStream_t st);
// The same on persistent CTA pairs (one cluster per SM pair walks the units,
// two TMEM accumulators: a unit's epilogue overlaps the next unit's MMAs).
cudaError_t k2_launch_c2p(const CUtensorMap &mx_hi, const CUtensorMap &mt2_hi, const K2Params &p, cudaStream_t st);
// The BF16 hi/lo split on persistent CTA pairs (TMEM runs of p.range K blocks
// drained into FP32 register sums, as k2_launch with nprod 3). p.ntile_c
// counts tile pairs; mt2_hi / mt2_lo: T over [nkb * 256][32], box 32 x 128.
cudaError_t k2_launch_c2s(const CUtensorMap &mx_hi, const CUtensorMap &mx_lo, const CUtensorMap &mt2_hi,
                          const CUtensorMap &mt2_lo, const K2Params &p, cudaStream_t st);
// Encodes a 2-D bf16 tensor map (inner dimension first). Rows of the box of
// 64 bytes (box0 = 32) take the 64-byte swizzle, rows of 128 bytes (box0 = 64)
// the 128-byte swizzle.
cudaError_t encode_bf16_2d(CUtensorMap *map, const void *base, unsigned long long dim0, unsigned long long dim1,
                           unsigned long long stride1_bytes, unsigned box0, unsigned box1);

// ---------------------------------------------------------------------------
// K3: MIMO on the tensor cores (k3_mimo_tc.cu). Tiles of 1024 output times
// (128 rows x 8 phases) x 16 outputs; K = inputs x taps in blocks of 32.
//   D[r][16 p + o] = sum_i sum_k' xr_i[s0 + 8 r + k'] * B_i[k'][16 p + o],
//   B_i[k'][16 p + o] = h_{o,i}[k' - p], xr_i[j] = x_i[R - j].
// ---------------------------------------------------------------------------
struct K3Params {
    int nin;                 // inputs
    int ntile;               // 1024-output tiles of the launch (a multiple of k3_tiles_per_cta)
    int nkbp;                // K blocks per input (multiple of the chunk)
    int nsplit, kb_per;      // K parts per tile over nin * nkbp blocks (kb_per a multiple of the chunk)
    int range;               // K blocks per TMEM run
    const void *xr_hi, *xr_lo;  // reversed inputs, bf16 [nin][xr_pitch]
    long long xr_pitch;      // elements, a multiple of 8, >= k3_xr_span
    float *partial;          // [ntile][nsplit][128][128]
    int *err;
};
int k3_kblocks_per_input(long long L);
int k3_chunk_blocks();
int k3_tiles_per_cta();       // ntile of a launch must be a multiple of it
long long k3_xr_span(int ntile, int nkbp);
// B tiles of one IR version: ir holds h_{o,i} at (o * nin + i) * set_stride.
cudaError_t k3_tprep_launch(const float *ir, long long set_stride, int nin, int nout, int L, int nkbp, void *bh,
                            void *bl, cudaStream_t st);
// xr_i[j] = x_i[R - j] (0 for samples >= n_end), j < span, bf16 hi/lo.
cudaError_t k3_rev_launch(const float *hist, long long pitch, long long base, int nin, long long R, long long n_end,
                          long long span, void *xh, void *xl, long long xr_pitch, cudaStream_t st);
size_t k3_smem_bytes(int nprod);
// Runs K3 then the K-part reduction into y[o * y_pitch + j], j < nout, o < nout_ch (<= 16).
cudaError_t k3_launch(const CUtensorMap &mb_hi, const CUtensorMap &mb_lo, const K3Params &p, int nprod, float *y,
                      long long y_pitch, int nout_ch, int nout, cudaStream_t st);

// Sets the calling thread's tc_last_error() message.
void set_last_error(const char *msg);

// Counts kernel launches issued by this library.
void count_launch(int n = 1);
// Failure injection (tc_test_inject): true when this pass through `site` is
// the one armed to fail.
bool inject_take(int site);
void inject_arm(int site, int nth);
// TC_NO_ROLE_SWAP=1 in the environment keeps the one-shot convolutions in the
// caller's roles (for comparison timings); read at each call.
bool no_role_swap();

// Stream-ordered allocation from the library's pool on the current device
// (keeps freed memory for the next call); free with cudaFreeAsync.
cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t st);
// Releases the current device's pool memory above the 2 GiB it keeps (called
// by tc_close and tc_server_close after their frees).
void pool_trim();

// tc_convolve: the one-shot convolution with scratch from the stream-ordered
// allocator (defined beside tc_convolve_noalloc, which shares its code).
tc_status oneshot_alloc(const float *x, size_t N, const float *h, size_t L, float *y, void *cuda_stream);

// Server groups (C channels, one shared IR, any precision): a group stream
// with its own CUDA stream, its device footprint in bytes, device-pointer
// pushes (x and y [C][n]) that only enqueue work, its device error word and
// its CUDA stream.
tc_status group_open(size_t channels, size_t L, size_t max_push, int precision, tc_stream **out, size_t *bytes);
tc_status group_push(tc_stream *s, const float *x, size_t n, float *y);
int *group_err(tc_stream *s);
void *group_stream(tc_stream *s);
uint64_t launches();

}  // namespace tc
