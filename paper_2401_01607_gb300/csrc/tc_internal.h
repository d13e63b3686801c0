// tc_internal.h -- host/device structures shared by the kernels and the C ABI
// implementation. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tc {

// ---------------------------------------------------------------------------
// K1: FP32 output-side gather (per-stream IRs, or any IR layout).
//
// The launch computes, for every item c (a channel, or a MIMO output) and every
// output sample t0 <= m < t0 + nout,
//     y_c[m] = sum_{i < nin} sum_{k < L} h_{c,i,v(m-k)}[k] * x_{c,i}[m-k],
// where x_{c,i} is a row of the input history and v(n) the IR version of
// input sample n (Eq. 4 with per-sample versions).
//
// Work split: output tiles of K1_MO = 128 samples x tap chunks of KC taps.
// One CTA per (item, tile, input, chunk). A CTA sums its tap chunk in FP32
// registers. Tap sub-segments are combined by a pairwise tree of warp
// shuffles and shared memory, and the chunk partials by a pairwise tree run
// by the last CTA of the tile.
// ---------------------------------------------------------------------------
constexpr int K1_MO = 128;         // outputs per tile
constexpr int K1_THREADS = 256;    // 8 output groups of 16 x 32 tap sub-segments
constexpr int K1_MAX_CHUNKS = 256; // nin * nchunk per tile, upper bound
constexpr int K1_KC_MAX = 32 * 260;  // largest tap chunk of any variant

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
    // vstart ascending; the version with the largest vstart <= n owns n.
    const long long *vstart;
    const int *vslot;
    const int *nver;
    int vt_item;             // 0: one table shared by all items

    int nitems;
    int nin;
    long long t0;            // first output sample of the launch
    int nout;                // outputs per item
    int ntile;               // ceil(nout / K1_MO)
    int nchunk;              // tap chunks per input
    int e;                   // tap shift so that chunk starts are 16-byte aligned

    float *y;                // output of item c, sample t0 + j: y[c * y_pitch + j]
    long long y_pitch;

    float *partial;          // [nitems][ntile][nin*nchunk][K1_MO]
    unsigned *counter;       // [nitems][ntile], zero between launches
    int *err;                // device error word
};

// Variants: taps per thread S (a multiple of 20 with S/4 odd, for the
// register window rotation and conflict-free 128-bit shared loads).
enum K1Variant { K1_S20 = 0, K1_S60 = 1, K1_S100 = 2, K1_S260 = 3, K1_NVARIANTS = 4 };
int k1_taps_per_thread(int variant);
int k1_chunk_taps(int variant);   // KC = 32 * S
size_t k1_smem_bytes(int variant);

// Chunk alignment shift for a launch starting at output t0 with history base.
inline int k1_shift_e(long long t0, long long base)
{
    long long d = ((t0 + 1 - base) % 4 + 4) % 4;
    return (int)((4 - d) & 3);
}

cudaError_t k1_launch(const K1Params &p, int variant, cudaStream_t st);

// ---------------------------------------------------------------------------
// IR preparation: writes the four shifted copies of each IR row into a slot.
//   dst[r * row_stride + e * phase + j] = (0 <= j - e < n) ? src[r * src_pitch + j - e] : 0
// for j in [0, Lpad). Rows r in [0, rows).
// ---------------------------------------------------------------------------
cudaError_t ir_prep_launch(const float *src, long long src_pitch, long long n, int rows,
                           float *dst, long long row_stride, long long phase, long long Lpad,
                           cudaStream_t st);

// Sets the calling thread's tc_last_error() message.
void set_last_error(const char *msg);

// Counts kernel launches issued by this library.
void count_launch(int n = 1);
uint64_t launches();

}  // namespace tc
