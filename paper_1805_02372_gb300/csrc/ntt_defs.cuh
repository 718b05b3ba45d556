// Shared definitions of the exact transform path: limits, work-item encoding, the
// launch's tile and block descriptors, the per-device twiddle tables and the
// per-field launch entry points (each prime field's persistent kernel is compiled
// in a translation unit of its own).
#pragma once

#include <algorithm>
#include <stdint.h>

#include "common.cuh"
#include "ntt_field.cuh"
#include "tiles.cuh"

namespace pa {

constexpr int kLogSmallMax = 12;      // one-CTA transforms up to 2^12
constexpr int kLogR1Max = 11;         // strided-pass columns of at most 2^11 points
constexpr int kThreads = 512;
// Two CTAs of 512 threads per SM for the 32-bit field (<= 64 registers), one for 64-bit.
template <class F>
constexpr int kMinBlocks = sizeof(typename F::T) == 4 ? 2 : 1;

// Transform-domain accumulation limits: tile pairs of one block (host tables) and
// spectra bytes of one block (about 22 bytes per key bit with l = 10%: n = 3e9 holds 67 GB).
constexpr uint64_t kFdMaxPairs = uint64_t(1) << 22;
constexpr uint64_t kFdMaxBytes = uint64_t(96) << 30;
// Segmented accumulation (blocks beyond the resident cap): spectra of one segment at most
// kSegMaxBytes by default (pa_opts.seg_cap_gib overrides), at most kSegMax segments.
constexpr uint64_t kSegMaxBytes = uint64_t(32) << 30;
constexpr uint64_t kSegMax = 1u << 16;

// Work-item types (bits 60..63 of an item; bits 32..59 tile index, 0..31 sub-index).
enum : uint32_t {
    IT_SMALL = 0,
    IT_P1 = 1,
    IT_P2 = 2,
    IT_P3 = 3,
    IT_FD_P1 = 4,
    IT_FD_P2 = 5,
    IT_FD_SUM = 6,
    IT_FD_P3 = 7,
    IT_FD_STREAM = 8,
    IT_FD_OUTER = 9,
    IT_FD_INV2 = 10
};

// A transform of a launch: a standard tile pair, an fd spectrum or an fd output sum.
struct NttTile {
    TilePair p;       // geometry (fd key spectrum: its key tile; window: a pair with
                      // that offset; output sum: the pair (I, 0))
    uint64_t ws_off;  // element offset of the spectrum (standard: the key spectrum, the
                      // window spectrum follows)
    uint64_t scale;   // final scale as the bits of F::Tw
    uint32_t logN, logR1, logR2;
    uint32_t g1;      // pass-1 column groups (per input)
    uint32_t g2;      // pass-2 row groups
    uint32_t logC1;   // pass-1/3 columns per item (log2)
    uint32_t logC2;   // pass-2 rows per item (log2)
    uint32_t which;   // fd spectra: 0 key tile, 1 seed window
    uint32_t fd;      // fd spectra and sums: index of the fd block
    uint32_t out;     // fd sums: output tile index I
    uint32_t jlo, jhi;  // fd sums: the key tiles J in [jlo, jhi) this sum covers
    // Outer convolutions (tiles of IT_FD_OUTER items, one per sum group and output slice):
    // the sums Z_I = sum_J X_J W_{d0+I-J} of output tiles out .. out + nout - 1 over key
    // tiles [jlo, jhi) are, bin by bin, a convolution over the tile index, computed with
    // transforms of 2^logT points over it, 2^logCo bins per item; windows from index wb.
    uint32_t logT, logCo, nout;
    int32_t wb;
    uint32_t octr;    // outer tiles: tile index of the sum tile of output `out` (the slice's
                      // sums follow it); sum tiles of an outer group: tile index of their
                      // outer tile, whose pass-1 counter counts the outer items done
    uint32_t pad;
};

// Outer convolutions: transform sizes up to 2^kLogOuterMax over the tile index.
constexpr int kLogOuterMax = 9;
// Bins per outer item (log2): the forward tile holds 2 x 2^logCo columns and the product
// tile 2^logCo, 3 x 2^(logT + logCo) elements in all (at most 12288 words of 32 bits).
__host__ __device__ inline int outer_log_cols(int logT, size_t elem) {
    const int budget = elem == 4 ? 12 : 11;  // log2 of T x C
    const int minc = elem == 4 ? 3 : 2;      // rows of at least 32 bytes
    return budget - logT > minc ? budget - logT : minc;
}

// One block under transform-domain accumulation.
// Streamed blocks (one output tile) skip the separate forward pass 2: their sum items
// run it on the key-tile and window rows they read.
struct FdBlock {
    uint64_t x_off;   // element offset of key spectrum 0 (key spectra at stride N)
    uint64_t w_off;   // element offset of window spectrum 0 (stride N)
    uint64_t wmap;    // first entry of the block's P x Q window-index table
    uint32_t Q;       // key tiles
    uint32_t nfwd2;   // forward pass-2 items of the block (all precede every sum)
    uint32_t nfwd1;   // forward pass-1 items of the block (streamed sums wait for all)
    uint32_t P;       // output tiles (per group of sums: sum tiles g P .. g P + P - 1)
    uint32_t consec;  // 1: the window of (I, J) is wmap[0][0] + I - J (equal key and output
                      // tiles: offsets (I - J) M), so sums can slide along J
    uint32_t outer;   // 1: the sums are outer convolutions (IT_FD_OUTER, then IT_FD_INV2)
    uint32_t pad;
};

// Four-step split N = R1 R2 of a two-pass transform: R1 = 2^ceil(logN/2) up to 2^22, and
// above that R1 = 2^11 with the contiguous pass taking the rest (R2 = 2^12 at 2^23), so
// that a pass-1 item keeps its 2^11-point columns.
__host__ __device__ inline void split_r(int logN, int *logR1, int *logR2) {
    *logR1 = (logN + 1) / 2 < kLogR1Max ? (logN + 1) / 2 : kLogR1Max;
    *logR2 = logN - *logR1;
}

// Columns per pass-1/3 item and rows per pass-2 item (log2): at least one 32-byte row
// segment, and enough to give a 512-thread CTA about 8192 (32-bit) elements per item in
// pass 2 and 16384 in passes 1 and 3 (two radix-16 groups per thread and round, for
// latency hiding; pass-2 items hold two or three column sets and stay at 8192).
inline void pass_columns(int logN, size_t elem, int *logC1, int *logC2) {
    int logR1 = 0, logR2 = 0;
    split_r(logN, &logR1, &logR2);
    const int logS = logN - logR1;
    const int target = elem == 4 ? 13 : 12;
    int c1 = std::max(elem == 4 ? 3 : 2, target + 1 - logR1);
    int c2 = std::max(elem == 4 ? 2 : 1, target - logR2);
    *logC1 = std::min(c1, logS);
    *logC2 = std::min(c2, logR1);
}

// Output tiles per transform-domain sum item (ntt_kernel.cuh, body_sum4_inv_last); each
// item covers 2048 elements of every one of them.
constexpr int kSum4Out = 4;

// Words of the pass-1 twiddle tables of a forward item (p1tw_build in ntt_kernel.cuh):
// per segment column 32 + R1/32 entries, and 32 + R1/32 shared ones (needs R1 >= 32).
__host__ __device__ constexpr int p1tw_words(int logR1, int seglog) {
    return ((1 << seglog) + 1) * (32 + (1 << (logR1 - 5)));
}

// Per-device tables: fwd[e] = w^e, inv[e] = w^-e for e < 2^(kLogMax-1), w of order 2^kLogMax.
struct Tables {
    void *fwd = nullptr, *inv = nullptr;
    void *stage = nullptr;  // compact stage tables, see stage_table()
};
constexpr int kStageBlock = 4096;  // entries per (direction, log2 R) block

// The tables of a field on the current device, built and uploaded on first use.
int ntt_tables(int field, Tables *out);

// One persistent launch of a field's work list (ntt_f28.cu, ntt_f29.cu, ntt_f31.cu,
// ntt_f64.cu).
#define PA_NTT_LAUNCH_ARGS const NttLayout &lay, void *ws, const BlockPtrs *blks, \
    const BlockPtrs &one, int *status, Prof *prof, cudaStream_t s
int ntt_launch_f28(PA_NTT_LAUNCH_ARGS);
int ntt_launch_f29(PA_NTT_LAUNCH_ARGS);
int ntt_launch_f31(PA_NTT_LAUNCH_ARGS);
int ntt_launch_f64(PA_NTT_LAUNCH_ARGS);

}  // namespace pa
