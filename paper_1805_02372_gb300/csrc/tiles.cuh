// Tile geometry shared by the transform paths (Sec. 3, Eq. Ti / Eq. Tij with the
// output-column split): one key tile x[j0, j0+L) against one output tile y[i0, i0+M).
// With a[t] = x[j0+t] and w[u] = s[n-1+i0-j0-L+u], output row i0+v is coefficient
// L+v of the linear convolution a*w; a cyclic convolution of size N >= L+M holds it
// unaliased. Tiles' bits are XORed into the output (Eq. finalkey).
#pragma once

#include <stdint.h>

#include <vector>

#include "internal.h"

namespace pa {

struct TilePair {
    int64_t key_bit0;   // first key bit of the tile
    uint64_t key_len;   // valid key bits in the tile
    int64_t win_bit0;   // seed bit of window position 0 (may be negative)
    uint64_t win_len;   // window positions read (beyond: 0)
    uint64_t out_bit0;  // first output row of the tile (multiple of 64)
    uint32_t out_len;   // valid output rows
    uint32_t K0;        // convolution index of output row out_bit0
    uint32_t blk;       // block index (batched launches)
    uint32_t pad;
};

struct BlockPtrs {
    const uint32_t *key32;
    const uint32_t *seed32;
    uint32_t *out32;
    uint64_t n, m;
};


__device__ __forceinline__ uint32_t get_bit(const uint32_t *__restrict__ v, uint64_t pos) {
    return (__ldg(v + (pos >> 5)) >> (pos & 31)) & 1u;
}

__device__ __forceinline__ uint32_t key_bit(const TilePair &pr, const BlockPtrs &bp, uint64_t t) {
    return t < pr.key_len ? get_bit(bp.key32, uint64_t(pr.key_bit0) + t) : 0u;
}

__device__ __forceinline__ uint32_t win_bit(const TilePair &pr, const BlockPtrs &bp, uint64_t u) {
    if (u >= pr.win_len) return 0u;
    const int64_t p = pr.win_bit0 + static_cast<int64_t>(u);
    if (p < 0 || static_cast<uint64_t>(p) >= bp.n + bp.m - 1) return 0u;
    return get_bit(bp.seed32, static_cast<uint64_t>(p));
}


__device__ __forceinline__ BlockPtrs pick(const BlockPtrs *blks, const BlockPtrs &one, uint32_t b) {
    return blks ? blks[b] : one;
}

// Pair descriptors of one block, in (output tile, key tile) order, for output tiles
// [I0, I1) and key tiles [J0, J1) (I1 = 0: all output tiles; J1 = 0: all key tiles).
inline void make_pairs(uint64_t n, uint64_t m, const TransformCfg &c, uint32_t blk,
                       std::vector<TilePair> *out, uint64_t I0 = 0, uint64_t I1 = 0,
                       uint64_t J0 = 0, uint64_t J1 = 0) {
    if (!I1) I1 = c.tiles_out;
    if (!J1) J1 = c.tiles_in;
    for (uint64_t I = I0; I < I1; ++I) {
        for (uint64_t J = J0; J < J1; ++J) {
            TilePair p{};
            const uint64_t i0 = I * c.M, j0 = J * c.L;
            p.key_bit0 = static_cast<int64_t>(j0);
            p.key_len = (n - j0 < c.L) ? n - j0 : c.L;
            p.K0 = static_cast<uint32_t>(c.L);
            p.win_bit0 = static_cast<int64_t>(n) - 1 + static_cast<int64_t>(i0) -
                         static_cast<int64_t>(j0) - static_cast<int64_t>(c.L);
            p.win_len = c.L + c.M;
            p.out_bit0 = i0;
            p.out_len = static_cast<uint32_t>((m - i0 < c.M) ? m - i0 : c.M);
            p.blk = blk;
            out->push_back(p);
        }
    }
}

}  // namespace pa
