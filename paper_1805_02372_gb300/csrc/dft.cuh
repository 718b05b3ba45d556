// Shared-memory R-point transforms over a ring policy F (a prime field or complex
// floating point): F::T element, F::Tw twiddle, and the two butterflies
// F::dif_bfly(a, b, w): (a, b) <- (a + b, (a - b) w) and
// F::dit_bfly(a, b, w): (a, b) <- (a + b w, a - b w), each up to the representation of
// residues the field keeps (canonical, or lazily reduced).
//
// Forward = decimation in frequency (natural order in, bit-reversed out); inverse =
// decimation in time (bit-reversed in, natural out, unnormalised). Every radix-2
// butterfly is the textbook one: (a, b) -> (a + b, (a - b) w) forward, and
// (a, b) -> (a + b w^-1, a - b w^-1) inverse, with w = w_{2h}^(i mod h) for the stage of
// half-size h. A round holds a group of 2^S elements (i0 + k q, k < 2^S) in registers
// and performs S consecutive stages on it, so shared memory is read and written once
// per S stages. Rounds are ordered so the group stride q is >= 256, 16 or 1.
//
// Twiddles come from stage tables st[h - 1 + j] = w_{2h}^(+-j), j < h (R - 1 entries).
//
// Bank-conflict-free layouts of a tile with R rows and C columns:
//   RowMajor: element (r, c) at slot(r) * C + c, where slot rotates the rows inside each
//             aligned group of four by (r >> 4) (C * sizeof(T) = 32 bytes per row);
//   ColMajor: element (r, c) at c * (R + R/16) + r + (r >> 4) (one word of skew per 16);
//   ColChunk: 32-bit elements, columns of R words whose 16-byte chunks (4 rows) stay whole,
//             swizzled instead of skewed (see the struct).
#pragma once

#include <type_traits>
#include <utility>

#include "ntt_field.cuh"  // compile-time roots of the prime fields (root16_tw)

namespace pa {

// addrs<LQ, K>(i0, c, a): addresses of rows i0 + k 2^LQ (k < K) of column c, for the
// strides the rounds use (LQ = 0 with i0 a multiple of 16 and K <= 16, LQ = 4, LQ >= 8).
struct RowMajor {
    int logC;
    __device__ __forceinline__ int at(int r, int c) const {
        const int slot = (r & ~3) | ((r + (r >> 4)) & 3);
        return (slot << logC) + c;
    }
    template <int LQ, int K>
    __device__ __forceinline__ void addrs(int i0, int c, int (&a)[K]) const {
        if (LQ >= 8) {
            const int b = at(i0, c);
#pragma unroll
            for (int k = 0; k < K; ++k) a[k] = b + (k << (LQ + logC));
        } else {
            const int rot0 = (i0 + (i0 >> 4)) & 3;
            const int b = ((i0 & ~3) << logC) + c;
#pragma unroll
            for (int k = 0; k < K; ++k)
                a[k] = b + ((LQ == 0 ? (k & ~3) : (k << LQ)) << logC) + (((rot0 + k) & 3) << logC);
        }
    }
    static __host__ __device__ __forceinline__ int words(int R, int C) { return R * C; }
};

struct ColMajor {
    int cs;  // column stride R + R/16
    __device__ __forceinline__ int at(int r, int c) const { return c * cs + r + (r >> 4); }
    template <int LQ, int K>
    __device__ __forceinline__ void addrs(int i0, int c, int (&a)[K]) const {
        const int b = at(i0, c);
        const int step = LQ == 0 ? 1 : (1 << LQ) + (1 << (LQ - 4));
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] = b + k * step;
    }
    static __host__ __device__ __forceinline__ int stride(int R) { return R + (R >> 4); }
    static __host__ __device__ __forceinline__ int words(int R, int C) { return C * stride(R); }
};

// Column tile of 32-bit elements (R = 2^logR >= 64 rows) for the contiguous passes of the
// NTT. Rows of a column are stored in 64-byte lines of 16; element (r, c) lies in line
// P = c R/16 + ((r >> 4) ^ fl), fl = ((r >> 8) ^ c) & 1 (adjacent 256-row blocks, and
// adjacent columns, sit in opposite halves of a 128-byte bank row), at chunk
// ((r >> 2) & 3) ^ ((P >> 1) & 3) of the line (the XOR spreads the chunks of eight
// consecutive lines over the eight 16-byte bank groups), word r & 3. The 16-byte chunks of
// four consecutive rows stay whole, so rows move with 16-byte copies and the stride-1
// groups read and write four chunks; the rounds of stride 16 and >= 256 (one word per
// lane), the stride-1 groups and the row copies (one chunk per lane, consecutive lanes on
// consecutive chunks or groups) all meet 32 distinct banks per wavefront. A column set
// starting at a multiple of 128 words and an even column keeps the swizzle, so
// at(r, C0 + c) = C0 R + at(r, c) for even C0 with C0 R a multiple of 128.
struct ColChunk {
    int logR;
    int cs;  // column stride: R words, no padding
    __host__ __device__ __forceinline__ int at(int r, int c) const {
        const int fl = ((r >> 8) ^ c) & 1;
        const int P = (c << (logR - 4)) + ((r >> 4) ^ fl);
        return (P << 4) + ((((r >> 2) & 3) ^ ((P >> 1) & 3)) << 2) + (r & 3);
    }
    // rows i0 + k 2^LQ, k < K, of column c: LQ = 4 (i0 = B + j, j < 16, the K rows within one
    // 256-row block) or LQ >= 8
    template <int LQ, int K>
    __host__ __device__ __forceinline__ void addrs(int i0, int c, int (&a)[K]) const {
        static_assert(LQ == 4 || LQ >= 8, "stride-1 groups use chunks()");
        if constexpr (LQ == 4) {
            // line (i0 >> 4) + k, flipped by fl (constant over k); the chunk XOR takes
            // ((P >> 1) & 3) = h ^ ((k >> 1) & 3), h from the group's first line
            const int j = i0 & 15, B = i0 - j;
            const int fl = ((i0 >> 8) ^ c) & 1;
            const int h = ((((c << (logR - 4)) + (B >> 4)) >> 1) & 3);
            const int q1 = ((j >> 2) & 3) ^ h;
            const int base = (c << logR) + B + (j & 3);
            const int be = base + 16 * fl, bo = base - 16 * fl;
#pragma unroll
            for (int k = 0; k < K; ++k) a[k] = ((k & 1) ? bo : be) + 16 * k + 4 * (q1 ^ ((k >> 1) & 3));
        } else {
            // the chunk XOR is the same for every k; at LQ = 8 fl alternates with k, which
            // moves the line by +-16 words on odd k
            const int a0 = at(i0, c);
            const int d = LQ == 8 ? 16 * (1 - 2 * (((i0 >> 4) ^ (((i0 >> 8) ^ c) & 1)) & 1)) : 0;
#pragma unroll
            for (int k = 0; k < K; ++k) a[k] = a0 + (k << LQ) + ((k & 1) ? d : 0);
        }
    }
    // the four 16-byte chunks of rows i0 .. i0 + 15 (i0 a multiple of 16) of column c
    __host__ __device__ __forceinline__ void chunks(int i0, int c, int (&a)[4]) const {
        const int fl = ((i0 >> 8) ^ c) & 1;
        const int P = (c << (logR - 4)) + ((i0 >> 4) ^ fl);
        const int f = (P >> 1) & 3;
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = (P << 4) + ((u ^ f) << 2);
    }
    static __host__ __device__ __forceinline__ int stride(int R) { return R; }
    static __host__ __device__ __forceinline__ int words(int R, int C) { return C * R; }
    static __host__ __device__ __forceinline__ ColChunk make(int logR) { return ColChunk{logR, 1 << logR}; }
};

// Rows i0 .. i0 + 15 of column c of a tile (a stride-1 group): sixteen words, or for
// ColChunk four 16-byte chunks.
template <class Lay>
struct Rows16 {
    int a[16];
    __device__ __forceinline__ Rows16(const Lay &lay, int i0, int c) { lay.template addrs<0, 16>(i0, c, a); }
    template <class T>
    __device__ __forceinline__ void load(const T *sm, T (&x)[16]) const {
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = sm[a[k]];
    }
    template <class T>
    __device__ __forceinline__ void store(T *sm, const T (&x)[16]) const {
#pragma unroll
        for (int k = 0; k < 16; ++k) sm[a[k]] = x[k];
    }
};
template <>
struct Rows16<ColChunk> {
    int a[4];
    __device__ __forceinline__ Rows16(const ColChunk &lay, int i0, int c) { lay.chunks(i0, c, a); }
    template <class T>
    __device__ __forceinline__ void load(const T *sm, T (&x)[16]) const {
        static_assert(sizeof(T) == 4, "ColChunk holds 32-bit elements");
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint4 v = *reinterpret_cast<const uint4 *>(sm + a[u]);
            x[4 * u] = v.x;
            x[4 * u + 1] = v.y;
            x[4 * u + 2] = v.z;
            x[4 * u + 3] = v.w;
        }
    }
    template <class T>
    __device__ __forceinline__ void store(T *sm, const T (&x)[16]) const {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            *reinterpret_cast<uint4 *>(sm + a[u]) = make_uint4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]);
    }
};

// Stage tables of an R-point transform into shared memory: st[h-1+j] = w_{2h}^(+-j),
// read from a table of the 2^logmax-th roots (first half).
template <class F>
__device__ void load_stage_tables(typename F::Tw *st, const typename F::Tw *__restrict__ tab,
                                  int logR, int logmax) {
    const int R = 1 << logR;
    for (int idx = threadIdx.x; idx < R - 1; idx += blockDim.x) {
        const int lh = 31 - __clz(idx + 1);
        const uint32_t j = static_cast<uint32_t>(idx + 1 - (1 << lh));
        st[idx] = tab[j << (logmax - 1 - lh)];
    }
}

// S decimation-in-frequency stages on x[0 .. 2^S) (element k at row i0 + k q), with the
// field's own butterflies.
template <class F, int S>
__device__ __forceinline__ void dif_group_plain(typename F::T (&x)[1 << S], const typename F::Tw *tw,
                                          int j, int q) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int half = 1 << (S - 1 - s);   // pair distance in k
        const int h = q * half;              // stage half-size in rows
#pragma unroll
        for (int k = 0; k < (1 << S); ++k) {
            if (k & half) continue;
            const typename F::Tw w = tw[h - 1 + j + (k & (half - 1)) * q];
            F::dif_bfly(x[k], x[k + half], w);
        }
    }
}

// The inverse of dif_group_plain (times 2^S) with inverse stage tables.
template <class F, int S>
__device__ __forceinline__ void dit_group_plain(typename F::T (&x)[1 << S], const typename F::Tw *tw,
                                          int j, int q) {
#pragma unroll
    for (int s = S - 1; s >= 0; --s) {
        const int half = 1 << (S - 1 - s);
        const int h = q * half;
#pragma unroll
        for (int k = 0; k < (1 << S); ++k) {
            if (k & half) continue;
            const typename F::Tw w = tw[h - 1 + j + (k & (half - 1)) * q];
            F::dit_bfly(x[k], x[k + half], w);
        }
    }
}

// Fields whose 16th roots of unity are compile-time constants (F::kRoot16).
template <class F, class = void>
struct HasRoot16 {
    static constexpr bool value = false;
};
template <class F>
struct HasRoot16<F, decltype(void(F::kRoot16))> {
    static constexpr bool value = true;
};

// Fields with lazily reduced residues (LazyField: F::kRoom, F::kIoDif, F::kIoDit).
template <class F, class = void>
struct IsLazy {
    static constexpr bool value = false;
};
template <class F>
struct IsLazy<F, decltype(void(F::kRoom))> {
    static constexpr bool value = true;
};

// Bound bookkeeping of the lazy groups. Every value of a group is below B p, B known at
// compile time: LzPlan runs the group's butterflies on the bounds alone (constexpr) and
// records where a value must be lowered and by which step, and the device code expands
// that schedule with `if constexpr` (straight-line code, no bound arithmetic left).
// Lowering B to T (lz_steps): one conditional subtraction of T p when B <= 2T (after one
// of 2T p when B <= 4T), else Shoup's product by 1, which leaves x below 2p. Step codes:
// c > 0 subtracts c p if x >= c p, c = -1 is the product by 1.
struct LzSteps {
    int c[2] = {0, 0};
};
constexpr LzSteps lz_steps(int &B, int T) {
    LzSteps r{};
    if (B <= T) return r;
    int n = 0;
    if (B > 2 * T && B <= 4 * T) {
        r.c[n++] = 2 * T;
        B = 2 * T;
    }
    if (B <= 2 * T) {
        r.c[n++] = T;
        B = T;
        return r;
    }
    r.c[n++] = -1;
    B = 2;
    return r;
}
constexpr void lz_join(LzSteps &a, const LzSteps &b) {
    for (int i = 0; i < 2; ++i)
        if (b.c[i]) {
            if (!a.c[0])
                a.c[0] = b.c[i];
            else
                a.c[1] = b.c[i];
        }
}

// The schedule of one radix-2^S group (DIF or DIT; Q1: the stride-1 group of a field with
// compile-time 16th roots, whose butterflies with w = 1 skip the product). For butterfly k
// (k & half == 0) of stage s: steps on x[k] (pa) and x[k + half] (pb) before it, and K, the
// bound of the subtracted operand (the difference is formed as a - b + K p); after the last
// stage, steps bringing every output below the group's io bound.
template <int S>
struct LzPlan {
    LzSteps pa[4][16], pb[4][16], post[16];
    int K[4][16] = {};
};
constexpr bool lz_w1(int S, bool q1, int k, int half) { return q1 && S == 4 && (k & (half - 1)) == 0; }

template <int S>
constexpr LzPlan<S> lz_plan(bool dif, bool q1, int room, int io_dif, int io_dit) {
    LzPlan<S> p{};
    int b[16] = {};
    const int io = dif ? io_dif : io_dit;
    for (int k = 0; k < (1 << S); ++k) b[k] = io;
    for (int t = 0; t < S; ++t) {
        const int s = dif ? t : S - 1 - t;  // stage, numbered as in dif_group_plain
        const int half = 1 << (S - 1 - s);
        for (int k = 0; k < (1 << S); ++k) {
            if (k & half) continue;
            const int k2 = k + half;
            const bool w1 = lz_w1(S, q1, k, half);
            if (dif || w1) {
                // a + b and a - b + K p below room p: lower the larger operand (at most twice)
                for (int i = 0; i < 2; ++i)
                    if (b[k] + b[k2] > room) {
                        if (b[k] >= b[k2])
                            lz_join(p.pa[s][k], lz_steps(b[k], io_dif));
                        else
                            lz_join(p.pb[s][k], lz_steps(b[k2], io_dif));
                    }
                p.K[s][k] = b[k2];
                const int sum = b[k] + b[k2];
                b[k] = sum;
                b[k2] = w1 ? sum : (dif ? 2 : sum);
                if (!dif) b[k2] = sum;
            } else {
                // t = b w below 2p: a + t and a - t + 2p
                if (b[k] + 2 > room) lz_join(p.pa[s][k], lz_steps(b[k], io_dif));
                p.K[s][k] = 2;
                b[k] = b[k2] = b[k] + 2;
            }
        }
    }
    for (int k = 0; k < (1 << S); ++k) p.post[k] = lz_steps(b[k], io);
    return p;
}

template <class F, int C>
__device__ __forceinline__ void lz_step(typename F::T &x) {
    if constexpr (C > 0)
        x = min(x, x - static_cast<uint32_t>(C) * F::P);
    else if constexpr (C < 0)
        x = F::red2(x);
}

// A lazy group: LzPlan's schedule, expanded at compile time.
template <class F, int S, bool DIF, bool Q1>
struct LzGroup {
    using T = typename F::T;
    using Tw = typename F::Tw;
    static constexpr LzPlan<S> kPlan = lz_plan<S>(DIF, Q1, F::kRoom, F::kIoDif, F::kIoDit);

    template <int s, int k>
    __device__ static __forceinline__ void bfly(T (&x)[1 << S], const Tw *tw, int j, int q) {
        constexpr int half = 1 << (S - 1 - s);
        if constexpr ((k & half) == 0) {
            constexpr int k2 = k + half;
            lz_step<F, kPlan.pa[s][k].c[0]>(x[k]);
            lz_step<F, kPlan.pa[s][k].c[1]>(x[k]);
            lz_step<F, kPlan.pb[s][k].c[0]>(x[k2]);
            lz_step<F, kPlan.pb[s][k].c[1]>(x[k2]);
            constexpr uint32_t KP = static_cast<uint32_t>(kPlan.K[s][k]) * F::P;
            constexpr bool w1 = lz_w1(S, Q1, k, half);
            constexpr int e = Q1 ? (k & (half - 1)) * (8 / half) : 0;
            if constexpr (DIF) {
                const T a = x[k], b = x[k2];
                x[k] = a + b;
                if constexpr (w1) {
                    x[k2] = a + (KP - b);
                } else {
                    Tw w;
                    if constexpr (Q1)
                        w = root16_tw<F, e>();
                    else
                        w = tw[q * half - 1 + j + (k & (half - 1)) * q];
                    x[k2] = F::mul_tw(a + (KP - b), w);
                }
            } else {
                T t;
                if constexpr (w1) {
                    t = x[k2];
                } else {
                    Tw w;
                    if constexpr (Q1)
                        w = root16_tw<F, 16 - e>();
                    else
                        w = tw[q * half - 1 + j + (k & (half - 1)) * q];
                    t = F::mul_tw(x[k2], w);
                }
                const T a = x[k];
                x[k] = a + t;
                x[k2] = a + (KP - t);
            }
        }
    }
    template <int s, int... ks>
    __device__ static __forceinline__ void stage(T (&x)[1 << S], const Tw *tw, int j, int q,
                                                 std::integer_sequence<int, ks...>) {
        (bfly<s, ks>(x, tw, j, q), ...);
    }
    template <int... ts>
    __device__ static __forceinline__ void stages(T (&x)[1 << S], const Tw *tw, int j, int q,
                                                  std::integer_sequence<int, ts...>) {
        (stage<(DIF ? ts : S - 1 - ts)>(x, tw, j, q, std::make_integer_sequence<int, (1 << S)>{}), ...);
    }
    template <int k>
    __device__ static __forceinline__ void post(T (&x)[1 << S]) {
        lz_step<F, kPlan.post[k].c[0]>(x[k]);
        lz_step<F, kPlan.post[k].c[1]>(x[k]);
    }
    template <int... ks>
    __device__ static __forceinline__ void posts(T (&x)[1 << S], std::integer_sequence<int, ks...>) {
        (post<ks>(x), ...);
    }
    __device__ static __forceinline__ void run(T (&x)[1 << S], const Tw *tw, int j, int q) {
        stages(x, tw, j, q, std::make_integer_sequence<int, S>{});
        posts(x, std::make_integer_sequence<int, (1 << S)>{});
    }
};

// dif_group on a lazy field: inputs below kIoDif p, outputs below kIoDif p.
template <class F, int S, bool Q1>
__device__ __forceinline__ void dif_group_lazy(typename F::T (&x)[1 << S], const typename F::Tw *tw,
                                               int j, int q) {
    LzGroup<F, S, true, Q1>::run(x, tw, j, q);
}

// dit_group on a lazy field: inputs below kIoDit p, outputs below kIoDit p.
template <class F, int S, bool Q1>
__device__ __forceinline__ void dit_group_lazy(typename F::T (&x)[1 << S], const typename F::Tw *tw,
                                               int j, int q) {
    LzGroup<F, S, false, Q1>::run(x, tw, j, q);
}

// S decimation-in-frequency stages on x[0 .. 2^S) (element k at row i0 + k q).
template <class F, int S>
__device__ __forceinline__ void dif_group(typename F::T (&x)[1 << S], const typename F::Tw *tw,
                                          int j, int q) {
    if constexpr (IsLazy<F>::value)
        dif_group_lazy<F, S, false>(x, tw, j, q);
    else
        dif_group_plain<F, S>(x, tw, j, q);
}

// The inverse of dif_group (times 2^S) with inverse stage tables.
template <class F, int S>
__device__ __forceinline__ void dit_group(typename F::T (&x)[1 << S], const typename F::Tw *tw,
                                          int j, int q) {
    if constexpr (IsLazy<F>::value)
        dit_group_lazy<F, S, false>(x, tw, j, q);
    else
        dit_group_plain<F, S>(x, tw, j, q);
}

// dif_group / dit_group of a stride-1 group (q = 1, j = 0): the twiddle of stage half-size
// h at position k' < h is w_{2h}^(+-k') = w16^(+-8k'/h), fixed. For S = 4 and a field with
// compile-time roots the twiddles are constants and the butterflies with w = 1 skip the
// product; otherwise the stage tables are read as usual.
template <class F, int S>
__device__ __forceinline__ void dif_group_q1(typename F::T (&x)[1 << S], const typename F::Tw *tw) {
    if constexpr (S == 4 && HasRoot16<F>::value && IsLazy<F>::value) {
        dif_group_lazy<F, 4, true>(x, tw, 0, 1);
    } else if constexpr (S == 4 && HasRoot16<F>::value) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int half = 8 >> s;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (k & half) continue;
                const int e = (k & (half - 1)) * (8 / half);
                if (e == 0)
                    F::dif_bfly1(x[k], x[k + half]);
                else
                    F::dif_bfly(x[k], x[k + half], root16_tw<F>(e));
            }
        }
    } else {
        dif_group<F, S>(x, tw, 0, 1);
    }
}

template <class F, int S>
__device__ __forceinline__ void dit_group_q1(typename F::T (&x)[1 << S], const typename F::Tw *tw) {
    if constexpr (S == 4 && HasRoot16<F>::value && IsLazy<F>::value) {
        dit_group_lazy<F, 4, true>(x, tw, 0, 1);
    } else if constexpr (S == 4 && HasRoot16<F>::value) {
#pragma unroll
        for (int s = 3; s >= 0; --s) {
            const int half = 8 >> s;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (k & half) continue;
                const int e = (k & (half - 1)) * (8 / half);
                if (e == 0)
                    F::dit_bfly1(x[k], x[k + half]);
                else
                    F::dit_bfly(x[k], x[k + half], root16_tw<F>(16 - e));
            }
        }
    } else {
        dit_group<F, S>(x, tw, 0, 1);
    }
}

// One round of S stages over every column: groups g = (block, j), i0 = block 2^S q + j.
// CF: consecutive threads take consecutive columns (RowMajor), else consecutive groups.
template <class F, int S, bool DIF, bool CF, class Lay, int LQ>
__device__ __forceinline__ void round_s(typename F::T *sm, const Lay &lay, int logR, int logC,
                                        int lq_rt, const typename F::Tw *tw) {
    using T = typename F::T;
    const int lq = LQ >= 0 ? LQ : lq_rt;
    const int logG = logR - S;
    const int total = 1 << (logG + logC);
    const int q = 1 << lq;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        int c, g;
        if (CF) {
            c = w & ((1 << logC) - 1);
            g = w >> logC;
        } else {
            g = w & ((1 << logG) - 1);
            c = w >> logG;
        }
        const int j = g & (q - 1);
        const int i0 = ((g >> lq) << (lq + S)) + j;
        T x[1 << S];
        if constexpr (LQ == 0 && S == 4 && std::is_same<Lay, ColChunk>::value) {
            // a stride-1 group of a chunked tile: four 16-byte chunks
            const Rows16<Lay> rows(lay, i0, c);
            rows.load(sm, x);
            if (DIF)
                dif_group_q1<F, S>(x, tw);
            else
                dit_group_q1<F, S>(x, tw);
            rows.store(sm, x);
        } else {
            int a[1 << S];
            if constexpr (LQ >= 0 && !(LQ == 0 && std::is_same<Lay, ColChunk>::value)) {
                lay.template addrs<LQ, (1 << S)>(i0, c, a);
            } else {
#pragma unroll
                for (int k = 0; k < (1 << S); ++k) a[k] = lay.at(i0 + k * q, c);
            }
#pragma unroll
            for (int k = 0; k < (1 << S); ++k) x[k] = sm[a[k]];
            if (LQ == 0) {  // q = 1, j = 0
                if (DIF)
                    dif_group_q1<F, S>(x, tw);
                else
                    dit_group_q1<F, S>(x, tw);
            } else if (DIF) {
                dif_group<F, S>(x, tw, j, q);
            } else {
                dit_group<F, S>(x, tw, j, q);
            }
#pragma unroll
            for (int k = 0; k < (1 << S); ++k) sm[a[k]] = x[k];
        }
    }
}

template <class F, int S, bool DIF, bool CF, class Lay>
__device__ __forceinline__ void round_q(typename F::T *sm, const Lay &lay, int logR, int logC,
                                        int lq, const typename F::Tw *tw) {
    // strides 1, 16, 256 have compile-time addressing (rounds of transforms with R >= 16)
    if (logR >= 4 && lq == 0)
        round_s<F, S, DIF, CF, Lay, 0>(sm, lay, logR, logC, lq, tw);
    else if (logR >= 4 && lq == 4)
        round_s<F, S, DIF, CF, Lay, 4>(sm, lay, logR, logC, lq, tw);
    else if (logR >= 4 && lq == 8)
        round_s<F, S, DIF, CF, Lay, 8>(sm, lay, logR, logC, lq, tw);
    else
        round_s<F, S, DIF, CF, Lay, -1>(sm, lay, logR, logC, lq, tw);
}

template <class F, bool DIF, bool CF, class Lay>
__device__ __forceinline__ void round_any(int S, typename F::T *sm, const Lay &lay, int logR,
                                          int logC, int lq, const typename F::Tw *tw) {
    switch (S) {
        case 1: round_q<F, 1, DIF, CF, Lay>(sm, lay, logR, logC, lq, tw); break;
        case 2: round_q<F, 2, DIF, CF, Lay>(sm, lay, logR, logC, lq, tw); break;
        case 3: round_q<F, 3, DIF, CF, Lay>(sm, lay, logR, logC, lq, tw); break;
        default: round_q<F, 4, DIF, CF, Lay>(sm, lay, logR, logC, lq, tw); break;
    }
    __syncthreads();
}

// Warp-local low rounds (ColMajor tiles of 32-bit elements, R >= 256). The rounds of
// stride 16 and 1 (stage half-sizes 128 .. 1) keep every aligned 256-row block of a column
// to itself, so a warp can take whole (column, block) pairs, one per half-warp, with lane j
// running group j of both rounds, and order the two rounds with __syncwarp instead of a
// barrier of the whole CTA. The two pairs of a warp are (c, b), (c, b + 1), or (c, 0),
// (c + 1, 0) when R = 256: 272 words, 16 banks, apart, so every access of both rounds is
// conflict-free. Pairs are numbered p = (c << (logR - 8)) + b.
template <class F, class Lay>
struct WarpLocal {
    static constexpr bool value = sizeof(typename F::T) == 4 && std::is_same<Lay, ColChunk>::value;
};

template <class F, bool DIF, class Lay>
__device__ __forceinline__ void wl_round16(typename F::T *sm, const Lay &lay, int c, int blk,
                                           int j, const typename F::Tw *tw) {
    typename F::T x[16];
    int a[16];
    lay.template addrs<4, 16>((blk << 8) + j, c, a);
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = sm[a[k]];
    if (DIF)
        dif_group<F, 4>(x, tw, j, 16);
    else
        dit_group<F, 4>(x, tw, j, 16);
#pragma unroll
    for (int k = 0; k < 16; ++k) sm[a[k]] = x[k];
}

template <class F, bool DIF, class Lay>
__device__ __forceinline__ void wl_round1(typename F::T *sm, const Lay &lay, int c, int i0,
                                          const typename F::Tw *tw) {
    typename F::T x[16];
    const Rows16<Lay> rows(lay, i0, c);
    rows.load(sm, x);
    if (DIF)
        dif_group_q1<F, 4>(x, tw);
    else
        dit_group_q1<F, 4>(x, tw);
    rows.store(sm, x);
}

// Runs body(c, blk, l16) for every (column, block) pair of ncols columns, a half-warp per
// pair (pairs beyond the last: on = false, the lanes still reach every __syncwarp).
template <class Body>
__device__ __forceinline__ void wl_pairs(int logR, int ncols, Body body) {
    const int lane = threadIdx.x & 31;
    const int lb = logR - 8;
    const int npairs = ncols << lb;
    for (int p0 = (threadIdx.x >> 5) * 2; p0 < npairs; p0 += (blockDim.x >> 5) * 2) {
        const int p = p0 + (lane >> 4);
        body(p < npairs, p >> lb, p & ((1 << lb) - 1), lane & 15);
    }
}

// The eight low stages of an R-point transform on every column, warp-local (no CTA
// barrier inside; the caller's barriers order them against the other rounds).
template <class F, bool DIF, class Lay>
__device__ __forceinline__ void low_rounds_warp(typename F::T *sm, const Lay &lay, int logR, int ncols,
                                const typename F::Tw *tw) {
    wl_pairs(logR, ncols, [&](bool on, int c, int blk, int j) {
        if (DIF) {
            if (on) wl_round16<F, true, Lay>(sm, lay, c, blk, j, tw);
            __syncwarp();
            if (on) wl_round1<F, true, Lay>(sm, lay, c, (blk << 8) + (j << 4), tw);
        } else {
            if (on) wl_round1<F, false, Lay>(sm, lay, c, (blk << 8) + (j << 4), tw);
            __syncwarp();
            if (on) wl_round16<F, false, Lay>(sm, lay, c, blk, j, tw);
        }
    });
}

// The forward rounds above the low eight stages (stride >= 256), each ending in a barrier.
template <class F, bool CF, class Lay>
__device__ __forceinline__ void dif_top_rounds(typename F::T *sm, const Lay &lay, int logR, int logC,
                                               const typename F::Tw *tw) {
    int done = 0;
    const int s0 = logR & 3;
    if (s0 && logR > 8) {
        round_any<F, true, CF>(s0, sm, lay, logR, logC, logR - s0, tw);
        done = s0;
    }
    for (; done < logR - 8; done += 4) round_any<F, true, CF>(4, sm, lay, logR, logC, logR - done - 4, tw);
}

// The inverse rounds above the low eight stages, in the order dit_columns runs them.
template <class F, bool CF, class Lay>
__device__ __forceinline__ void dit_top_rounds(typename F::T *sm, const Lay &lay, int logR, int logC,
                                               const typename F::Tw *tw) {
    const int s0 = logR & 3;
    for (int done = logR - 8; done > s0; done -= 4)
        round_any<F, false, CF>(4, sm, lay, logR, logC, logR - done, tw);
    if (s0 && logR > 8) round_any<F, false, CF>(s0, sm, lay, logR, logC, logR - s0, tw);
}

// Forward R-point DIF on every column: a top round of logR mod 4 stages (if any), then
// rounds of four stages down to the stage of half-size 1.
template <class F, bool CF, class Lay>
__device__ __forceinline__ void dif_columns(typename F::T *sm, const Lay &lay, int logR, int logC,
                            const typename F::Tw *tw) {
    if constexpr (!CF && WarpLocal<F, Lay>::value) {
        if (logR >= 8) {
            dif_top_rounds<F, CF>(sm, lay, logR, logC, tw);
            low_rounds_warp<F, true>(sm, lay, logR, 1 << logC, tw);
            __syncthreads();
            return;
        }
    }
    int done = 0;
    const int s0 = logR & 3;
    if (s0) {
        round_any<F, true, CF>(s0, sm, lay, logR, logC, logR - s0, tw);
        done = s0;
    }
    for (; done < logR; done += 4) round_any<F, true, CF>(4, sm, lay, logR, logC, logR - done - 4, tw);
}

// Inverse R-point DIT on every column: the rounds of dif_columns in reverse order.
template <class F, bool CF, class Lay>
__device__ __forceinline__ void dit_columns(typename F::T *sm, const Lay &lay, int logR, int logC,
                            const typename F::Tw *tw) {
    if constexpr (!CF && WarpLocal<F, Lay>::value) {
        if (logR >= 8) {
            low_rounds_warp<F, false>(sm, lay, logR, 1 << logC, tw);
            __syncthreads();
            dit_top_rounds<F, CF>(sm, lay, logR, logC, tw);
            return;
        }
    }
    const int s0 = logR & 3;
    for (int done = logR; done > s0; done -= 4)
        round_any<F, false, CF>(4, sm, lay, logR, logC, logR - done, tw);
    if (s0) round_any<F, false, CF>(s0, sm, lay, logR, logC, logR - s0, tw);
}

// dif_columns without its first stage (half-size R/2), for a caller that ran that stage
// while loading the tile: the remaining stages, half-sizes R/4 .. 1, in rounds of
// (logR - 1) mod 4 (if any) and then four stages.
template <class F, bool CF, class Lay>
__device__ __forceinline__ void dif_columns_after_first(typename F::T *sm, const Lay &lay, int logR, int logC,
                                        const typename F::Tw *tw) {
    const int rem = logR - 1, s0 = rem & 3;
    int done = 0;
    if (s0) {
        round_any<F, true, CF>(s0, sm, lay, logR, logC, rem - s0, tw);
        done = s0;
    }
    for (; done < rem; done += 4) round_any<F, true, CF>(4, sm, lay, logR, logC, rem - done - 4, tw);
}

// dit_columns without its last stage (half-size R/2), for a caller that runs that stage on
// the rows it writes out: stages of half-size 1 .. R/4, in the reverse order of
// dif_columns_after_first.
template <class F, bool CF, class Lay>
__device__ __forceinline__ void dit_columns_but_last(typename F::T *sm, const Lay &lay, int logR, int logC,
                                     const typename F::Tw *tw) {
    const int rem = logR - 1, s0 = rem & 3;
    for (int done = rem; done > s0; done -= 4)
        round_any<F, false, CF>(4, sm, lay, logR, logC, rem - done, tw);
    if (s0) round_any<F, false, CF>(s0, sm, lay, logR, logC, rem - s0, tw);
}

// The forward rounds of dif_columns except the last (the four stages of half-size 8..1),
// and the inverse rounds of dit_columns except the first: the caller runs those two in
// registers around the pointwise product (product_round). Needs logR >= 4.
template <class F, bool CF, class Lay>
__device__ __forceinline__ void dif_columns_head(typename F::T *sm, const Lay &lay, int logR, int logC,
                                 const typename F::Tw *tw) {
    int done = 0;
    const int s0 = logR & 3;
    if (s0) {
        round_any<F, true, CF>(s0, sm, lay, logR, logC, logR - s0, tw);
        done = s0;
    }
    for (; done < logR - 4; done += 4)
        round_any<F, true, CF>(4, sm, lay, logR, logC, logR - done - 4, tw);
}

template <class F, bool CF, class Lay>
__device__ __forceinline__ void dit_columns_tail(typename F::T *sm, const Lay &lay, int logR, int logC,
                                 const typename F::Tw *tw) {
    const int s0 = logR & 3;
    for (int done = logR - 4; done > s0; done -= 4)
        round_any<F, false, CF>(4, sm, lay, logR, logC, logR - done, tw);
    if (s0) round_any<F, false, CF>(s0, sm, lay, logR, logC, logR - s0, tw);
}

// One group of 16 consecutive rows from i0 of key column cx and window column cy: the last
// four forward stages of both, the pointwise product Mul, the first four inverse stages of
// the product, written over the window column.
template <class F, class Lay, class Mul>
__device__ __forceinline__ void product_group(typename F::T *sm, const Lay &lay, int i0, int cx, int cy,
                                              const typename F::Tw *twf, const typename F::Tw *twi,
                                              Mul mul) {
    using T = typename F::T;
    T x[16], y[16];
    const Rows16<Lay> rx(lay, i0, cx), ry(lay, i0, cy);
    rx.load(sm, x);
    ry.load(sm, y);
    dif_group_q1<F, 4>(x, twf);
    dif_group_q1<F, 4>(y, twf);
#pragma unroll
    for (int k = 0; k < 16; ++k) y[k] = mul(x[k], y[k]);
    dit_group_q1<F, 4>(y, twi);
    ry.store(sm, y);
}

// One group of 16 consecutive rows from i0: the last four forward stages of key column cx
// and window column cy, and column cz += their pointwise product Mul (field addition Add).
template <class F, class Lay, class Mul, class Add>
__device__ __forceinline__ void product_acc_group(typename F::T *sm, const Lay &lay, int i0, int cx,
                                                  int cy, int cz, const typename F::Tw *twf, Mul mul,
                                                  Add add) {
    using T = typename F::T;
    T x[16], y[16], z[16];
    const Rows16<Lay> rx(lay, i0, cx), ry(lay, i0, cy), rz(lay, i0, cz);
    rx.load(sm, x);
    ry.load(sm, y);
    dif_group_q1<F, 4>(x, twf);
    dif_group_q1<F, 4>(y, twf);
#pragma unroll
    for (int k = 0; k < 16; ++k) y[k] = mul(x[k], y[k]);
    rz.load(sm, z);
#pragma unroll
    for (int k = 0; k < 16; ++k) z[k] = add(z[k], y[k]);
    rz.store(sm, z);
}

// For each of C column pairs (key column c, window column C + c): product_group on every
// group of 16 rows.
template <class F, class Lay, class Mul>
__device__ __forceinline__ void product_round(typename F::T *sm, const Lay &lay, int logR, int logC,
                              const typename F::Tw *twf, const typename F::Tw *twi, Mul mul) {
    const int logG = logR - 4;
    const int C = 1 << logC;
    const int total = 1 << (logG + logC);
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int g = w & ((1 << logG) - 1), c = w >> logG;
        product_group<F>(sm, lay, g << 4, c, C + c, twf, twi, mul);
    }
    __syncthreads();
}

// For each of C column pairs: product_acc_group into the accumulator column acc_col0 + c.
template <class F, class Lay, class Mul, class Add>
__device__ __forceinline__ void product_acc_round(typename F::T *sm, const Lay &lay, int logR, int logC,
                                  int acc_col0, const typename F::Tw *twf, Mul mul, Add add) {
    const int logG = logR - 4;
    const int C = 1 << logC;
    const int total = 1 << (logG + logC);
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int g = w & ((1 << logG) - 1), c = w >> logG;
        product_acc_group<F>(sm, lay, g << 4, c, C + c, acc_col0 + c, twf, mul, add);
    }
    __syncthreads();
}

// Forward transforms of C key columns and C window columns (column C + c), their pointwise
// products, and the inverse transforms of the products over the window columns: for
// R >= 256 (32-bit elements) the stages below half-size 256 of both spectra, the product
// and the first inverse stages run warp-local per (column, block) pair, between the
// CTA-wide top rounds.
template <class F, class Lay, class Mul>
__device__ __forceinline__ void product_columns(typename F::T *sm, const Lay &lay, int logR, int logC,
                                const typename F::Tw *twf, const typename F::Tw *twi, Mul mul) {
    const int C = 1 << logC;
    if constexpr (WarpLocal<F, Lay>::value) {
        if (logR >= 8) {
            dif_top_rounds<F, false>(sm, lay, logR, logC + 1, twf);
            wl_pairs(logR, C, [&](bool on, int c, int blk, int j) {
                if (on) {
                    wl_round16<F, true, Lay>(sm, lay, c, blk, j, twf);
                    wl_round16<F, true, Lay>(sm, lay, C + c, blk, j, twf);
                }
                __syncwarp();
                if (on) product_group<F>(sm, lay, (blk << 8) + (j << 4), c, C + c, twf, twi, mul);
                __syncwarp();
                if (on) wl_round16<F, false, Lay>(sm, lay, C + c, blk, j, twi);
            });
            __syncthreads();
            dit_top_rounds<F, false>(sm + C * lay.cs, lay, logR, logC, twi);
            return;
        }
    }
    dif_columns_head<F, false>(sm, lay, logR, logC + 1, twf);
    product_round<F>(sm, lay, logR, logC, twf, twi, mul);
    dit_columns_tail<F, false>(sm + C * lay.cs, lay, logR, logC, twi);
}

// Forward transforms of C key and C window columns and acc[c] += their pointwise products
// (accumulator column acc_col0 + c), warp-local below the top rounds as in product_columns.
template <class F, class Lay, class Mul, class Add>
__device__ __forceinline__ void product_acc_columns(typename F::T *sm, const Lay &lay, int logR, int logC,
                                    int acc_col0, const typename F::Tw *twf, Mul mul, Add add) {
    const int C = 1 << logC;
    if constexpr (WarpLocal<F, Lay>::value) {
        if (logR >= 8) {
            dif_top_rounds<F, false>(sm, lay, logR, logC + 1, twf);
            wl_pairs(logR, C, [&](bool on, int c, int blk, int j) {
                if (on) {
                    wl_round16<F, true, Lay>(sm, lay, c, blk, j, twf);
                    wl_round16<F, true, Lay>(sm, lay, C + c, blk, j, twf);
                }
                __syncwarp();
                if (on)
                    product_acc_group<F>(sm, lay, (blk << 8) + (j << 4), c, C + c, acc_col0 + c, twf,
                                         mul, add);
            });
            __syncthreads();
            return;
        }
    }
    dif_columns_head<F, false>(sm, lay, logR, logC + 1, twf);
    product_acc_round<F>(sm, lay, logR, logC, acc_col0, twf, mul, add);
}

}  // namespace pa
