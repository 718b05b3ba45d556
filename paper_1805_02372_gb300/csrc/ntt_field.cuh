// Prime fields of the exact transform path.
//
// Every convolution coefficient the path reads is a count of at most n bit products,
// so for n < p the residue IS the integer and its low bit is the hash bit.
// F29: p = 7 * 2^26 + 1 (2-adicity 26), for n < p. Residues are kept lazily in
//      [0, 4p) (4p < 2^31): a butterfly needs one conditional subtraction instead of
//      three (Harvey's lazy butterflies for Shoup multiplication); values are made
//      canonical only when the hash bit is taken.
// F28: p = 5 * 2^25 + 1 (2-adicity 25), as F29 for n < p, with room for 25p in 32 bits:
//      the rounds of a transform subtract far less often (LazyField).
// F31: p = 15 * 2^27 + 1 (2-adicity 27), canonical residues, for n < p.
//      Twiddles carry Shoup quotients (one high-half multiply per twiddle product);
//      the pointwise product is a Montgomery product.
// F64: p = 2^64 - 2^32 + 1 (2-adicity 32); products reduced with 2^64 = 2^32 - 1 mod p.
#pragma once

#include <stdint.h>

namespace pa {

// Compile-time modular arithmetic for the 32-bit fields (p < 2^32, products fit 64 bits).
constexpr uint64_t cx_powmod(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1;
    a %= p;
    while (e) {
        if (e & 1) r = r * a % p;
        a = a * a % p;
        e >>= 1;
    }
    return r;
}
// The primitive 16th root of unity the twiddle tables use: g^((p-1)/16) for the smallest
// generator g >= 2 (g^((p-1)/f) != 1 for f = 2 and the odd primes f1, f2 of p - 1; f2 = 0:
// none), the same search as the host tables' root of order 2^23, whose 2^19-th power it is.
constexpr uint32_t cx_root16(uint64_t p, uint64_t f1, uint64_t f2) {
    for (uint64_t g = 2;; ++g) {
        if (cx_powmod(g, (p - 1) / 2, p) == 1) continue;
        if (cx_powmod(g, (p - 1) / f1, p) == 1) continue;
        if (f2 && cx_powmod(g, (p - 1) / f2, p) == 1) continue;
        return static_cast<uint32_t>(cx_powmod(g, (p - 1) / 16, p));
    }
}

// Inverse of an odd 32-bit modulus mod 2^32 (Newton iteration, 3 -> 6 -> ... -> 96 bits).
constexpr uint32_t inverse_mod_2_32(uint32_t p) {
    uint32_t x = p;
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    return x;
}

struct F31 {
    using T = uint32_t;
    struct Tw {
        uint32_t w, q;  // value and Shoup quotient floor(w * 2^32 / p)
    };
    static constexpr uint32_t P = 2013265921u;
    static constexpr int kTwoAdicity = 27;
    static constexpr uint32_t PINV = inverse_mod_2_32(2013265921u);  // p^-1 mod 2^32
    static_assert(PINV * 2013265921u == 1u, "Montgomery inverse");

    __device__ static __forceinline__ T add(T a, T b) {
        T s = a + b;
        return min(s, s - P);
    }
    __device__ static __forceinline__ T sub(T a, T b) {
        T d = a + (P - b);
        return min(d, d - P);
    }
    __device__ static __forceinline__ T mul_tw(T a, Tw w) {
        uint32_t q = __umulhi(a, w.q);
        uint32_t r = a * w.w - q * P;  // in [0, 2p)
        return min(r, r - P);
    }
    // a * b * 2^-32 mod p.
    __device__ static __forceinline__ T mont(T a, T b) {
        uint32_t lo = a * b, hi = __umulhi(a, b);
        uint32_t mq = lo * PINV;
        uint32_t r = hi - __umulhi(mq, P);  // (ab - mq p) / 2^32, in (-p, p)
        return static_cast<int32_t>(r) < 0 ? r + P : r;
    }
    __device__ static __forceinline__ uint32_t low_bit(T a) { return a & 1u; }
    // A twiddle in the form mul_full expects: w * 2^32 mod p (Montgomery form).
    static constexpr uint32_t R_MOD = static_cast<uint32_t>((uint64_t(1) << 32) % 2013265921u);
    static constexpr uint32_t R_Q = static_cast<uint32_t>((uint64_t(R_MOD) << 32) / 2013265921u);
    __device__ static __forceinline__ T full_form(Tw w) {
        Tw r;
        r.w = R_MOD;
        r.q = R_Q;
        return mul_tw(w.w, r);
    }
    // a * w for w in full form (no precomputed quotient): Montgomery product.
    __device__ static __forceinline__ T mul_full(T a, T wf) { return mont(a, wf); }
    // next twiddle in full form: wf * step
    __device__ static __forceinline__ T step_full(T wf, Tw step) { return mul_tw(wf, step); }
    __device__ static __forceinline__ Tw neg_tw(Tw w) {
        // -w mod p with its own quotient: floor((p - w) 2^32 / p) = 2^32 - 1 - q for w != 0.
        Tw r;
        r.w = w.w ? P - w.w : 0u;
        r.q = w.w ? 0xFFFFFFFFu - w.q : 0u;
        return r;
    }
    __device__ static __forceinline__ void dif_bfly(T &a, T &b, Tw w) {
        const T s = add(a, b);
        b = mul_tw(sub(a, b), w);
        a = s;
    }
    __device__ static __forceinline__ void dit_bfly(T &a, T &b, Tw w) {
        const T t = mul_tw(b, w);
        b = sub(a, t);
        a = add(a, t);
    }
    // the same butterflies with w = 1
    __device__ static __forceinline__ void dif_bfly1(T &a, T &b) {
        const T s = add(a, b);
        b = sub(a, b);
        a = s;
    }
    __device__ static __forceinline__ void dit_bfly1(T &a, T &b) {
        const T t = b;
        b = sub(a, t);
        a = add(a, t);
    }
    static constexpr uint32_t kRoot16 = cx_root16(2013265921u, 3, 5);
};

// Lazily reduced residues of a prime p < 2^29 (Harvey, "Faster arithmetic for
// number-theoretic transforms", 2014): Shoup's product of any 32-bit a by a canonical
// twiddle w with quotient floor(w 2^32 / p) lies in [0, 2p), so values need not be
// canonical between operations, only below 2^32. The single-operation butterflies below
// keep them in [0, 4p) with one conditional subtraction each. The radix-2^S rounds of
// dft.cuh instead track, at compile time, a bound B p on every value of a group and
// subtract only where a sum or difference could pass kRoom p (the largest multiple of p
// below 2^32): values between forward rounds are below kIoDif p, between inverse rounds
// below kIoDit p. Every consumer of an inverse round's output is a product (Shoup or
// Montgomery: any 32-bit input) or another inverse round, so kIoDit may exceed 4.
//   P = 7 * 2^26 + 1 (29-bit, 2-adicity 26): kRoom 9, kIoDit 4;
//   P = 5 * 2^25 + 1 (28-bit, 2-adicity 25): kRoom 25, kIoDit 12 (an inverse round of four
//   stages adds at most 8p, and 12 + 8 <= 25).
template <uint32_t kP, int kAdic, uint32_t kOdd, int kDitIo>
struct LazyField {
    using T = uint32_t;
    using Tw = F31::Tw;  // value and Shoup quotient
    static constexpr uint32_t P = kP;
    static constexpr uint32_t P2 = 2 * P, P4 = 4 * P;
    static constexpr int kTwoAdicity = kAdic;
    static constexpr uint32_t PINV = inverse_mod_2_32(kP);
    static_assert(PINV * kP == 1u, "Montgomery inverse");
    static_assert(uint64_t(8) * kP < (uint64_t(1) << 32), "8p fits 32 bits");
    static constexpr int kRoom = static_cast<int>((uint64_t(1) << 32) / kP);
    static constexpr int kIoDif = 4, kIoDit = kDitIo;
    static_assert(kIoDit >= 4 && kIoDit + 2 <= kRoom, "an inverse stage adds 2p at most");
    // floor(2^32 / p): the Shoup quotient of the twiddle 1
    static constexpr uint32_t kShoup1 = static_cast<uint32_t>((uint64_t(1) << 32) / kP);

    // [0, 4p) + [0, 4p) -> [0, 4p)
    __device__ static __forceinline__ T add(T a, T b) {
        const T s = a + b;
        return min(s, s - P4);
    }
    __device__ static __forceinline__ T sub(T a, T b) {
        const T d = a + (P4 - b);
        return min(d, d - P4);
    }
    // any 32-bit a -> [0, 2p)
    __device__ static __forceinline__ T mul_tw(T a, Tw w) {
        const uint32_t q = __umulhi(a, w.q);
        return a * w.w - q * P;
    }
    // any 32-bit a -> [0, 2p) (Shoup's product by 1)
    __device__ static __forceinline__ T red2(T a) { return a - __umulhi(a, kShoup1) * P; }
    // a b 2^-32: (ab - mq p) / 2^32 lies in (-p, ab / 2^32), plus p: (0, p + ab / 2^32),
    // e.g. below 2.75p (29-bit p) or 1.7p (28-bit p) for a, b < 4p, below 3p for any
    // 32-bit a and b < 2p
    __device__ static __forceinline__ T mont(T a, T b) {
        const uint32_t lo = a * b, hi = __umulhi(a, b);
        const uint32_t mq = lo * PINV;
        return hi - __umulhi(mq, P) + P;
    }
    // canonical residue of a in [0, 4p), then its low bit
    __device__ static __forceinline__ uint32_t low_bit(T a) {
        a = min(a, a - P2);
        a = min(a, a - P);
        return a & 1u;
    }
    static constexpr uint32_t R_MOD = static_cast<uint32_t>((uint64_t(1) << 32) % kP);
    static constexpr uint32_t R_Q = static_cast<uint32_t>((uint64_t(R_MOD) << 32) / kP);
    // w 2^32 mod p in [0, 2p)
    __device__ static __forceinline__ T full_form(Tw w) {
        Tw r;
        r.w = R_MOD;
        r.q = R_Q;
        return mul_tw(w.w, r);
    }
    // a < 2^32 times wf < 2p: (0, 3p) after the Montgomery reduction
    __device__ static __forceinline__ T mul_full(T a, T wf) { return mont(a, wf); }
    __device__ static __forceinline__ T step_full(T wf, Tw step) { return mul_tw(wf, step); }
    __device__ static __forceinline__ Tw neg_tw(Tw w) {
        Tw r;
        r.w = w.w ? P - w.w : 0u;
        r.q = w.w ? 0xFFFFFFFFu - w.q : 0u;
        return r;
    }
    // Gentleman-Sande: (a + b, (a - b) w); a, b in [0, 4p) -> [0, 4p), [0, 2p)
    __device__ static __forceinline__ void dif_bfly(T &a, T &b, Tw w) {
        const T s = a + b;
        b = mul_tw(a + (P4 - b), w);
        a = min(s, s - P4);
    }
    // Cooley-Tukey: (a + b w, a - b w); a < kIoDit p -> both below kIoDit p
    __device__ static __forceinline__ void dit_bfly(T &a, T &b, Tw w) {
        const T t = mul_tw(b, w);
        const T a2 = min(a, a - P2);
        a = a2 + t;
        b = a2 + (P2 - t);
    }
    // the same butterflies with w = 1 (no product: a conditional subtraction keeps the
    // ranges of the general ones)
    __device__ static __forceinline__ void dif_bfly1(T &a, T &b) {
        const T s = a + b, d = a + (P4 - b);
        b = min(d, d - P4);
        a = min(s, s - P4);
    }
    __device__ static __forceinline__ void dit_bfly1(T &a, T &b) {
        const T t = min(b, b - P2);
        const T a2 = min(a, a - P2);
        a = a2 + t;
        b = a2 + (P2 - t);
    }
    static constexpr uint32_t kRoot16 = cx_root16(kP, kOdd, 0);
};

using F29 = LazyField<469762049u, 26, 7, 4>;
using F28 = LazyField<167772161u, 25, 5, 12>;

// Twiddle w16^E of a field with a compile-time 16th root (value and Shoup quotient).
template <class F, int E>
__device__ __forceinline__ typename F::Tw root16_tw() {
    constexpr uint32_t w = static_cast<uint32_t>(cx_powmod(F::kRoot16, E & 15, F::P));
    constexpr uint32_t q = static_cast<uint32_t>((uint64_t(w) << 32) / F::P);
    typename F::Tw t;
    t.w = w;
    t.q = q;
    return t;
}
template <class F>
__device__ __forceinline__ typename F::Tw root16_tw(int e) {
    switch (e & 15) {
        case 1: return root16_tw<F, 1>();
        case 2: return root16_tw<F, 2>();
        case 3: return root16_tw<F, 3>();
        case 4: return root16_tw<F, 4>();
        case 5: return root16_tw<F, 5>();
        case 6: return root16_tw<F, 6>();
        case 7: return root16_tw<F, 7>();
        case 8: return root16_tw<F, 8>();
        case 9: return root16_tw<F, 9>();
        case 10: return root16_tw<F, 10>();
        case 11: return root16_tw<F, 11>();
        case 12: return root16_tw<F, 12>();
        case 13: return root16_tw<F, 13>();
        case 14: return root16_tw<F, 14>();
        case 15: return root16_tw<F, 15>();
        default: return root16_tw<F, 0>();
    }
}

struct F64 {
    using T = uint64_t;
    using Tw = uint64_t;
    static constexpr uint64_t P = 0xFFFFFFFF00000001ull;
    static constexpr uint64_t EPS = 0xFFFFFFFFull;  // 2^64 mod p
    static constexpr int kTwoAdicity = 32;

    __device__ static __forceinline__ T add(T a, T b) {
        T s = a + b;
        if (s < a) return s + EPS;  // wrapped: a+b-2^64+(2^32-1) < p
        return s >= P ? s - P : s;
    }
    __device__ static __forceinline__ T sub(T a, T b) {
        T d = a - b;
        return a < b ? d - EPS : d;  // a-b+2^64-(2^32-1) = a-b+p
    }
    __device__ static __forceinline__ T reduce128(uint64_t lo, uint64_t hi) {
        const uint64_t hh = hi >> 32, hl = hi & EPS;
        uint64_t t0 = lo - hh;
        if (lo < hh) t0 -= EPS;
        const uint64_t t1 = hl * EPS;
        uint64_t r = t0 + t1;
        if (r < t1) r += EPS;
        return r >= P ? r - P : r;
    }
    __device__ static __forceinline__ T mul(T a, T b) { return reduce128(a * b, __umul64hi(a, b)); }
    __device__ static __forceinline__ T mul_tw(T a, Tw w) { return mul(a, w); }
    __device__ static __forceinline__ T mont(T a, T b) { return mul(a, b); }
    __device__ static __forceinline__ uint32_t low_bit(T a) { return static_cast<uint32_t>(a & 1u); }
    __device__ static __forceinline__ T full_form(Tw w) { return w; }
    __device__ static __forceinline__ T mul_full(T a, T wf) { return mul(a, wf); }
    __device__ static __forceinline__ T step_full(T wf, Tw step) { return mul(wf, step); }
    __device__ static __forceinline__ Tw neg_tw(Tw w) { return w ? P - w : 0; }
    __device__ static __forceinline__ void dif_bfly(T &a, T &b, Tw w) {
        const T s = add(a, b);
        b = mul_tw(sub(a, b), w);
        a = s;
    }
    __device__ static __forceinline__ void dit_bfly(T &a, T &b, Tw w) {
        const T t = mul_tw(b, w);
        b = sub(a, t);
        a = add(a, t);
    }
};

}  // namespace pa
