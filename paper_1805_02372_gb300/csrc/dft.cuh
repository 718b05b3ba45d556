// Shared-memory R-point transforms over a ring policy F (a prime field or complex
// floating point): F::T element, F::Tw twiddle, F::add, F::sub, F::mul_tw.
// Forward = decimation in frequency (natural order in, bit-reversed out); inverse =
// decimation in time (bit-reversed in, natural out, unnormalised), each round doing
// two radix-2 stages on a group of four elements held in registers.
#pragma once

namespace pa {

// Stage tables of an R-point transform into shared memory: st[h-1+j] = w_{2h}^(+-j).
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

// Element (r, c) of a shared tile at base[r*rs + c*cs]. CF: consecutive threads take
// consecutive columns (when cs == 1), else consecutive rows (when rs == 1).
template <class F, bool CF>
__device__ __forceinline__ void dif_round4(typename F::T *sm, int logR, int logC, int rs, int cs,
                                           int lq, const typename F::Tw *tw) {
    using T = typename F::T;
    const int q = 1 << lq, h = 2 * q;
    const int logG = logR - 2;
    const int total = 1 << (logG + logC);
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
        const int i0 = ((g >> lq) << (lq + 2)) + j;
        T *b = sm + c * cs;
        const T x0 = b[i0 * rs], x1 = b[(i0 + q) * rs], x2 = b[(i0 + 2 * q) * rs],
                x3 = b[(i0 + 3 * q) * rs];
        const typename F::Tw w1 = tw[h - 1 + j], w2 = tw[h - 1 + j + q], w3 = tw[q - 1 + j];
        const T y0 = F::add(x0, x2), y2 = F::mul_tw(F::sub(x0, x2), w1);
        const T y1 = F::add(x1, x3), y3 = F::mul_tw(F::sub(x1, x3), w2);
        b[i0 * rs] = F::add(y0, y1);
        b[(i0 + q) * rs] = F::mul_tw(F::sub(y0, y1), w3);
        b[(i0 + 2 * q) * rs] = F::add(y2, y3);
        b[(i0 + 3 * q) * rs] = F::mul_tw(F::sub(y2, y3), w3);
    }
}

template <class F, bool CF>
__device__ __forceinline__ void dit_round4(typename F::T *sm, int logR, int logC, int rs, int cs,
                                           int lq, const typename F::Tw *tw) {
    using T = typename F::T;
    const int q = 1 << lq, h = 2 * q;
    const int logG = logR - 2;
    const int total = 1 << (logG + logC);
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
        const int i0 = ((g >> lq) << (lq + 2)) + j;
        T *b = sm + c * cs;
        const T z0 = b[i0 * rs], z1 = b[(i0 + q) * rs], z2 = b[(i0 + 2 * q) * rs],
                z3 = b[(i0 + 3 * q) * rs];
        const typename F::Tw w1 = tw[h - 1 + j], w2 = tw[h - 1 + j + q], w3 = tw[q - 1 + j];
        T t = F::mul_tw(z1, w3);
        const T y0 = F::add(z0, t), y1 = F::sub(z0, t);
        t = F::mul_tw(z3, w3);
        const T y2 = F::add(z2, t), y3 = F::sub(z2, t);
        t = F::mul_tw(y2, w1);
        b[i0 * rs] = F::add(y0, t);
        b[(i0 + 2 * q) * rs] = F::sub(y0, t);
        t = F::mul_tw(y3, w2);
        b[(i0 + q) * rs] = F::add(y1, t);
        b[(i0 + 3 * q) * rs] = F::sub(y1, t);
    }
}

template <class F, bool CF, bool DIF>
__device__ __forceinline__ void round2(typename F::T *sm, int logR, int logC, int rs, int cs,
                                       const typename F::Tw *tw) {
    // single stage with half-size 1: pairs (2g, 2g+1), twiddle w_2^0 = 1
    using T = typename F::T;
    const int logG = logR - 1;
    const int total = 1 << (logG + logC);
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        int c, g;
        if (CF) {
            c = w & ((1 << logC) - 1);
            g = w >> logC;
        } else {
            g = w & ((1 << logG) - 1);
            c = w >> logG;
        }
        T *b = sm + c * cs;
        const T a = b[(2 * g) * rs], d = b[(2 * g + 1) * rs];
        b[(2 * g) * rs] = F::add(a, d);
        b[(2 * g + 1) * rs] = F::sub(a, d);
    }
    (void)tw;
}

// Forward R-point DIF on every column (natural in, bit-reversed out).
template <class F, bool CF>
__device__ void dif_columns(typename F::T *sm, int logR, int logC, int rs, int cs,
                            const typename F::Tw *tw) {
    int lq = logR - 2;
    for (; lq >= 0; lq -= 2) {
        dif_round4<F, CF>(sm, logR, logC, rs, cs, lq, tw);
        __syncthreads();
    }
    if (logR & 1) {
        round2<F, CF, true>(sm, logR, logC, rs, cs, tw);
        __syncthreads();
    }
}

// Inverse R-point DIT on every column (bit-reversed in, natural out, unnormalised).
template <class F, bool CF>
__device__ void dit_columns(typename F::T *sm, int logR, int logC, int rs, int cs,
                            const typename F::Tw *tw) {
    int lq = 0;
    if (logR & 1) {
        round2<F, CF, false>(sm, logR, logC, rs, cs, tw);
        __syncthreads();
        lq = 1;
    }
    for (; lq <= logR - 2; lq += 2) {
        dit_round4<F, CF>(sm, logR, logC, rs, cs, lq, tw);
        __syncthreads();
    }
}

}  // namespace pa
