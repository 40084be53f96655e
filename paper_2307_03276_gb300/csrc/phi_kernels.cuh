// Phi^(n) tile kernels (Algorithm 2 of arXiv 2307.03276, evaluated per
// nonzero as in Algorithm 3) and their two variants that share the same
// gather: MTTKRP (Experiment 8: no dot product, no division) and the
// log-likelihood sum (the dot product alone).
//
// Work decomposition.  Nonzeros of mode n are sorted by i_n.  A thread block
// takes one tile of `tile_nnz` consecutive sorted nonzeros.  Inside the tile
// a "group" of G lanes owns a contiguous run of nonzeros and walks it in
// order; each lane holds RPL consecutive ranks of every row it touches, so
// the G lanes of a group read a factor row (Rp = G * RPL entries) as one
// coalesced 16-byte-vector access, and the dot product <B[i_n], pi> is summed
// across the group with xor shuffles.  While consecutive nonzeros share a
// row the group adds v * pi into registers; when the row changes it flushes.
//
// Same-row reduction without atomics (the paper's atomic-mitigation idea of
// Algorithm 4 taken to three levels):
//   1. a row that starts and ends inside a group's run is stored directly;
//   2. a row cut by group boundaries leaves a head or tail partial in shared
//      memory; after a barrier the block adds each chain of partials in group
//      order and stores the row if it ends inside the tile;
//   3. a row cut by a tile boundary leaves a per-tile partial in the carry
//      buffer and counts it on the row's counter; the tile whose partial
//      arrives last adds all of them in tile order (a fixed order, so results
//      are bit-reproducible) and stores the row.
// Rows without nonzeros are never touched.  With reduction = ATOMIC, levels
// 2 and 3 are replaced by atomic adds into a zeroed output.
//
// A tile's coordinates and values are first staged in shared memory by bulk
// asynchronous copies, so that a batch reads them with a few vector shared
// loads and only the factor-row gathers go to L1/L2.  The rows are not
// streamed per nonzero: the tile stages the row-start bits of its positions
// (one bit per nonzero) and the list of its rows (one entry per row), and a
// group walks its run by counting row starts.
//
// The KKT violation max_{i,r} |min(B, 1 - Phi)| of the MU loop is folded in:
// whoever writes a final Phi row also reduces its violation, and one atomicMax
// per block publishes it (non-negative doubles order like their bit patterns).
//
// FP32 form: gathers, Khatri-Rao products, dot and scale in FP32; a run of
// same-row nonzeros is summed in plain FP32 over two interleaved
// accumulators, the sums of partial rows across groups and tiles are
// Kahan-compensated; the violation is taken in FP32 (its maximum is exact)
// and published, like the log-likelihood partials, in FP64.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace cpapr {

constexpr int kMaxNm1 = kMaxModes - 1;

struct PhiArgs {
    int64_t nnz;
    int32_t T;       // nonzeros per tile
    int32_t ntiles;
    int32_t Rp;
    int32_t In;
    int32_t nm1;     // number of gathered modes (N - 1)
    int32_t atomic;  // 1: partial rows are added with atomics into a zeroed output
    const uint32_t *rstart;  // row-start bits of the sorted positions: bit p set where a row begins at p
    const int32_t *nzrow;    // the rows holding nonzeros, increasing
    const int32_t *krow;     // [ntiles + 1] index in nzrow of the row holding each tile's first nonzero
    const int32_t *idx[kMaxNm1];
    const void *val;
    const void *A[kMaxNm1];
    const void *B;
    void *out;
    void *carry;     // head partials [ntiles][Rp], then tail partials [ntiles][Rp]
    const int32_t *split;   // [nsplit][3]: rows that span tiles (row, first tile, last tile)
    const int32_t *tsplit;  // [ntiles][2]: split of the tile's head partial, of its tail partial (-1: none)
    int32_t *splitcnt;      // [nsplit]: partials arrived in this launch (zero between launches)
    int32_t nsplit;
    double eps;
    InnerState *inner;  // null for a one-off Phi (no KKT bookkeeping)
    double *llpart;     // OP_LL: one partial per tile
    int32_t *err;       // set to 1 when a bounded wait gives up
    const void *pi;     // materialised Khatri-Rao rows [nnz][Rp] in mode-n order, or null
    uint32_t stage_extra;  // bytes the staging barrier expects beyond the copies: 0, or 16
                           // when the host injects a staging-wait failure (tests)
    // FP32 form: FP64 masters of B and of the gathered factors, which the
    // log-likelihood reads where an FP32 model value underflows (else null)
    const double *Bm;
    const double *Am[kMaxNm1];
    int32_t dfdot;  // FP64 Phi: 1 = the kernel with the dot product on the FP32 pipe (df_dot)
};

// ---- compensated sums --------------------------------------------------------
template <typename T> struct KSum {
    T s, c;
    __device__ __forceinline__ void zero() { s = T(0); c = T(0); }
    __device__ __forceinline__ void add(T x) { s += x; }
    __device__ __forceinline__ void fma_add(T v, T p) { s = fma(v, p, s); }
    __device__ __forceinline__ T value() const { return s; }
};
template <> struct KSum<float> {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    // Kahan (1965): carry the rounding error of every addition in c
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ void fma_add(float v, float p) { add(v * p); }
    __device__ __forceinline__ float value() const { return s - c; }
};

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// |min(B, 1 - Phi)| in the working precision.  Its maximum is exact in any
// precision; only 1 - Phi rounds, which is far below any KKT tolerance.
template <typename T> __device__ __forceinline__ T viol_t(T b, T phi) {
    const T om = T(1) - phi;
    const T m = b < om ? b : om;
    return m < T(0) ? -m : m;
}

// x >= 0 as a float hi <= x within 2^-23 relative (its leading 24 bits, by
// integer operations); false where x is outside the float range
__device__ __forceinline__ bool hi_of(double x, float &hi) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const uint32_t H = (uint32_t)(bits >> 32), L = (uint32_t)bits;
    const uint32_t e = H >> 20;
    hi = bits ? __uint_as_float(__funnelshift_l(L, H, 3) - (896u << 23)) : 0.f;
    return bits == 0ull || (e >= 1023u - 126u && e < 1023u + 127u);
}

// The running KKT maximum k of an FP64 Phi kernel takes the exact term
// |min(b, 1 - phi)| only where an FP32 estimate from the leading 24 bits of b
// (b_hi) and of phi could exceed it: the estimate is within 2^-22 (1 + phi + b)
// of the term (b_hi and phi_hi are within 2^-23 relative, 1 - phi_hi rounds
// once, min and |.| are 1-Lipschitz), so with twice that margin no term above
// k is skipped and the maximum stays exact.  kf is a float <= k.
__device__ __forceinline__ bool kkt_candidate(float b_hi, double phi, float kf) {
    float ph;
    if (!hi_of(phi, ph)) return true;
    const float m = fminf(b_hi, 1.f - ph);
    return fabsf(m) + 0x1p-21f * (1.f + ph + b_hi) >= kf;
}
__device__ __forceinline__ float float_below(double k) {
    float h;
    if (hi_of(k, h)) return h;
    return ((unsigned long long)__double_as_longlong(k) >> 52) < 1023ull ? 0.f : 3.4028234663852886e38f;
}

// x / max(s, eps) of Algorithm 2.
// FP64: s >= 0, so the maximum is taken on the bit patterns (integer ALU,
// not the FP64 pipe).  r0 is the hardware's approximate FP64 reciprocal of m
// (PTX rcp.approx.ftz.f64, relative error below 2^-19 measured on GB300; no
// conversions through FP32).  With e = 1 - m r0, 1/m = r0 / (1 - e) =
// r0 (1 + e + e^2 + ...); the third-order step r1 = r0 + r0 (e + e^2)
// leaves the relative error e^3 (below 2^-57) plus a few FP64 roundings:
// four FP64 operations with the final x * r1, instead of the longer IEEE
// division on GB300's narrow FP64 pipe, far inside the 1e-12 parity bound.
// Where m lies outside [2^-1000, 2^1000] the IEEE division runs.
// FP32: the fast reciprocal-based division (within 2 ulp, far inside the
// FP32 path's 1e-5 tolerance).
__device__ __forceinline__ double phi_divide(double x, double s, double eps) {
    const double m = __longlong_as_double(max(__double_as_longlong(s), __double_as_longlong(eps)));
    const unsigned ex = ((unsigned)__double2hiint(m) >> 20) & 0x7ffu;  // biased exponent (sign is 0)
    if (ex - 23u >= 2000u) return x / m;  // zero, subnormal, tiny or huge, inf, NaN
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(m));
    const double e = fma(-m, r, 1.0);
    r = fma(r, fma(e, e, e), r);
    return x * r;
}
__device__ __forceinline__ float phi_divide(float x, float s, float eps) { return __fdividef(x, s > eps ? s : eps); }

// ---- the FP64 form's dot product on the FP32 pipe ---------------------------------
//
// GB300 issues 64 FP32 FMAs for every FP64 FMA.  In the FP64 Phi kernel the dot
// s = <B[i_n], pi> is the divisor of x and only has to be accurate relative to
// max(s, eps), so it runs on the FP32 pipe: each FP64 operand is cut into two
// floats hi + lo holding its leading 48 significant bits (integer operations),
// each product hi_a hi_b is taken exactly with an FMA (Dekker's product p + e),
// the products p are added with Knuth's two-sum (the rounding error of every
// addition is kept), and the errors e, the cross products hi_a lo_b + lo_a hi_b
// and the two-sum errors are summed in plain FP32.  For k terms, all >= 0,
// with u = 2^-24 (first order):
//   operands cut to 48 bits:                 <= 2.5 * 2^-47 s
//   e and cross terms (3k sums of terms <= 3u s):  <= 9k u^2 s
//   two-sum errors (k sums of terms <= u s):        <= k^2 u^2 s
//   operands below 2^-126 dropped:           < k 2^31 2^-126 (absolute)
// For k = 8 ranks per lane: |s_df - s| <= 5.2e-13 s + 2^-92, i.e. below 6e-13
// relative to max(s, eps) for eps >= 2^-43.  The lanes' partials are added
// as hi/lo pairs (df_add) and x / max(s, eps) is taken on the FP32 pipe as well
// (df_divide, within 2^-43 relative), so v = x / max(s, eps) is within 7.5e-13
// relative, inside the FP64 form's 1e-12 parity bound (Phi inherits the
// relative error of its v, its terms being >= 0); the batch's FP64 operations
// are one addition per division and the scale-add.  An operand >= 2^31
// (beyond the exponents the cut assumes) or a value x outside {0} and
// [2^-20, 2^31) makes the group redo the batch with the FP64 dot and division.

// x >= 0 as hi + lo, its leading 48 significant bits (integer operations and
// one integer-to-float conversion); x < 2^-126 gives 0 + 0, x >= 2^31 sets big.
__device__ __forceinline__ void df_cut(double x, float &hi, float &lo, bool &big) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const uint32_t H = (uint32_t)(bits >> 32), L = (uint32_t)bits;
    const int e = (int)(H >> 20);  // biased exponent (x >= 0)
    big = big || e >= 1023 + 31;
    const bool keep = e >= 1023 - 126;
    // hi: the first 23 fraction bits with the exponent rebased from bias 1023
    // to bias 127 (896 less in the exponent field)
    hi = keep ? __uint_as_float(__funnelshift_l(L, H, 3) - (896u << 23)) : 0.f;
    // lo: the next 29 fraction bits (24 kept) times 2^(e - 1075), scaled in
    // two exact steps that stay in the float range
    const float m = __uint2float_rz(L & 0x1fffffffu);
    lo = keep ? m * __uint_as_float((uint32_t)(e - 1075 + 64 + 127) << 23) * 0x1p-64f : 0.f;
}

// the float f as a double (integer operations; 0 for zero and subnormal f)
__device__ __forceinline__ double df_widen(float f) {
    const uint32_t b = __float_as_uint(f);
    const unsigned long long d = (((unsigned long long)(b & 0x7fffffffu) << 29) + (896ull << 52)) |
                                 ((unsigned long long)(b & 0x80000000u) << 32);
    return (b & 0x7f800000u) ? __longlong_as_double((long long)d) : 0.0;
}

// a + b for hi/lo float pairs with |lo| <= ulp(hi) / 2 (Knuth's two-sum of the
// highs, then a fast two-sum that renormalises); the result is such a pair
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float z = s - a.x;
    const float e = ((a.x - (s - z)) + (b.x - z)) + (a.y + b.y);
    const float h = s + e;
    return make_float2(h, e - (h - s));
}

// sum_r a_r b_r with a given as hi/lo floats (cut once per B row) and b in
// FP64, as a renormalised hi/lo float pair
template <int K>
__device__ __forceinline__ float2 df_dot(const float (&ahi)[K], const float (&alo)[K], const double (&b)[K],
                                         bool &big) {
    float S = 0.f, C = 0.f, D = 0.f;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        float bh, bl;
        df_cut(b[r], bh, bl, big);
        const float p = ahi[r] * bh;
        D = fmaf(ahi[r], bh, -p) + D;
        D = fmaf(ahi[r], bl, D);
        D = fmaf(alo[r], bh, D);
        const float t = S + p;
        const float z = t - S;
        C += (S - (t - z)) + (p - z);
        S = t;
    }
    const float E = C + D;
    const float h = S + E;  // |E| << S: fast two-sum
    return make_float2(h, E - (h - S));
}

// x / max(s, eps) in FP64 from the pair s = s.x + s.y and eps = eh + el, on the
// FP32 pipe: q0 = x_hi / m_hi to single precision (the hardware reciprocal
// estimate), then the classical correction of a double-length division
// (Dekker): the residual x - q0 m, formed exactly to first order with the FMA
// product q0 m_hi = p + pe (x_hi - p is exact: p is within a factor of two of
// x_hi), divided by m_hi gives q1, and q0 + q1 is the quotient.  |q1| <= 2^-21
// q0 and q1 carries a relative error of about 2^-22 (estimate, rounding), so
// the quotient is within 2^-43 relative; x enters with its 48 leading bits
// (2^-48).  One FP64 addition widens it.  Needs x = 0 or 2^-20 <= x < 2^31
// (checked by df_check_x), eps >= 2^-43 and s < 2^66 (eight operands < 2^31 per
// lane, up to 16 lanes), so that q0 and q1 are normal floats.
__device__ __forceinline__ double df_divide(double x, float2 s, float eh, float el) {
    float xh, xl;
    bool unused = false;
    df_cut(x, xh, xl, unused);
    const bool use_s = (s.x - eh) + (s.y - el) >= 0.f;  // s.x - eh is exact where they are close
    const float mh = use_s ? s.x : eh, ml = use_s ? s.y : el;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(mh));
    const float q0 = xh * r;
    const float p = q0 * mh;
    const float pe = fmaf(q0, mh, -p);
    const float res = ((xh - p) - pe) + fmaf(-q0, ml, xl);
    return df_widen(q0) + df_widen(res * r);
}

// sets big unless x = 0 or 2^-20 <= x < 2^31 (the range df_divide handles);
// integer operations on the bits of x >= 0
__device__ __forceinline__ void df_check_x(double x, bool &big) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(bits >> 52);
    big = big || (bits != 0ull && (e < 1023u - 20u || e >= 1023u + 31u));
}

// the reduce-scatter below for hi/lo float pairs (two shuffles per pair)
template <int G, int U>
__device__ __forceinline__ float2 group_reduce_scatter_df(float2 (&s)[U], int lane, unsigned gmask) {
    static_assert(U <= G, "reduce-scatter needs U <= G");
    int o = G / 2;
#pragma unroll
    for (int h = U / 2; h >= 1; h >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float2 send = upper ? s[i] : s[i + h];
            const float2 keep = upper ? s[i + h] : s[i];
            s[i] = df_add(keep, make_float2(__shfl_xor_sync(gmask, send.x, o), __shfl_xor_sync(gmask, send.y, o)));
        }
        o >>= 1;
    }
    float2 tot = s[0];
#pragma unroll
    for (int oo = G / (2 * U); oo > 0; oo >>= 1)
        tot = df_add(tot, make_float2(__shfl_xor_sync(gmask, tot.x, oo), __shfl_xor_sync(gmask, tot.y, oo)));
    return tot;
}

// On entry each of the G lanes of a group holds U partial dot products (its
// RPL ranks) of the group's U nonzeros.  A reduce-scatter halves the set at
// every exchange, so that afterwards lane l holds the complete sum for
// nonzero u = l / (G / U) -- each lane divides once per batch instead of U
// times.  Requires U <= G (G > 1).
template <typename T, int G, int U>
__device__ __forceinline__ T group_reduce_scatter(T (&s)[U], int lane, unsigned gmask) {
    static_assert(U <= G, "reduce-scatter needs U <= G");
    int o = G / 2;
#pragma unroll
    for (int h = U / 2; h >= 1; h >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = upper ? s[i] : s[i + h];
            const T keep = upper ? s[i + h] : s[i];
            s[i] = keep + __shfl_xor_sync(gmask, send, o);
        }
        o >>= 1;
    }
    T tot = s[0];
#pragma unroll
    for (int oo = G / (2 * U); oo > 0; oo >>= 1) tot += __shfl_xor_sync(gmask, tot, oo);
    return tot;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduces the block's violation (in FP64) and publishes it into inner->kkt[l & 1].
template <int THREADS>
__device__ __forceinline__ void publish_kkt(double v, InnerState *inner, double *sm) {
    v = warp_max(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; ++w) m = fmax(m, sm[w]);
        if (m > 0.0) atomicMax(&inner->kkt[inner->l & 1], ordered_bits(m));
    }
}

template <typename T, int RPL>
__device__ __forceinline__ void load_row(const T *__restrict__ base, T (&dst)[RPL]) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    const V *p = reinterpret_cast<const V *>(base);
#pragma unroll
    for (int v = 0; v < RPL / VN; ++v) {
        V x = __ldg(p + v);
        if constexpr (VN == 4) {
            dst[4 * v + 0] = x.x;
            dst[4 * v + 1] = x.y;
            dst[4 * v + 2] = x.z;
            dst[4 * v + 3] = x.w;
        } else {
            dst[2 * v + 0] = x.x;
            dst[2 * v + 1] = x.y;
        }
    }
}

// load_row for data read once (evict-first: the materialised Pi streams
// through L2 without displacing the factor rows)
template <typename T, int RPL>
__device__ __forceinline__ void load_row_stream(const T *__restrict__ base, T (&dst)[RPL]) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    const V *p = reinterpret_cast<const V *>(base);
#pragma unroll
    for (int v = 0; v < RPL / VN; ++v) {
        V x = __ldcs(p + v);
        if constexpr (VN == 4) {
            dst[4 * v + 0] = x.x;
            dst[4 * v + 1] = x.y;
            dst[4 * v + 2] = x.z;
            dst[4 * v + 3] = x.w;
        } else {
            dst[2 * v + 0] = x.x;
            dst[2 * v + 1] = x.y;
        }
    }
}

template <typename T, int RPL>
__device__ __forceinline__ void mul_row(const T *__restrict__ base, T (&dst)[RPL]) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    const V *p = reinterpret_cast<const V *>(base);
#pragma unroll
    for (int v = 0; v < RPL / VN; ++v) {
        V x = __ldg(p + v);
        if constexpr (VN == 4) {
            dst[4 * v + 0] *= x.x;
            dst[4 * v + 1] *= x.y;
            dst[4 * v + 2] *= x.z;
            dst[4 * v + 3] *= x.w;
        } else {
            dst[2 * v + 0] *= x.x;
            dst[2 * v + 1] *= x.y;
        }
    }
}

// <row at base, v> with the row read through L1 (used by the FP64 kernels
// where registers are short; one FMA chain, see dot_regs)
template <typename T, int RPL>
__device__ __forceinline__ T dot_global(const T *__restrict__ base, const T (&v)[RPL]) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    const V *p = reinterpret_cast<const V *>(base);
    T d = T(0);
#pragma unroll
    for (int k = 0; k < RPL / VN; ++k) {
        V x = __ldg(p + k);
        if constexpr (VN == 4) {
            d = fma(x.x, v[4 * k + 0], d);
            d = fma(x.y, v[4 * k + 1], d);
            d = fma(x.z, v[4 * k + 2], d);
            d = fma(x.w, v[4 * k + 3], d);
        } else {
            d = fma(x.x, v[2 * k + 0], d);
            d = fma(x.y, v[2 * k + 1], d);
        }
    }
    return d;
}

// <a, b>.  FP32 with 8 or more ranks per lane: four independent partial sums
// (short dependency chains); otherwise one FMA chain -- for FP64 because on
// this GPU the FP64 pipe itself is the limit and every extra add costs a
// pipe slot.
template <typename T, int RPL>
__device__ __forceinline__ T dot_regs(const T (&a)[RPL], const T (&b)[RPL]) {
    if constexpr (RPL < 8 || sizeof(T) == 8) {
        T d = T(0);
#pragma unroll
        for (int r = 0; r < RPL; ++r) d = fma(a[r], b[r], d);
        return d;
    } else {
        T d[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int r = 0; r < RPL; ++r) d[r & 3] = fma(a[r], b[r], d[r & 3]);
        return (d[0] + d[1]) + (d[2] + d[3]);
    }
}

template <typename T, int RPL>
__device__ __forceinline__ void store_row(T *__restrict__ base, const T (&src)[RPL]) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    V *p = reinterpret_cast<V *>(base);
#pragma unroll
    for (int v = 0; v < RPL / VN; ++v) {
        V x;
        if constexpr (VN == 4) {
            x.x = src[4 * v + 0];
            x.y = src[4 * v + 1];
            x.z = src[4 * v + 2];
            x.w = src[4 * v + 3];
        } else {
            x.x = src[2 * v + 0];
            x.y = src[2 * v + 1];
        }
        p[v] = x;
    }
}

// ---- staging of a tile's streams in shared memory ------------------------------
//
// A tile's row ids, its N-1 coordinate streams and its values are contiguous
// runs in HBM.  One thread copies each run into shared memory with a bulk
// asynchronous copy (cp.async.bulk; completion is counted in bytes on an
// mbarrier) and the block waits on the barrier.  The wait is bounded in time:
// if the copies have not landed after kStageWaitNs the block records the
// failure in *a.err, waits once more for its copies and skips the tile (the
// host then reports CPAPR_E_TIMEOUT).

// The limit is a hang guard, not a performance bound: a tile's copies land in
// microseconds, so only a copy that can never complete (or a GPU so starved
// that one tile's few kilobytes take a second) reaches it, and then the call
// reports CPAPR_E_TIMEOUT instead of hanging the GPU.
constexpr uint64_t kStageWaitNs = 1000000000ull;  // 1 s

// entries reserved per staged stream (a multiple of 4: 16-byte rows)
__host__ __device__ constexpr int stage_cap(int T) { return (T + 3) & ~3; }

// 32-bit words of row-start bits a tile stages (from the 16-byte group that
// holds its first position through the word of the position after its last),
// with room to spare; the same count holds the set bits before each word.
__host__ __device__ constexpr int stage_words(int T) { return (((T + 31) >> 5) + 8 + 3) & ~3; }

// shared-memory bytes of a tile of T nonzeros: the tile's rows, the staged
// streams (N-1 coordinates, values), the row-start bits and their word
// counts, then the partial-row slots of the segmented reduction (2 per group
// of lanes) and a few words of bookkeeping
__host__ __device__ constexpr size_t phi_smem_bytes(int T, int nm1, int esize, int threads, int rpl) {
    return (size_t)(stage_cap(T) + 8) * 4 + (size_t)stage_cap(T) * (size_t)(4 * nm1 + esize) +
           (size_t)stage_words(T) * 8 + (size_t)2 * threads * rpl * esize + (size_t)2 * threads * 4 + 32;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void stage_barrier_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void stage_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}


// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void stage_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"((uint64_t)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool stage_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true once the phase with this parity has completed; false after
// kStageWaitNs (or 2^26 polls) without completion
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity) {
    if (stage_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (stage_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kStageWaitNs) break;
    }
    return false;
}

// U consecutive staged entries starting at a multiple of U (vector loads)
template <int U>
__device__ __forceinline__ void lds_u(const int32_t *p, int32_t (&d)[U]) {
    if constexpr (U == 4) {
        const int4 v = *reinterpret_cast<const int4 *>(p);
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    } else if constexpr (U == 2) {
        const int2 v = *reinterpret_cast<const int2 *>(p);
        d[0] = v.x;
        d[1] = v.y;
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) d[u] = p[u];
    }
}
template <int U>
__device__ __forceinline__ void lds_u(const float *p, float (&d)[U]) {
    if constexpr (U == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    } else if constexpr (U == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        d[0] = v.x;
        d[1] = v.y;
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) d[u] = p[u];
    }
}
template <int U>
__device__ __forceinline__ void lds_u(const double *p, double (&d)[U]) {
    if constexpr (U % 2 == 0) {
#pragma unroll
        for (int h = 0; h < U / 2; ++h) {
            const double2 v = reinterpret_cast<const double2 *>(p)[h];
            d[2 * h] = v.x;
            d[2 * h + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) d[u] = p[u];
    }
}

// <B[row], pi> recomputed in FP64 from the FP64 masters of B and of the
// factors: the FP32 log-likelihood uses it where the FP32 product underflows
// (m < 2^-96), so the value is the FP64 model's even where FP32 copies of
// factor entries are zero.
template <typename T, int RPL, int MAXK>
__device__ __forceinline__ double dot_fp64(const PhiArgs &a, const int32_t (&ii)[MAXK], int32_t row, int col0, int nm1) {
    const double *Bm = a.Bm + (int64_t)row * a.Rp + col0;
    double d = 0.0;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        double p = __ldg(Bm + r);
#pragma unroll
        for (int k = 0; k < MAXK; ++k)
            if (k < nm1) p *= __ldg(a.Am[k] + (int64_t)ii[k] * a.Rp + col0 + r);
        d += p;
    }
    return d;
}

// NM1: number of gathered modes (exact), or 0 for "runtime count up to kMaxNm1".
// U: nonzeros whose gathers are issued together (memory-level parallelism).
//
// One tile (t) of one tensor (a) by the whole block.  Every thread of the
// block calls it with the same arguments.  smem_raw holds phi_smem_bytes();
// red is NWARPS doubles; bar is the block's staging barrier (initialised) and
// phase the parity of its next phase (flipped here whenever a tile is staged).
// Returns false if the staging wait gave up (the caller stops).
// PI: the Khatri-Rao rows are read from the materialised Pi (a.pi, one row
// per nonzero in mode-n order) instead of being formed from the factors; the
// stage then holds only the row ids and the values.
// DF: the FP64 Phi (8 or fewer ranks per lane) takes its dot on the FP32 pipe.
template <typename T, int NM1, int RPL, int G, int OP, int THREADS, int U, bool PI = false, bool DF = false>
__device__ __forceinline__ bool phi_tile_body(const PhiArgs &a, const int t, unsigned char *smem_raw, double *red,
                                              uint64_t *bar, uint32_t &phase) {
    static_assert(U == 1 || U == 2 || U == 4, "batches of 1, 2 or 4 nonzeros");
    static_assert(!PI || OP == OP_PHI || (OP == OP_LL && sizeof(T) == 8),
                  "the materialised Pi serves Phi and the FP64 log-likelihood");
    constexpr int NG = THREADS / G;
    constexpr int NWARPS = THREADS / 32;
    constexpr int MAXK = NM1 > 0 ? NM1 : kMaxNm1;
    // the tile's first and last row in nzrow, read first so that their latency
    // passes while the block checks its state and synchronises
    int32_t k0 = 0, k1 = 0;
    // FP64 Phi on the FP32 pipe: the KKT maximum published so far (both slots
    // and the iteration index, read at once), which seeds the running maximum
    constexpr bool KSEED = DF && sizeof(T) == 8 && OP == OP_PHI;
    unsigned long long kslot0 = 0ull, kslot1 = 0ull;
    int32_t kl = 0;
    if (threadIdx.x == 0) {
        k0 = __ldg(a.krow + t);
        k1 = __ldg(a.krow + t + 1);
        if (KSEED && a.inner) {
            kl = *((volatile int32_t *)&a.inner->l);
            kslot0 = *((volatile unsigned long long *)&a.inner->kkt[0]);
            kslot1 = *((volatile unsigned long long *)&a.inner->kkt[1]);
        }
    }
    if (a.inner && a.inner->done) return true;
    const int nm1 = PI ? 0 : (NM1 > 0 ? NM1 : a.nm1);  // staged coordinate streams
    const int tid = threadIdx.x;
    const int g = tid / G, lane = tid % G;
    const int warp = tid >> 5, wlane = tid & 31;
    const int Rp = RPL * G;
    const int64_t p0 = (int64_t)t * a.T;
    const int64_t p1 = min(p0 + (int64_t)a.T, a.nnz);
    const int n = (int)(p1 - p0);
    const int col0 = lane * RPL;
    const unsigned gmask = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << ((wlane / G) * G));

    const int cap = stage_cap(a.T);
    const int W = stage_words(a.T);
    int32_t *s_rows = reinterpret_cast<int32_t *>(smem_raw);  // [cap + 8]: the tile's rows (from nzrow)
    int32_t *s_idx = s_rows + cap + 8;                          // [nm1][cap]
    T *s_val = reinterpret_cast<T *>(s_idx + (int64_t)nm1 * cap);
    uint32_t *s_bits = reinterpret_cast<uint32_t *>(s_val + cap);  // [W]: row-start bits from word w0
    int32_t *s_cnt = reinterpret_cast<int32_t *>(s_bits + W);      // [W]: set bits before each staged word
    T *slot_val = reinterpret_cast<T *>(s_cnt + W);                 // [2 * NG][Rp]
    int32_t *slot_row = reinterpret_cast<int32_t *>(slot_val + 2 * NG * Rp);  // [2 * NG]
    int32_t *slot_fin = slot_row + 2 * NG;  // [2]: rows spanning tiles this block finishes
    int32_t *s_meta = slot_fin + 2;         // [2]: s_rows index of the tile's first row; rows after it;
                                            // then 8 bytes: the KKT maximum published so far
    // the staged bits start at the 16-byte group holding bit p0 and run
    // through the word holding bit p1 (whether the last row goes on)
    const int64_t w0 = (p0 >> 5) & ~(int64_t)3;
    const int nw = (int)((((p1 >> 5) - w0 + 1) + 3) & ~(int64_t)3);

    // the previous tile of a persistent block may still read the stage and the slots
    __syncthreads();
    if (tid == 0) {
        // order this block's earlier generic accesses of the stage before the async writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the tile's rows: nzrow[k0 .. k1], k0 holding p0 and k1 holding p1
        // (or the last row), copied from the 16-byte group holding k0
        const int32_t k0a = k0 & ~3;
        const uint32_t br = (uint32_t)((k1 - k0a + 1 + 3) & ~3) * 4u;
        const uint32_t bw = (uint32_t)nw * 4u;
        const uint32_t b4 = (uint32_t)(((int64_t)n * 4 + 15) & ~(int64_t)15);
        const uint32_t bv = (uint32_t)(((int64_t)n * (int64_t)sizeof(T) + 15) & ~(int64_t)15);
        stage_expect(bar, br + bw + b4 * (uint32_t)nm1 + bv + a.stage_extra);
        stage_copy(s_bits, a.rstart + w0, bw, bar);
        for (int k = 0; k < nm1; ++k) stage_copy(s_idx + (int64_t)k * cap, a.idx[k] + p0, b4, bar);
        stage_copy(s_val, reinterpret_cast<const T *>(a.val) + p0, bv, bar);
        stage_copy(s_rows, a.nzrow + k0a, br, bar);
        s_meta[0] = k0 - k0a;
        s_meta[1] = k1 - k0;
        // the maximum published so far: terms below it cannot change the result
        *reinterpret_cast<unsigned long long *>(s_meta + 2) = (kl & 1) ? kslot1 : kslot0;
    }
    const bool segmented = (OP != OP_LL) && !a.atomic;
    if (segmented) {
        for (int s = tid; s < 2 * NG; s += THREADS) slot_row[s] = -1;
        if (tid < 2) slot_fin[tid] = -1;
    }
    const bool landed = stage_wait(bar, phase);
    phase ^= 1u;
    // set bits before each staged word (one warp, a running warp scan; the
    // block barrier below publishes them with the stage)
    if (warp == 0 && __all_sync(0xffffffffu, landed)) {
        int carry = 0;
        for (int base = 0; base < nw; base += 32) {
            const int w = base + wlane;
            const int c = w < nw ? __popc(s_bits[w]) : 0;
            int x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (wlane >= o) x += y;
            }
            if (w < nw) s_cnt[w] = carry + x - c;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    if (__syncthreads_or(!landed)) {
        if (tid == 0) atomicExch(a.err, 1);
        if (!landed) stage_wait(bar, phase ^ 1u);  // let the copies finish before the block moves on
        return false;
    }
    // position q of the tile is bit boff + q of the staged words
    const int boff = (int)(p0 - (w0 << 5));
    // row-start bit of tile position q (0 <= q <= n), and the row starts at
    // or before it counted from the tile's first staged word
    auto bit_at = [&](int q) -> uint32_t { return (s_bits[(boff + q) >> 5] >> ((boff + q) & 31)) & 1u; };
    auto starts_upto = [&](int q) -> int {
        const int b = boff + q;
        return s_cnt[b >> 5] + __popc(s_bits[b >> 5] & (0xffffffffu >> (31 - (b & 31))));
    };
    // s_rows index of the row holding tile position q: the tile's first row
    // plus the row starts in (p0, p0 + q]
    const int rbase = s_meta[0] - starts_upto(0);

    const T *__restrict__ Bm = reinterpret_cast<const T *>(a.B);
    T *__restrict__ out = reinterpret_cast<T *>(a.out);
    const T eps = (T)a.eps;
    float eps_hi = 0.f, eps_lo = 0.f;  // eps as a hi/lo float pair (FP32-pipe division)
    {
        bool unused = false;
        df_cut(a.eps, eps_hi, eps_lo, unused);
    }

    // Contiguous run [la, lb) of the tile for this group.  Runs start on
    // multiples of U (vector loads of a batch).  With one lane per group an
    // FP32 run length is made odd so that the 32 threads of a warp read 32
    // banks; FP64 keeps equal runs (its FP64 pipe hides the bank conflicts,
    // a longer run would not be hidden).
    int vlen = (a.T + NG - 1) / NG;
    if (G == 1) {
        if (sizeof(T) == 4) vlen |= 1;
    } else {
        vlen = (vlen + U - 1) / U * U;
    }
    const int la = min(g * vlen, n), lb = min(la + vlen, n);

    // running KKT maximum, from the one published so far (FP64 Phi on the FP32 pipe)
    T kkt = T(0);
    if constexpr (KSEED) kkt = (T)__longlong_as_double(*reinterpret_cast<const long long *>(s_meta + 2));
    double ll = 0.0;
    // with G > 1 lanes each lane finishes one nonzero of the batch: u_mine
    constexpr int LPU = G > 1 ? G / U : 1;  // lanes per nonzero after the reduce-scatter
    const int u_mine = G > 1 ? lane / LPU : 0;
    const int gbase = (wlane / G) * G;
    // B rows held in registers (reused along a row), except for wide FP64
    // lanes, whose registers go to the Khatri-Rao row and the accumulator:
    // there the dot reads the B row through L1 for every nonzero
    constexpr bool BREG = (OP != OP_MTTKRP) && !(sizeof(T) == 8 && (RPL >= 16 || U >= 4));
    // FP64 Phi with up to 8 ranks per lane may take its dot on the FP32 pipe
    // (df_dot); a B row in registers is then kept as hi/lo floats
    constexpr bool DFDOT = DF && sizeof(T) == 8 && OP == OP_PHI && RPL <= 8;
    constexpr bool BREGD = BREG && !DFDOT;  // B row in registers in the working type
    constexpr int BR = BREGD ? RPL : 1;
    constexpr int BF = (BREG && DFDOT) ? RPL : 1;

    if (la < lb) {
        // does the row at la begin before the run, the row at lb - 1 go on after it?
        const bool head_open = p0 + la > 0 && !bit_at(la);
        const bool tail_open = p0 + lb < a.nnz && !bit_at(lb);
        int kcur = rbase + starts_upto(la);  // s_rows index of the current row
        int32_t cur = s_rows[kcur];
        bool first_run = true;
        // Run accumulation (segmented, plain FMA).  FP32 interleaves two
        // accumulators so that each sums at most half of a run; the row sums
        // across groups and tiles are the compensated ones.
        constexpr int NACC = sizeof(T) == 4 ? 2 : 1;
        T acc[NACC][RPL];
#pragma unroll
        for (int h = 0; h < NACC; ++h)
#pragma unroll
            for (int r = 0; r < RPL; ++r) acc[h][r] = T(0);
        T brow[BR];  // B row of `brow_row` (loaded once per row, not per nonzero)
        float bhi[BF], blo[BF];  // or that row cut into hi/lo floats (df_dot)
        bool bbig = false;       // the cut row has an entry >= 2^31
        int32_t brow_row = cur;
        auto load_brow = [&]() {
            if constexpr (BREGD) {
                load_row<T, BR>(Bm + (int64_t)cur * Rp + col0, brow);
            } else if constexpr (BREG && DFDOT) {
                T t[RPL];
                load_row<T, RPL>(Bm + (int64_t)cur * Rp + col0, t);
                bbig = false;
#pragma unroll
                for (int r = 0; r < RPL; ++r) df_cut((double)t[r], bhi[r], blo[r], bbig);
            }
        };
        load_brow();

        auto flush = [&](int32_t frow, bool first, bool last) {
            T v[RPL];
#pragma unroll
            for (int r = 0; r < RPL; ++r) v[r] = NACC == 2 ? acc[0][r] + acc[NACC - 1][r] : acc[0][r];
            const bool before = first && head_open, after = last && tail_open;
            if (!before && !after) {
                store_row<T, RPL>(out + (int64_t)frow * Rp + col0, v);
                if (OP == OP_PHI && a.inner) {
                    if constexpr (BREG && DFDOT) {
                        // the exact FP64 term only where it could raise the running maximum
                        // (flushes diverge across a warp's groups, and each FP64 warp
                        // instruction costs the FP64 pipe the same with two lanes or 32)
                        if (frow == brow_row && !bbig) {
                            const float kf = float_below((double)kkt);
#pragma unroll
                            for (int r = 0; r < RPL; ++r)
                                if (kkt_candidate(bhi[r], (double)v[r], kf))
                                    kkt = tmax(kkt, viol_t(__ldg(Bm + (int64_t)frow * Rp + col0 + r), v[r]));
                            return;
                        }
                    }
                    if constexpr (BREGD) {
                        if (frow == brow_row) {
#pragma unroll
                            for (int r = 0; r < RPL; ++r) kkt = tmax(kkt, viol_t(brow[r], v[r]));
                            return;
                        }
                    }
#pragma unroll
                    for (int r = 0; r < RPL; ++r)
                        kkt = tmax(kkt, viol_t(__ldg(Bm + (int64_t)frow * Rp + col0 + r), v[r]));
                }
            } else if (a.atomic) {
#pragma unroll
                for (int r = 0; r < RPL; ++r) atomicAdd(out + (int64_t)frow * Rp + col0 + r, v[r]);
            } else {
                const int s = before ? 2 * g : 2 * g + 1;
                if (lane == 0) slot_row[s] = frow;
                store_row<T, RPL>(slot_val + (int64_t)s * Rp + col0, v);
            }
        };

        for (int q = la; q < lb; q += U) {
            int32_t rr[U];
            int32_t ii[U][MAXK];
            T xx[U];
            bool fast;  // every nonzero of the batch in the current row (the common case)
            if constexpr (G == 1) {
                // row starts among the batch's positions (the U bits may straddle two
                // words: one-lane runs need not start on multiples of U)
                const int bq = boff + q;
                uint32_t starts = __funnelshift_r(s_bits[bq >> 5], s_bits[(bq >> 5) + 1], bq & 31) & ((1u << U) - 1u);
                if (q == la) starts &= ~1u;                       // the run's first row is cur
                if (q + U > lb) starts &= (1u << (lb - q)) - 1u;  // past the run: not this group's
                fast = q + U <= lb && starts == 0u;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int qq = min(q + u, lb - 1);
                    if (fast) {
                        rr[u] = cur;
                    } else {
                        if ((starts >> u) & 1u) ++kcur;
                        rr[u] = s_rows[kcur];
                    }
                    xx[u] = s_val[qq];
#pragma unroll
                    for (int k = 0; k < MAXK; ++k)
                        if (k < nm1) ii[u][k] = s_idx[(int64_t)k * cap + qq];
                }
            } else {
                // row starts among the batch's positions: q is a multiple of U and
                // p0 of 4, so the batch's U bits lie in one word
                const int bq = boff + q;
                uint32_t starts = (s_bits[bq >> 5] >> (bq & 31)) & ((1u << U) - 1u);
                if (q == la) starts &= ~1u;                       // the run's first row is cur
                if (q + U > lb) starts &= (1u << (lb - q)) - 1u;  // past the run: not this group's
                fast = q + U <= lb && starts == 0u;
                if (!fast) {
                    // the batch's rows: the current one, advanced at each row start
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if ((starts >> u) & 1u) ++kcur;
                        rr[u] = s_rows[kcur];
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < U; ++u) rr[u] = cur;
                }
                lds_u<U>(s_val + q, xx);
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    if (k < nm1) {
                        int32_t tmp[U];
                        lds_u<U>(s_idx + (int64_t)k * cap + q, tmp);
#pragma unroll
                        for (int u = 0; u < U; ++u) ii[u][k] = tmp[u];
                    }
                }
                if (q + U > lb) {  // ragged end of the run: repeat its first entry (never accumulated)
#pragma unroll
                    for (int u = 1; u < U; ++u) {
                        if (q + u >= lb) {
                            rr[u] = rr[0];
                            xx[u] = xx[0];
#pragma unroll
                            for (int k = 0; k < MAXK; ++k) ii[u][k] = ii[0][k];
                        }
                    }
                }
            }

            T pi[U][RPL];
            if constexpr (PI) {
                // consecutive rows of the materialised Pi, streamed (read once per Phi)
                const T *P = reinterpret_cast<const T *>(a.pi) + (p0 + q) * Rp + col0;
#pragma unroll
                for (int u = 0; u < U; ++u) load_row_stream<T, RPL>(P + (int64_t)min(u, lb - 1 - q) * Rp, pi[u]);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    load_row<T, RPL>(reinterpret_cast<const T *>(a.A[0]) + (int64_t)ii[u][0] * Rp + col0, pi[u]);
#pragma unroll
                    for (int k = 1; k < MAXK; ++k)
                        if (k < nm1)
                            mul_row<T, RPL>(reinterpret_cast<const T *>(a.A[k]) + (int64_t)ii[u][k] * Rp + col0, pi[u]);
                }
            }
            T v[U];
            if (OP == OP_MTTKRP) {
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = xx[u];
            } else {
                T s[U];
                bool fp64dot = true;
                if constexpr (DFDOT) {
                    // <B[i_n], pi>, the lanes' sum and x / max(s, eps) on the FP32 pipe,
                    // unless an operand or x is outside their ranges somewhere in the group
                    float2 s2[U];
                    bool big = false;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        df_check_x((double)xx[u], big);
                        // one dot for fast and slow groups alike (converged across the warp)
                        float bh[RPL], bl[RPL];
                        if (BREG && fast) {
                            if constexpr (BREG) {
#pragma unroll
                                for (int r = 0; r < RPL; ++r) {
                                    bh[r] = bhi[r];
                                    bl[r] = blo[r];
                                }
                            }
                        } else {
                            T brw[RPL];
                            load_row<T, RPL>(Bm + (int64_t)rr[u] * Rp + col0, brw);
#pragma unroll
                            for (int r = 0; r < RPL; ++r) df_cut((double)brw[r], bh[r], bl[r], big);
                        }
                        s2[u] = df_dot<RPL>(bh, bl, pi[u], big);
                    }
                    if constexpr (BREG) big = big || (fast && bbig);
                    fp64dot = __any_sync(gmask, big);
                    if (!fp64dot) {
                        if constexpr (G == 1) {
#pragma unroll
                            for (int u = 0; u < U; ++u) v[u] = (T)df_divide((double)xx[u], s2[u], eps_hi, eps_lo);
                        } else {
                            const float2 tot = group_reduce_scatter_df<G, U>(s2, lane, gmask);
                            T xm = xx[0];
#pragma unroll
                            for (int u = 1; u < U; ++u)
                                if (u_mine == u) xm = xx[u];
                            const T vm = (T)df_divide((double)xm, tot, eps_hi, eps_lo);
#pragma unroll
                            for (int u = 0; u < U; ++u) v[u] = __shfl_sync(gmask, vm, gbase + u * LPU);
                        }
                    }
                }
                if (fp64dot) {
                    if (BREGD && fast) {
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if constexpr (BREGD) s[u] = dot_regs<T, RPL>(brow, pi[u]);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            s[u] = dot_global<T, RPL>(Bm + (int64_t)rr[u] * Rp + col0, pi[u]);
                    }
                }
                if (!fp64dot) {
                    // v done on the FP32 pipe above
                } else if constexpr (G == 1) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (OP == OP_PHI) {
                            v[u] = phi_divide(xx[u], s[u], eps);
                        } else if (q + u < lb) {  // OP_LL: x log(m), m = <lambda o A^(n)[i_n], pi>
                            if constexpr (sizeof(T) == 8) {
                                ll += (double)xx[u] * log((double)s[u]);
                            } else if (s[u] < 0x1p-96f) {
                                ll += (double)xx[u] * log(dot_fp64<T, RPL, MAXK>(a, ii[u], rr[u], col0, nm1));
                            } else {
                                ll += (double)xx[u] * (double)logf((float)s[u]);
                            }
                        }
                    }
                } else {
                    const T tot = group_reduce_scatter<T, G, U>(s, lane, gmask);
                    T xm = xx[0];
#pragma unroll
                    for (int u = 1; u < U; ++u)
                        if (u_mine == u) xm = xx[u];
                    if (OP == OP_PHI) {
                        const T vm = phi_divide(xm, tot, eps);
#pragma unroll
                        for (int u = 0; u < U; ++u) v[u] = __shfl_sync(gmask, vm, gbase + u * LPU);
                    } else if constexpr (sizeof(T) == 8) {
                        if (q + u_mine < lb && (lane % LPU) == 0) ll += (double)xm * log((double)tot);
                    } else {
                        // FP32 log of the model value (FP64 logs would load the
                        // FP64 pipe); where the FP32 value underflows, the
                        // group's dots are redone in FP64 (all its lanes join)
                        double lm = (double)logf((float)tot);
                        if (__any_sync(gmask, tot < 0x1p-96f)) {
                            double d[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) d[u] = dot_fp64<T, RPL, MAXK>(a, ii[u], rr[u], col0, nm1);
#pragma unroll
                            for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
                                for (int u = 0; u < U; ++u) d[u] += __shfl_xor_sync(gmask, d[u], o);
                            if (tot < 0x1p-96f) {
                                double m = d[0];
#pragma unroll
                                for (int u = 1; u < U; ++u)
                                    if (u_mine == u) m = d[u];
                                lm = log(m);
                            }
                        }
                        if (q + u_mine < lb && (lane % LPU) == 0) ll += (double)xm * lm;
                    }
                }
            }
            if constexpr (DF && sizeof(T) == 8) {
                // Row changes (slow batches only) flush the run's sum; the scale-add
                // itself runs for every group of the warp together, fast or slow, a
                // nonzero past the run's end adding 0 * pi: each FP64 warp
                // instruction costs the FP64 pipe the same with two lanes or 32.
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (!fast && q + u < lb && rr[u] != cur) {
                        if (OP != OP_LL) {
                            flush(cur, first_run, false);
#pragma unroll
                            for (int h = 0; h < NACC; ++h)
#pragma unroll
                                for (int r = 0; r < RPL; ++r) acc[h][r] = T(0);
                        }
                        first_run = false;
                        cur = rr[u];
                    }
                    if (OP != OP_LL) {
                        const T w = (fast || q + u < lb) ? v[u] : T(0);
#pragma unroll
                        for (int r = 0; r < RPL; ++r) acc[u % NACC][r] = fma(w, pi[u][r], acc[u % NACC][r]);
                    }
                }
            } else if (fast) {
                if (OP != OP_LL) {
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int r = 0; r < RPL; ++r) acc[u % NACC][r] = fma(v[u], pi[u][r], acc[u % NACC][r]);
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (q + u < lb) {
                        if (rr[u] != cur) {
                            if (OP != OP_LL) {
                                flush(cur, first_run, false);
#pragma unroll
                                for (int h = 0; h < NACC; ++h)
#pragma unroll
                                    for (int r = 0; r < RPL; ++r) acc[h][r] = T(0);
                            }
                            first_run = false;
                            cur = rr[u];
                        }
                        if (OP != OP_LL) {
#pragma unroll
                            for (int r = 0; r < RPL; ++r) acc[u % NACC][r] = fma(v[u], pi[u][r], acc[u % NACC][r]);
                        }
                    }
                }
            }
            if constexpr (BREG) {
                if (!fast && cur != brow_row) {
                    load_brow();
                    brow_row = cur;
                }
            }
        }
        if (OP != OP_LL) flush(cur, first_run, true);
    }

    if (OP == OP_LL) {
        double v = warp_sum(ll);
        if (wlane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NWARPS; ++w) s += red[w];
            a.llpart[t] = s;
        }
        return true;
    }

    if (segmented) {
        __syncthreads();
        // chains of partials: slot 0 (a row that began before the tile) and
        // every tail slot start a chain that continues through the head slots
        // of the following groups while they hold the same row
        T *carry = reinterpret_cast<T *>(a.carry);
        T *carry_head = carry + (int64_t)t * Rp;
        T *carry_tail = carry + ((int64_t)a.ntiles + t) * Rp;
        // row at the next tile's start if it goes on from this tile (nzrow[k1]), else -1
        const int32_t next_row = (p1 < a.nnz && !bit_at(n)) ? s_rows[s_meta[0] + s_meta[1]] : -1;
        for (int s = warp; s < 2 * NG; s += NWARPS) {
            if (!(s == 0 || (s & 1))) continue;
            const int32_t crow = slot_row[s];
            if (crow < 0) continue;
            const int gs = s >> 1;
            int gend = gs + 1;
            while (gend < NG && slot_row[2 * gend] == crow) ++gend;
            const bool complete = s != 0 && crow != next_row;
            for (int c = wlane; c < Rp; c += 32) {
                KSum<T> sum;
                sum.zero();
                sum.add(slot_val[(int64_t)s * Rp + c]);
                for (int k = gs + 1; k < gend; ++k) sum.add(slot_val[(int64_t)(2 * k) * Rp + c]);
                const T v = sum.value();
                if (s == 0) {
                    carry_head[c] = v;
                } else if (complete) {
                    out[(int64_t)crow * Rp + c] = v;
                    if (OP == OP_PHI) kkt = tmax(kkt, viol_t(__ldg(Bm + (int64_t)crow * Rp + c), v));
                } else {
                    carry_tail[c] = v;
                }
            }
            if (s == 0 || !complete) {
                // a partial of a row that spans tiles: publish it, and if it
                // is the row's last partial to arrive this block adds them up
                __threadfence();
                __syncwarp();
                if (wlane == 0) {
                    const int32_t si = __ldg(a.tsplit + 2 * t + (s == 0 ? 0 : 1));
                    if (si >= 0 && si < a.nsplit) {  // always, by construction of the table
                        const int32_t parts = __ldg(a.split + 3 * si + 2) - __ldg(a.split + 3 * si + 1) + 1;
                        if (atomicAdd(a.splitcnt + si, 1) == parts - 1) slot_fin[s == 0 ? 0 : 1] = si;
                    }
                }
            }
        }
        __syncthreads();
        // Rows that span tiles, finished by the tile whose partial came last:
        // the partials (tail of the first tile, heads of the others) are
        // added in tile order, so the result does not depend on which tile
        // finishes.  Columns are split into chunks of tiles across the block
        // and the chunk sums combined in chunk order.
#pragma unroll 1
        for (int f = 0; f < 2; ++f) {
            const int32_t si = slot_fin[f];
            if (si < 0) continue;
            __threadfence();
            const int32_t crow = __ldg(a.split + 3 * si + 0);
            const int32_t t0 = __ldg(a.split + 3 * si + 1);
            const int npart = __ldg(a.split + 3 * si + 2) - t0 + 1;
            auto part = [&](int k, int c) -> T {
                const int64_t off = k == 0 ? ((int64_t)a.ntiles + t0) * Rp : (int64_t)(t0 + k) * Rp;
                return __ldcg(carry + off + c);
            };
            if (Rp < THREADS) {
                const int nch = THREADS / Rp, c = tid % Rp, chunk = tid / Rp;
                KSum<T> sum;
                sum.zero();
                for (int k = chunk; k < npart; k += nch) sum.add(part(k, c));
                slot_val[tid] = sum.s;
                slot_val[THREADS + tid] = sum.c;
                __syncthreads();
                if (tid < Rp) {
                    KSum<T> tot;
                    tot.zero();
                    for (int k = 0; k < nch; ++k) {
                        tot.add(slot_val[k * Rp + c]);
                        tot.add(-slot_val[THREADS + k * Rp + c]);
                    }
                    const T v = tot.value();
                    out[(int64_t)crow * Rp + c] = v;
                    if (OP == OP_PHI) kkt = tmax(kkt, viol_t(__ldg(Bm + (int64_t)crow * Rp + c), v));
                }
                __syncthreads();
            } else {
                for (int c = tid; c < Rp; c += THREADS) {
                    KSum<T> sum;
                    sum.zero();
                    for (int k = 0; k < npart; ++k) sum.add(part(k, c));
                    const T v = sum.value();
                    out[(int64_t)crow * Rp + c] = v;
                    if (OP == OP_PHI) kkt = tmax(kkt, viol_t(__ldg(Bm + (int64_t)crow * Rp + c), v));
                }
            }
            if (tid == 0) a.splitcnt[si] = 0;  // ready for the next launch
        }
        // Rows without nonzeros are never written here: their Phi row is zero
        // in a buffer that starts zeroed, and their KKT term min(B, 1) is
        // added once per inner loop by empty_kkt_kernel (after the first
        // update those B rows are zero).
    }
    if (OP == OP_PHI && a.inner && !a.atomic) publish_kkt<THREADS>(kkt, a.inner, red);
    return true;
}

// One block per tile of one tensor.
template <typename T, int NM1, int RPL, int G, int OP, int THREADS, int U, bool PI>
__global__ void __launch_bounds__(THREADS) phi_tile_kernel(const PhiArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[THREADS / 32];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) stage_barrier_init(&bar);
    __syncthreads();
    uint32_t phase = 0;
    phi_tile_body<T, NM1, RPL, G, OP, THREADS, U, PI>(a, blockIdx.x, smem_raw, red, &bar, phase);
}

// The FP64 Phi kernel with the divisor on the FP32 pipe.  With four or more
// lanes per nonzero it runs at five blocks per SM (registers held to 96, a
// few spilled): measured on GB300 4-6% faster on the 3-way R = 32 and 5-way
// R = 32 and 64 tensors; with two lanes (R = 16, whose 2048-nonzero stages
// would then take 213 KB of an SM's shared memory) it was 3-4% slower, so
// those are held to four blocks (128 registers).
template <typename T, int NM1, int RPL, int G, int OP, int THREADS, int U, bool PI>
__global__ void __launch_bounds__(THREADS, G >= 4 ? 5 : 4) phi_tile_kernel_df(const PhiArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[THREADS / 32];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) stage_barrier_init(&bar);
    __syncthreads();
    uint32_t phase = 0;
    phi_tile_body<T, NM1, RPL, G, OP, THREADS, U, PI, true>(a, blockIdx.x, smem_raw, red, &bar, phase);
}

// The same with registers held to four resident blocks per SM (64 per
// thread at 256 threads): measured on GB300 the better trade for FP32 with
// one float4 per lane, where more warps hide more gather latency.
template <typename T, int NM1, int RPL, int G, int OP, int THREADS, int U, bool PI>
__global__ void __launch_bounds__(THREADS, 4) phi_tile_kernel_occ4(const PhiArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[THREADS / 32];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) stage_barrier_init(&bar);
    __syncthreads();
    uint32_t phase = 0;
    phi_tile_body<T, NM1, RPL, G, OP, THREADS, U, PI>(a, blockIdx.x, smem_raw, red, &bar, phase);
}

// Materialised Khatri-Rao rows, the paper's Pi (Algorithm 3 reads Pi[j][r]):
// Pi[p][:] = A^(m_0)[i_m0(p), :] * A^(m_1)[i_m1(p), :] * ... over the modes
// m != n, for every nonzero p in mode-n order.  The products are taken in the
// same order as the fused tile kernel forms them, so a Phi from the
// materialised Pi equals the fused one bit for bit.  One thread per 16-byte
// vector of a row (elements e0, e0 + step, ... below e1); rows are written
// with evict-first stores (read once per inner iteration, they are not worth
// keeping in L2).
template <typename T, int NM1>
__device__ __forceinline__ void pi_build_range(const PhiArgs &a, T *__restrict__ pi, int64_t e0, int64_t e1,
                                               int64_t step) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    constexpr int MAXK = NM1 > 0 ? NM1 : kMaxNm1;
    const int nm1 = NM1 > 0 ? NM1 : a.nm1;
    const int vpr = a.Rp / VN;  // vectors per row, a power of two (Rp is one)
    const int lg = 31 - __clz(vpr);
    for (int64_t e = e0; e < e1; e += step) {
        const int64_t p = e >> lg;
        const int c = (int)(e & (vpr - 1)) * VN;
        V x = __ldg(reinterpret_cast<const V *>(reinterpret_cast<const T *>(a.A[0]) +
                                                (int64_t)__ldg(a.idx[0] + p) * a.Rp + c));
#pragma unroll
        for (int k = 1; k < MAXK; ++k) {
            if (k < nm1) {
                const V y = __ldg(reinterpret_cast<const V *>(reinterpret_cast<const T *>(a.A[k]) +
                                                              (int64_t)__ldg(a.idx[k] + p) * a.Rp + c));
                if constexpr (VN == 4) {
                    x.x *= y.x;
                    x.y *= y.y;
                    x.z *= y.z;
                    x.w *= y.w;
                } else {
                    x.x *= y.x;
                    x.y *= y.y;
                }
            }
        }
        __stcs(reinterpret_cast<V *>(pi + p * a.Rp + c), x);
    }
}

template <typename T, int NM1>
__global__ void __launch_bounds__(256) pi_build_kernel(const PhiArgs a, T *__restrict__ pi) {
    const int64_t total = a.nnz * (a.Rp / Vec16<T>::n);
    pi_build_range<T, NM1>(a, pi, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, total,
                           (int64_t)gridDim.x * blockDim.x);
}

// FP32 with one float4 per lane runs at four blocks per SM
template <typename T, int RPL>
__host__ __device__ constexpr bool phi_occ4() {
    return sizeof(T) == 4 && RPL <= 4;
}

// KKT term of the rows without nonzeros, |min(B, 1 - 0)|, published into
// the slot of the first inner iteration (run after the S/B kernel, which
// cleared that slot).  Later iterations need no term: the first update sets
// those B rows to B * 0 = 0.
template <typename T>
__global__ void __launch_bounds__(256) empty_kkt_kernel(const int32_t *__restrict__ erows, int64_t nempty, int Rp,
                                                         const T *__restrict__ B, InnerState *inner) {
    __shared__ double red[8];
    const int lg = 31 - __clz(Rp);  // Rp is a power of two
    T v = T(0);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nempty * Rp;
         q += (int64_t)gridDim.x * blockDim.x)
        v = tmax(v, viol_t(B[(int64_t)erows[q >> lg] * Rp + (q & (Rp - 1))], T(0)));
    publish_kkt<256>((double)v, inner, red);
}

// Writes zeros into the rows without nonzeros.
template <typename T>
__global__ void zero_rows_kernel(const int32_t *__restrict__ erows, int64_t nempty, int Rp, T *__restrict__ out) {
    const int lg = 31 - __clz(Rp);  // Rp is a power of two
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nempty * Rp;
         q += (int64_t)gridDim.x * blockDim.x)
        out[(int64_t)erows[q >> lg] * Rp + (q & (Rp - 1))] = T(0);
}

// KKT violation over all rows (used after the atomic reduction).
template <typename T>
__global__ void __launch_bounds__(256) kkt_rows_kernel(const T *__restrict__ B, const T *__restrict__ P, int64_t n,
                                                        InnerState *inner) {
    if (inner->done) return;
    __shared__ double red[8];
    double v = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v = fmax(v, (double)viol_t(B[e], P[e]));
    publish_kkt<256>(v, inner, red);
}

}  // namespace cpapr
