// sx_device.cuh -- device helpers shared by libsx's kernels: the element operations of the
// four STREAM kernels (Section 5, Listing 4), raw vector loads/stores, the seeded generator.
#pragma once

#include <cstdint>

#include "sx.h"

namespace sx {
namespace dev {

// ---- element arithmetic --------------------------------------------------------------------
// One IEEE operation each, rounded to nearest even.  The _rn intrinsics are never contracted
// into a fused multiply-add, so Triad keeps its two roundings.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

template <int OP>
__host__ __device__ constexpr bool has_y() { return OP == SX_OP_ADD || OP == SX_OP_TRIAD; }

// ---- binary64 product on the integer units ----------------------------------------------------
// B300's FP64 pipe issues about two operations per clock per SM, which is what bounds an FP64
// Triad (one multiply and one add per 24 bytes) below the HBM rate.  This computes the same
// correctly rounded product RN(c*q) from the IEEE-754 definition with 64-bit integer
// arithmetic: the 53-bit significands multiply to a 105/106-bit product (high word by
// __umul64hi, low word for the sticky bit), which is normalised and rounded to nearest even.
// Whenever c or q is zero, subnormal, infinite or NaN, or the rounded result would be
// subnormal or overflow, it defers to the FP64 pipe (__dmul_rn), so the result is bit-identical
// to __dmul_rn for every input.
//
// The fallback sits in a function that is never inlined: an inlined DMUL would be if-converted
// into a predicated instruction that still occupies the FP64 pipe for every element.
static __device__ __noinline__ double dmul_fallback(double c, double q) { return __dmul_rn(c, q); }

//
// SHORT selects, at compile time, the path for a scalar whose significand has at most 11
// significant bits (q = 3.0 has two): the caller guarantees it (see q_short_significand).
template <bool SHORT>
__device__ __forceinline__ double mul_rn_int(double c, double q) {
    const uint64_t cb = (uint64_t)__double_as_longlong(c);
    const uint64_t qb = (uint64_t)__double_as_longlong(q);
    const uint32_t ce = (uint32_t)(cb >> 52) & 0x7FFu;
    const uint32_t qe = (uint32_t)(qb >> 52) & 0x7FFu;
    // q-only quantities (loop invariant): q = Qs * 2^tz * 2^(qe-1075) with Qs odd
    const uint64_t qsig = (qb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const uint32_t tz = (uint32_t)__ffsll((long long)qsig) - 1u;
    const uint64_t qs = qsig >> tz;
    const uint32_t L = 64u - (uint32_t)__clzll((long long)qs);  // bits of Qs, 1..53
    const uint64_t mc = (cb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    uint64_t m;
    int e;
    if constexpr (SHORT) {
        // short significand (q = 3 has two bits): Mc*Qs < 2^64 is exact in one word
        const uint64_t p = mc * qs;                         // in [2^(51+L), 2^(53+L))
        const uint32_t top = (uint32_t)(p >> (52u + L)) & 1u;
        const uint32_t s = L - 1u + top;                    // bits dropped to keep 53
        m = p >> s;
        const uint64_t rb = s ? (p >> (s - 1u)) & 1u : 0u;
        const uint64_t st = s > 1u ? p & ((1ull << (s - 1u)) - 1u) : 0u;
        m += rb & ((st != 0) | (m & 1u));                   // ties to even
        e = (int)ce + (int)qe + (int)s + (int)tz - 1075;
    } else {
        const uint64_t a = mc << 11;                        // leading bit at 63
        const uint64_t b = qsig << 11;
        const uint64_t hi = __umul64hi(a, b);               // product / 2^64, in [2^62, 2^64)
        const uint64_t lo = a * b;
        const uint32_t top = (uint32_t)(hi >> 63);          // product significand in [2, 4)
        const uint32_t sh = 10u + top;
        m = hi >> sh;                                       // 53 bits
        const uint64_t rb = (hi >> (sh - 1)) & 1u;          // first dropped bit
        const uint64_t st = (hi & ((1ull << (sh - 1)) - 1)) | lo;
        m += rb & ((st != 0) | (m & 1u));                   // ties to even
        e = (int)ce + (int)qe - 1023 + (int)top;            // biased exponent before the carry
    }
    const int ef = e + (int)(m >> 53);
    const bool ok = (ce - 1u < 2046u) & (qe - 1u < 2046u) & (e >= 1) & (ef <= 2046);
    if (!ok) return dmul_fallback(c, q);
    const uint64_t bits = ((uint64_t)e << 52) + (m - (1ull << 52));  // a carry bumps the exponent
    return __longlong_as_double((long long)(bits | ((cb ^ qb) & 0x8000000000000000ull)));
}

// Product used by SCALE/TRIAD, by kernel variant MM:
//   0 = FP64 pipe; 1 = integer units; 2 = integer units and FP64 pipe alternating by the parity
//   of `k` (the word index within a thread's vector); 3 and 4 = as 1 and 2 with the
//   short-significand path.  The host picks MM from the launch's fp64_mul and q (mul_variant).
template <int MM, class T>
__device__ __forceinline__ T mul_sel(T x, T q, int k) {
    if constexpr (sizeof(T) == 8 && MM == 1) return mul_rn_int<false>(x, q);
    else if constexpr (sizeof(T) == 8 && MM == 2) return (k & 1) ? mul_rn(x, q) : mul_rn_int<false>(x, q);
    else if constexpr (sizeof(T) == 8 && MM == 3) return mul_rn_int<true>(x, q);
    else if constexpr (sizeof(T) == 8 && MM == 4) return (k & 1) ? mul_rn(x, q) : mul_rn_int<true>(x, q);
    else return mul_rn(x, q);
}

// COPY out=x, SCALE out=x*q, ADD out=x+y, TRIAD out=x+y*q.
template <int OP, class T>
__device__ __forceinline__ T apply_op(T x, T y, T q) {
    if constexpr (OP == SX_OP_COPY) return x;
    else if constexpr (OP == SX_OP_SCALE) return mul_rn(x, q);
    else if constexpr (OP == SX_OP_ADD) return add_rn(x, y);
    else return add_rn(x, mul_rn(y, q));
}

// apply_op with the product taken by mul_sel<MM>.
template <int OP, int MM, class T>
__device__ __forceinline__ T apply_op_mm(T x, T y, T q, int k) {
    if constexpr (OP == SX_OP_COPY) return x;
    else if constexpr (OP == SX_OP_SCALE) return mul_sel<MM>(x, q, k);
    else if constexpr (OP == SX_OP_ADD) return add_rn(x, y);
    else return add_rn(x, mul_sel<MM>(y, q, k));
}

// The op on one 64-bit word: one binary64 element or two binary32 elements.  `k` is the word's
// index within the thread's vector (selects the product unit when MM == 2).
template <int OP, class T, int MM = 0>
__device__ __forceinline__ uint64_t op_word(uint64_t xw, uint64_t yw, T q, int k = 0) {
    if constexpr (OP == SX_OP_COPY) {
        return xw;
    } else if constexpr (sizeof(T) == 8) {
        double r = apply_op_mm<OP, MM, double>(__longlong_as_double((long long)xw),
                                               __longlong_as_double((long long)yw), q, k);
        return (uint64_t)__double_as_longlong(r);
    } else {
        float r0 = apply_op<OP, float>(__uint_as_float((uint32_t)xw), __uint_as_float((uint32_t)yw), q);
        float r1 = apply_op<OP, float>(__uint_as_float((uint32_t)(xw >> 32)),
                                       __uint_as_float((uint32_t)(yw >> 32)), q);
        return (uint64_t)__float_as_uint(r0) | ((uint64_t)__float_as_uint(r1) << 32);
    }
}

// ---- vector loads and stores (inline PTX) ---------------------------------------------------
// HINT 0: read-only path (ld.global.nc), default stores.
// HINT 1: streaming: read-only path without L1 allocation and a 256-byte L2 prefetch hint,
//         evict-first (.cs) stores.
// HINT 2: coherent loads (ld.global), used when the output aliases an input.
template <int VB, int HINT>
__device__ __forceinline__ void ldv(const char *p, uint64_t (&w)[VB / 8]) {
    if constexpr (VB == 16) {
        if constexpr (HINT == 0)
            asm volatile("ld.global.nc.v2.u64 {%0,%1}, [%2];" : "=l"(w[0]), "=l"(w[1]) : "l"(p));
        else if constexpr (HINT == 1)
            asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v2.u64 {%0,%1}, [%2];"
                         : "=l"(w[0]), "=l"(w[1]) : "l"(p));
        else
            asm volatile("ld.global.v2.u64 {%0,%1}, [%2];" : "=l"(w[0]), "=l"(w[1]) : "l"(p));
    } else {
        if constexpr (HINT == 0)
            asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3]) : "l"(p));
        else if constexpr (HINT == 1)
            asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3]) : "l"(p));
        else
            asm volatile("ld.global.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3]) : "l"(p));
    }
}

template <int VB, int HINT>
__device__ __forceinline__ void stv(char *p, const uint64_t (&w)[VB / 8]) {
    if constexpr (VB == 16) {
        if constexpr (HINT == 1)
            asm volatile("st.global.cs.v2.u64 [%0], {%1,%2};" ::"l"(p), "l"(w[0]), "l"(w[1]) : "memory");
        else
            asm volatile("st.global.v2.u64 [%0], {%1,%2};" ::"l"(p), "l"(w[0]), "l"(w[1]) : "memory");
    } else {
        if constexpr (HINT == 1)
            asm volatile("st.global.cs.v4.u64 [%0], {%1,%2,%3,%4};" ::"l"(p), "l"(w[0]), "l"(w[1]),
                         "l"(w[2]), "l"(w[3]) : "memory");
        else
            asm volatile("st.global.v4.u64 [%0], {%1,%2,%3,%4};" ::"l"(p), "l"(w[0]), "l"(w[1]),
                         "l"(w[2]), "l"(w[3]) : "memory");
    }
}

// ---- seeded construction: SplitMix64 in counter form ----------------------------------------
// Word i under `seed` is the (i+1)-th output of SplitMix64 (Steele, Lea & Flood 2014, with
// Vigna's 64-bit finaliser) started from state `seed`: splitmix_mix(seed + (i+1) gamma).
constexpr uint64_t kSplitmixGamma = 0x9E3779B97F4A7C15ull;

// The finaliser on 32-bit halves: each z ^ (z >> s) (s < 32) is one funnel shift and one shift
// with two XORs; the products stay 64-bit.
__device__ __forceinline__ void xorshift_halves(uint32_t &lo, uint32_t &hi, int s) {
    lo ^= __funnelshift_r(lo, hi, s);
    hi ^= hi >> s;
}
// HIGH_ONLY: the result is exact in bits 33..63 only.  The last step z ^ (z >> 31) leaves those
// bits as they are (the shifted term is zero there), so a caller that uses w >> 40 (binary32
// values) skips it.
template <bool HIGH_ONLY = false>
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    uint32_t lo = (uint32_t)z, hi = (uint32_t)(z >> 32);
    xorshift_halves(lo, hi, 30);
    z = (((uint64_t)hi << 32) | lo) * 0xBF58476D1CE4E5B9ull;
    lo = (uint32_t)z;
    hi = (uint32_t)(z >> 32);
    xorshift_halves(lo, hi, 27);
    z = (((uint64_t)hi << 32) | lo) * 0x94D049BB133111EBull;
    if (HIGH_ONLY) return z;
    lo = (uint32_t)z;
    hi = (uint32_t)(z >> 32);
    xorshift_halves(lo, hi, 31);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t splitmix_word(uint64_t seed, uint64_t i) {
    return splitmix_mix(seed + (i + 1) * kSplitmixGamma);
}

// lo + span*u with u = (w >> 11) 2^-53 (binary64) or (w >> 40) 2^-24 (binary32), each step
// rounded to nearest even; span = RN(hi - lo) is computed by the caller in the same type.
// The binary64 u is built exactly from the word's bits: with m the low 52 bits of w >> 11,
// D = 0.5 + m 2^-53 lies in [0.5, 1), and u = D when the top bit of w is set, else D - 0.5
// (exact by Sterbenz); one FP64 subtraction instead of a 64-bit conversion and a product.
__device__ __forceinline__ double seeded_u53(uint64_t w) {
    const uint32_t wl = (uint32_t)w, wh = (uint32_t)(w >> 32);
    const uint32_t dlo = __funnelshift_r(wl, wh, 11);
    const uint32_t dhi = ((wh >> 11) & 0xFFFFFu) | 0x3FE00000u;
    const uint32_t chi = (wh >> 31) ? 0u : 0x3FE00000u;  // 0.0 or 0.5
    return __dsub_rn(__hiloint2double((int)dhi, (int)dlo), __hiloint2double((int)chi, 0));
}
__device__ __forceinline__ double seeded_value(uint64_t w, double lo, double span) {
    return __dadd_rn(lo, __dmul_rn(span, seeded_u53(w)));
}
__device__ __forceinline__ float seeded_value(uint64_t w, float lo, float span) {
    const float u = __fmul_rn(__uint2float_rn((uint32_t)(w >> 40)), 0x1p-24f);
    return __fadd_rn(lo, __fmul_rn(span, u));
}

// The binary64 value for lo = -1, hi = 1.  There span = 2, RN(2u) = 2u and RN(-1 + 2u) =
// k * 2^-52 exactly, with k = (w >> 11) - 2^52 in [-2^52, 2^52) (k = 0 gives +0, as -1 + 1 does
// under round to nearest).  Two constructions, each bit-identical to seeded_value(w, -1.0, 2.0):
//
// seeded_value_pm1 assembles the double from |k|'s leading bit on the integer units.  When
// |k| >= 2^32 (all words but one in 2^20) the leading bit is in the high half and the
// normalising shift is one funnel shift; smaller |k| take the general path.
static __device__ __noinline__ double pm1_small(int64_t k) {
    if (k == 0) return 0.0;
    const uint64_t a = k < 0 ? (uint64_t)(-k) : (uint64_t)k;  // 1 .. 2^32 - 1
    const int e = 63 - __clzll((long long)a);
    const uint64_t frac = (a << (52 - e)) & 0x000FFFFFFFFFFFFFull;
    const uint64_t bits = ((uint64_t)(1023 + e - 52) << 52) | frac | (k < 0 ? 0x8000000000000000ull : 0ull);
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double seeded_value_pm1(uint64_t w) {
    const uint32_t wl = (uint32_t)w, wh = (uint32_t)(w >> 32);
    const uint32_t klo = __funnelshift_r(wl, wh, 11);
    const int32_t khi = (int32_t)(wh >> 11) - (1 << 20);
    const uint32_t sg = (uint32_t)(khi >> 31);  // all ones when k < 0
    const uint64_t k = ((uint64_t)(uint32_t)khi << 32) | klo;
    const uint64_t a = (k ^ ((uint64_t)sg << 32 | sg)) - ((uint64_t)sg << 32 | sg);  // |k|
    const uint32_t alo = (uint32_t)a, ahi = (uint32_t)(a >> 32);
    if (ahi == 0) return pm1_small((int64_t)k);
    const uint32_t c = __clz(ahi);  // 11 .. 31: |k| = 1.f * 2^(63 - c)
    const uint32_t sh = c - 11;     // moves the leading bit to bit 52
    const uint32_t mhi = __funnelshift_l(alo, ahi, sh);
    const uint32_t mlo = alo << sh;
    // the leading bit (bit 20 of mhi) adds one to the biased exponent (1034 - c) - 1
    const uint32_t hi = mhi - (c << 20) + ((1033u << 20) | (sg & 0x80000000u));
    return __hiloint2double((int)hi, (int)mlo);
}
// seeded_value_pm1_sub uses one FP64 subtraction instead.  With m the low 52 bits of w >> 11
// and D = 1 + m 2^-52, the value is D - 1 when the top bit of w is set and D - 2 otherwise;
// D lies in [1, 2), so both differences are exact (Sterbenz) and D - 1 is +0 for m = 0.
__device__ __forceinline__ double seeded_value_pm1_sub(uint64_t w) {
    const uint32_t wl = (uint32_t)w, wh = (uint32_t)(w >> 32);
    const uint32_t dlo = __funnelshift_r(wl, wh, 11);
    const uint32_t dhi = ((wh >> 11) & 0xFFFFFu) | 0x3FF00000u;
    const uint32_t chi = 0x40000000u - (wh >> 31) * 0x00100000u;  // 2.0 or 1.0
    return __dsub_rn(__hiloint2double((int)dhi, (int)dlo), __hiloint2double((int)chi, 0));
}

// Seeded construction of out[e] = value(seed, base + e), e in [0, cnt), by `nthr` cooperating
// threads (this one is `tid`): a scalar head up to a 32-byte boundary, a body of 32-byte stores
// with 8 (binary64) or 16 (binary32) consecutive elements per thread and step, and a scalar
// tail.  The counter advances by gamma from one element to the next.  PM1 selects lo = -1,
// hi = 1 (binary64 only), where 5 of every 8 elements take the subtraction and 3 the integer
// assembly, so that the FP64 pipe and the integer units share the work.
template <class T, bool PM1>
__device__ __forceinline__ T seed_one(uint64_t w, T lo, T span) {
    if constexpr (PM1) return seeded_value_pm1(w);
    else return seeded_value(w, lo, span);
}
template <class T, bool PM1>
__device__ __forceinline__ void seed_range(T *out, uint64_t cnt, uint64_t seed, uint64_t base, T lo,
                                           T span, uint64_t tid, uint64_t nthr) {
    constexpr int E = sizeof(T) == 8 ? 8 : 16;  // elements per thread and step: 64 bytes
    static_assert(!PM1 || sizeof(T) == 8, "lo = -1, hi = 1 construction is binary64");
    const uintptr_t mis = (uintptr_t)out % 32;
    uint64_t head = mis % sizeof(T) ? cnt : ((32 - mis) % 32) / sizeof(T);
    if (head > cnt) head = cnt;
    const uint64_t nrun = (cnt - head) / E;
    const uint64_t body_end = head + nrun * E;
    for (uint64_t e = tid; e < head + (cnt - body_end); e += nthr) {
        const uint64_t i = e < head ? e : body_end + (e - head);
        out[i] = seed_one<T, PM1>(splitmix_word(seed, base + i), lo, span);
    }
    for (uint64_t r = tid; r < nrun; r += nthr) {
        const uint64_t i0 = head + r * E;
        uint64_t z = seed + (base + i0 + 1) * kSplitmixGamma;
        uint64_t b[E * sizeof(T) / 8];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const uint64_t w = splitmix_mix<sizeof(T) == 4>(z);  // binary32 uses bits 40..63 only
            z += kSplitmixGamma;
            if constexpr (sizeof(T) == 8) {
                const double v = !PM1 ? seeded_value(w, (double)lo, (double)span)
                                      : (j % 8 < 5 ? seeded_value_pm1_sub(w) : seeded_value_pm1(w));
                b[j] = (uint64_t)__double_as_longlong(v);
            } else {
                const uint32_t v = __float_as_uint(seeded_value(w, (float)lo, (float)span));
                if (j % 2 == 0) b[j / 2] = v;
                else b[j / 2] |= (uint64_t)v << 32;
            }
        }
        char *p = reinterpret_cast<char *>(out + i0);
        stv<32, 0>(p, *reinterpret_cast<const uint64_t(*)[4]>(&b[0]));
        stv<32, 0>(p + 32, *reinterpret_cast<const uint64_t(*)[4]>(&b[4]));
    }
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace dev
}  // namespace sx
