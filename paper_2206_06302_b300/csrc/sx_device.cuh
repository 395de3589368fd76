// sx_device.cuh -- device helpers shared by libsx's kernels: the element operations of the
// four STREAM kernels (Section 5, Listing 4) and raw vector loads/stores.  The seeded generator
// is in sx_seed.cuh.
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

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace dev
}  // namespace sx
