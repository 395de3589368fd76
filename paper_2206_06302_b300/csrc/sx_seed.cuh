// sx_seed.cuh -- the seeded generator of libsx's bulk construction (sx_seed_uniform, the SEED
// items of batches and serving steps): SplitMix64 words in counter form, mapped to uniform
// values in [lo, hi) exactly as the host-side definition does.
#pragma once

#include <cstdint>

#include "sx_device.cuh"

namespace sx {
namespace dev {

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
// The same value with u assembled and the product taken on the integer units (mul_rn_int, exact
// round-to-nearest-even; SHORT when span's significand has at most 11 bits): only the sum uses
// the FP64 pipe.  u = M 2^-53 with M = w >> 11 < 2^53: for M > 0 its leading bit e gives the
// normal double 1.f 2^(e - 53).
__device__ __forceinline__ double seeded_u53_int(uint64_t w) {
    const uint64_t m = w >> 11;
    if (m == 0) return 0.0;
    const int e = 63 - __clzll((long long)m);  // 0 .. 52
    const uint64_t frac = (m << (52 - e)) & 0x000FFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(((uint64_t)(970 + e) << 52) | frac));
}
template <bool SHORT>
__device__ __forceinline__ double seeded_value_int(uint64_t w, double lo, double span) {
    return __dadd_rn(lo, mul_rn_int<SHORT>(seeded_u53_int(w), span));
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
// MV (binary64, general range): 0 = every element on the FP64 pipe; 1 and 3 = three of every
// four elements through seeded_value_int (3: span has a short significand), so that the FP64
// pipe (three operations for the others, one for these) and the integer units share the work:
// at n = 2^27 1.25-1.33 TB/s with every element on the FP64 pipe, 1.98 with one in two on the
// integer units, 2.35-2.45 with three in four, 2.15-2.26 with seven in eight.  All forms give
// the same bits.
template <class T, bool PM1, int MV = 0>
__device__ __forceinline__ T seed_one(uint64_t w, T lo, T span, uint64_t k = 0) {
    if constexpr (PM1) return seeded_value_pm1(w);
    else if constexpr (sizeof(T) == 8 && MV != 0)
        return (k & 3) ? seeded_value_int<MV == 3>(w, lo, span) : seeded_value(w, lo, span);
    else return seeded_value(w, lo, span);
}
template <class T, bool PM1, int MV = 0>
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
        out[i] = seed_one<T, PM1, MV>(splitmix_word(seed, base + i), lo, span, i);
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
                const double v = !PM1 ? seed_one<double, false, MV>(w, (double)lo, (double)span, j)
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

}  // namespace dev
}  // namespace sx
