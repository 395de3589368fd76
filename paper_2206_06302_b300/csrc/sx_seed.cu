// sx_seed.cu -- bulk construction on the device (Section 3.2: the allocator constructs the
// elements of a placed array in bulk; Section 4.2: on a GPU target by a kernel): a value for
// every element (sx_bulk_construct) or seeded uniform values in [lo, hi) (sx_seed_uniform).
// Construction writes only: it is bound by the integer units that compute the generator's words
// (sx_seed.cuh), not by HBM.
#include "sx_internal.h"
#include "sx_seed.cuh"

namespace sx {
namespace {

using namespace dev;

// ---- seeded bulk construction ---------------------------------------------------------------
// All threads of the grid share the range (seed_range); PM1: lo = -1, hi = 1 in binary64.
// Blocks of 256 threads that one SM holds at once: the bounds make the compiler keep each form's
// registers within them (the binary64 [-1, 1) form needs 38 registers: 6 blocks; the others fit
// 32: 8), and the grid-stride loop launches no more than that, so that no block waits for
// another to finish before it starts (such blocks would run the loop's last share alone).
template <class T, bool PM1>
constexpr int seed_blocks_per_sm() { return (sizeof(T) == 8 && PM1) ? 6 : 8; }

template <class T, bool PM1, int MV = 0>
__global__ void __launch_bounds__(256, seed_blocks_per_sm<T, PM1>())
    k_seed(T *out, uint64_t n, uint64_t seed, T lo, T span, uint64_t base) {
    seed_range<T, PM1, MV>(out, n, seed, base, lo, span, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                           (uint64_t)gridDim.x * blockDim.x);
}

// Blocks of 256 threads for `n` elements taken `per_thread` at a time: at most `per_sm` per SM of
// the current device.
unsigned seed_blocks(size_t n, int per_thread, int per_sm) {
    static std::atomic<int> sms[64];  // per device, 0 until first asked
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t nsm = 148;
    if (dev >= 0 && dev < 64) {
        int v = sms[dev].load(std::memory_order_relaxed);
        if (v == 0) {
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
            if (v <= 0) v = 148;
            sms[dev].store(v, std::memory_order_relaxed);
        }
        nsm = (uint64_t)v;
    }
    uint64_t b = (n + 256ull * per_thread - 1) / (256ull * per_thread);
    if (b > nsm * per_sm) b = nsm * per_sm;
    return b == 0 ? 1u : (unsigned)b;
}

// ---- construction with one value: stores only ------------------------------------------------
// Elements [0, head) and [head + nvec * 32 / sizeof(T), n) one by one by the first threads of the
// grid; the body is nvec 32-byte vector stores of `word` (the value's bits repeated over 8 bytes),
// in tiles of two stores per thread, one tile per block (a grid-stride loop over tiles only
// beyond 2^31 blocks).  Measured on B300 at 1 GiB: one tile per block 7.3 TB/s, a grid-stride
// loop over 16 blocks per SM 6.8 TB/s.
constexpr int kFillThreads = 256, kFillUnroll = 2;
template <class T>
__global__ void __launch_bounds__(kFillThreads) k_fill(T *out, uint64_t n, uint64_t head, uint64_t nvec, T v,
                                                       uint64_t word) {
    constexpr uint64_t EPV = 32 / sizeof(T);
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t body_end = head + nvec * EPV;
    if (gtid < head + (n - body_end)) out[gtid < head ? gtid : body_end + (gtid - head)] = v;
    char *b = reinterpret_cast<char *>(out + head);
    const uint64_t w[4] = {word, word, word, word};
    const uint64_t tile = (uint64_t)blockDim.x * kFillUnroll;
    for (uint64_t base = (uint64_t)blockIdx.x * tile; base < nvec; base += (uint64_t)gridDim.x * tile) {
#pragma unroll
        for (int u = 0; u < kFillUnroll; ++u) {
            const uint64_t k = base + (uint64_t)u * blockDim.x + threadIdx.x;
            if (k < nvec) stv<32, 0>(b + 32 * k, w);
        }
    }
}

template <class T>
int fill_t(cudaStream_t s, T *out, size_t n, T v, uint64_t word) {
    const uintptr_t mis = (uintptr_t)out % 32;
    uint64_t head = mis % sizeof(T) ? n : ((32 - mis) % 32) / sizeof(T);
    if (head > n) head = n;
    const uint64_t nvec = (n - head) * sizeof(T) / 32;
    const uint64_t edge = n - nvec * 32 / sizeof(T);
    const uint64_t tile = (uint64_t)kFillThreads * kFillUnroll;
    uint64_t b = (nvec + tile - 1) / tile;
    if (b > 0x7fffffffull) b = 0x7fffffffull;  // then a grid-stride loop over the tiles
    const uint64_t eb = (edge + kFillThreads - 1) / kFillThreads;
    if (b < eb) b = eb;
    if (b == 0) b = 1;
    if (b > 0x7fffffffull) return fail(SX_ERR_INVALID, "bulk_construct: array too long for its edge elements");
    k_fill<T><<<(unsigned)b, kFillThreads, 0, s>>>(out, n, head, nvec, v, word);
    return SX_OK;
}

}  // namespace

int launch_fill(cudaStream_t s, int dtype, void *out, size_t n, double value) {
    if (n == 0) return SX_OK;
    if (dtype == SX_F64) {
        uint64_t w;
        std::memcpy(&w, &value, 8);
        SX_TRY(fill_t<double>(s, (double *)out, n, value, w));
    } else if (dtype == SX_F32) {
        const float f = (float)value;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        SX_TRY(fill_t<float>(s, (float *)out, n, f, ((uint64_t)u << 32) | u));
    } else if (dtype == SX_U8) {
        const uint8_t c = (uint8_t)value;
        SX_TRY(fill_t<uint8_t>(s, (uint8_t *)out, n, c, 0x0101010101010101ull * c));
    } else {
        return fail(SX_ERR_DTYPE, "bulk_construct: unsupported dtype %d", dtype);
    }
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

int launch_seed(cudaStream_t s, int dtype, void *out, size_t n, uint64_t seed, double lo, double hi,
                uint64_t index_base) {
    if (n == 0) return SX_OK;
    if (dtype == SX_F64) {
        const double span = hi - lo;
        const unsigned b = seed_blocks(n, 8, seed_blocks_per_sm<double, false>());
        const unsigned b_pm1 = seed_blocks(n, 8, seed_blocks_per_sm<double, true>());
        // general range: most products on the integer units (not for a zero, subnormal, infinite
        // or NaN span, which the integer product would only send back to the FP64 pipe)
        const int mv = mul_variant(1, span);
        if (lo == -1.0 && hi == 1.0)
            k_seed<double, true><<<b_pm1, 256, 0, s>>>((double *)out, n, seed, lo, span, index_base);
        else if (mv == 3)
            k_seed<double, false, 3><<<b, 256, 0, s>>>((double *)out, n, seed, lo, span, index_base);
        else if (mv == 1)
            k_seed<double, false, 1><<<b, 256, 0, s>>>((double *)out, n, seed, lo, span, index_base);
        else
            k_seed<double, false, 0><<<b, 256, 0, s>>>((double *)out, n, seed, lo, span, index_base);
    } else if (dtype == SX_F32) {
        const float lo32 = (float)lo, hi32 = (float)hi;
        const float span = hi32 - lo32;
        k_seed<float, false><<<seed_blocks(n, 16, seed_blocks_per_sm<float, false>()), 256, 0, s>>>(
            (float *)out, n, seed, lo32, span, index_base);
    } else {
        return fail(SX_ERR_DTYPE, "seed_uniform takes F32 or F64 (got dtype %d)", dtype);
    }
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

}  // namespace sx
