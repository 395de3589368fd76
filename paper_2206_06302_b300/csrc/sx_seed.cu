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
template <class T, bool PM1, int MV = 0>
__global__ void __launch_bounds__(256) k_seed(T *out, uint64_t n, uint64_t seed, T lo, T span, uint64_t base) {
    seed_range<T, PM1, MV>(out, n, seed, base, lo, span, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                           (uint64_t)gridDim.x * blockDim.x);
}

// Blocks of 256 threads for `n` elements taken `per_thread` at a time: up to 8 per SM.
unsigned seed_blocks(size_t n, int per_thread) {
    uint64_t b = (n + 256ull * per_thread - 1) / (256ull * per_thread);
    if (b > 148ull * 8) b = 148ull * 8;
    return b == 0 ? 1u : (unsigned)b;
}

template <class T>
__global__ void k_fill(T *out, uint64_t n, T v) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = v;
}

unsigned setup_blocks(size_t n) {
    uint64_t b = (n + 255) / 256;
    if (b > 148ull * 32) b = 148ull * 32;
    return b == 0 ? 1u : (unsigned)b;
}

}  // namespace

int launch_fill(cudaStream_t s, int dtype, void *out, size_t n, double value) {
    if (n == 0) return SX_OK;
    const unsigned b = setup_blocks(n);
    if (dtype == SX_F64) k_fill<double><<<b, 256, 0, s>>>((double *)out, n, value);
    else if (dtype == SX_F32) k_fill<float><<<b, 256, 0, s>>>((float *)out, n, (float)value);
    else if (dtype == SX_U8) k_fill<uint8_t><<<b, 256, 0, s>>>((uint8_t *)out, n, (uint8_t)value);
    else return fail(SX_ERR_DTYPE, "bulk_construct: unsupported dtype %d", dtype);
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

int launch_seed(cudaStream_t s, int dtype, void *out, size_t n, uint64_t seed, double lo, double hi,
                uint64_t index_base) {
    if (n == 0) return SX_OK;
    if (dtype == SX_F64) {
        const double span = hi - lo;
        const unsigned b = seed_blocks(n, 8);
        // general range: most products on the integer units (not for a zero, subnormal, infinite
        // or NaN span, which the integer product would only send back to the FP64 pipe)
        const int mv = mul_variant(1, span);
        if (lo == -1.0 && hi == 1.0)
            k_seed<double, true><<<b, 256, 0, s>>>((double *)out, n, seed, lo, span, index_base);
        else if (mv == 3)
            k_seed<double, false, 3><<<b, 256, 0, s>>>((double *)out, n, seed, lo, span, index_base);
        else if (mv == 1)
            k_seed<double, false, 1><<<b, 256, 0, s>>>((double *)out, n, seed, lo, span, index_base);
        else
            k_seed<double, false, 0><<<b, 256, 0, s>>>((double *)out, n, seed, lo, span, index_base);
    } else if (dtype == SX_F32) {
        const float lo32 = (float)lo, hi32 = (float)hi;
        const float span = hi32 - lo32;
        k_seed<float, false><<<seed_blocks(n, 16), 256, 0, s>>>((float *)out, n, seed, lo32, span, index_base);
    } else {
        return fail(SX_ERR_DTYPE, "seed_uniform takes F32 or F64 (got dtype %d)", dtype);
    }
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

}  // namespace sx
