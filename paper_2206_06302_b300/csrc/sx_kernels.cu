// sx_kernels.cu -- the STREAM element kernels (Section 5, Listing 4) for sm_103a.
//
// Copy c=a, Scale b=c*q, Add c=a+b, Triad a=b+c*q, with the library operand convention
// COPY out=x, SCALE out=x*q, ADD out=x+y, TRIAD out=x+y*q.  Every arithmetic operation is
// one IEEE operation rounded to nearest even through __dmul_rn/__dadd_rn/__fmul_rn/__fadd_rn,
// which the compiler never fuses into a multiply-add; the library is also built with
// -fmad=false and without fast-math (no flush-to-zero).  Results are therefore bit-identical
// to a serial CPU loop.
//
// Nothing here is a contraction; the kernels are bound by HBM bandwidth.  The VECTOR family
// moves 16 or 32 bytes per thread access (32-byte ld/st.global.v4.u64 are new with sm_100),
// issues all loads of a tile before its stores so each thread keeps `unroll` vectors per
// input in flight, and walks the array with a grid-stride loop or one tile per block.
// The BULK family (sx_bulk.cu) stages tiles through shared memory with TMA bulk copies.
#include "sx_device.cuh"
#include "sx_internal.h"

#include <cstdio>
#include <type_traits>

namespace sx {
namespace {

using namespace dev;

// ---- VECTOR kernel -------------------------------------------------------------------------
// Elements [0, head) and [head + nvec*EPV, n) are done one by one by the first threads of the
// grid; the body [head, head + nvec*EPV) is nvec vectors of VB bytes, all VB-aligned.
template <int OP, class T, int VB, int U, int HINT, int MM>
__global__ void __launch_bounds__(1024)
k_stream_vec(const T *x, const T *y, T *out, uint64_t n, uint64_t head, uint64_t nvec, T q) {
    constexpr int W = VB / 8;
    constexpr int EPV = VB / (int)sizeof(T);
    constexpr bool HAS_Y = (OP == SX_OP_ADD || OP == SX_OP_TRIAD);

    // Launched as a programmatic dependent of the kernel before it on the stream: wait until
    // that kernel has completed and its stores are visible (at once otherwise), then allow the
    // next kernel's blocks to be scheduled, so that its launch overlaps this kernel's tail.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t body_end = head + nvec * EPV;
    if (gtid < head + (n - body_end)) {
        const uint64_t i = gtid < head ? gtid : body_end + (gtid - head);
        const T yv = HAS_Y ? y[i] : T(0);
        out[i] = apply_op<OP, T>(x[i], yv, q);
    }

    const char *xb = reinterpret_cast<const char *>(x + head);
    const char *yb = HAS_Y ? reinterpret_cast<const char *>(y + head) : nullptr;
    char *ob = reinterpret_cast<char *>(out + head);
    const uint64_t tile = (uint64_t)blockDim.x * U;
    const uint64_t stride = (uint64_t)gridDim.x * tile;
    for (uint64_t base = (uint64_t)blockIdx.x * tile; base < nvec; base += stride) {
        uint64_t xw[U][W], yw[U][W];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t v = base + (uint64_t)u * blockDim.x + threadIdx.x;
#pragma unroll
            for (int k = 0; k < W; ++k) yw[u][k] = 0;
            if (v < nvec) {
                ldv<VB, HINT>(xb + v * VB, xw[u]);
                if constexpr (HAS_Y) ldv<VB, HINT>(yb + v * VB, yw[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t v = base + (uint64_t)u * blockDim.x + threadIdx.x;
            if (v < nvec) {
                uint64_t r[W];
#pragma unroll
                for (int k = 0; k < W; ++k) r[k] = op_word<OP, T, MM>(xw[u][k], yw[u][k], q, k);
                stv<VB, HINT>(ob + v * VB, r);
            }
        }
    }
}

// Element-by-element fallback when the arrays do not share an alignment modulo 16 bytes.
template <int OP, class T>
__global__ void __launch_bounds__(256) k_stream_scalar(const T *x, const T *y, T *out, uint64_t n, T q) {
    constexpr bool HAS_Y = (OP == SX_OP_ADD || OP == SX_OP_TRIAD);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const T yv = HAS_Y ? y[i] : T(0);
        out[i] = apply_op<OP, T>(x[i], yv, q);
    }
}

struct VecLaunch {
    unsigned blocks, threads;
    cudaStream_t s;
    uint64_t n, head, nvec;
    bool pdl;  // launch as a programmatic dependent of the stream's previous kernel
};

// Launches one k_stream_vec instantiation with the shape of `l`.
template <int OP, class T, int VB, int U, int HINT, int MM>
cudaError_t launch_vec_one(const VecLaunch &l, const T *x, const T *y, T *out, T q) {
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(l.blocks);
    lc.blockDim = dim3(l.threads);
    lc.stream = l.s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = l.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&lc, k_stream_vec<OP, T, VB, U, HINT, MM>, x, y, out, l.n, l.head, l.nvec, q);
}

template <int OP, class T, int VB, int U, int HINT>
cudaError_t launch_vec_mm(int mm, const VecLaunch &l, const T *x, const T *y, T *out, T q) {
    // the product unit only matters for binary64 SCALE and TRIAD
    // (aliased outputs, HINT 2, keep the FP64 pipe: a rare case not worth more instantiations)
    constexpr bool MUL64 = sizeof(T) == 8 && (OP == SX_OP_SCALE || OP == SX_OP_TRIAD) && HINT != 2;
    if constexpr (MUL64) {
        switch (mm) {
            case 1: return launch_vec_one<OP, T, VB, U, HINT, 1>(l, x, y, out, q);
            case 2: return launch_vec_one<OP, T, VB, U, HINT, 2>(l, x, y, out, q);
            case 3: return launch_vec_one<OP, T, VB, U, HINT, 3>(l, x, y, out, q);
            case 4: return launch_vec_one<OP, T, VB, U, HINT, 4>(l, x, y, out, q);
            default: break;
        }
    }
    return launch_vec_one<OP, T, VB, U, HINT, 0>(l, x, y, out, q);
}

template <int OP, class T, int VB, int U>
cudaError_t launch_vec_hint(int hint, int mm, const VecLaunch &l, const T *x, const T *y, T *out, T q) {
    switch (hint) {
        case 0: return launch_vec_mm<OP, T, VB, U, 0>(mm, l, x, y, out, q);
        case 1: return launch_vec_mm<OP, T, VB, U, 1>(mm, l, x, y, out, q);
        default: return launch_vec_mm<OP, T, VB, U, 2>(mm, l, x, y, out, q);
    }
}

template <int OP, class T, int VB>
cudaError_t launch_vec_unroll(int unroll, int hint, int mm, const VecLaunch &l, const T *x, const T *y, T *out, T q) {
    switch (unroll) {
        case 1: return launch_vec_hint<OP, T, VB, 1>(hint, mm, l, x, y, out, q);
        case 2: return launch_vec_hint<OP, T, VB, 2>(hint, mm, l, x, y, out, q);
        default: return launch_vec_hint<OP, T, VB, 4>(hint, mm, l, x, y, out, q);
    }
}

bool ranges_overlap(const void *a, const void *b, size_t bytes) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + bytes && pb < pa + bytes;
}

template <int OP, class T>
int launch_vector(const sx_target *t, cudaStream_t s, const T *x, const T *y, T *out, size_t n, T q,
                  const sx_launch_cfg &c) {
    constexpr bool HAS_Y = (OP == SX_OP_ADD || OP == SX_OP_TRIAD);
    const size_t bytes = n * sizeof(T);
    int hint = c.cache_hint == 1 ? 1 : 0;
    if (ranges_overlap(x, out, bytes) || (HAS_Y && ranges_overlap(y, out, bytes))) hint = 2;

    const int VB = c.vec_bytes;
    const uintptr_t mis = (uintptr_t)out % VB;
    const bool same_mis = ((uintptr_t)x % VB == mis) && (!HAS_Y || (uintptr_t)y % VB == mis);
    if (!same_mis || mis % sizeof(T) != 0) {
        const unsigned threads = 256;
        uint64_t blocks = (n + threads - 1) / threads;
        const uint64_t cap = (uint64_t)t->sm_count * 8;
        if (blocks > cap) blocks = cap;
        if (blocks == 0) blocks = 1;
        k_stream_scalar<OP, T><<<(unsigned)blocks, threads, 0, s>>>(x, y, out, n, q);
        SX_CUDA(cudaGetLastError());
        return SX_OK;
    }
    const size_t epv = VB / sizeof(T);
    size_t head = ((VB - mis) % VB) / sizeof(T);
    if (head > n) head = n;
    const uint64_t nvec = (n - head) / epv;
    const uint64_t nedge = n - nvec * epv;
    const unsigned threads = (unsigned)c.threads;
    const uint64_t tile = (uint64_t)threads * c.unroll;
    uint64_t blocks = (nvec + tile - 1) / tile;
    if (c.blocks_per_sm > 0) {
        const uint64_t cap = (uint64_t)t->sm_count * c.blocks_per_sm;
        if (blocks > cap) blocks = cap;
    }
    const uint64_t edge_blocks = (nedge + threads - 1) / threads;
    if (blocks < edge_blocks) blocks = edge_blocks;
    if (blocks == 0) blocks = 1;
    if (blocks > 0x7fffffffull) return fail(SX_ERR_INVALID, "grid too large (%llu blocks)", (unsigned long long)blocks);
    // programmatic dependent launch on the library's and callers' streams; the default streams
    // keep plain serialisation
    const bool pdl = s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
    const VecLaunch l{(unsigned)blocks, threads, s, n, head, nvec, pdl};
    const int mm = mul_variant(c.fp64_mul, (double)q);
    cudaError_t e = VB == 16 ? launch_vec_unroll<OP, T, 16>(c.unroll, hint, mm, l, x, y, out, q)
                             : launch_vec_unroll<OP, T, 32>(c.unroll, hint, mm, l, x, y, out, q);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "k_stream_vec launch");
    }
    return SX_OK;
}

template <class T>
int dispatch_op(const sx_target *t, cudaStream_t s, int op, const void *x, const void *y, void *out,
                size_t n, double q, const sx_launch_cfg &c) {
    const T *xt = static_cast<const T *>(x);
    const T *yt = static_cast<const T *>(y);
    T *ot = static_cast<T *>(out);
    const T qt = (T)q;
    switch (op) {
        case SX_OP_COPY: return launch_vector<SX_OP_COPY, T>(t, s, xt, yt, ot, n, qt, c);
        case SX_OP_SCALE: return launch_vector<SX_OP_SCALE, T>(t, s, xt, yt, ot, n, qt, c);
        case SX_OP_ADD: return launch_vector<SX_OP_ADD, T>(t, s, xt, yt, ot, n, qt, c);
        case SX_OP_TRIAD: return launch_vector<SX_OP_TRIAD, T>(t, s, xt, yt, ot, n, qt, c);
        default: return fail(SX_ERR_INVALID, "unknown op %d", op);
    }
}

// ---- fused STREAM passes ---------------------------------------------------------------------
// Element i's chain of roundings over `iters` passes depends only on a[i]: Copy sets c=a,
// Scale b=RN(c*q), Add c=RN(a+b), Triad a=RN(b+RN(c*q)).  One kernel can run the whole chain
// per element from one read of a and write a, b, c once, bit-identical to four launches per
// pass.
template <int MM, class T>
__device__ __forceinline__ void fused_pass(T &a, T &b, T &c, T q, int lane) {
    c = a;
    b = mul_sel<MM>(c, q, lane);
    c = add_rn(a, b);
    a = add_rn(b, mul_sel<MM>(c, q, lane + 1));
}

template <int MM, class T>
__device__ __forceinline__ void fused_chain(T &a, T &b, T &c, T q, int iters, int lane) {
    for (int k = 0; k < iters; ++k) fused_pass<MM>(a, b, c, q, lane);
}

template <class T, int MM>
__global__ void __launch_bounds__(256) k_stream_fused(T *a, T *b, T *c, uint64_t n, T q, int iters) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        T av = a[i], bv, cv;
        fused_chain<MM>(av, bv, cv, q, iters, 0);
        a[i] = av;
        b[i] = bv;
        c[i] = cv;
    }
}

// 16-byte vector form of the fused kernel for arrays that are all 16-byte aligned.
template <class T, int MM>
__global__ void __launch_bounds__(256) k_stream_fused_v(T *a, T *b, T *c, uint64_t nvec, T q, int iters) {
    constexpr int EPV = 16 / sizeof(T);
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec;
         v += (uint64_t)gridDim.x * blockDim.x) {
        V av = reinterpret_cast<const V *>(a)[v];
        T ae[EPV], be[EPV], ce[EPV];
        memcpy(ae, &av, 16);
#pragma unroll
        for (int k = 0; k < EPV; ++k) fused_chain<MM>(ae[k], be[k], ce[k], q, iters, k);
        V ao, bo, co;
        memcpy(&ao, ae, 16);
        memcpy(&bo, be, 16);
        memcpy(&co, ce, 16);
        reinterpret_cast<V *>(a)[v] = ao;
        reinterpret_cast<V *>(b)[v] = bo;
        reinterpret_cast<V *>(c)[v] = co;
    }
}

// ---- generic byte transform: a registry of device callables (Listing 3's to_upper) ---------
struct ToUpper {
    __device__ __forceinline__ uint32_t operator()(uint32_t w) const {
        // bytes in 'a'..'z' lose 0x20; SIMD-within-a-word compares give 0xff per true byte
        const uint32_t m = __vcmpgeu4(w, 0x61616161u) & __vcmpleu4(w, 0x7a7a7a7au);
        return w - (m & 0x20202020u);
    }
    __device__ __forceinline__ uint8_t operator()(uint8_t ch) const {
        return (ch >= 'a' && ch <= 'z') ? (uint8_t)(ch - 0x20) : ch;
    }
};
struct ToLower {
    __device__ __forceinline__ uint32_t operator()(uint32_t w) const {
        const uint32_t m = __vcmpgeu4(w, 0x41414141u) & __vcmpleu4(w, 0x5a5a5a5au);
        return w + (m & 0x20202020u);
    }
    __device__ __forceinline__ uint8_t operator()(uint8_t ch) const {
        return (ch >= 'A' && ch <= 'Z') ? (uint8_t)(ch + 0x20) : ch;
    }
};

template <class F>
__global__ void __launch_bounds__(256) k_u8_transform(const uint8_t *in, uint8_t *out, uint64_t n, uint64_t head, uint64_t nvec) {
    F f;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t body_end = head + nvec * 16;
    if (gtid < head + (n - body_end)) {
        const uint64_t i = gtid < head ? gtid : body_end + (gtid - head);
        out[i] = f(in[i]);
    }
    const uint4 *vi = reinterpret_cast<const uint4 *>(in + head);
    uint4 *vo = reinterpret_cast<uint4 *>(out + head);
    for (uint64_t v = gtid; v < nvec; v += (uint64_t)gridDim.x * blockDim.x) {
        uint4 w = vi[v];
        w.x = f(w.x);
        w.y = f(w.y);
        w.z = f(w.z);
        w.w = f(w.w);
        vo[v] = w;
    }
}

}  // namespace

// ---- dispatch ----------------------------------------------------------------------------------
int launch_stream_op(const sx_target *t, cudaStream_t s, int op, int dtype, const void *x, const void *y,
                     void *out, size_t n, double q, const sx_launch_cfg &c) {
    if (n == 0) return SX_OK;
    if (c.variant == SX_VARIANT_BULK || c.variant == SX_VARIANT_TMA || c.variant == SX_VARIANT_TMA_TENSOR)
        return launch_bulk_op(t, s, op, dtype, x, y, out, n, q, c);
    if (dtype == SX_F64) return dispatch_op<double>(t, s, op, x, y, out, n, q, c);
    if (dtype == SX_F32) return dispatch_op<float>(t, s, op, x, y, out, n, q, c);
    return fail(SX_ERR_DTYPE, "STREAM kernels take F32 or F64 (got dtype %d)", dtype);
}

int launch_stream_fused(const sx_target *t, cudaStream_t s, int dtype, void *a, void *b, void *c,
                        size_t n, double q, int iters, int mm) {
    if (n == 0 || iters <= 0) return SX_OK;
    const size_t es = dtype_size(dtype);
    const uint64_t sms = (uint64_t)t->sm_count;
    double *a8 = (double *)a, *b8 = (double *)b, *c8 = (double *)c;
    if (dtype == SX_F64 && n <= 1024 * sms) {
        // Few elements per SM: the time is that of each warp's chain of dependent operations.
        // On B300 a dependent FP64 add or multiply takes ~80 cycles and an SM sub-partition's
        // FP64 unit ~64 cycles per warp instruction, so one element per thread in blocks of two
        // warps spreads the chains over as many sub-partitions as there are warps; up to one
        // warp per sub-partition the products stay on the FP64 pipe (the integer-unit product
        // has the longer dependent latency), beyond that they move to the integer units.
        if (mm < 0) mm = n <= 128 * sms ? 0 : 1;
        const int v = mul_variant(mm, q);
        const unsigned threads = 64;
        const unsigned g = (unsigned)((n + threads - 1) / threads);
        if (v == 1 || v == 2) k_stream_fused<double, 1><<<g, threads, 0, s>>>(a8, b8, c8, n, q, iters);
        else if (v == 3 || v == 4) k_stream_fused<double, 3><<<g, threads, 0, s>>>(a8, b8, c8, n, q, iters);
        else k_stream_fused<double, 0><<<g, threads, 0, s>>>(a8, b8, c8, n, q, iters);
        SX_CUDA(cudaGetLastError());
        return SX_OK;
    }
    if (mm < 0) mm = 1;  // many elements per SM: the products go to the integer units
    const bool aligned = ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0) &&
                         ((uintptr_t)c % 16 == 0) && ((n * es) % 16 == 0);
    const uint64_t cap = sms * 8;
    const int v = dtype == SX_F64 ? mul_variant(mm, q) : 0;
    // Each thread's chains are arithmetic (the FP64 pipe and the integer units), so small arrays
    // are spread over as many SMs as possible: blocks shrink from 256 to 32 threads until the
    // grid has a block per SM.
    const uint64_t units = aligned ? n * es / 16 : n;
    unsigned threads = 256;
    while (threads > 32 && (units + threads - 1) / threads < sms) threads /= 2;
    uint64_t blocks = (units + threads - 1) / threads;
    if (blocks > cap) blocks = cap;
    const unsigned g = (unsigned)blocks;
    if (aligned) {
        const uint64_t nvec = units;
        if (dtype == SX_F32)
            k_stream_fused_v<float, 0><<<g, threads, 0, s>>>((float *)a, (float *)b, (float *)c, nvec, (float)q, iters);
        else if (v == 1) k_stream_fused_v<double, 1><<<g, threads, 0, s>>>(a8, b8, c8, nvec, q, iters);
        else if (v == 2) k_stream_fused_v<double, 2><<<g, threads, 0, s>>>(a8, b8, c8, nvec, q, iters);
        else if (v == 3) k_stream_fused_v<double, 3><<<g, threads, 0, s>>>(a8, b8, c8, nvec, q, iters);
        else if (v == 4) k_stream_fused_v<double, 4><<<g, threads, 0, s>>>(a8, b8, c8, nvec, q, iters);
        else k_stream_fused_v<double, 0><<<g, threads, 0, s>>>(a8, b8, c8, nvec, q, iters);
    } else {
        if (dtype == SX_F32)
            k_stream_fused<float, 0><<<g, threads, 0, s>>>((float *)a, (float *)b, (float *)c, n, (float)q, iters);
        else if (v == 1 || v == 2) k_stream_fused<double, 1><<<g, threads, 0, s>>>(a8, b8, c8, n, q, iters);
        else if (v == 3 || v == 4) k_stream_fused<double, 3><<<g, threads, 0, s>>>(a8, b8, c8, n, q, iters);
        else k_stream_fused<double, 0><<<g, threads, 0, s>>>(a8, b8, c8, n, q, iters);
    }
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

int launch_u8_transform(const sx_target *t, cudaStream_t s, int fn, const void *in, void *out, size_t n) {
    if (n == 0) return SX_OK;
    const uintptr_t mis = (uintptr_t)out % 16;
    uint64_t head, nvec;
    if ((uintptr_t)in % 16 == mis) {
        head = (16 - mis) % 16;
        if (head > n) head = n;
        nvec = (n - head) / 16;
    } else {
        head = n;  // everything one byte at a time
        nvec = 0;
    }
    const uint64_t edge = n - nvec * 16;
    uint64_t blocks = (nvec + 255) / 256;
    const uint64_t cap = (uint64_t)t->sm_count * 8;
    if (blocks > cap) blocks = cap;
    const uint64_t eb = (edge + 255) / 256;
    if (blocks < eb) blocks = eb;
    if (blocks == 0) blocks = 1;
    if (blocks > 0x7fffffffull) return fail(SX_ERR_INVALID, "u8 transform: array too long for the byte path");
    const uint8_t *ip = (const uint8_t *)in;
    uint8_t *op = (uint8_t *)out;
    if (fn == SX_FN_TO_UPPER) k_u8_transform<ToUpper><<<(unsigned)blocks, 256, 0, s>>>(ip, op, n, head, nvec);
    else if (fn == SX_FN_TO_LOWER) k_u8_transform<ToLower><<<(unsigned)blocks, 256, 0, s>>>(ip, op, n, head, nvec);
    else return fail(SX_ERR_INVALID, "unknown callable %d", fn);
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

}  // namespace sx
