// sx_batch.cu -- bulk execution of many independent STREAM instances in one persistent launch
// (Listing 2's bulk_execute over a shape of instances), captured once in a CUDA graph.
//
// The host cuts every item into work tiles of about `chunk_bytes` moved bytes (all of the item's
// arrays counted), a multiple of 64 elements so that vector alignment is kept from tile to tile,
// and lists the tiles item by item.  A batch built by sx_batch_create lists the items with the
// fewest bytes first (shortest job first: an item's completion waits only for items no larger than
// itself; the total work is the same in any order); the allocation-free launch keeps the caller's
// order.  A persistent grid (SMs x blocks_per_sm; for sx_batch_create's batches and the serving
// steps capped at the blocks the SMs hold at once, so that every block's share of a round runs in
// that round) walks the list round-robin: block b takes tiles b, b + grid, b + 2*grid, ...  Tiles
// are of equal bytes except each item's last, so the static assignment balances the byte load
// without a work queue.
// Inside a tile the block runs the same 16/32-byte vector loop as the VECTOR kernels, or an
// element loop when the item's pointers do not share the vector alignment.
//
// Optional completion recording: after its last tile of an item, a block bumps the item's
// counter; the block that completes the item writes %globaltimer.  The counters and stamps are
// scratch memory of the batch, cleared by a memset node in the same graph before the kernel.
#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "sx_device.cuh"
#include "sx_internal.h"
#include "sx_seed.cuh"

namespace sx {
namespace {

using namespace dev;

struct DevItem {
    uint32_t op, dtype;
    uint64_t n;
    const void *x;
    const void *y;
    void *out;
    double q, q2;
    uint64_t seed, index_base;
    uint32_t tile_elems, ntiles;
    uint32_t mulv;  // product variant of FP64 SCALE/TRIAD (0, 2 or 4; see mul_sel)
    uint32_t pad;   // serving steps: bit 0 dependent, bit 1 construct-then-operate, bits 8.. 1 + completion word
    uint64_t seed2; // construct-then-operate: seed of y (seed: of x)
    double q3;      // construct-then-operate: upper end of the inputs' range (q2: lower end; q: the op's scalar)
};
constexpr uint32_t kPadDependent = 1u, kPadConstructThenOp = 2u;

// Batches split each FP64 product between the integer units and the FP64 pipe.
inline uint32_t item_mul_variant(const sx_batch_item &it) {
    const bool mul64 = it.dtype == SX_F64 && (it.op == SX_OP_SCALE || it.op == SX_OP_TRIAD);
    return mul64 ? (uint32_t)mul_variant(2, it.q) : 0u;
}

struct DevTile {
    uint32_t item;
    uint32_t index;  // tile index within the item
};

template <int OP, class T, int VB, int MM>
__device__ __forceinline__ void tile_vector(const DevItem &it, uint64_t start, uint64_t cnt) {
    constexpr int W = VB / 8;
    constexpr int EPV = VB / (int)sizeof(T);
    constexpr bool HY = has_y<OP>();
    const T q = (T)it.q;
    const T *x = static_cast<const T *>(it.x) + start;
    const T *y = HY ? static_cast<const T *>(it.y) + start : nullptr;
    T *o = static_cast<T *>(it.out) + start;
    const uintptr_t mis = (uintptr_t)o % VB;
    const bool vec_ok = ((uintptr_t)x % VB == mis) && (!HY || (uintptr_t)y % VB == mis) && mis % sizeof(T) == 0;
    uint64_t head = 0, nvec = 0;
    if (vec_ok) {
        head = ((VB - mis) % VB) / sizeof(T);
        if (head > cnt) head = cnt;
        nvec = (cnt - head) / EPV;
    } else {
        head = cnt;
    }
    const uint64_t body_end = head + nvec * EPV;
    for (uint64_t e = threadIdx.x; e < head + (cnt - body_end); e += blockDim.x) {
        const uint64_t i = e < head ? e : body_end + (e - head);
        const T yv = HY ? y[i] : T(0);
        o[i] = apply_op_mm<OP, MM, T>(x[i], yv, q, 0);
    }
    const char *xb = reinterpret_cast<const char *>(x + head);
    const char *yb = HY ? reinterpret_cast<const char *>(y + head) : nullptr;
    char *ob = reinterpret_cast<char *>(o + head);
    // 32 bytes per input in flight per thread: two 16-byte vectors or one 32-byte vector (one
    // 16-byte vector with the integer product).  More would raise the register demand of the
    // whole kernel, which holds every op's tile code, past 64 and make it spill.
    constexpr uint64_t PER = (MM == 0 && VB == 16) ? 2 : 1;
    for (uint64_t v = threadIdx.x; v < nvec; v += PER * blockDim.x) {
        const uint64_t v2 = v + blockDim.x;
        uint64_t xa[W], ya[W], xc[W], yc[W];
#pragma unroll
        for (int k = 0; k < W; ++k) ya[k] = yc[k] = 0;
        ldv<VB, 0>(xb + v * VB, xa);
        if constexpr (HY) ldv<VB, 0>(yb + v * VB, ya);
        const bool two = PER == 2 && v2 < nvec;
        if (two) {
            ldv<VB, 0>(xb + v2 * VB, xc);
            if constexpr (HY) ldv<VB, 0>(yb + v2 * VB, yc);
        }
        uint64_t r[W];
#pragma unroll
        for (int k = 0; k < W; ++k) r[k] = op_word<OP, T, MM>(xa[k], ya[k], q, k);
        stv<VB, 0>(ob + v * VB, r);
        if (two) {
#pragma unroll
            for (int k = 0; k < W; ++k) r[k] = op_word<OP, T, MM>(xc[k], yc[k], q, k);
            stv<VB, 0>(ob + v2 * VB, r);
        }
    }
}

// Seeded construction of a tile by the block's threads (seed_range); PM1: lo = -1, hi = 1.
template <class T, bool PM1>
__device__ __forceinline__ void tile_seed(const DevItem &it, uint64_t start, uint64_t cnt) {
    const T lo = (T)it.q;
    const T span = (T)it.q2 - lo;  // RN(hi - lo) in T, as the host-side generator defines it
    seed_range<T, PM1>(static_cast<T *>(it.out) + start, cnt, it.seed, it.index_base + start, lo, span,
                       threadIdx.x, blockDim.x);
}

template <int VB>
__device__ __forceinline__ void run_tile(const DevItem &it, uint64_t start, uint64_t cnt) {
    const bool f64 = it.dtype == SX_F64;
    switch (it.op) {
        case SX_OP_COPY:
            if (f64) tile_vector<SX_OP_COPY, double, VB, 0>(it, start, cnt);
            else tile_vector<SX_OP_COPY, float, VB, 0>(it, start, cnt);
            break;
        case SX_OP_SCALE:
            if (!f64) tile_vector<SX_OP_SCALE, float, VB, 0>(it, start, cnt);
            else if (it.mulv == 4) tile_vector<SX_OP_SCALE, double, VB, 4>(it, start, cnt);
            else if (it.mulv == 2) tile_vector<SX_OP_SCALE, double, VB, 2>(it, start, cnt);
            else tile_vector<SX_OP_SCALE, double, VB, 0>(it, start, cnt);
            break;
        case SX_OP_ADD:
            if (f64) tile_vector<SX_OP_ADD, double, VB, 0>(it, start, cnt);
            else tile_vector<SX_OP_ADD, float, VB, 0>(it, start, cnt);
            break;
        case SX_OP_TRIAD:
            if (!f64) tile_vector<SX_OP_TRIAD, float, VB, 0>(it, start, cnt);
            else if (it.mulv == 4) tile_vector<SX_OP_TRIAD, double, VB, 4>(it, start, cnt);
            else if (it.mulv == 2) tile_vector<SX_OP_TRIAD, double, VB, 2>(it, start, cnt);
            else tile_vector<SX_OP_TRIAD, double, VB, 0>(it, start, cnt);
            break;
        case SX_OP_SEED:
            if (f64 && it.q == -1.0 && it.q2 == 1.0) tile_seed<double, true>(it, start, cnt);
            else if (f64) tile_seed<double, false>(it, start, cnt);
            else tile_seed<float, false>(it, start, cnt);
            break;
        default: break;
    }
}

// Construct-then-operate piece of a serving step: each element's inputs are drawn from their
// seeds in registers and stored, and the operation is applied to those register values and
// stored.  The result has the bits of constructing the inputs and then running the operation
// over memory (the operation would read back exactly the values stored), without reading the
// inputs back and without a barrier between the two: the tile's DRAM traffic is its stores.
//
// Binary64 inputs on [-1, 1): kFusedPm1Sub of every four elements take the FP64-subtraction
// form of the value and the others the integer-unit assembly (the same bits either way).  The
// operation's additions (and half of its products) already occupy the FP64 pipe, so fewer of
// these pieces' values go there than in plain construction (5 of 8): on the served workload 0 or
// 1 of 4 moved 8.5-8.8 TB/s, 2 of 4 8.2-8.8, 3 of 4 7.7-8.1, 4 of 4 7.2-7.5.
constexpr int kFusedPm1Sub = 1;

template <class T, bool PM1>
__device__ __forceinline__ T fused_input(uint64_t z, T lo, T span, int j) {
    if constexpr (sizeof(T) == 4) {
        return seeded_value(splitmix_mix<true>(z), (float)lo, (float)span);  // uses bits 40..63 only
    } else if constexpr (PM1) {
        const uint64_t w = splitmix_mix(z);
        return (j & 3) < kFusedPm1Sub ? seeded_value_pm1_sub(w) : seeded_value_pm1(w);
    } else {
        return seeded_value(splitmix_mix(z), (double)lo, (double)span);
    }
}

template <int OP, class T, bool PM1, int MM>
__device__ __forceinline__ void tile_fused(const DevItem &it, uint64_t start, uint64_t cnt) {
    constexpr bool HY = has_y<OP>();
    constexpr int E = 32 / (int)sizeof(T);  // elements per thread and step: one 32-byte vector per array
    T *x = static_cast<T *>(const_cast<void *>(it.x)) + start;
    T *y = HY ? static_cast<T *>(const_cast<void *>(it.y)) + start : nullptr;
    T *o = static_cast<T *>(it.out) + start;
    const T lo = (T)it.q2;
    const T span = (T)it.q3 - lo;  // RN(hi - lo) in T, as the host-side generator defines it
    const T q = (T)it.q;
    const uint64_t base = it.index_base + start;  // generator index of element 0 of the tile
    const uintptr_t mis = (uintptr_t)o % 32;
    const bool vec_ok = ((uintptr_t)x % 32 == mis) && (!HY || (uintptr_t)y % 32 == mis) && mis % sizeof(T) == 0;
    uint64_t head = vec_ok ? ((32 - mis) % 32) / sizeof(T) : cnt;
    if (head > cnt) head = cnt;
    const uint64_t nrun = (cnt - head) / E;
    const uint64_t body_end = head + nrun * E;
    for (uint64_t e = threadIdx.x; e < head + (cnt - body_end); e += blockDim.x) {
        const uint64_t i = e < head ? e : body_end + (e - head);
        const uint64_t z = (base + i + 1) * kSplitmixGamma;
        const T xv = fused_input<T, PM1>(it.seed + z, lo, span, (int)i);
        x[i] = xv;
        T yv = T(0);
        if constexpr (HY) {
            yv = fused_input<T, PM1>(it.seed2 + z, lo, span, (int)i);
            y[i] = yv;
        }
        o[i] = apply_op_mm<OP, MM, T>(xv, yv, q, (int)i);
    }
    for (uint64_t r = threadIdx.x; r < nrun; r += blockDim.x) {
        const uint64_t i0 = head + r * E;
        const uint64_t z0 = (base + i0 + 1) * kSplitmixGamma;
        T xv[E], yv[E], ov[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            xv[j] = fused_input<T, PM1>(it.seed + z0 + (uint64_t)j * kSplitmixGamma, lo, span, j);
            yv[j] = T(0);
            if constexpr (HY) yv[j] = fused_input<T, PM1>(it.seed2 + z0 + (uint64_t)j * kSplitmixGamma, lo, span, j);
        }
        stv<32, 0>(reinterpret_cast<char *>(x + i0), *reinterpret_cast<const uint64_t(*)[4]>(xv));
        if constexpr (HY) stv<32, 0>(reinterpret_cast<char *>(y + i0), *reinterpret_cast<const uint64_t(*)[4]>(yv));
#pragma unroll
        for (int j = 0; j < E; ++j) ov[j] = apply_op_mm<OP, MM, T>(xv[j], yv[j], q, j);
        stv<32, 0>(reinterpret_cast<char *>(o + i0), *reinterpret_cast<const uint64_t(*)[4]>(ov));
    }
}

template <int OP>
__device__ __forceinline__ void fused_tile_op(const DevItem &it, uint64_t start, uint64_t cnt) {
    constexpr bool MUL = OP == SX_OP_SCALE || OP == SX_OP_TRIAD;
    if (it.dtype != SX_F64) {
        tile_fused<OP, float, false, 0>(it, start, cnt);
    } else if (it.q2 == -1.0 && it.q3 == 1.0) {
        if (MUL && it.mulv == 4) tile_fused<OP, double, true, 4>(it, start, cnt);
        else if (MUL && it.mulv == 2) tile_fused<OP, double, true, 2>(it, start, cnt);
        else tile_fused<OP, double, true, 0>(it, start, cnt);
    } else {
        if (MUL && it.mulv == 4) tile_fused<OP, double, false, 4>(it, start, cnt);
        else if (MUL && it.mulv == 2) tile_fused<OP, double, false, 2>(it, start, cnt);
        else tile_fused<OP, double, false, 0>(it, start, cnt);
    }
}

__device__ __forceinline__ void fused_tile(const DevItem &it, uint64_t start, uint64_t cnt) {
    switch (it.op) {
        case SX_OP_COPY: fused_tile_op<SX_OP_COPY>(it, start, cnt); break;
        case SX_OP_SCALE: fused_tile_op<SX_OP_SCALE>(it, start, cnt); break;
        case SX_OP_ADD: fused_tile_op<SX_OP_ADD>(it, start, cnt); break;
        case SX_OP_TRIAD: fused_tile_op<SX_OP_TRIAD>(it, start, cnt); break;
        default: break;
    }
}

template <int VB>
__global__ void __launch_bounds__(1024)
k_batch(const DevItem *__restrict__ items, const DevTile *__restrict__ tiles, uint64_t ntiles,
        uint32_t *done_count, uint64_t *done_ns, uint64_t *t_start) {
    if (done_count && threadIdx.x == 0) atomicMin((unsigned long long *)t_start, (unsigned long long)global_ns());
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const DevTile tl = tiles[t];
        const DevItem it = items[tl.item];
        const uint64_t start = (uint64_t)tl.index * it.tile_elems;
        const uint64_t cnt = min((uint64_t)it.tile_elems, it.n - start);
        run_tile<VB>(it, start, cnt);
        if (done_count) {
            __syncthreads();  // every thread's stores of this tile are issued
            if (threadIdx.x == 0) {
                __threadfence();
                if (atomicAdd(&done_count[tl.item], 1u) + 1 == it.ntiles)
                    done_ns[tl.item] = global_ns();
            }
        }
    }
}

// Blocks of `kern` (blocks of `threads` threads, no dynamic shared memory) that one SM of the
// current device holds at once, cached per (device, kernel, threads).  The persistent grids walk
// their tiles round-robin and assume every block is resident: a block that is not starts only when
// a resident one has finished all of its tiles, so its share of every round (the first rounds'
// tiles included) would be done last.  Their grids are capped at this many blocks per SM.
int resident_blocks(const void *kern, int threads) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    const auto key = std::make_tuple(dev, kern, threads);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    cache[key] = occ;
    return occ;
}

}  // namespace
}  // namespace sx

using namespace sx;

struct sx_batch {
    sx_target *t = nullptr;
    std::vector<sx_batch_item> items;
    // The order items run in: fewest bytes first, ties in the caller's order (both launch kinds).
    std::vector<uint32_t> order;
    sx_batch_cfg cfg{};
    uint64_t ntiles = 0, bytes = 0;
    DevItem *d_items = nullptr;
    DevTile *d_tiles = nullptr;
    // completion-recording scratch: counters, stamps, start stamp
    uint32_t *d_done = nullptr;
    uint64_t *d_ns = nullptr;
    bool record = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // per-call baseline completion events
    std::vector<cudaEvent_t> call_events;
    cudaEvent_t call_start = nullptr;
    bool last_was_percall = false;
};

namespace sx {
namespace {

double item_bytes(const sx_batch_item &it) {
    return (double)op_arrays(it.op) * (double)it.n * (double)dtype_size(it.dtype);
}

int check_items(const sx_batch_item *items, size_t count) {
    for (size_t i = 0; i < count; ++i) {
        const auto &it = items[i];
        if (it.op < SX_OP_COPY || it.op > SX_OP_SEED) return fail(SX_ERR_INVALID, "item %zu: bad op %d", i, it.op);
        if (it.dtype != SX_F32 && it.dtype != SX_F64) return fail(SX_ERR_DTYPE, "item %zu: dtype %d", i, it.dtype);
        if (it.n == 0) continue;
        const bool hy = it.op == SX_OP_ADD || it.op == SX_OP_TRIAD;
        const bool hx = it.op != SX_OP_SEED;
        if (!it.out || (hx && !it.x) || (hy && !it.y)) return fail(SX_ERR_INVALID, "item %zu: NULL pointer", i);
        const size_t es = dtype_size(it.dtype);
        if ((uintptr_t)it.out % es || (hx && (uintptr_t)it.x % es) || (hy && (uintptr_t)it.y % es))
            return fail(SX_ERR_INVALID, "item %zu: pointer not aligned to its element type", i);
        if (it.n > (1ull << 40)) return fail(SX_ERR_INVALID, "item %zu: n too large", i);
    }
    return SX_OK;
}

sx_batch_cfg resolve_batch_cfg(const sx_target *t, const sx_batch_item *items, size_t count,
                               const sx_batch_cfg *req) {
    sx_batch_cfg c{};
    double total = 0;
    for (size_t i = 0; i < count; ++i) total += item_bytes(items[i]);
    const double mean = count ? total / count : 0;
    if (!req || (req->chunk_bytes == 0 && req->threads == 0 && req->blocks_per_sm == 0 && req->vec_bytes == 0)) {
        if (!tune_batch_lookup(t, mean, &c)) c = sx_batch_cfg{};
    } else {
        c = *req;
    }
    // the fastest shape measured on the 4096-instance FP64 batch among those whose blocks are all
    // resident at once (the kernel's 54 registers allow 36 warps per SM; 28 ran fastest)
    if (c.chunk_bytes == 0) c.chunk_bytes = 512 * 1024;
    if (c.threads == 0) c.threads = 128;
    if (c.blocks_per_sm == 0) c.blocks_per_sm = 7;
    if (c.vec_bytes == 0) c.vec_bytes = 32;
    return c;
}

int validate_batch_cfg(const sx_batch_cfg &c) {
    if (c.chunk_bytes < 16384 || c.chunk_bytes > (8 << 20))
        return fail(SX_ERR_INVALID, "chunk_bytes=%d out of [16 KiB, 8 MiB]", c.chunk_bytes);
    if (c.threads < 64 || c.threads > 1024 || c.threads % 32)
        return fail(SX_ERR_INVALID, "threads=%d: multiple of 32 in [64, 1024]", c.threads);
    if (c.blocks_per_sm < 1 || c.blocks_per_sm > 32 || c.blocks_per_sm * c.threads > 2048)
        return fail(SX_ERR_INVALID, "blocks_per_sm=%d with %d threads exceeds an SM", c.blocks_per_sm, c.threads);
    if (c.vec_bytes != 16 && c.vec_bytes != 32) return fail(SX_ERR_INVALID, "vec_bytes=%d: 16 or 32", c.vec_bytes);
    return SX_OK;
}

void free_device(sx_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_done) cudaFree(b->d_done);
    if (b->d_ns) cudaFree(b->d_ns);
    b->d_items = nullptr;
    b->d_tiles = nullptr;
    b->d_done = nullptr;
    b->d_ns = nullptr;
}

const void *batch_kernel(int vec_bytes) {
    return vec_bytes == 16 ? (const void *)k_batch<16> : (const void *)k_batch<32>;
}

int enqueue_kernel(sx_batch *b, cudaStream_t s) {
    const size_t count = b->items.size();
    if (b->record) {
        SX_CUDA(cudaMemsetAsync(b->d_done, 0, count * sizeof(uint32_t), s));
        SX_CUDA(cudaMemsetAsync(b->d_ns, 0xFF, sizeof(uint64_t), s));  // t_start = max, then atomicMin
        SX_CUDA(cudaMemsetAsync(b->d_ns + 1, 0, count * sizeof(uint64_t), s));
    }
    if (b->ntiles == 0) return SX_OK;
    const int bps = std::min(b->cfg.blocks_per_sm, resident_blocks(batch_kernel(b->cfg.vec_bytes), b->cfg.threads));
    uint64_t grid = (uint64_t)b->t->sm_count * bps;
    if (grid > b->ntiles) grid = b->ntiles;
    uint32_t *dc = b->record ? b->d_done : nullptr;
    uint64_t *dn = b->record ? b->d_ns + 1 : nullptr;
    uint64_t *ts = b->record ? b->d_ns : nullptr;
    if (b->cfg.vec_bytes == 16)
        k_batch<16><<<(unsigned)grid, b->cfg.threads, 0, s>>>(b->d_items, b->d_tiles, b->ntiles, dc, dn, ts);
    else
        k_batch<32><<<(unsigned)grid, b->cfg.threads, 0, s>>>(b->d_items, b->d_tiles, b->ntiles, dc, dn, ts);
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

int capture(sx_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    resident_blocks(batch_kernel(b->cfg.vec_bytes), b->cfg.threads);  // queried outside the capture
    cudaStream_t cs;
    SX_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int st = SX_OK;
    if (e == cudaSuccess) {
        st = enqueue_kernel(b, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
    }
    if (e == cudaSuccess && st == SX_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (st != SX_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
    return SX_OK;
}

// Elements per work tile of an item for tiles of about `tile_bytes` moved bytes: a multiple of
// 64 elements, so vector alignment carries from one tile to the next.
uint64_t tile_elems_for(const sx_batch_item &it, int tile_bytes) {
    const size_t per_elem = (size_t)op_arrays(it.op) * dtype_size(it.dtype);
    const uint64_t te = (uint64_t)tile_bytes / per_elem;
    return std::max<uint64_t>(64, te / 64 * 64);
}

// Fill the device-layout item table and append the item-major tile list.
// One item in the device layout; returns its tile count.
uint64_t fill_item(const sx_batch_item &it, int tile_bytes, DevItem &d) {
    d.op = (uint32_t)it.op;
    d.dtype = (uint32_t)it.dtype;
    d.n = it.n;
    d.x = it.x;
    d.y = it.y;
    d.out = it.out;
    d.q = it.q;
    d.q2 = it.q2;
    d.seed = it.seed;
    d.index_base = it.index_base;
    d.mulv = item_mul_variant(it);
    d.pad = 0;
    d.seed2 = 0;
    d.q3 = 0.0;
    const uint64_t te = tile_elems_for(it, tile_bytes);
    d.tile_elems = (uint32_t)te;
    const uint64_t nt = (it.n + te - 1) / te;
    d.ntiles = (uint32_t)std::min<uint64_t>(nt, 0xffffffffull);
    return nt;
}

int fill_tables(const sx_batch_item *items, size_t count, int tile_bytes, DevItem *di, DevTile *tiles,
                size_t tile_cap, size_t *ntiles, uint64_t *bytes) {
    size_t nt_total = 0;
    uint64_t by = 0;
    for (size_t i = 0; i < count; ++i) {
        const auto &it = items[i];
        const uint64_t nt = fill_item(it, tile_bytes, di[i]);
        if (nt > 0xffffffffull) return fail(SX_ERR_INVALID, "item %zu has too many tiles", i);
        if (nt_total + nt > tile_cap) return fail(SX_ERR_INVALID, "tile table overflow");
        for (uint64_t k = 0; k < nt; ++k) tiles[nt_total + k] = DevTile{(uint32_t)i, (uint32_t)k};
        nt_total += nt;
        by += (uint64_t)item_bytes(it);
    }
    *ntiles = nt_total;
    if (bytes) *bytes = by;
    return SX_OK;
}

size_t count_tiles(const sx_batch_item *items, size_t count, int tile_bytes) {
    size_t nt = 0;
    for (size_t i = 0; i < count; ++i) {
        const uint64_t te = tile_elems_for(items[i], tile_bytes);
        nt += (items[i].n + te - 1) / te;
    }
    return nt;
}

// (Re)build the device tables and the graph for the batch's items under b->cfg.
int build(sx_batch *b) {
    free_device(b);
    const size_t count = b->items.size();
    std::vector<DevItem> di(count);
    std::vector<DevTile> tiles(count_tiles(b->items.data(), count, b->cfg.chunk_bytes));
    size_t nt = 0;
    SX_TRY(fill_tables(b->items.data(), count, b->cfg.chunk_bytes, di.data(), tiles.data(), tiles.size(),
                       &nt, &b->bytes));
    b->ntiles = nt;
    // List the tiles in the batch's run order (the tile list is item-major, so a stable sort on
    // the item's rank keeps each item's tiles in index order).
    std::vector<uint32_t> rank(count);
    for (size_t k = 0; k < count; ++k) rank[b->order[k]] = (uint32_t)k;
    std::stable_sort(tiles.begin(), tiles.begin() + nt,
                     [&](const DevTile &l, const DevTile &r) { return rank[l.item] < rank[r.item]; });
    SX_CUDA(cudaMalloc(&b->d_items, std::max<size_t>(1, count) * sizeof(DevItem)));
    SX_CUDA(cudaMalloc(&b->d_tiles, std::max<size_t>(1, tiles.size()) * sizeof(DevTile)));
    SX_CUDA(cudaMalloc(&b->d_done, std::max<size_t>(1, count) * sizeof(uint32_t)));
    SX_CUDA(cudaMalloc(&b->d_ns, (count + 1) * sizeof(uint64_t)));
    if (count) SX_CUDA(cudaMemcpy(b->d_items, di.data(), count * sizeof(DevItem), cudaMemcpyHostToDevice));
    if (!tiles.empty())
        SX_CUDA(cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(DevTile), cudaMemcpyHostToDevice));
    return capture(b);
}

}  // namespace

// ---- item lists built per launch (the serving loop's steps) ------------------------------------
size_t step_tile_count(const sx_batch_item *items, size_t count, int tile_bytes) {
    return count_tiles(items, count, tile_bytes);
}

void step_slot_free(StepSlot &s) {
    if (s.h_items) cudaFreeHost(s.h_items);
    if (s.h_tiles) cudaFreeHost(s.h_tiles);
    if (s.d_items) cudaFree(s.d_items);
    if (s.d_tiles) cudaFree(s.d_tiles);
    if (s.done) cudaEventDestroy(s.done);
    s = StepSlot{};
}

int step_slot_reserve(StepSlot &s, size_t items, size_t tiles) {
    if (!s.done) SX_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    if (items > s.cap_items) {
        const size_t cap = std::max<size_t>(items, 2 * s.cap_items);
        if (s.h_items) cudaFreeHost(s.h_items);
        if (s.d_items) cudaFree(s.d_items);
        s.h_items = s.d_items = nullptr;
        s.cap_items = 0;
        SX_CUDA(cudaMallocHost(&s.h_items, cap * sizeof(DevItem)));
        SX_CUDA(cudaMalloc(&s.d_items, cap * sizeof(DevItem)));
        s.cap_items = cap;
    }
    if (tiles > s.cap_tiles) {
        const size_t cap = std::max<size_t>(tiles, 2 * s.cap_tiles);
        if (s.h_tiles) cudaFreeHost(s.h_tiles);
        if (s.d_tiles) cudaFree(s.d_tiles);
        s.h_tiles = s.d_tiles = nullptr;
        s.cap_tiles = 0;
        SX_CUDA(cudaMallocHost(&s.h_tiles, cap * sizeof(DevTile)));
        SX_CUDA(cudaMalloc(&s.d_tiles, cap * sizeof(DevTile)));
        s.cap_tiles = cap;
    }
    return SX_OK;
}

// A step's items travel in the launch's own parameter space (up to 32 KB per launch on sm_70+
// with CUDA 12.1+), so a step costs one launch and no table copies.  Each item's first global
// tile is in `prefix`; a block finds the item of its tile by binary search over that array.
constexpr uint32_t kStepMaxItems = 256;
struct StepParams {
    uint32_t count, total_tiles;
    // completion report (last launch of a step only): the block that finishes last writes `seq`
    // to the host-mapped word `done`; `counter` is the step slot's device counter of finished
    // blocks, left at zero for the slot's next use
    uint64_t seq;
    unsigned long long *done;
    unsigned int *counter;
    // per-piece completion words (pieces with pad bits 8..): the warp that finishes the piece's
    // last part (ntiles x warps per block parts, one per warp and tile) sets fin_host[w]
    // (host-mapped) to 1; fin_count[w] counts the finished parts and is left at zero for the
    // word's next use
    unsigned long long *fin_host;
    unsigned int *fin_count;
    uint32_t prefix[kStepMaxItems + 1];
    DevItem items[kStepMaxItems];
};
static_assert(sizeof(StepParams) <= 32764, "kernel parameter space limit");

// Steps may overlap through programmatic dependent launch: every block allows the next step
// to launch as soon as it starts (all of a step's blocks are then resident or done, so the next
// step's blocks only take SM slots this step frees), waits for the previous step before its
// first tile of an item marked dependent (DevItem.pad bit 0: the operation phase of a request
// whose inputs were constructed in a step not yet known complete), and waits for it before
// exiting, so that a step's completion implies its predecessor's.  Without a programmatic
// predecessor griddepcontrol.wait returns at once.
template <int VB>
__global__ void __launch_bounds__(1024) k_batch_step(const __grid_constant__ StepParams p) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    bool waited = false;
    for (uint32_t t = blockIdx.x; t < p.total_tiles; t += gridDim.x) {
        uint32_t lo = 0, hi = p.count;  // prefix[lo] <= t < prefix[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (p.prefix[mid] <= t) lo = mid;
            else hi = mid;
        }
        const DevItem &it = p.items[lo];
        if ((it.pad & kPadDependent) && !waited) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            waited = true;
        }
        const uint64_t start = (uint64_t)(t - p.prefix[lo]) * it.tile_elems;
        const uint64_t cnt = min((uint64_t)it.tile_elems, it.n - start);
        if (it.pad & kPadConstructThenOp) fused_tile(it, start, cnt);
        else run_tile<VB>(it, start, cnt);
        const uint32_t w = it.pad >> 8;
        if (w) {
            // Each warp counts its part of the tile (no block-wide barrier per tile): its lanes'
            // stores are ordered before lane 0's device-scope fence, and the last of the piece's
            // ntiles x warps parts publishes it (as the step's last block does below).
            __syncwarp();
            if ((threadIdx.x & 31u) == 0) {
                __threadfence();
                const uint32_t parts = it.ntiles * (blockDim.x >> 5);
                if (atomicAdd(p.fin_count + (w - 1), 1u) == parts - 1) {
                    p.fin_count[w - 1] = 0u;
                    __threadfence_system();
                    *(volatile unsigned long long *)(p.fin_host + (w - 1)) = 1ull;
                }
            }
        }
    }
    if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
    if (p.done) {
        // every block's stores are issued; the last block to get here publishes the step
        // (blocks exit only after the previous step completed, so the word only grows)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(p.counter, 1u) == gridDim.x - 1) {
                *p.counter = 0u;
                __threadfence_system();
                *(volatile unsigned long long *)p.done = p.seq;
            }
        }
    }
}

int step_warm(cudaStream_t stream) {
    static thread_local StepParams p;
    std::memset(&p, 0, sizeof p);  // no items, no tiles, no report: the kernel only returns
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(1);
    lc.blockDim = dim3(32);
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    SX_CUDA(cudaLaunchKernelEx(&lc, k_batch_step<16>, p));
    SX_CUDA(cudaLaunchKernelEx(&lc, k_batch_step<32>, p));
    SX_CUDA(cudaStreamSynchronize(stream));
    return SX_OK;
}

int step_launch(const sx_target *t, cudaStream_t stream, StepSlot &s, const StepItem *items, size_t count,
                const sx_batch_cfg &cfg, bool overlap, const StepReport *report) {
    if (!report) SX_TRY(step_slot_reserve(s, 0, 0));  // the completion event
    static thread_local StepParams p;   // 23 KB: kept off the stack
    // the launch that carries the completion report: the last one that has work
    size_t last = 0;
    for (size_t first = 0; first < count; first += kStepMaxItems) {
        const size_t m = std::min<size_t>(kStepMaxItems, count - first);
        for (size_t i = 0; i < m; ++i)
            if (items[first + i].item.n) last = first;
    }
    bool reported = false;
    for (size_t first = 0; first < count; first += kStepMaxItems) {
        const size_t m = std::min<size_t>(kStepMaxItems, count - first);
        uint32_t tiles = 0;
        for (size_t i = 0; i < m; ++i) {
            const StepItem &si = items[first + i];
            DevItem &d = p.items[i];
            uint64_t nti = fill_item(si.item, cfg.chunk_bytes, d);
            if (si.flags & kStepConstructThenOp) {
                // tiles sized by the bytes of both phases: inputs written, then every array of the op
                const sx_batch_item &it = si.item;
                const bool hy = it.op == SX_OP_ADD || it.op == SX_OP_TRIAD;
                const size_t per = (size_t)((hy ? 2 : 1) + op_arrays(it.op)) * dtype_size(it.dtype);
                const uint64_t te = std::max<uint64_t>(64, (uint64_t)cfg.chunk_bytes / per / 64 * 64);
                d.tile_elems = (uint32_t)te;
                nti = (it.n + te - 1) / te;
                d.ntiles = (uint32_t)std::min<uint64_t>(nti, 0xffffffffull);
                d.seed2 = si.seed2;
                d.q3 = si.hi;
            }
            if ((uint64_t)tiles + nti > 0xffffffffull) return fail(SX_ERR_INVALID, "step has too many tiles");
            if (si.fin_word && (!report || !report->fin_host || si.fin_word >= (1u << 24)))
                return fail(SX_ERR_INVALID, "piece completion word without report words");
            if (si.fin_word && nti * (uint64_t)(cfg.threads / 32) >= (1ull << 32))
                return fail(SX_ERR_INVALID, "piece with a completion word has too many tiles");
            d.pad = (si.flags & kStepDependent ? kPadDependent : 0u) |
                    (si.flags & kStepConstructThenOp ? kPadConstructThenOp : 0u) | (si.fin_word << 8);
            p.prefix[i] = tiles;
            tiles += (uint32_t)nti;
        }
        p.fin_host = report ? report->fin_host : nullptr;
        p.fin_count = report ? report->fin_count : nullptr;
        p.prefix[m] = tiles;
        p.count = (uint32_t)m;
        p.total_tiles = tiles;
        if (tiles == 0) continue;
        const bool carries = report && first == last;
        p.seq = carries ? report->seq : 0;
        p.done = carries ? report->done : nullptr;
        p.counter = carries ? report->counter : nullptr;
        reported |= carries;
        const void *kern = cfg.vec_bytes == 16 ? (const void *)k_batch_step<16> : (const void *)k_batch_step<32>;
        const int bps = std::min(cfg.blocks_per_sm, resident_blocks(kern, cfg.threads));
        uint64_t grid = (uint64_t)t->sm_count * bps;
        if (grid > tiles) grid = tiles;
        cudaLaunchConfig_t lc{};
        lc.gridDim = dim3((unsigned)grid);
        lc.blockDim = dim3((unsigned)cfg.threads);
        lc.dynamicSmemBytes = 0;
        lc.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = overlap ? 1 : 0;
        lc.attrs = attr;
        lc.numAttrs = 1;
        if (cfg.vec_bytes == 16) SX_CUDA(cudaLaunchKernelEx(&lc, k_batch_step<16>, p));
        else SX_CUDA(cudaLaunchKernelEx(&lc, k_batch_step<32>, p));
    }
    if (!report) {
        SX_CUDA(cudaEventRecord(s.done, stream));
    } else if (!reported) {
        // nothing ran: publish the step from the host side of the stream's order
        return fail(SX_ERR_INVALID, "step without work");
    }
    return SX_OK;
}

}  // namespace sx

extern "C" {

int sx_batch_create(sx_target *t, const sx_batch_item *items, size_t count, const sx_batch_cfg *cfg,
                    sx_batch **out) {
    if (!t || !out || (!items && count)) return fail(SX_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (count > 0xffffffffull) return fail(SX_ERR_INVALID, "too many items");
    SX_TRY(check_items(items, count));
    sx_batch_cfg c = resolve_batch_cfg(t, items, count, cfg);
    SX_TRY(validate_batch_cfg(c));
    DeviceScope ds(t->device);
    // the shape that runs (sx_batch_info reports it): no more blocks per SM than an SM holds
    c.blocks_per_sm = std::min(c.blocks_per_sm, resident_blocks(batch_kernel(c.vec_bytes), c.threads));
    sx_batch *b = new (std::nothrow) sx_batch();
    if (!b) return fail(SX_ERR_OOM, "host allocation failed");
    b->t = t;
    b->items.assign(items, items + count);
    b->order.resize(count);
    for (size_t i = 0; i < count; ++i) b->order[i] = (uint32_t)i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](uint32_t l, uint32_t r) {
        return item_bytes(b->items[l]) < item_bytes(b->items[r]);
    });
    b->cfg = c;
    const int st = build(b);
    if (st != SX_OK) {
        free_device(b);
        delete b;
        return st;
    }
    *out = b;
    return SX_OK;
}

int sx_batch_launch(sx_batch *b) {
    TraceRange tr("sx_batch_launch");
    if (!b) return fail(SX_ERR_INVALID, "batch is NULL");
    DeviceScope ds(b->t->device);
    SX_CUDA(cudaGraphLaunch(b->exec, b->t->stream));
    b->last_was_percall = false;
    return SX_OK;
}

int sx_batch_launch_async(sx_batch *b, sx_future **fut) {
    TraceRange tr("sx_batch_launch_async");
    if (!b || !fut) return fail(SX_ERR_INVALID, "NULL argument");
    *fut = nullptr;
    DeviceScope ds(b->t->device);
    sx_future *f = nullptr;
    SX_TRY(new_future(b->t, &f));
    cudaError_t e = cudaEventRecord(f->start, b->t->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->t->stream);
    if (e == cudaSuccess) e = cudaEventRecord(f->end, b->t->stream);
    if (e != cudaSuccess) {
        sx_future_destroy(f);
        return cuda_fail(e, "batch launch");
    }
    b->last_was_percall = false;
    *fut = f;
    return SX_OK;
}

int sx_batch_launch_percall(sx_batch *b, const sx_launch_cfg *cfg) {
    TraceRange tr("sx_batch_launch_percall");
    if (!b) return fail(SX_ERR_INVALID, "batch is NULL");
    DeviceScope ds(b->t->device);
    cudaStream_t s = b->t->stream;
    const size_t count = b->items.size();
    if (b->record) {
        if (b->call_events.size() != count) {
            for (auto ev : b->call_events) cudaEventDestroy(ev);
            b->call_events.assign(count, nullptr);
            for (auto &ev : b->call_events) SX_CUDA(cudaEventCreate(&ev));
        }
        if (!b->call_start) SX_CUDA(cudaEventCreate(&b->call_start));
        SX_CUDA(cudaEventRecord(b->call_start, s));
    }
    for (size_t k = 0; k < count; ++k) {
        const size_t i = b->order[k];
        const auto &it = b->items[i];
        if (it.op == SX_OP_SEED) {
            SX_TRY(launch_seed(s, it.dtype, it.out, it.n, it.seed, it.q, it.q2, it.index_base));
        } else {
            sx_launch_cfg c = resolve_cfg(b->t, it.op, it.dtype, it.n, cfg);
            SX_TRY(validate_cfg(b->t, it.op, c));
            SX_TRY(launch_stream_op(b->t, s, it.op, it.dtype, it.x, it.y, it.out, it.n, it.q, c));
        }
        if (b->record) SX_CUDA(cudaEventRecord(b->call_events[i], s));
    }
    b->last_was_percall = true;
    return SX_OK;
}

int sx_batch_set_record(sx_batch *b, int record) {
    if (!b) return fail(SX_ERR_INVALID, "batch is NULL");
    if ((record != 0) == b->record) return SX_OK;
    DeviceScope ds(b->t->device);
    SX_CUDA(cudaStreamSynchronize(b->t->stream));
    b->record = record != 0;
    return capture(b);
}

int sx_batch_completion_ns(sx_batch *b, uint64_t *t_ns, size_t count) {
    if (!b || (!t_ns && count)) return fail(SX_ERR_INVALID, "NULL argument");
    if (!b->record) return fail(SX_ERR_STATE, "completion recording is off (sx_batch_set_record)");
    if (count > b->items.size()) return fail(SX_ERR_INVALID, "count exceeds the item count");
    DeviceScope ds(b->t->device);
    SX_CUDA(cudaStreamSynchronize(b->t->stream));
    if (b->last_was_percall) {
        for (size_t i = 0; i < count; ++i) {
            float ms = 0;
            SX_CUDA(cudaEventElapsedTime(&ms, b->call_start, b->call_events[i]));
            t_ns[i] = (uint64_t)((double)ms * 1e6);
        }
        return SX_OK;
    }
    std::vector<uint64_t> h(b->items.size() + 1);
    SX_CUDA(cudaMemcpy(h.data(), b->d_ns, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    const uint64_t t0 = h[0];
    for (size_t i = 0; i < count; ++i) t_ns[i] = (h[i + 1] >= t0 && h[i + 1] != 0) ? h[i + 1] - t0 : 0;
    return SX_OK;
}

int sx_batch_info(const sx_batch *b, sx_batch_cfg *cfg, uint64_t *tiles, uint64_t *bytes) {
    if (!b) return fail(SX_ERR_INVALID, "batch is NULL");
    if (cfg) *cfg = b->cfg;
    if (tiles) *tiles = b->ntiles;
    if (bytes) *bytes = b->bytes;
    return SX_OK;
}

int sx_batch_destroy(sx_batch *b) {
    if (!b) return fail(SX_ERR_INVALID, "batch is NULL");
    {
        DeviceScope ds(b->t->device);
        cudaStreamSynchronize(b->t->stream);
        free_device(b);
        for (auto ev : b->call_events) cudaEventDestroy(ev);
        if (b->call_start) cudaEventDestroy(b->call_start);
    }
    delete b;
    return SX_OK;
}

int sx_tune_batch(sx_batch *b, sx_batch_cfg *best_out, float *ms_out) {
    if (!b) return fail(SX_ERR_INVALID, "batch is NULL");
    DeviceScope ds(b->t->device);
    cudaStream_t s = b->t->stream;
    const bool rec = b->record;
    b->record = false;
    cudaEvent_t e0, e1;
    SX_CUDA(cudaEventCreate(&e0));
    SX_CUDA(cudaEventCreate(&e1));
    auto time_cfg = [&](sx_batch_cfg &c, float *ms) -> int {
        // blocks beyond those an SM holds are capped at launch: record the shape that runs
        c.blocks_per_sm = std::min(c.blocks_per_sm, resident_blocks(batch_kernel(c.vec_bytes), c.threads));
        b->cfg = c;
        SX_TRY(build(b));
        SX_CUDA(cudaGraphLaunch(b->exec, s));  // warm
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0, s);
            SX_CUDA(cudaGraphLaunch(b->exec, s));
            cudaEventRecord(e1, s);
            SX_CUDA(cudaEventSynchronize(e1));
            float m = 0;
            cudaEventElapsedTime(&m, e0, e1);
            best = std::min(best, m);
        }
        *ms = best;
        return SX_OK;
    };
    sx_batch_cfg best = b->cfg;
    float best_ms = 1e30f;
    int st = SX_OK;
    auto try_cfg = [&](sx_batch_cfg c) -> int {
        if (validate_batch_cfg(c) != SX_OK) {
            clear_error();
            return SX_OK;
        }
        float ms = 0;
        SX_TRY(time_cfg(c, &ms));
        if (ms < best_ms) best_ms = ms, best = c;
        return SX_OK;
    };
    // pass 1: tile size x residency; pass 2: block size and vector width at the best of pass 1
    // (same threads per SM); pass 3: blocks per SM from 1 to all an SM holds, for blocks of 64 to
    // 512 threads (on the 4096-instance FP64 batch 28 warps per SM ran 2-4% faster than 32 or 36,
    // and 36 is all the kernel's registers allow); pass 4: the tile size again at that shape
    for (int chunk : {64 << 10, 128 << 10, 256 << 10, 512 << 10, 1 << 20, 2 << 20})
        for (int bps : {1, 2, 4, 8})
            if (st == SX_OK) st = try_cfg(sx_batch_cfg{chunk, 256, bps, 32});
    if (st == SX_OK) {
        const sx_batch_cfg p1 = best;
        for (int th : {64, 128, 256, 512, 1024})
            for (int vb : {16, 32})
                if (st == SX_OK)
                    st = try_cfg(sx_batch_cfg{p1.chunk_bytes, th,
                                              std::max(1, std::min(p1.blocks_per_sm * 256 / th, 2048 / th)), vb});
    }
    if (st == SX_OK) {
        const sx_batch_cfg p2 = best;
        for (int th : {64, 128, 256, 512}) {
            const int most = std::min(resident_blocks(batch_kernel(p2.vec_bytes), th), 2048 / th);
            for (int bps = 1; bps <= most && st == SX_OK; ++bps)
                if (th != p2.threads || bps != p2.blocks_per_sm)
                    st = try_cfg(sx_batch_cfg{p2.chunk_bytes, th, bps, p2.vec_bytes});
        }
    }
    if (st == SX_OK) {
        const sx_batch_cfg p3 = best;
        for (int chunk : {64 << 10, 128 << 10, 256 << 10, 512 << 10, 1 << 20, 2 << 20})
            if (chunk != p3.chunk_bytes && st == SX_OK)
                st = try_cfg(sx_batch_cfg{chunk, p3.threads, p3.blocks_per_sm, p3.vec_bytes});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cfg = best;
    b->record = rec;
    const int st2 = build(b);
    if (st != SX_OK) return st;
    if (st2 != SX_OK) return st2;
    double total = 0;
    for (const auto &it : b->items) total += item_bytes(it);
    tune_batch_store(b->t, b->items.empty() ? 0 : total / b->items.size(), best);
    if (best_out) *best_out = best;
    if (ms_out) *ms_out = best_ms;
    return SX_OK;
}

}  // extern "C"

// ---- a batch launch that allocates nothing -------------------------------------------------------
// Some callers must not allocate device memory: a process whose device memory already belongs
// to another allocator (a framework's caching pool that has reserved what is free, so
// cudaMalloc would fail or fragment it), or a latency-bound loop that cannot pay for cudaMalloc
// and cudaFree, which may synchronize the whole device.  sx_batch_run_noalloc serves them with
// the same batched kernel as sx_batch_launch, its item and tile tables kept in the static array
// below instead of in memory allocated per batch.  The array is part of the library's device
// image, so every GPU that loads the library holds it until the process exits.
namespace sx {
namespace {

constexpr size_t kNoAllocMaxItems = SX_NOALLOC_MAX_ITEMS;
constexpr size_t kNoAllocMaxTiles = SX_NOALLOC_MAX_TILES;
constexpr size_t kNoAllocItemBytes = kNoAllocMaxItems * sizeof(DevItem);
constexpr size_t kNoAllocBytes = kNoAllocItemBytes + kNoAllocMaxTiles * sizeof(DevTile);
static_assert(kNoAllocBytes == SX_NOALLOC_SCRATCH_BYTES, "header states the scratch size");
static_assert(kNoAllocItemBytes % 256 == 0, "tile table stays 256-byte aligned");

// Device scratch: the item table, then the tile table.  In host code this name is only a
// stand-in for the symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host staging of the tables (static too: the call allocates no host memory either), the
// per-device scratch addresses, and a lock that makes calls from several threads take turns.
constexpr int kNoAllocMaxDevices = 64;
DevItem g_noalloc_host_items[kNoAllocMaxItems];
DevTile g_noalloc_host_tiles[kNoAllocMaxTiles];
void *g_noalloc_dev_ptr[kNoAllocMaxDevices];
int g_noalloc_dev_sms[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// Set-up, once per device, with that device current: look up the scratch's device address.
int noalloc_setup(int dev) {
    if (g_noalloc_dev_ptr[dev]) return SX_OK;
    void *p = nullptr;
    SX_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    int sms = 0;
    SX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    g_noalloc_dev_sms[dev] = sms;
    g_noalloc_dev_ptr[dev] = p;
    return SX_OK;
}

}  // namespace
}  // namespace sx

extern "C" int sx_batch_run_noalloc(void *stream, const sx_batch_item *items, size_t count,
                                    const sx_batch_cfg *cfg) {
    if (!items && count) return fail(SX_ERR_INVALID, "items is NULL");
    if (count > kNoAllocMaxItems)
        return fail(SX_ERR_INVALID, "%zu items exceed the %zu that the static scratch holds; split the batch",
                    count, kNoAllocMaxItems);
    SX_TRY(check_items(items, count));
    sx_batch_cfg c = cfg ? *cfg : sx_batch_cfg{};
    if (c.chunk_bytes == 0) c.chunk_bytes = 256 * 1024;
    if (c.threads == 0) c.threads = 512;
    if (c.blocks_per_sm == 0) c.blocks_per_sm = 4;
    if (c.vec_bytes == 0) c.vec_bytes = 32;
    SX_TRY(validate_batch_cfg(c));
    const size_t want = count_tiles(items, count, c.chunk_bytes);
    if (want > kNoAllocMaxTiles)
        return fail(SX_ERR_INVALID, "the batch needs %zu work tiles but the static scratch holds %zu; "
                    "raise chunk_bytes or split the batch", want, kNoAllocMaxTiles);
    cudaStream_t s = (cudaStream_t)stream;
    // The table copies below read the static host staging when they execute.  Captured into a
    // graph, they would read it at every replay, after later calls had refilled it with their
    // own items (whose arrays may since have been freed), so a capturing stream is refused.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce == cudaErrorStreamCaptureImplicit || (ce == cudaSuccess && cap != cudaStreamCaptureStatusNone)) {
        cudaGetLastError();
        return fail(SX_ERR_STATE, "the stream is being captured into a CUDA graph; this call copies its "
                    "tables from host staging that the next call overwrites, so it cannot be captured");
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamIsCapturing");
    int dev = 0;
    SX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SX_ERR_INVALID, "device %d out of range", dev);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    SX_TRY(noalloc_setup(dev));
    size_t nt = 0;
    // every call writes the whole part of the tables it uses; nothing is read before written
    SX_TRY(fill_tables(items, count, c.chunk_bytes, g_noalloc_host_items, g_noalloc_host_tiles,
                       kNoAllocMaxTiles, &nt, nullptr));
    if (nt == 0) return SX_OK;
    char *base = static_cast<char *>(g_noalloc_dev_ptr[dev]);
    DevItem *d_items = reinterpret_cast<DevItem *>(base);
    DevTile *d_tiles = reinterpret_cast<DevTile *>(base + kNoAllocItemBytes);
    // copies from pageable host memory: the staging arrays may be refilled once these return
    // (the driver stages pageable data before returning, and may wait for the stream's earlier
    // work to do so)
    SX_CUDA(cudaMemcpyAsync(d_items, g_noalloc_host_items, count * sizeof(DevItem), cudaMemcpyHostToDevice, s));
    SX_CUDA(cudaMemcpyAsync(d_tiles, g_noalloc_host_tiles, nt * sizeof(DevTile), cudaMemcpyHostToDevice, s));
    uint64_t grid = (uint64_t)g_noalloc_dev_sms[dev] * c.blocks_per_sm;
    if (grid > nt) grid = nt;
    if (c.vec_bytes == 16)
        k_batch<16><<<(unsigned)grid, c.threads, 0, s>>>(d_items, d_tiles, nt, nullptr, nullptr, nullptr);
    else
        k_batch<32><<<(unsigned)grid, c.threads, 0, s>>>(d_items, d_tiles, nt, nullptr, nullptr, nullptr);
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}
