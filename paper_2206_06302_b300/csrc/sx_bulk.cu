// sx_bulk.cu -- BULK family of the STREAM kernels: tiles staged through shared memory by the
// Tensor Memory Accelerator's bulk copies (sm_90+ cp.async.bulk, no tensor map needed).
//
// One persistent block per SM (or two) walks its share of the tiles through a ring of `stages`
// shared-memory slots.  Thread 0 is the producer: for each tile it arms the slot's mbarrier
// with the expected byte count and issues one cp.async.bulk global->shared per input array.
// All threads wait on the slot's mbarrier, apply the element operation in shared memory (in
// place, in the first input's buffer), fence the generic-proxy writes for the async proxy, and
// thread 0 writes the slot back with cp.async.bulk shared->global (a bulk async-group).  A slot
// is refilled only once its store has finished reading it (cp.async.bulk.wait_group.read).
//
// Waits are bounded: each mbarrier wait gives up after ~2 s of %globaltimer, records a code in
// the target's device error word, and the block leaves the loop together (the decision is
// made with __syncthreads_or so no thread is left at a barrier); before leaving, thread 0 waits
// (again bounded) for the loads it issued and for its stores.  Nothing traps.
//
// Alignment: every bulk copy starts on a 16-byte boundary and moves a multiple of 16 bytes.
// Elements before the first 16-byte boundary and after the last whole 16 bytes are done one
// by one.  Arrays whose addresses differ modulo 16 bytes take the VECTOR family instead.
#include "sx_device.cuh"
#include "sx_internal.h"

namespace sx {
namespace {

constexpr int kMaxStages = 8;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kErrBulkWait = 0x101;
constexpr int kErrBulkDrain = 0x102;

using namespace dev;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return done != 0;
}

// Bounded wait: true once the phase completed, false after the time limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint64_t limit_ns) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, phase)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int OP, class T, int MM>
__global__ void __launch_bounds__(1024)
k_stream_bulk(const T *x, const T *y, T *out, uint64_t n, uint64_t head, uint64_t nbody,
              uint32_t tile_elems, int stages, T q, int *err) {
    constexpr bool HAS_Y = (OP == SX_OP_ADD || OP == SX_OP_TRIAD);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kMaxStages];

    // scalar edges: [0, head) and [head + nbody, n)
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t body_end = head + nbody;
    if (gtid < head + (n - body_end)) {
        const uint64_t i = gtid < head ? gtid : body_end + (gtid - head);
        const T yv = HAS_Y ? y[i] : T(0);
        out[i] = apply_op<OP, T>(x[i], yv, q);
    }

    const uint64_t ntiles = (nbody + tile_elems - 1) / tile_elems;
    const uint64_t nlocal = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (nlocal == 0) return;  // uniform across the block
    if constexpr (OP == SX_OP_COPY) {
        if (threadIdx.x != 0) return;  // a copy needs no compute: one thread drives the engine
    }

    const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(T);
    const T *xb = x + head;
    const T *yb = HAS_Y ? y + head : nullptr;
    T *ob = out + head;
    auto slot_x = [&](int s) { return smem + (size_t)s * (HAS_Y ? 2u : 1u) * tile_bytes; };
    auto slot_y = [&](int s) { return smem + (size_t)s * 2u * tile_bytes + tile_bytes; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if constexpr (OP != SX_OP_COPY) __syncthreads();

    uint64_t issued = 0;  // producer only: tiles whose loads were issued
    auto issue = [&](uint64_t j) {
        const int s = (int)(j % (uint64_t)stages);
        const uint64_t start = (blockIdx.x + j * gridDim.x) * (uint64_t)tile_elems;
        const uint64_t cnt = min((uint64_t)tile_elems, nbody - start);
        const uint32_t bytes = (uint32_t)(cnt * sizeof(T));
        mbar_expect_tx(&full[s], HAS_Y ? 2 * bytes : bytes);
        bulk_load(slot_x(s), xb + start, bytes, &full[s]);
        if constexpr (HAS_Y) bulk_load(slot_y(s), yb + start, bytes, &full[s]);
        issued = j + 1;
    };
    if (threadIdx.x == 0)
        for (uint64_t j = 0; j < (uint64_t)stages && j < nlocal; ++j) issue(j);

    bool aborted = false;
    uint64_t j = 0;
    for (; j < nlocal; ++j) {
        const int s = (int)(j % (uint64_t)stages);
        const uint32_t phase = (uint32_t)((j / (uint64_t)stages) & 1);
        const bool ok = mbar_wait_bounded(&full[s], phase, kWaitLimitNs);
        if constexpr (OP == SX_OP_COPY) {
            if (!ok) {
                aborted = true;
                break;
            }
        } else {
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
        }
        const uint64_t start = (blockIdx.x + j * gridDim.x) * (uint64_t)tile_elems;
        const uint64_t cnt = min((uint64_t)tile_elems, nbody - start);
        const uint32_t bytes = (uint32_t)(cnt * sizeof(T));
        if constexpr (OP != SX_OP_COPY) {
            uint64_t *px = reinterpret_cast<uint64_t *>(slot_x(s));
            const uint64_t *py = HAS_Y ? reinterpret_cast<const uint64_t *>(slot_y(s)) : nullptr;
            const uint32_t nv = bytes / 16;
            for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) {
                uint64_t a0, a1, b0 = 0, b1 = 0;
                asm volatile("ld.shared.v2.u64 {%0,%1}, [%2];" : "=l"(a0), "=l"(a1) : "r"(smem_addr(px + 2 * v)));
                if constexpr (HAS_Y)
                    asm volatile("ld.shared.v2.u64 {%0,%1}, [%2];" : "=l"(b0), "=l"(b1) : "r"(smem_addr(py + 2 * v)));
                const uint64_t r0 = op_word<OP, T, MM>(a0, b0, q, 0), r1 = op_word<OP, T, MM>(a1, b1, q, 1);
                asm volatile("st.shared.v2.u64 [%0], {%1,%2};" ::"r"(smem_addr(px + 2 * v)), "l"(r0), "l"(r1)
                             : "memory");
            }
            fence_async_smem();
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            bulk_store(ob + start, slot_x(s), bytes);
            bulk_commit();
            if (j >= 1 && j - 1 + (uint64_t)stages < nlocal) {
                bulk_wait_read_1();  // the store of tile j-1 has read its slot
                issue(j - 1 + (uint64_t)stages);
            }
        }
    }
    if (threadIdx.x == 0) {
        if (aborted) {
            atomicExch(err, kErrBulkWait);
            // wait, bounded, for the loads still in flight before shared memory is released
            for (uint64_t k = j; k < issued; ++k) {
                const int s = (int)(k % (uint64_t)stages);
                if (!mbar_wait_bounded(&full[s], (uint32_t)((k / (uint64_t)stages) & 1), kWaitLimitNs)) {
                    atomicExch(err, kErrBulkDrain);
                    break;
                }
            }
        }
        bulk_wait_all();
    }
}

template <int OP, class T>
int launch_bulk_t(const sx_target *t, cudaStream_t st, const T *x, const T *y, T *out, size_t n, T q,
                  const sx_launch_cfg &c) {
    constexpr bool HAS_Y = (OP == SX_OP_ADD || OP == SX_OP_TRIAD);
    const uintptr_t mis = (uintptr_t)out % 16;
    const bool same = ((uintptr_t)x % 16 == mis) && (!HAS_Y || (uintptr_t)y % 16 == mis);
    const bool alias = (x == out) || (HAS_Y && y == out);
    if (!same || alias) {
        // bulk copies need a common 16-byte alignment; aliased outputs take the coherent path
        sx_launch_cfg v = resolve_cfg(t, OP, sizeof(T) == 8 ? SX_F64 : SX_F32, n, nullptr);
        if (v.variant != SX_VARIANT_VECTOR) {
            v = sx_launch_cfg{};
            v.variant = SX_VARIANT_VECTOR;
            v = resolve_cfg(t, OP, sizeof(T) == 8 ? SX_F64 : SX_F32, n, &v);
        }
        return launch_stream_op(t, st, OP, sizeof(T) == 8 ? SX_F64 : SX_F32, x, y, out, n, (double)q, v);
    }
    const size_t es = sizeof(T);
    size_t head = ((16 - mis) % 16) / es;
    if (head > n) head = n;
    const uint64_t nbody = ((n - head) * es / 16) * 16 / es;
    const uint32_t tile_elems = (uint32_t)(c.tile_bytes / es);
    const size_t smem = (size_t)c.stages * (HAS_Y ? 2 : 1) * c.tile_bytes;
    constexpr bool MUL64 = sizeof(T) == 8 && (OP == SX_OP_SCALE || OP == SX_OP_TRIAD);
    auto kern = k_stream_bulk<OP, T, 0>;
    if constexpr (MUL64) {
        switch (mul_variant(c.fp64_mul, (double)q)) {
            case 1: kern = k_stream_bulk<OP, T, 1>; break;
            case 2: kern = k_stream_bulk<OP, T, 2>; break;
            case 3: kern = k_stream_bulk<OP, T, 3>; break;
            case 4: kern = k_stream_bulk<OP, T, 4>; break;
            default: break;
        }
    }
    // raise this instantiation's dynamic shared memory limit (cheap; repeated per launch so
    // that every device the kernel runs on has it)
    SX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    SX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, c.threads, smem));
    if (occ < 1) return fail(SX_ERR_INVALID, "BULK shape does not fit on an SM (%zu B shared)", smem);
    const int bps = c.blocks_per_sm < occ ? c.blocks_per_sm : occ;
    const uint64_t ntiles = (nbody + tile_elems - 1) / tile_elems;
    uint64_t grid = (uint64_t)t->sm_count * bps;
    if (grid > ntiles) grid = ntiles;
    if (grid == 0) grid = 1;
    kern<<<(unsigned)grid, c.threads, smem, st>>>(x, y, out, n, head, nbody, tile_elems, c.stages, q, t->d_err);
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

template <class T>
int dispatch_bulk(const sx_target *t, cudaStream_t s, int op, const void *x, const void *y, void *out,
                  size_t n, double q, const sx_launch_cfg &c) {
    const T *xt = static_cast<const T *>(x);
    const T *yt = static_cast<const T *>(y);
    T *ot = static_cast<T *>(out);
    switch (op) {
        case SX_OP_COPY: return launch_bulk_t<SX_OP_COPY, T>(t, s, xt, yt, ot, n, (T)q, c);
        case SX_OP_SCALE: return launch_bulk_t<SX_OP_SCALE, T>(t, s, xt, yt, ot, n, (T)q, c);
        case SX_OP_ADD: return launch_bulk_t<SX_OP_ADD, T>(t, s, xt, yt, ot, n, (T)q, c);
        case SX_OP_TRIAD: return launch_bulk_t<SX_OP_TRIAD, T>(t, s, xt, yt, ot, n, (T)q, c);
        default: return fail(SX_ERR_INVALID, "unknown op %d", op);
    }
}

}  // namespace

int validate_bulk_cfg(const sx_target *t, int op, const sx_launch_cfg &c) {
    if (c.threads < 32 || c.threads > 1024 || c.threads % 32)
        return fail(SX_ERR_INVALID, "BULK threads=%d: need a multiple of 32 in [32, 1024]", c.threads);
    if (c.tile_bytes < 1024 || c.tile_bytes > 65536 || c.tile_bytes % 1024)
        return fail(SX_ERR_INVALID, "BULK tile_bytes=%d: need a multiple of 1024 in [1024, 65536]", c.tile_bytes);
    if (c.stages < 2 || c.stages > kMaxStages)
        return fail(SX_ERR_INVALID, "BULK stages=%d: need 2..%d", c.stages, kMaxStages);
    if (c.blocks_per_sm < 1 || c.blocks_per_sm > 4)
        return fail(SX_ERR_INVALID, "BULK blocks_per_sm=%d: need 1..4", c.blocks_per_sm);
    if (c.fp64_mul < 0 || c.fp64_mul > 2)
        return fail(SX_ERR_INVALID, "fp64_mul=%d: need 0, 1 or 2", c.fp64_mul);
    const int nin = (op == SX_OP_ADD || op == SX_OP_TRIAD) ? 2 : 1;
    const long smem = (long)c.stages * nin * c.tile_bytes;
    if (smem > (long)t->max_smem_block - 1024)
        return fail(SX_ERR_INVALID, "BULK needs %ld B of shared memory per block (limit %d)", smem,
                    t->max_smem_block - 1024);
    return SX_OK;
}

int launch_bulk_op(const sx_target *t, cudaStream_t s, int op, int dtype, const void *x, const void *y,
                   void *out, size_t n, double q, const sx_launch_cfg &c) {
    SX_TRY(validate_bulk_cfg(t, op, c));
    if (dtype == SX_F64) return dispatch_bulk<double>(t, s, op, x, y, out, n, q, c);
    if (dtype == SX_F32) return dispatch_bulk<float>(t, s, op, x, y, out, n, q, c);
    return fail(SX_ERR_DTYPE, "STREAM kernels take F32 or F64 (got dtype %d)", dtype);
}

}  // namespace sx
