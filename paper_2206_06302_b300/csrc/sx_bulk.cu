// sx_bulk.cu -- BULK family of the STREAM kernels: input tiles staged through shared memory by
// the Tensor Memory Accelerator's bulk copies (sm_90+ cp.async.bulk, no tensor map needed), with
// warp-specialised blocks.
//
// Persistent blocks (one or two per SM) walk their share of the tiles through a ring of `stages`
// shared-memory slots, each with two mbarriers: `full` (armed by the producer with the slot's
// byte count, completed by the bulk copies) and `empty` (one arrival per consumer warp).
//   producer  lane 0 of warp 0: for each tile, wait until the slot is empty, arm `full`, issue
//             one cp.async.bulk global->shared per input array;
//   consumers the other warps: wait until the slot is full, read it (16-byte shared loads),
//             apply the element operation and write the result straight to global memory with
//             16-byte streaming stores, then each warp arrives on `empty`.
// Loads of later tiles overlap the consumers' work on earlier ones, and a slot is free as soon as
// it has been read (the stores leave from registers, so no bulk-store completion is awaited).
//
// Waits are bounded: a wait gives up after ~2 s of %globaltimer or as soon as another role has
// given up (a shared abort flag), records a code in the target's device error word, and every
// role leaves its loop; after the block's final barrier thread 0 waits (again bounded) for the
// loads still in flight before shared memory is released.  Nothing traps.
//
// TMA family (k_stream_tma): the same pipeline with the results written back by bulk stores as
// well, and a third role.  Consumers (warps 2..) compute each tile in place in its input slot
// (x slot <- op(x, y)), make their shared-memory writes visible to the async proxy
// (fence.proxy.async) and arrive on the slot's `done` mbarrier (one arrival per warp).  The
// storer, lane 0 of warp 1, waits for `done`, issues one cp.async.bulk shared->global store of
// the tile, and once the store of the tile before has finished reading its slot
// (cp.async.bulk.wait_group.read 1) hands that slot back to the producer (`empty`, one arrival).
// For copy there is nothing to compute: the storer takes each slot as soon as it is full, so a
// tile crosses the SM without passing through a register.  Before the block exits the storer
// waits until its stores are complete.
//
// TMA_TENSOR is the same kernel with 2-D tensor-map copies (cp.async.bulk.tensor.2d): each array's
// body is described to the TMA unit as rows of 256 elements, a tile is a box of tile/256 rows, and
// every copy starts at column 0 of its first row (so the 16-byte rule on the innermost coordinate
// always holds).  The last tile may reach past the last row: the load fills those rows with zeros
// and still completes the full box's byte count, the store writes only rows inside the array.
// Elements after the last whole row are done one by one, like the unaligned head.

// Alignment: every bulk copy starts on a 16-byte boundary and moves a multiple of 16 bytes.
// Elements before the first 16-byte boundary and after the last whole 16 bytes are done one
// by one.  Arrays whose addresses differ modulo 16 bytes take the VECTOR family instead.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <map>
#include <mutex>
#include <utility>

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

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait that also gives up once *abort is set: true once the phase completed.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t phase, const volatile int *abort) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 32; ++k)
            if (mbar_try_wait(bar, phase)) return true;
        if (*abort || global_ns() - t0 > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src_smem)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the bulk stores of all but the most recent group have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_but_one() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// all bulk stores issued by this thread are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// The tensor maps of a TMA_TENSOR launch (kernel parameters; unused otherwise).
struct TmaMaps {
    CUtensorMap x, y, out;
};

// Box at (column c0, row c1) of `map` into shared memory, completing on `bar` (tx bytes).
__device__ __forceinline__ void tensor_load_2d(void *dst_smem, const CUtensorMap *map, int32_t c0, int32_t c1,
                                               uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst_smem)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

// Shared memory to the box at (column c0, row c1) of `map` (rows past the array are not written).
__device__ __forceinline__ void tensor_store_2d(const CUtensorMap *map, int32_t c0, int32_t c1, const void *src_smem) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(smem_addr(src_smem))
                 : "memory");
}

template <int OP, class T, int MM>
__global__ void __launch_bounds__(1024, 1)
k_stream_bulk(const T *x, const T *y, T *out, uint64_t n, uint64_t head, uint64_t nbody,
              uint32_t tile_elems, int stages, T q, int *err) {
    constexpr bool HAS_Y = (OP == SX_OP_ADD || OP == SX_OP_TRIAD);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kMaxStages];
    __shared__ __align__(8) uint64_t empty[kMaxStages];
    __shared__ int abort_flag;

    // launched as a programmatic dependent of the kernel before it on the stream (as the VECTOR
    // kernels are): wait until that kernel has completed and its stores are visible, then let
    // the next kernel's blocks be scheduled while this one runs
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

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

    const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(T);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t consumer_warps = blockDim.x / 32 - 1;
    const T *xb = x + head;
    const T *yb = HAS_Y ? y + head : nullptr;
    T *ob = out + head;
    auto slot_x = [&](int s) { return smem + (size_t)s * (HAS_Y ? 2u : 1u) * tile_bytes; };
    auto slot_y = [&](int s) { return smem + (size_t)s * 2u * tile_bytes + tile_bytes; };
    auto tile_start = [&](uint64_t j) { return (blockIdx.x + j * gridDim.x) * (uint64_t)tile_elems; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], consumer_warps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    __syncthreads();
    volatile int *abort_v = &abort_flag;

    uint64_t issued = 0;  // producer only: tiles whose loads were issued
    if (warp == 0) {
        if (lane == 0) {
            for (uint64_t j = 0; j < nlocal; ++j) {
                const int s = (int)(j % (uint64_t)stages);
                if (j >= (uint64_t)stages &&
                    !mbar_wait_or_abort(&empty[s], (uint32_t)((j / (uint64_t)stages - 1) & 1), abort_v)) {
                    *abort_v = 1;
                    break;
                }
                const uint64_t start = tile_start(j);
                const uint32_t bytes = (uint32_t)(min((uint64_t)tile_elems, nbody - start) * sizeof(T));
                mbar_expect_tx(&full[s], HAS_Y ? 2 * bytes : bytes);
                bulk_load(slot_x(s), xb + start, bytes, &full[s]);
                if constexpr (HAS_Y) bulk_load(slot_y(s), yb + start, bytes, &full[s]);
                issued = j + 1;
            }
        }
    } else {
        const uint32_t ctid = threadIdx.x - 32, ncons = blockDim.x - 32;
        for (uint64_t j = 0; j < nlocal; ++j) {
            const int s = (int)(j % (uint64_t)stages);
            // one decision per warp (every lane's wait returns within the limit), so that no lane
            // leaves the loop while the others go on to the warp barrier below
            const bool ok = mbar_wait_or_abort(&full[s], (uint32_t)((j / (uint64_t)stages) & 1), abort_v);
            if (!__all_sync(0xffffffffu, ok)) {
                *abort_v = 1;
                break;
            }
            const uint64_t start = tile_start(j);
            const uint32_t nv = (uint32_t)(min((uint64_t)tile_elems, nbody - start) * sizeof(T) / 16);
            const uint32_t sx0 = smem_addr(slot_x(s));
            const uint32_t sy0 = HAS_Y ? smem_addr(slot_y(s)) : 0u;
            char *og = reinterpret_cast<char *>(ob + start);
            // two 16-byte vectors per thread and step; a lone last vector on its own (no work
            // on words that are not there)
            auto vec = [&](uint32_t v, uint64_t (&r)[2]) {
                uint64_t a0, a1, b0 = 0, b1 = 0;
                asm volatile("ld.shared.v2.u64 {%0,%1}, [%2];" : "=l"(a0), "=l"(a1) : "r"(sx0 + 16 * v));
                if constexpr (HAS_Y)
                    asm volatile("ld.shared.v2.u64 {%0,%1}, [%2];" : "=l"(b0), "=l"(b1) : "r"(sy0 + 16 * v));
                r[0] = op_word<OP, T, MM>(a0, b0, q, 0);
                r[1] = op_word<OP, T, MM>(a1, b1, q, 1);
            };
            auto put = [&](uint32_t v, const uint64_t (&r)[2]) {
                asm volatile("st.global.cs.v2.u64 [%0], {%1,%2};" ::"l"(og + 16 * (uint64_t)v), "l"(r[0]), "l"(r[1])
                             : "memory");
            };
            uint32_t v = ctid;
            for (; v + ncons < nv; v += 2 * ncons) {
                uint64_t r0[2], r1[2];
                vec(v, r0);
                vec(v + ncons, r1);
                put(v, r0);
                put(v + ncons, r1);
            }
            if (v < nv) {
                uint64_t r0[2];
                vec(v, r0);
                put(v, r0);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // this warp has read the slot
        }
    }
    __syncthreads();  // every role has left its loop (all waits above are bounded)
    if (threadIdx.x == 0 && *abort_v) {
        atomicExch(err, kErrBulkWait);
        // the most recent load into each slot, if any is still in flight, lands before the
        // block's shared memory is released
        const uint64_t first = issued > (uint64_t)stages ? issued - (uint64_t)stages : 0;
        for (uint64_t k = first; k < issued; ++k) {
            const int s = (int)(k % (uint64_t)stages);
            if (!mbar_wait_bounded(&full[s], (uint32_t)((k / (uint64_t)stages) & 1), kWaitLimitNs)) {
                atomicExch(err, kErrBulkDrain);
                break;
            }
        }
    }
}

constexpr uint32_t kRowElems = 256;  // TMA_TENSOR: elements per row of the 2-D view

template <int OP, class T, int MM, bool TENSOR>
__global__ void __launch_bounds__(1024, 1)
k_stream_tma(const T *x, const T *y, T *out, uint64_t n, uint64_t head, uint64_t nbody,
             uint32_t tile_elems, int stages, T q, int *err, const __grid_constant__ TmaMaps maps) {
    constexpr bool HAS_Y = (OP == SX_OP_ADD || OP == SX_OP_TRIAD);
    constexpr bool COMPUTE = OP != SX_OP_COPY;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kMaxStages];
    __shared__ __align__(8) uint64_t done[kMaxStages];
    __shared__ __align__(8) uint64_t empty[kMaxStages];
    __shared__ int abort_flag;

    asm volatile("griddepcontrol.wait;" ::: "memory");  // as in k_stream_bulk
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // scalar edges: [0, head) and [head + nbody, n) (up to 255 elements after the last row)
    const uint64_t body_end = head + nbody;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < head + (n - body_end);
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = e < head ? e : body_end + (e - head);
        const T yv = HAS_Y ? y[i] : T(0);
        out[i] = apply_op<OP, T>(x[i], yv, q);
    }

    const uint64_t ntiles = (nbody + tile_elems - 1) / tile_elems;
    const uint64_t nlocal = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (nlocal == 0) return;  // uniform across the block

    const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(T);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t consumer_warps = COMPUTE ? blockDim.x / 32 - 2 : 0;
    auto tile_row = [&](uint64_t j) { return (int32_t)((blockIdx.x + j * gridDim.x) * (uint64_t)(tile_elems / kRowElems)); };
    const T *xb = x + head;
    const T *yb = HAS_Y ? y + head : nullptr;
    T *ob = out + head;
    auto slot_x = [&](int s) { return smem + (size_t)s * (HAS_Y ? 2u : 1u) * tile_bytes; };
    auto slot_y = [&](int s) { return smem + (size_t)s * 2u * tile_bytes + tile_bytes; };
    auto tile_start = [&](uint64_t j) { return (blockIdx.x + j * gridDim.x) * (uint64_t)tile_elems; };
    auto tile_len = [&](uint64_t j) { return (uint32_t)(min((uint64_t)tile_elems, nbody - tile_start(j)) * sizeof(T)); };
    auto phase = [&](uint64_t j) { return (uint32_t)((j / (uint64_t)stages) & 1); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            if (COMPUTE) mbar_init(&done[s], consumer_warps);
            mbar_init(&empty[s], 1);  // the storing thread hands each slot back
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    __syncthreads();
    volatile int *abort_v = &abort_flag;

    uint64_t issued = 0;  // producer only: tiles whose loads were issued
    if (warp == 0) {
        if (lane == 0) {
            for (uint64_t j = 0; j < nlocal; ++j) {
                const int s = (int)(j % (uint64_t)stages);
                if (j >= (uint64_t)stages && !mbar_wait_or_abort(&empty[s], phase(j) ^ 1u, abort_v)) {
                    *abort_v = 1;
                    break;
                }
                if constexpr (TENSOR) {
                    // a box always completes its full size, rows past the array filled with zeros
                    mbar_expect_tx(&full[s], HAS_Y ? 2 * tile_bytes : tile_bytes);
                    tensor_load_2d(slot_x(s), &maps.x, 0, tile_row(j), &full[s]);
                    if constexpr (HAS_Y) tensor_load_2d(slot_y(s), &maps.y, 0, tile_row(j), &full[s]);
                } else {
                    const uint32_t bytes = tile_len(j);
                    mbar_expect_tx(&full[s], HAS_Y ? 2 * bytes : bytes);
                    bulk_load(slot_x(s), xb + tile_start(j), bytes, &full[s]);
                    if constexpr (HAS_Y) bulk_load(slot_y(s), yb + tile_start(j), bytes, &full[s]);
                }
                issued = j + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // storer: a tile leaves once it is computed (copy: once it has arrived); its slot goes
            // back to the producer when the store of the next tile has been issued and this one's
            // has finished reading shared memory
            for (uint64_t j = 0; j < nlocal; ++j) {
                const int s = (int)(j % (uint64_t)stages);
                if (!mbar_wait_or_abort(COMPUTE ? &done[s] : &full[s], phase(j), abort_v)) {
                    *abort_v = 1;
                    break;
                }
                if constexpr (TENSOR) tensor_store_2d(&maps.out, 0, tile_row(j), slot_x(s));
                else bulk_store(ob + tile_start(j), slot_x(s), tile_len(j));
                bulk_commit();
                bulk_wait_read_but_one();
                if (j >= 1) mbar_arrive(&empty[(int)((j - 1) % (uint64_t)stages)]);
            }
            bulk_wait_all();  // the stores are complete before the block exits
        }
    } else if (COMPUTE) {
        const uint32_t ctid = threadIdx.x - 64, ncons = blockDim.x - 64;
        for (uint64_t j = 0; j < nlocal; ++j) {
            const int s = (int)(j % (uint64_t)stages);
            // one decision per warp, as in k_stream_bulk
            const bool ok = mbar_wait_or_abort(&full[s], phase(j), abort_v);
            if (!__all_sync(0xffffffffu, ok)) {
                *abort_v = 1;
                break;
            }
            const uint32_t nv = tile_len(j) / 16;
            const uint32_t sx0 = smem_addr(slot_x(s));
            const uint32_t sy0 = HAS_Y ? smem_addr(slot_y(s)) : 0u;
            // two 16-byte vectors per thread and step (both loaded before either is computed, so
            // each thread waits on shared memory once per two vectors), a lone last one on its own
            auto ld2 = [](uint32_t a, uint64_t &w0, uint64_t &w1) {
                asm volatile("ld.shared.v2.u64 {%0,%1}, [%2];" : "=l"(w0), "=l"(w1) : "r"(a));
            };
            auto st2 = [](uint32_t a, uint64_t w0, uint64_t w1) {
                asm volatile("st.shared.v2.u64 [%0], {%1,%2};" ::"r"(a), "l"(w0), "l"(w1) : "memory");
            };
            uint32_t v = ctid;
            for (; v + ncons < nv; v += 2 * ncons) {
                const uint32_t u = v + ncons;
                uint64_t a0, a1, c0, c1, b0 = 0, b1 = 0, d0 = 0, d1 = 0;
                ld2(sx0 + 16 * v, a0, a1);
                ld2(sx0 + 16 * u, c0, c1);
                if constexpr (HAS_Y) {
                    ld2(sy0 + 16 * v, b0, b1);
                    ld2(sy0 + 16 * u, d0, d1);
                }
                st2(sx0 + 16 * v, op_word<OP, T, MM>(a0, b0, q, 0), op_word<OP, T, MM>(a1, b1, q, 1));
                st2(sx0 + 16 * u, op_word<OP, T, MM>(c0, d0, q, 0), op_word<OP, T, MM>(c1, d1, q, 1));
            }
            if (v < nv) {
                uint64_t a0, a1, b0 = 0, b1 = 0;
                ld2(sx0 + 16 * v, a0, a1);
                if constexpr (HAS_Y) ld2(sy0 + 16 * v, b0, b1);
                st2(sx0 + 16 * v, op_word<OP, T, MM>(a0, b0, q, 0), op_word<OP, T, MM>(a1, b1, q, 1));
            }
            fence_async_smem();  // this thread's results are visible to the bulk store
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[s]);
        }
    }
    __syncthreads();  // every role has left its loop (all waits above are bounded)
    if (threadIdx.x == 0 && *abort_v) {
        atomicExch(err, kErrBulkWait);
        const uint64_t first = issued > (uint64_t)stages ? issued - (uint64_t)stages : 0;
        for (uint64_t k = first; k < issued; ++k) {
            const int s = (int)(k % (uint64_t)stages);
            if (!mbar_wait_bounded(&full[s], phase(k), kWaitLimitNs)) {
                atomicExch(err, kErrBulkDrain);
                break;
            }
        }
    }
}

// Per device and kernel instantiation: the dynamic shared memory limit already raised, and the
// resident blocks per SM of each (threads, shared memory) shape.  Setting the attribute and
// querying occupancy cost several microseconds of host time, more than a small launch runs.
struct BulkKernelState {
    size_t smem_limit = 0;
    std::map<std::pair<int, size_t>, int> occupancy;
};
std::mutex g_bulk_mu;
std::map<std::pair<int, const void *>, BulkKernelState> g_bulk_state;

int bulk_prepare(int device, const void *kern, int threads, size_t smem, int *occ) {
    std::lock_guard<std::mutex> g(g_bulk_mu);
    BulkKernelState &st = g_bulk_state[{device, kern}];
    if (smem > st.smem_limit) {
        SX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        st.smem_limit = smem;
    }
    auto it = st.occupancy.find({threads, smem});
    if (it == st.occupancy.end()) {
        int o = 0;
        SX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, smem));
        it = st.occupancy.emplace(std::make_pair(threads, smem), o).first;
    }
    *occ = it->second;
    return SX_OK;
}

// Kernel instantiation for the product unit `mv` (mul_variant; binary64 SCALE and TRIAD only).
template <int OP, class T>
auto bulk_kernel(int mv) {
    constexpr bool MUL64 = sizeof(T) == 8 && (OP == SX_OP_SCALE || OP == SX_OP_TRIAD);
    auto k = k_stream_bulk<OP, T, 0>;
    if constexpr (MUL64) {
        switch (mv) {
            case 1: k = k_stream_bulk<OP, T, 1>; break;
            case 2: k = k_stream_bulk<OP, T, 2>; break;
            case 3: k = k_stream_bulk<OP, T, 3>; break;
            case 4: k = k_stream_bulk<OP, T, 4>; break;
            default: break;
        }
    }
    return k;
}

template <int OP, class T, bool TENSOR>
auto tma_kernel(int mv) {
    constexpr bool MUL64 = sizeof(T) == 8 && (OP == SX_OP_SCALE || OP == SX_OP_TRIAD);
    auto k = k_stream_tma<OP, T, 0, TENSOR>;
    if constexpr (MUL64) {
        switch (mv) {
            case 1: k = k_stream_tma<OP, T, 1, TENSOR>; break;
            case 2: k = k_stream_tma<OP, T, 2, TENSOR>; break;
            case 3: k = k_stream_tma<OP, T, 3, TENSOR>; break;
            case 4: k = k_stream_tma<OP, T, 4, TENSOR>; break;
            default: break;
        }
    }
    return k;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (the library does
// not link the driver library itself).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

// The 2-D view of `nrows` rows of kRowElems elements from `base` (16-byte aligned), in boxes of
// `box_rows` rows; loads past the last row read zeros.
int encode_row_map(CUtensorMap *m, const void *base, size_t es, uint64_t nrows, uint32_t box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(SX_ERR_STATE, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[2] = {kRowElems, nrows};
    const cuuint64_t strides[1] = {kRowElems * es};
    const cuuint32_t box[2] = {kRowElems, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                           const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SX_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return SX_OK;
}

template <int OP, class T>
int launch_bulk_t(const sx_target *t, cudaStream_t st, const T *x, const T *y, T *out, size_t n, T q,
                  const sx_launch_cfg &c) {
    constexpr bool HAS_Y = (OP == SX_OP_ADD || OP == SX_OP_TRIAD);
    constexpr bool MUL64 = sizeof(T) == 8 && (OP == SX_OP_SCALE || OP == SX_OP_TRIAD);
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
    const bool tensor = c.variant == SX_VARIANT_TMA_TENSOR;
    // the body: whole 16-byte units, or whole rows of the 2-D view
    const uint64_t nrows = (n - head) / kRowElems;
    const uint64_t nbody = tensor ? nrows * kRowElems : ((n - head) * es / 16) * 16 / es;
    if (tensor && nrows >= (1ull << 31)) return fail(SX_ERR_INVALID, "array too long for the 2-D tensor view");
    const uint32_t tile_elems = (uint32_t)(c.tile_bytes / es);
    const size_t smem = (size_t)c.stages * (HAS_Y ? 2 : 1) * c.tile_bytes;
    const int mv = MUL64 ? mul_variant(c.fp64_mul, (double)q) : 0;
    const void *kfn = c.variant == SX_VARIANT_BULK ? (const void *)bulk_kernel<OP, T>(mv)
                      : tensor                     ? (const void *)tma_kernel<OP, T, true>(mv)
                                                   : (const void *)tma_kernel<OP, T, false>(mv);
    int occ = 0;
    SX_TRY(bulk_prepare(t->device, kfn, c.threads, smem, &occ));
    if (occ < 1) return fail(SX_ERR_INVALID, "BULK/TMA shape does not fit on an SM (%zu B shared)", smem);
    const int bps = c.blocks_per_sm < occ ? c.blocks_per_sm : occ;
    const uint64_t ntiles = (nbody + tile_elems - 1) / tile_elems;
    uint64_t grid = (uint64_t)t->sm_count * bps;
    if (grid > ntiles) grid = ntiles;
    if (grid == 0) grid = 1;
    // programmatic dependent launch on the library's and callers' streams (the default streams
    // keep plain serialisation), as for the VECTOR kernels
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3((unsigned)c.threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) ? 1 : 0;
    cudaError_t e;
    if (c.variant == SX_VARIANT_BULK) {
        e = cudaLaunchKernelEx(&lc, bulk_kernel<OP, T>(mv), x, y, out, (uint64_t)n, (uint64_t)head, (uint64_t)nbody,
                               tile_elems, c.stages, q, t->d_err);
    } else {
        TmaMaps maps;
        std::memset(&maps, 0, sizeof maps);
        if (tensor && nrows > 0) {
            const uint32_t box_rows = tile_elems / kRowElems;
            SX_TRY(encode_row_map(&maps.x, x + head, es, nrows, box_rows));
            SX_TRY(encode_row_map(&maps.y, HAS_Y ? y + head : x + head, es, nrows, box_rows));
            SX_TRY(encode_row_map(&maps.out, out + head, es, nrows, box_rows));
        }
        e = cudaLaunchKernelEx(&lc, tensor ? tma_kernel<OP, T, true>(mv) : tma_kernel<OP, T, false>(mv), x, y, out,
                               (uint64_t)n, (uint64_t)head, (uint64_t)nbody, tile_elems, c.stages, q, t->d_err, maps);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "bulk-copy kernel launch");
    }
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
    if (c.threads < 64 || c.threads > 1024 || c.threads % 32)
        return fail(SX_ERR_INVALID, "BULK/TMA threads=%d: need a multiple of 32 in [64, 1024] (a producer warp "
                    "and at least one consumer warp)", c.threads);
    const bool tma = c.variant == SX_VARIANT_TMA || c.variant == SX_VARIANT_TMA_TENSOR;
    if (tma && c.threads < 96)
        return fail(SX_ERR_INVALID, "TMA threads=%d: need at least 96 (producer, storer and consumer warps)",
                    c.threads);
    if (c.variant == SX_VARIANT_TMA_TENSOR && c.tile_bytes % 2048)
        return fail(SX_ERR_INVALID, "TMA_TENSOR tile_bytes=%d: need whole rows of 256 binary64 elements "
                    "(a multiple of 2048)", c.tile_bytes);
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
