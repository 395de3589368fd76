/*
 * sx.h -- C ABI of libsx, STREAM over execution targets on one B300 GPU (sm_103a).
 *
 * What the library does.  Heller, Kaiser, Diehl, Fey, Schweitzer, "Closing the Performance
 * Gap with Modern C++", propose three ingredients for co-locating data and work: a *target*
 * (an opaque handle to a place in the system, Section 3.1), an *allocator* that places arrays
 * on a target and constructs them in bulk there (Section 3.2, Listing 1), and an *executor*
 * that runs work on a target, with async_execute as its one required operation and
 * execute / apply_execute / bulk_execute / bulk_async_execute derived from it (Section 3.3,
 * Listing 2).  Parallel algorithms (copy, transform) then run on a vector placed on a target
 * through a policy bound to an executor (Section 3.4, Listing 3).  The CUDA realisation makes a
 * target a device number plus a stream, offloads bulk construction to the GPU and copies
 * host<->device with CUDA memcpy (Section 4.2).  Section 5 (Listing 4) ports STREAM onto it:
 * Copy c=a, Scale b=c*q, Add c=a+b, Triad a=b+c*q with q=3.0.
 *
 * This header is that design as a C ABI.  Plain pointers and sizes only; no C++ or torch
 * types.  Every function returns an int status (SX_OK on success); no exception crosses the
 * ABI.  On failure sx_last_error() returns a message for the calling thread.
 *
 * Arithmetic: every element operation is one IEEE-754 operation, round to nearest even, with
 * no fused multiply-add and no flush-to-zero; Triad is two roundings (c*q, then b+that).
 * Results are therefore bit-identical to a serial CPU loop in the same precision.  Generated
 * NaNs (e.g. inf*0) have an unspecified sign and payload; copied NaNs keep their bits.
 *
 * Ownership: the caller owns every handle it creates and destroys it.  Destroy arrays,
 * executors, futures, batches and servers before the target they were made on.  Memory the
 * caller lends (sx_array_wrap, a borrowed stream) is never freed by the library.
 *
 * Threads: handles are not thread-safe unless stated (the server's submit/poll/wait/read/
 * release are).  Distinct targets may be used from distinct threads.
 */
#ifndef SX_H_
#define SX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
enum {
    SX_OK = 0,
    SX_ERR_INVALID = 1,   /* bad argument: NULL handle, size mismatch, bad config value     */
    SX_ERR_OOM = 2,       /* target budget (host-side accounting) or device memory exhausted */
    SX_ERR_DTYPE = 3,     /* operands of different or unsupported element types            */
    SX_ERR_OVERLAP = 4,   /* output partially overlaps an input (exact aliasing is allowed)  */
    SX_ERR_TIMEOUT = 5,   /* a host-side wait ran past its limit                             */
    SX_ERR_CUDA = 6,      /* a CUDA runtime call failed; sx_last_error() carries its text    */
    SX_ERR_NOT_READY = 7, /* non-blocking test: the work has not completed yet               */
    SX_ERR_DEVICE = 8,    /* a kernel's bounded device-side wait expired; outputs invalid    */
    SX_ERR_STATE = 9      /* the call is not valid in the object's current state            */
};

/* Message of the last failing call on this thread ("" if none).  Valid until the next call. */
const char *sx_last_error(void);
/* Static name of a status code ("SX_OK", "SX_ERR_OOM", ...). */
const char *sx_status_string(int status);
/* Library version, as major*10000 + minor*100 + patch. */
int sx_version(void);

/* ---- element types, operations, policies ------------------------------------------- */
typedef enum sx_dtype { SX_F32 = 1, SX_F64 = 2, SX_U8 = 3 } sx_dtype;

/* The four STREAM kernels (Section 5, Listing 4) with the library's operand convention:
 *   COPY  out = x            SCALE out = x * q
 *   ADD   out = x + y        TRIAD out = x + y * q
 * SEED (batch/server items only) writes out[i] = the seeded uniform value of element
 * (index_base + i), see sx_seed_uniform. */
typedef enum sx_op {
    SX_OP_COPY = 0, SX_OP_SCALE = 1, SX_OP_ADD = 2, SX_OP_TRIAD = 3, SX_OP_SEED = 4
} sx_op;

/* Execution policy bound to an executor (Section 3.4: par.on(exec); Listing 2's execute vs
 * async_execute).  SX_PAR: the algorithm calls return after the work has completed on the
 * device.  SX_PAR_TASK: they return once the work is enqueued on the target's stream; order
 * follows the stream; completion is observed with futures or sx_executor_wait. */
typedef enum sx_policy { SX_PAR = 1, SX_PAR_TASK = 2 } sx_policy;

/* Kernel family.  VECTOR: grid-stride loop of 16- or 32-byte vector loads/stores per thread.
 * BULK: a persistent, warp-specialised kernel that stages input tiles through shared memory
 * with the Tensor Memory Accelerator's bulk copies (a producer warp issues cp.async.bulk
 * global->shared per pipeline stage; consumer warps compute from shared memory and store to
 * global memory).
 * TMA: the BULK pipeline with the results written back by bulk copies as well: consumer warps
 * compute each tile in place in shared memory and a storer warp issues one cp.async.bulk
 * shared->global per tile (copy: the storer takes each tile as it arrives, no consumer work).
 * TMA_TENSOR: TMA with 2-D tensor-map copies (cp.async.bulk.tensor.2d; tensor maps encoded per
 * call): each array's body is a view of rows of 256 elements, a tile is a box of whole rows
 * (tile_bytes a multiple of 2048), elements after the last whole row are done one by one.
 * AUTO: the autotuner's choice for (op, dtype, size) if it has one, else a fixed default. */
typedef enum sx_variant {
    SX_VARIANT_AUTO = 0, SX_VARIANT_VECTOR = 1, SX_VARIANT_BULK = 2, SX_VARIANT_TMA = 3,
    SX_VARIANT_TMA_TENSOR = 4
} sx_variant;

/* Launch configuration of one algorithm call.  A zero field means "default".
 *   threads        threads per block (multiple of 32; VECTOR: 32..1024; BULK: 64..1024, a producer
 *                  warp and consumer warps; TMA, TMA_TENSOR: 96..1024, a producer warp, a storer
 *                  warp and consumer warps, which copy leaves idle)
 *   blocks_per_sm  VECTOR: grid = SMs * blocks_per_sm with a grid-stride loop; 0 = one tile
 *                  per block (grid covers the array).  BULK, TMA*: persistent blocks per SM (1..4)
 *   vec_bytes      VECTOR: 16 or 32 bytes per thread access
 *   unroll         VECTOR: vector accesses per thread per tile (1, 2 or 4)
 *   cache_hint     VECTOR: 0 = default caching, 1 = streaming (L1 no-allocate loads with an
 *                  L2 256-byte prefetch hint, evict-first stores)
 *   tile_bytes     BULK, TMA*: bytes per array per pipeline stage (multiple of 1024, 1024..65536;
 *                  TMA_TENSOR: of 2048)
 *   stages         BULK, TMA*: pipeline depth (2..8); shared memory = stages*tile_bytes*inputs
 *   fp64_mul       FP64 SCALE and TRIAD: where the product c*q is computed.  0 = the FP64
 *                  pipe; 1 = the integer units (an exact round-to-nearest-even binary64 multiply
 *                  that defers to the FP64 pipe for zero, subnormal, infinite and NaN operands
 *                  and for subnormal or overflowing results); 2 = half of the elements each.
 *                  All three give bit-identical results.  Ignored for FP32.
 *   reserved       must be 0 */
typedef struct sx_launch_cfg {
    int32_t variant;
    int32_t threads;
    int32_t blocks_per_sm;
    int32_t vec_bytes;
    int32_t unroll;
    int32_t cache_hint;
    int32_t tile_bytes;
    int32_t stages;
    int32_t fp64_mul;
    int32_t reserved;
} sx_launch_cfg;

/* ---- targets: Section 3.1 (a place in the system) and Section 4.2 (CUDA target =
 *      device number + stream) ----------------------------------------------------------- */
typedef struct sx_target sx_target;

typedef struct sx_target_info {
    int32_t device;          /* CUDA device ordinal                                      */
    int32_t sm_count;        /* streaming multiprocessors                                 */
    int32_t cc_major, cc_minor;
    int64_t l2_bytes;        /* L2 cache size                                             */
    int64_t hbm_total;       /* device memory, bytes                                      */
    int64_t hbm_free;        /* free device memory at the time of the call                */
    int64_t budget;          /* allocation budget of this target (bytes)                  */
    int64_t used;            /* bytes currently allocated through this target             */
    int32_t max_smem_block;  /* opt-in shared memory per block, bytes                     */
    int32_t sm_clock_khz;    /* maximum SM clock                                          */
    char name[128];          /* device name                                               */
} sx_target_info;

/* Number of visible CUDA devices (the paper's get_targets() for GPUs). */
int sx_target_count(int *count);
/* A target on `device` with its own non-blocking stream; budget = total device memory. */
int sx_target_create(int device, sx_target **out);
/* A target that borrows `stream` (a cudaStream_t; NULL = create an owned stream) and caps
 * allocation through it at `budget_bytes` (0 = total device memory).  The stream must
 * outlive the target.  To borrow the legacy default stream (the one other libraries use when
 * they name stream 0), pass its handle cudaStreamLegacy, (void *)0x1. */
int sx_target_create_ext(int device, void *stream, size_t budget_bytes, sx_target **out);
/* Wait for the target's stream, then free the target (and its stream if it owns it). */
int sx_target_destroy(sx_target *t);
/* The target's properties and allocation accounting (hbm_free as of the call). */
int sx_target_info_get(const sx_target *t, sx_target_info *out);
/* The cudaStream_t the target enqueues on. */
int sx_target_stream(const sx_target *t, void **stream);
/* Wait for all work on the target's stream, then check the device error word that bounded
 * device-side waits set (SX_ERR_DEVICE if one expired; the word is then cleared). */
int sx_target_synchronize(sx_target *t);
/* Self-test of the device-side failure path: enqueues a kernel whose bounded wait on a flag that
 * nothing sets runs out after limit_us microseconds (1..1000000).  It records its code in the
 * target's device error word, so the next sx_target_synchronize returns SX_ERR_DEVICE (and clears
 * the word); the context stays usable.  Returns once the kernel is enqueued. */
int sx_target_selftest(sx_target *t, int64_t limit_us);

/* ---- arrays and the allocator: Section 3.2, Listing 1 (allocator_traits::target,
 *      bulk_construct, bulk_destroy) and Section 4.2 (construction offloaded to the GPU) ---- */
typedef struct sx_array sx_array;

/* Allocate n elements of `dtype` on the target.  The data pointer is 256-byte aligned and
 * followed by 256 guard bytes filled with 0xA5 (see sx_array_guard_ok).  The bytes are charged
 * to the target's budget; if they do not fit, SX_ERR_OOM is returned without calling into the
 * CUDA allocator.  Contents are undefined until constructed.  n = 0 is allowed. */
int sx_alloc(sx_target *t, sx_dtype dtype, size_t n, sx_array **out);
/* Borrow n elements of device memory at `device_ptr` (e.g. a torch tensor's storage).  Not
 * charged to the budget, never freed.  Any alignment of the element type is accepted. */
int sx_array_wrap(sx_target *t, sx_dtype dtype, void *device_ptr, size_t n, sx_array **out);
/* Release an array and, for owned arrays, its device memory. */
int sx_free(sx_array *a);
/* The array's device pointer, element count and sx_dtype (any output may be NULL). */
int sx_array_data(const sx_array *a, void **device_ptr, size_t *n, int *dtype);
/* Owned arrays: *ok = 1 if the 256 guard bytes past the last element are untouched.  Waits
 * for the target's stream first.  Borrowed arrays: *ok = 1. */
int sx_array_guard_ok(const sx_array *a, int *ok);
/* bulk_construct with one value: every element = (T)value.  Enqueued on the target stream. */
int sx_bulk_construct(sx_array *a, double value);
/* bulk_construct with seeded uniform values: element i = lo + (hi - lo) * u_i, evaluated in the
 * array's type as RN(lo + RN(RN(hi - lo) * u_i)) with lo/hi first rounded to that type, where
 * u_i = (w_i >> 11) * 2^-53 (F64) or (w_i >> 40) * 2^-24 (F32) and w_i is the (i+1)-th output
 * of SplitMix64 (Steele, Lea & Flood 2014; Vigna's 64-bit finaliser) started from state
 * `seed`.  Enqueued on the target stream. */
int sx_seed_uniform(sx_array *a, uint64_t seed, double lo, double hi);
/* sx_seed_uniform with the generator indices shifted: element i takes the value that element
 * (index_base + i) of sx_seed_uniform's array from the same seed would take.  So an array that
 * holds elements [off, off + n) of a longer logical array (one block of sx_block_partition)
 * is constructed with index_base = off and equals that slice of the whole.  SX_ERR_INVALID if
 * index_base + n - 1 overflows 64 bits.  Enqueued on the target stream. */
int sx_seed_uniform_at(sx_array *a, uint64_t seed, double lo, double hi, uint64_t index_base);
/* bulk_destroy (Section 3.2, Listing 1: ends the lifetime of the array's elements on its
 * target, never fails for a valid array).  The element types here are trivially destructible,
 * so nothing runs on the device and no memory is freed (sx_free does that); the call exists so
 * that code written against the allocator interface pairs each bulk construction with its
 * destruction.  SX_ERR_INVALID only for a NULL array. */
int sx_bulk_destroy(sx_array *a);

/* ---- block partition of one logical array over several targets: Section 4.1 (the block
 *      allocator divides the bytes evenly over a vector of targets; the executor runs each
 *      block's work on the target that holds it) ------------------------------------------- */
/* The block of part `part` (0..parts-1) when n elements are divided over `parts` targets in
 * contiguous blocks of ceil(n / parts) elements: *offset = min(n, part * ceil(n / parts)),
 * *count = min(n, *offset + ceil(n / parts)) - *offset.  The blocks of parts 0..parts-1 tile
 * [0, n) exactly, in order; trailing parts may be empty when parts does not divide n.  Host
 * arithmetic only.  SX_ERR_INVALID for parts < 1, part outside [0, parts), n >= 2^63 or a NULL
 * output. */
int sx_block_partition(uint64_t n, int parts, int part, uint64_t *offset, uint64_t *count);

/* ---- host<->device copy: Section 4.2 (copy specialised to CUDA memcpy) ---------------- */
/* Copy n elements between host memory and the array, starting at element 0.  The blocking
 * forms return once the copy has finished; the _async forms return once it is enqueued on the
 * target's stream and need pinned (page-locked) host memory that stays valid until then. */
int sx_copy_h2d(sx_array *dst, const void *host, size_t n);
int sx_copy_d2h(void *host, const sx_array *src, size_t n);
int sx_copy_h2d_async(sx_array *dst, const void *host, size_t n);
int sx_copy_d2h_async(void *host, const sx_array *src, size_t n);

/* ---- executors: Section 3.3, Listing 2 and Section 4.2 (CUDA executor) ---------------- */
typedef struct sx_executor sx_executor;
/* `cfg` NULL (or variant AUTO) lets each call pick its launch shape (autotuner table first,
 * then the built-in default).  The executor keeps a copy of *cfg, checked here as for a
 * one-input call (SX_ERR_INVALID); a BULK or TMA shape whose shared memory fits one input array
 * but not two is refused by each two-input call (add, triad) with SX_ERR_INVALID. */
int sx_executor_create(sx_target *t, sx_policy policy, const sx_launch_cfg *cfg, sx_executor **out);
/* Free the executor and the CUDA graphs it keeps (work it enqueued is not waited for). */
int sx_executor_destroy(sx_executor *e);
/* Block until all work enqueued on the executor's target has finished (then as
 * sx_target_synchronize). */
int sx_executor_wait(sx_executor *e);
/* The launch configuration a call of (op, dtype, n) would use on this executor. */
int sx_executor_resolve(const sx_executor *e, sx_op op, sx_dtype dtype, size_t n, sx_launch_cfg *out);

/* ---- futures: async_execute's return value (Listing 2; Section 4.2 completes it from the
 *      stream).  Backed by CUDA events, so they also give the device time of the work. ------- */
typedef struct sx_future sx_future;
/* SX_OK once complete, SX_ERR_TIMEOUT if timeout_ms (>= 0) elapsed first; < 0 waits forever.
 * Also reports SX_ERR_DEVICE as sx_target_synchronize does. */
int sx_future_wait(sx_future *f, int64_t timeout_ms);
/* SX_OK if complete, SX_ERR_NOT_READY if not. */
int sx_future_test(sx_future *f);
/* Device time between the start and the end of the future's work (complete futures only). */
int sx_future_elapsed_ms(sx_future *f, float *ms);
int sx_future_destroy(sx_future *f);

/* ---- parallel algorithms on placed arrays: Section 3.4 and Section 5, Listing 4 ------- */
/* All arrays of one call must live on the executor's target, have the same element type
 * (F32 or F64) and the same length.  `out` may be the same array as an input; a partial
 * overlap is SX_ERR_OVERLAP.  n = 0 is a no-op.  q is converted to the element type once.
 * The call follows the executor's policy (see sx_policy). */
int sx_copy(sx_executor *e, const sx_array *src, sx_array *dst);                        /* dst = src       */
int sx_transform_scale(sx_executor *e, const sx_array *in, sx_array *out, double q);    /* out = in * q    */
int sx_transform_add(sx_executor *e, const sx_array *x, const sx_array *y, sx_array *out); /* out = x + y */
int sx_transform_triad(sx_executor *e, const sx_array *x, const sx_array *y, sx_array *out,
                       double q);                                                         /* out = x + y*q  */
/* Any of the four by code (y ignored for COPY and SCALE; may be NULL). */
int sx_execute(sx_executor *e, sx_op op, const sx_array *x, const sx_array *y, sx_array *out, double q);
/* async_execute: always returns once enqueued.  If `fut` is not NULL a future is created for
 * the work (the caller destroys it); NULL gives apply_execute's fire-and-forget. */
int sx_execute_async(sx_executor *e, sx_op op, const sx_array *x, const sx_array *y,
                     sx_array *out, double q, sx_future **fut);
/* Listing 4's stream(): `iters` passes of Copy c=a, Scale b=c*q, Add c=a+b, Triad a=b+c*q,
 * four kernels per pass in stream order.  Follows the executor's policy.  With iters >= 2 the
 * passes are replayed from CUDA graphs of up to 16 passes, captured on the executor's first
 * call for these arrays, q and launch shapes and kept by the executor (the 8 most recent), so
 * that small arrays are not bound by per-kernel launch cost; same kernels, same bits.  A single
 * pass, or a call while the target's stream is being captured, launches the kernels directly. */
int sx_stream_iter(sx_executor *e, sx_array *a, sx_array *b, sx_array *c, double q, int iters);
/* The same `iters` passes computed by one kernel that reads a once and writes a, b, c once;
 * bit-identical results (each element's chain of roundings is the same). */
int sx_stream_fused(sx_executor *e, sx_array *a, sx_array *b, sx_array *c, double q, int iters);
/* End to end from host memory: copy a (n elements, pinned or pageable host memory) to the
 * target's array, run `iters` passes of sx_stream_iter, copy a, b and c back.  A pass writes c
 * (Copy) and b (Scale) before it reads them, so their start values are not copied in unless
 * iters is 0 (then all three make the round trip).
 * The work goes in 32 MiB chunks over three internal streams (every element's passes are
 * independent), so copies in both directions and the kernels overlap; with pinned host memory
 * the two link directions run at once.  Same bits as the unchunked sequence.  Returns after the
 * results are in host memory. */
int sx_stream_host(sx_executor *e, void *host_a, void *host_b, void *host_c, sx_array *a,
                   sx_array *b, sx_array *c, double q, int iters);

/* Generic element transform with a device callable chosen from a registry (Section 3.4,
 * Listing 3's transform(par.on(exec), s, to_upper); Section 4.2: any __device__ callable).
 * Built-in callables for U8 arrays: SX_FN_TO_UPPER (ASCII a-z -> A-Z), SX_FN_TO_LOWER. */
enum { SX_FN_TO_UPPER = 1, SX_FN_TO_LOWER = 2 };
int sx_transform_u8(sx_executor *e, int fn, const sx_array *in, sx_array *out);
/* Element transform with any device callable, given as CUDA C++ source (Section 4.2: the CUDA
 * executor runs any callable marked __device__).  `src` defines
 *     __device__ sx_t sx_fn(sx_t x)
 * where sx_t is the arrays' element type (float, double or unsigned char); out[i] = sx_fn(in[i]).
 * The source is compiled at run time for the target's GPU (NVRTC, no fused multiply-add, no fast
 * math) on first use and kept per (device, type, source).  `out` may be `in`.  SX_ERR_INVALID,
 * with the compiler's log in sx_last_error(), if the source does not compile; SX_ERR_STATE if
 * run-time compilation is not available.  Follows the executor's policy. */
int sx_transform_src(sx_executor *e, const char *src, const sx_array *in, sx_array *out);

/* ---- bulk execution over many independent instances (Listing 2's bulk_execute, one
 *      persistent launch captured in a CUDA graph) -------------------------------------- */
/* One instance: device pointers, all `n` elements long (72 bytes). */
typedef struct sx_batch_item {
    int32_t op;            /* sx_op (COPY..TRIAD, or SEED)                                */
    int32_t dtype;         /* SX_F32 or SX_F64                                            */
    uint64_t n;            /* elements                                                     */
    const void *x;         /* first input (unused for SEED)                                */
    const void *y;         /* second input (ADD, TRIAD; unused otherwise)                  */
    void *out;             /* output                                                       */
    double q;              /* scalar of SCALE and TRIAD; SEED: lo                          */
    double q2;             /* SEED: hi                                                     */
    uint64_t seed;         /* SEED: generator state (see sx_seed_uniform)                  */
    uint64_t index_base;   /* SEED: generator index of out[0]                              */
} sx_batch_item;

/* Launch shape of a batch.  chunk_bytes: bytes moved per work tile (all arrays), the unit a
 * block takes at a time (16 KiB..8 MiB); threads per block; blocks_per_sm of the persistent
 * grid, capped at the blocks of that size an SM holds at once (the grid walks its tiles
 * round-robin, which assumes every block is resident); vec_bytes 16/32.  Zero fields = the
 * values sx_tune_batch stored for a similar item mix, else 512 KiB tiles, 128 threads, 7 blocks
 * per SM, 32-byte vectors. */
typedef struct sx_batch_cfg {
    int32_t chunk_bytes;
    int32_t threads;
    int32_t blocks_per_sm;
    int32_t vec_bytes;
} sx_batch_cfg;

typedef struct sx_batch sx_batch;
/* Build a batch: copies `items` into device memory, cuts every item into byte-balanced work
 * tiles and captures the persistent kernel into a CUDA graph.  The items' pointers must stay
 * valid while the batch is used.  Items must not write memory another item reads or writes.
 * Both launch kinds run the items shortest first (fewest STREAM bytes; equal sizes in the
 * order given), which lowers the items' mean completion time and leaves the total unchanged. */
int sx_batch_create(sx_target *t, const sx_batch_item *items, size_t count,
                    const sx_batch_cfg *cfg, sx_batch **out);
/* Run every item once: one graph launch on the target's stream (returns once enqueued). */
int sx_batch_launch(sx_batch *b);
/* bulk_async_execute (Listing 2): the same launch, returning in *fut a future that completes
 * when every item has run (sx_future_wait / _test / _elapsed_ms, destroyed by the caller). */
int sx_batch_launch_async(sx_batch *b, sx_future **fut);
/* Baseline: run every item with its own kernel launch, in the batch's order, on the same stream. */
int sx_batch_launch_percall(sx_batch *b, const sx_launch_cfg *cfg);
/* Completion times.  With recording on (sx_batch_set_record(b, 1), then a launch of either
 * kind), sx_batch_completion_ns gives, after that launch has completed, each item's
 * completion time in ns of the device global timer relative to the launch's first work. */
int sx_batch_set_record(sx_batch *b, int record);
int sx_batch_completion_ns(sx_batch *b, uint64_t *t_ns, size_t count);
/* The batch's launch shape (as it runs: blocks per SM capped at those an SM holds), number of
 * work tiles and STREAM bytes of one launch. */
int sx_batch_info(const sx_batch *b, sx_batch_cfg *cfg, uint64_t *tiles, uint64_t *bytes);
/* Wait for the target's stream, then free the batch's graph and tables. */
int sx_batch_destroy(sx_batch *b);

/* ---- a batch launch that allocates nothing ---------------------------------------------
 * The paper has no counterpart to this call.  It is for callers that must not allocate device
 * memory: a process whose device memory already belongs to another allocator (for instance a
 * framework's caching pool that has reserved the free memory, so cudaMalloc would fail), or a
 * latency-bound loop that cannot afford cudaMalloc/cudaFree, which may synchronize the whole
 * device.  It runs `items` once, like sx_batch_create + sx_batch_launch with the same shape,
 * but needs no target and allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine): the item and tile tables go to a static device array of SX_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads this library holds until the process exits.
 *   stream   cudaStream_t to launch on (NULL = the legacy default stream), on the current device
 *   items    count instances as for sx_batch_create (device pointers, caller-owned); at most
 *            SX_NOALLOC_MAX_ITEMS items cut into at most SX_NOALLOC_MAX_TILES work tiles of
 *            cfg->chunk_bytes, else SX_ERR_INVALID before anything is launched
 *   cfg      launch shape as sx_batch_cfg (NULL or zero fields = 256 KiB tiles, 512 threads,
 *            4 blocks per SM, 32-byte vectors; the autotuner's table is not consulted)
 * Returns once the work is enqueued.  The tables are copied to the device from static pageable
 * host staging, which the driver stages before the copy call returns: the call may therefore
 * block the host until the stream's earlier work has drained, and the staging may be refilled
 * by the next call at once.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  While `stream` is being captured into a CUDA graph the call is
 * refused with SX_ERR_STATE before anything is enqueued: a captured copy would read the host
 * staging at every replay, after later calls had put their own items there.  All calls share
 * the one array and each overwrites the tables it uses: calls whose work overlaps on the GPU
 * (different streams, no ordering between them) race and give wrong results; calls on one
 * stream, or otherwise ordered, are safe, with no synchronization between them.  Calls from
 * several host threads take turns on a lock. */
#define SX_NOALLOC_MAX_ITEMS 4096
#define SX_NOALLOC_MAX_TILES 65536
#define SX_NOALLOC_SCRATCH_BYTES 950272 /* 4096 items x 104 B + 65536 tiles x 8 B */
int sx_batch_run_noalloc(void *stream, const sx_batch_item *items, size_t count, const sx_batch_cfg *cfg);

/* ---- autotuner ------------------------------------------------------------------------ */
/* The tuners time launches on the target's stream with CUDA events: other work on the same GPU
 * at the same time skews which shape wins (never the results computed under it).  sx_tune and
 * sx_tune_pass allocate scratch arrays on the target and free them before returning;
 * sx_tune_batch runs the batch's own items. */
/* Time the candidate launch shapes (the three families, vector widths, unroll, block counts,
 * cache hints, bulk tile sizes and pipeline depths) for (op, dtype, n) on scratch arrays the tuner allocates on the
 * target, keep the fastest in the in-process table (keyed by device name, op, dtype and
 * log2(n) bucket) and return it.  *gbs = its bandwidth (STREAM byte count). */
int sx_tune(sx_target *t, sx_op op, sx_dtype dtype, size_t n, sx_launch_cfg *best, float *gbs);
/* Tune the four kernels of a STREAM pass together, where they run: copy c = a, scale b = q c,
 * add c = a + b, triad a = b + q c in turn over three arrays (Section 5, Listing 4).  Each
 * kernel starts from its shape for (op, dtype, n) (the table's entry, else the defaults); the
 * VECTOR kernels' cache hint (0 or 1) is tried in every combination over the four, timing whole
 * passes on scratch arrays of n elements the call allocates on the target (seeded uniform in
 * [-1, 1) again before each trial; best of three trials).  A kernel's hint sets how much of its
 * output is still in L2 when it ends and what the next kernel finds there, so the best hints in
 * a pass need not be those of the kernel timed alone.  The fastest combination is stored in the
 * table for the four (op, dtype, log2(n) bucket) entries and returned in best[0..3] (copy,
 * scale, add, triad; may be NULL); *gbs (may be NULL) = the pass's STREAM bandwidth (10 n
 * elements moved).  SX_ERR_INVALID for n = 0 or a NULL target, SX_ERR_DTYPE unless F32/F64,
 * SX_ERR_OOM if three arrays of n do not fit the target's budget. */
int sx_tune_pass(sx_target *t, sx_dtype dtype, size_t n, sx_launch_cfg *best, float *gbs);
/* Tune the batch launch shape (chunk bytes, threads, blocks per SM, vector width) on `b`'s own
 * items (outputs are overwritten), store it for batches with a similar item mix, rebuild `b`
 * with it and return it.  *ms = device time of one launch with the best shape. */
int sx_tune_batch(sx_batch *b, sx_batch_cfg *best, float *ms);
/* Look up the table: SX_OK and *cfg = the entry of the nearest tuned log2(n) bucket for
 * (this target's device, op, dtype), the larger bucket on a tie; SX_ERR_NOT_READY if none.
 * Executors whose launch configuration leaves the variant at AUTO use the same lookup. */
int sx_tune_lookup(const sx_target *t, sx_op op, sx_dtype dtype, size_t n, sx_launch_cfg *cfg);
/* Persist / restore the table as JSON (entries for other devices are kept as they are). */
int sx_tune_save(const char *path);
int sx_tune_load(const char *path);
/* Empty the table (launches then use the built-in defaults until entries are added again). */
int sx_tune_clear(void);

/* ---- serving loop: continuous batching of STREAM requests on device-resident arrays ---- */
typedef struct sx_server sx_server;

/* Modes.  CONTINUOUS: the server thread runs "steps"; each step is one launch of the batched
 * kernel holding a piece (a range of elements) of every scheduled request, the step's byte budget
 * shared out so that short requests finish in one step and long ones share the rest.  A piece
 * constructs its range of the inputs and then applies the operation to it, tile by tile (unless
 * split_phases: then requests over a quarter of the budget construct their inputs in one phase
 * and run the operation in a later one).  A request that a step takes whole, in one piece, is
 * DONE as soon as that piece's last tile has finished (the device sets a completion word),
 * before the rest of the step.  Requests that arrive while steps are on the GPU are admitted as
 * slots and arena memory free up and join the next step.  FIFO: the per-call baseline; each
 * admitted request is enqueued at once as its own launches (construct x, construct y, op) on the
 * stream, in arrival order. */
enum { SX_SERVE_CONTINUOUS = 0, SX_SERVE_FIFO = 1 };
typedef struct sx_server_cfg {
    uint64_t budget_bytes;   /* device arena the server allocates once; admission bound.  Large
                                requests (more than 1/16 of the arena) hold memory at most four
                                at a time, so the rest stays open to smaller ones             */
    int32_t mode;            /* SX_SERVE_CONTINUOUS or SX_SERVE_FIFO                          */
    int32_t max_active;      /* requests admitted at once (slots), 1..65536; 0 = 256          */
    int32_t chunk_bytes;     /* CONTINUOUS: byte budget of one step (1 MiB..2 GiB); 0 = 1 GiB   */
    int32_t steps_in_flight; /* CONTINUOUS: launched steps not yet completed (1..8); 0 = 2    */
    int32_t threads, blocks_per_sm, vec_bytes;  /* batched-kernel shape; 0 = 128, 8, 32     */
    int32_t tile_bytes;      /* CONTINUOUS: work-tile bytes of the batched kernel; 0 = 256 KiB */
    int32_t policy;          /* CONTINUOUS: how a step's budget is shared, SX_SERVE_POLICY_*  */
    int32_t serialize_steps; /* CONTINUOUS: 0 = a step may start while the previous one ends
                                (programmatic dependent launch; pieces that need the previous
                                step's data wait for it); 1 = steps run strictly one after another */
    int32_t split_phases;    /* CONTINUOUS: 0 = every piece constructs its range of the inputs and
                                applies the operation to it in the same pass (each element's
                                inputs are computed, stored and used from registers); 1 = requests
                                over a quarter of the step budget run in two phases, inputs first,
                                the operation in a later piece reading them back              */
    int32_t backlog_steps;   /* CONTINUOUS: steps launched beyond steps_in_flight while requests
                                wait for admission (a backlog: the depth of the GPU's queue then
                                bounds throughput and hides the host's planning time; with nobody
                                waiting, a new arrival's first step should not queue behind more
                                steps).  steps_in_flight + backlog_steps <= 8; 0 = 2, -1 = none */
} sx_server_cfg;

/* CONTINUOUS sharing policies.  SRPT (default): shortest remaining work first; each request in
 * that order gets all of its current phase's remaining work until the step budget is spent (it
 * keeps the fewest requests, and so the least arena memory, in the system).  FAIR: water-filling;
 * requests with less remaining work in their phase than an equal share of the step get all of
 * it, the others split the rest equally.  SHORT_FIRST: requests whose remaining work is at most
 * a quarter of the step budget go first, shortest first; the rest of the budget goes to the
 * others in admission order. */
enum { SX_SERVE_POLICY_SRPT = 0, SX_SERVE_POLICY_FAIR = 1, SX_SERVE_POLICY_SHORT_FIRST = 2 };

/* Request flags. */
enum { SX_REQ_AUTO_RELEASE = 1 /* free the arrays as soon as the request is DONE */ };

/* One request: construct its inputs on the device from seeds (x from seed_x, y from seed_y,
 * uniform in [lo, hi), see sx_seed_uniform), then run `op` into `out`.  x, y and out live in
 * the server's arena from admission until sx_server_release (or completion, with
 * SX_REQ_AUTO_RELEASE). */
typedef struct sx_request {
    int32_t op;      /* COPY..TRIAD */
    int32_t dtype;   /* SX_F32 / SX_F64 */
    uint64_t n;
    double q;
    uint64_t seed_x, seed_y;
    double lo, hi;
    uint32_t flags;  /* SX_REQ_* flags */
    uint32_t reserved;
} sx_request;

enum { SX_REQ_QUEUED = 0, SX_REQ_ACTIVE = 1, SX_REQ_DONE = 2, SX_REQ_REJECTED = 3,
       SX_REQ_RELEASED = 4, SX_REQ_CANCELLED = 5 };
typedef struct sx_request_status {
    int32_t state;        /* SX_REQ_*                                                      */
    int32_t status;       /* SX_OK, or why it was rejected (SX_ERR_OOM: larger than arena)  */
    double t_submit;      /* host monotonic seconds                                        */
    double t_admit;
    double t_done;        /* when the server saw its last step complete                    */
    const void *x, *y;    /* device pointers (valid from admission to release)             */
    void *out;
} sx_request_status;

typedef struct sx_server_stats {
    uint64_t submitted, admitted, completed, rejected, steps, launches;
    uint64_t bytes_moved;     /* STREAM byte count of completed work (seeding included)     */
    uint64_t arena_used, arena_peak, arena_bytes;
    double busy_seconds;      /* host time with at least one step in flight                 */
    double host_step_seconds;  /* CONTINUOUS: host time spent building and launching steps */
    double host_admit_seconds; /* host time spent in admission passes                      */
    uint64_t cancelled;        /* requests cancelled (sx_server_cancel)                     */
    uint64_t fused;            /* CONTINUOUS: requests run whole as one construct-then-operate
                                  piece                                                     */
    uint64_t early_done;       /* CONTINUOUS: of those, DONE from the piece's own completion
                                  word, before the step holding it had completed            */
    uint64_t steps_in_flight_peak;    /* CONTINUOUS: most steps launched and not yet completed */
    uint64_t backlog_launches;        /* CONTINUOUS: steps launched beyond steps_in_flight
                                         (requests were waiting for admission)               */
} sx_server_stats;

/* Start a server thread on the target (its stream carries every launch).  Thread-safe calls:
 * submit, poll, wait, read, release, stats. */
int sx_server_create(sx_target *t, const sx_server_cfg *cfg, sx_server **out);
/* Queue a request; *id identifies it.  Requests larger than the arena are rejected at once
 * (state REJECTED, status SX_ERR_OOM); others wait until slots and arena memory free up. */
int sx_server_submit(sx_server *s, const sx_request *r, uint64_t *id);
/* Open-loop load: a library thread submits reqs[k] at t_arrival[k] seconds (non-decreasing)
 * after this call; ids[k] receives each request's id at once.  Returns immediately. */
int sx_server_replay(sx_server *s, const sx_request *reqs, const double *t_arrival, size_t count,
                     uint64_t *ids);
/* The request's current state and timestamps, without waiting. */
int sx_server_poll(sx_server *s, uint64_t id, sx_request_status *st);
/* Wait until the request is DONE, REJECTED, RELEASED or CANCELLED (SX_ERR_TIMEOUT after
 * timeout_ms >= 0). */
int sx_server_wait(sx_server *s, uint64_t id, int64_t timeout_ms, sx_request_status *st);
/* Copy n elements of a DONE request's array (0 = x, 1 = y, 2 = out) to host memory; returns
 * once the copy is complete.  Reads from several threads may run at once. */
int sx_server_read(sx_server *s, uint64_t id, int which, void *host, size_t n);
/* Free a DONE (or REJECTED) request's arena memory.  The request is RELEASED at once (later
 * reads fail); if reads of it are in progress on other threads, the memory is freed when the
 * last of them ends. */
int sx_server_release(sx_server *s, uint64_t id);
/* Cancel a request.  QUEUED: it leaves the queue at once.  ACTIVE: no further work of it is
 * launched, and its arena memory is freed once the steps already holding its work have
 * completed; it is then CANCELLED (sx_server_wait returns).  Finished requests:
 * SX_ERR_STATE (release a DONE one instead).  Releasing a CANCELLED request does nothing. */
int sx_server_cancel(sx_server *s, uint64_t id);
/* Counters of the server since its creation (busy_seconds up to the call). */
int sx_server_stats_get(sx_server *s, sx_server_stats *st);
/* Finish all admitted work, reject what is still queued, stop the thread, free the arena. */
int sx_server_destroy(sx_server *s);

#ifdef __cplusplus
}
#endif
#endif /* SX_H_ */
