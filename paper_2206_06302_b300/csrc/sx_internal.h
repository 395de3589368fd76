// sx_internal.h -- shared declarations of libsx's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sx.h"

namespace sx {

// ---- errors --------------------------------------------------------------------------------
int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
void clear_error();
int cuda_fail(cudaError_t e, const char *what);

#define SX_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::sx::cuda_fail(e_, #call);       \
    } while (0)

#define SX_TRY(call)                      \
    do {                                  \
        int s_ = (call);                  \
        if (s_ != SX_OK) return s_;       \
    } while (0)

// An NVTX range named after the API call for its scope (header-only NVTX3: a no-op unless a
// tool such as ncu --nvtx is attached).  Profiles can then be filtered by call.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Makes the target's device current for the scope of one API call.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceScope() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// True if the binary64 q is normal and its significand has at most 11 significant bits.
inline bool q_short_significand(double q) {
    uint64_t b;
    std::memcpy(&b, &q, sizeof b);
    const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
    if (e == 0 || e == 0x7FF) return false;
    uint64_t s = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    s >>= __builtin_ctzll(s);
    return s < (1ull << 11);
}

// Kernel product variant (see mul_sel) for a launch's fp64_mul on q.  The integer path only
// pays off for normal q; for zero, subnormal, infinite or NaN q every element would fall back.
inline int mul_variant(int fp64_mul, double q) {
    uint64_t b;
    std::memcpy(&b, &q, sizeof b);
    const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
    if (fp64_mul == 0 || e == 0 || e == 0x7FF) return 0;
    return q_short_significand(q) ? fp64_mul + 2 : fp64_mul;
}

inline size_t dtype_size(int dt) {
    switch (dt) {
        case SX_F32: return 4;
        case SX_F64: return 8;
        case SX_U8: return 1;
        default: return 0;
    }
}

// Bytes one element of `op` moves (STREAM convention: every array read or written once).
inline int op_arrays(int op) {
    switch (op) {
        case SX_OP_COPY: return 2;
        case SX_OP_SCALE: return 2;
        case SX_OP_ADD: return 3;
        case SX_OP_TRIAD: return 3;
        case SX_OP_SEED: return 1;
        default: return 0;
    }
}

}  // namespace sx

// ---- handles -------------------------------------------------------------------------------
struct sx_target {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t l2_bytes = 0;
    size_t hbm_total = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    int max_smem_block = 0;
    int sm_clock_khz = 0;
    std::string name;
    // Device error word: kernels whose bounded waits expire write a non-zero code here.
    int *d_err = nullptr;
    // Streams and events of host<->device pipelines (sx_stream_host), created on first use.
    static constexpr int kPipe = 3;
    cudaStream_t pipe[kPipe] = {};
    cudaEvent_t pipe_ev[kPipe + 1] = {};
};

struct sx_array {
    sx_target *t = nullptr;
    int dtype = 0;
    size_t n = 0;
    void *ptr = nullptr;
    bool owned = false;
    size_t alloc_bytes = 0;  // owned: data bytes rounded to 256 + 256 guard bytes
    size_t data_bytes = 0;
};

// What the nodes of a captured run of STREAM passes bake in (zero-filled, compared bytewise).
struct sx_pass_graph_key {
    const void *a, *b, *c;
    size_t n;
    int dtype, passes;
    uint64_t q_bits;
    sx_launch_cfg cfg[4];  // copy, scale, add, triad
};

struct sx_executor {
    sx_target *t = nullptr;
    int policy = SX_PAR;
    bool fixed_cfg = false;
    sx_launch_cfg cfg{};
    // sx_stream_iter's CUDA graphs (most recent last) and the private stream they are captured on
    struct PassGraph {
        sx_pass_graph_key key;
        cudaGraphExec_t exec;
    };
    static constexpr size_t kMaxGraphs = 8;
    std::vector<PassGraph> graphs;
    cudaStream_t capture = nullptr;
};

struct sx_future {
    sx_target *t = nullptr;
    cudaEvent_t start = nullptr, end = nullptr;
};

namespace sx {

constexpr int kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

// ---- kernels (sx_kernels.cu) ----------------------------------------------------------------
// One STREAM kernel launch on `stream` with the resolved configuration `cfg` (variant VECTOR
// or BULK).  x, y, out are element pointers; y may be null for COPY/SCALE.
int launch_stream_op(const sx_target *t, cudaStream_t stream, int op, int dtype, const void *x,
                     const void *y, void *out, size_t n, double q, const sx_launch_cfg &cfg);
int launch_fill(cudaStream_t stream, int dtype, void *out, size_t n, double value);
int launch_seed(cudaStream_t stream, int dtype, void *out, size_t n, uint64_t seed, double lo,
                double hi, uint64_t index_base);
// fp64_mul < 0: the product unit is chosen by the elements per SM
int launch_stream_fused(const sx_target *t, cudaStream_t stream, int dtype, void *a, void *b,
                        void *c, size_t n, double q, int iters, int fp64_mul);
int launch_u8_transform(const sx_target *t, cudaStream_t stream, int fn, const void *in,
                        void *out, size_t n);
// TMA bulk-copy staging family (sx_bulk.cu).
int launch_bulk_op(const sx_target *t, cudaStream_t stream, int op, int dtype, const void *x,
                   const void *y, void *out, size_t n, double q, const sx_launch_cfg &cfg);
int validate_bulk_cfg(const sx_target *t, int op, const sx_launch_cfg &cfg);
// The configuration actually used for (op, dtype, n) when `req` leaves fields at 0.
sx_launch_cfg resolve_cfg(const sx_target *t, int op, int dtype, size_t n, const sx_launch_cfg *req);
// Checks a fully specified configuration; SX_ERR_INVALID with a message if unsupported.
int validate_cfg(const sx_target *t, int op, const sx_launch_cfg &cfg);
// Enqueues the failure-path self-test kernel (sx_target_selftest).
int launch_selftest(const sx_target *t, cudaStream_t stream, int64_t limit_us);
// Reads and clears the target's device error word.
int check_device_error(const sx_target *t);
// A future on target `t` with its two events created, not yet recorded (sx_runtime.cpp).
int new_future(sx_target *t, sx_future **out);

// ---- batched kernel over item lists built per launch (sx_batch.cu) ----------------------------
// Staging of one launch: pinned host tables, device tables, and an event recorded after the
// kernel.  A slot may be refilled once its event has completed.
struct StepSlot {
    void *h_items = nullptr, *h_tiles = nullptr, *d_items = nullptr, *d_tiles = nullptr;
    size_t cap_items = 0, cap_tiles = 0;
    cudaEvent_t done = nullptr;
};
int step_slot_reserve(StepSlot &s, size_t items, size_t tiles);
void step_slot_free(StepSlot &s);
// Number of work tiles `items` are cut into with tiles of `tile_bytes`.
size_t step_tile_count(const sx_batch_item *items, size_t count, int tile_bytes);
// One piece of a serving step: a batch item and how the step treats it.
//   kStepDependent        waits for the previous step to complete before its first tile
//   kStepConstructThenOp  a range of a request: each element's x (and y) is computed from item.seed
//                         (and seed2) over [item.q2, hi) in registers and stored, and item.op
//                         (scalar item.q) is applied to those values and stored; item.index_base is
//                         the generator index of element 0
// fin_word: 1 + index of the completion word the piece reports to when its last tile is done (0:
// none).
struct StepItem {
    sx_batch_item item{};
    uint32_t flags = 0;
    uint32_t fin_word = 0;
    uint64_t seed2 = 0;
    double hi = 0.0;
};
constexpr uint32_t kStepDependent = 1u, kStepConstructThenOp = 2u;
// Launch the batched kernel over `items` (tiles of cfg.chunk_bytes, items passed in the launch's
// parameters) on `stream` and record s.done after it.  With `overlap` the launch may start while
// the previous step still runs (programmatic dependent launch).
// With `report`, no event is recorded: the step's last block to finish writes report->seq to the
// host-mapped word report->done (report->counter: a zeroed device counter owned by the caller's
// slot), and pieces with a fin_word set fin_host[fin_word - 1] (host-mapped, device address) to 1
// when their last tile is done (fin_count: zeroed device counters, one per word).  The step must
// have work.
struct StepReport {
    uint64_t seq;
    unsigned long long *done;  // device address of a host-mapped word
    unsigned int *counter;
    unsigned long long *fin_host = nullptr;
    unsigned int *fin_count = nullptr;
};
int step_launch(const sx_target *t, cudaStream_t stream, StepSlot &s, const StepItem *items, size_t count,
                const sx_batch_cfg &cfg, bool overlap, const StepReport *report = nullptr);
// Launch the step kernels once with no work on `stream` and wait: module loading and other
// first-launch costs are paid here rather than by the first step of a latency-bound caller.
int step_warm(cudaStream_t stream);

// ---- autotuner table (sx_tune.cpp) ------------------------------------------------------
bool tune_table_lookup(const sx_target *t, int op, int dtype, size_t n, sx_launch_cfg *cfg);
bool tune_batch_lookup(const sx_target *t, double mean_item_bytes, sx_batch_cfg *cfg);
void tune_batch_store(const sx_target *t, double mean_item_bytes, const sx_batch_cfg &cfg);

// ---- monotonic host clock in seconds --------------------------------------------------------
double now_seconds();

}  // namespace sx
