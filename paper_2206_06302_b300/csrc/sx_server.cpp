// sx_server.cpp -- a serving loop for STREAM requests on device-resident arrays.
//
// A request asks for `op` over n elements whose inputs are constructed on the device from
// seeds (Section 3.2's bulk construction, offloaded to the GPU as in Section 4.2) and whose
// output stays resident until the client releases it.  The server thread owns one device arena
// of budget_bytes; a request is admitted when a slot is free and its arrays fit in the arena
// (first fit, address-ordered free list with coalescing), otherwise it waits.  Requests larger
// than the whole arena are rejected at submission.
//
// CONTINUOUS mode batches requests continuously.  A step is one launch of the batched kernel
// (sx_batch.cu) over a list of pieces, passed in the launch's parameters: for each active
// request a range of its elements.  By default every piece is a construct-then-operate piece:
// for each element the inputs are computed from their seeds in registers and stored, and the
// operation is applied to those register values and stored, so the operation's inputs are never
// read back from memory and the integer-bound construction of some blocks overlaps the stores
// of others on the same SM.  (With split_phases, as before, phase 0 constructs x and y and
// phase 1 runs the operation in a later piece; only short requests are fused.)  The step's byte
// budget goes by policy, shortest remaining work first by default, so short requests finish in
// the first step that takes them while long ones advance in the rest.  Up to steps_in_flight
// steps are queued on the stream (backlog_steps more while requests wait for admission) and
// consecutive steps overlap through programmatic dependent launch; a split-phase operation piece that needs the inputs built in a step not yet known
// complete waits for it on the device.  The thread builds the next step while the GPU runs the
// previous ones, admits arrivals between steps, and marks a request DONE when the step holding
// its last piece has completed.  A request that a step takes whole, in one piece, reports its
// own completion: the warp that finishes the piece's last part sets a host-mapped word, and the
// request is DONE as soon as the thread sees it, without waiting for the rest of the step.
//
// FIFO mode is the per-call baseline: each admitted request is enqueued at once as its own
// launches (construct x, construct y, operation) in arrival order, like a client calling the
// algorithms directly.
//
// The host waits by polling (the step completion word, FIFO events) and on condition variables.
// On the device a step waits for its predecessor only through programmatic dependent launch
// (griddepcontrol.wait, a dependency the hardware resolves when the previous kernel in the
// stream completes); no kernel spins on memory another kernel writes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sx_internal.h"
#include "sx_sched.h"

namespace sx {
namespace {

using sched::Arena;

struct Request {
    uint64_t id = 0;
    sx_request r{};
    int state = SX_REQ_QUEUED;
    int status = SX_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int narr = 0;             // arrays held: x (and y), out
    size_t off[3] = {0, 0, 0};
    size_t bytes[3] = {0, 0, 0};
    bool allocated = false;
    int phase = 0;            // 0: construct inputs, 1: operation, 2: all work launched
    uint64_t next = 0;        // next element of the current phase
    int bypassed = 0;         // admission: times a later request was admitted first
    uint64_t admit_seq = 0;   // order of admission
    uint64_t inputs_step = 0; // step that holds the last piece of the inputs construction
    bool cancel = false;      // sx_server_cancel: no further work; CANCELLED once none is in flight
    uint64_t last_step = 0;   // CONTINUOUS: the last step that holds a piece of this request
    int readers = 0;          // sx_server_read copies in progress from the request's arrays
    bool free_deferred = false;  // released while being read: the last reader frees the arrays
    int fin_word = -1;        // CONTINUOUS: completion word of its construct-then-operate piece
    uint64_t fin_step = 0;    // the step that holds that piece
};

bool has_y(int op) { return op == SX_OP_ADD || op == SX_OP_TRIAD; }

// STREAM byte count of a phase per element.
size_t phase_bytes_per_elem(const Request &q, int phase) {
    const size_t es = dtype_size(q.r.dtype);
    if (phase == 0) return (has_y(q.r.op) ? 2 : 1) * es;
    return (size_t)op_arrays(q.r.op) * es;
}

struct Step {
    uint64_t seq = 0;                 // CONTINUOUS: step number, from 1
    int slot = -1;                    // CONTINUOUS: staging slot; FIFO: -1
    cudaEvent_t ev = nullptr;         // FIFO: the request's completion event
    std::vector<Request *> finishing; // requests whose last work is in this step
    uint64_t bytes = 0;
    double t_launch = 0;
};

}  // namespace
}  // namespace sx

using namespace sx;

struct sx_server {
    sx_target *t = nullptr;
    sx_server_cfg cfg{};
    sx_batch_cfg kcfg{};
    char *base = nullptr;
    std::unique_ptr<Arena> arena;
    cudaStream_t read_stream = nullptr;

    std::mutex mu;
    std::condition_variable cv;       // wakes the server thread
    std::condition_variable done_cv;  // wakes waiters
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::deque<Request *> waiting;
    std::vector<Request *> active;
    std::vector<Request *> cancelling;  // cancelled mid-phase: freed once their last step retires
    std::deque<Step> inflight;
    std::vector<StepSlot> slots;
    // CONTINUOUS completion reports: the host-mapped word the last block of each step writes its
    // step number to, and one device counter of finished blocks per slot
    unsigned long long *done_host = nullptr, *done_dev = nullptr;
    unsigned int *counters = nullptr;
    // completion words of construct-then-operate pieces (host-mapped, set to 1 by the device) with
    // their device tile counters; words in use are watched through fin_watch (server thread only)
    unsigned long long *fin_host = nullptr, *fin_dev = nullptr;
    unsigned int *fin_count = nullptr;
    std::vector<int> free_fin;
    std::vector<Request *> fin_watch;
    std::vector<int> free_slots;
    std::vector<cudaEvent_t> free_events;
    uint64_t next_id = 1;
    bool stop = false;
    bool admit_dirty = false;  // arrivals, freed memory or slots since the last admission pass
    // threads (other than the server's) waiting for or holding the lock: the server thread
    // neither spins nor polls the GPU with the lock held while this is non-zero
    std::atomic<int> contenders{0};
    std::atomic<uint64_t> grants{0};  // lock acquisitions by such threads
    // bumped on every arrival and every release of arena memory: the server thread watches it
    // without the lock to know that admission has something to do
    std::atomic<uint64_t> arrivals{0};
    uint64_t step_seq = 0;     // steps launched
    uint64_t retired_seq = 0;  // every step up to this one is known complete
    int large_held = 0;        // large requests holding arena memory (see kMaxLarge)
    int error = SX_OK;
    std::string error_msg;
    sx_server_stats stats{};
    double busy_since = -1;

    std::thread th;
    std::vector<std::thread> replayers;
};

namespace sx {
namespace {

// True once the step numbered `seq` has completed (its last block wrote seq or later).
bool step_reported(const sx_server *s, uint64_t seq) {
    return *(volatile unsigned long long *)s->done_host >= seq;
}

// Large requests hold more than 1/16 of the arena.  At most kMaxLarge of them hold memory at a
// time, so the rest of the arena stays open to smaller requests: under fair sharing a long
// request keeps its memory for long, and without the cap a handful of them could fill the
// arena and stall every admission behind them.
constexpr int kMaxLarge = 4;

// Completion words for construct-then-operate pieces in flight (more such pieces wait for their
// step to retire instead).
constexpr int kFinWords = 4096;

bool fin_reported(const sx_server *s, const Request *q) {
    return ((volatile unsigned long long *)s->fin_host)[q->fin_word] != 0;
}

bool is_large(const sx_server *s, const Request *q) {
    return (q->bytes[0] + q->bytes[1] + q->bytes[2]) * 16 > s->arena->size();
}

void release_arrays(sx_server *s, Request *q) {
    if (!q->allocated) return;
    if (is_large(s, q)) s->large_held--;
    for (int k = 0; k < 3; ++k)
        if (q->bytes[k]) s->arena->release(q->off[k], q->bytes[k]);
    q->allocated = false;
    s->stats.arena_used = s->arena->used();
}

void *ptr_of(sx_server *s, const Request *q, int k) { return q->bytes[k] ? s->base + q->off[k] : nullptr; }

// Arena bytes of a request: x, y (ADD/TRIAD), out.
void request_sizes(const sx_request &r, size_t bytes[3]) {
    const size_t b = (size_t)r.n * dtype_size(r.dtype);
    bytes[0] = b;
    bytes[1] = has_y(r.op) ? b : 0;
    bytes[2] = b;
}

size_t rounded_total(const size_t bytes[3]) {
    size_t t = 0;
    for (int k = 0; k < 3; ++k)
        if (bytes[k]) t += sched::arena_bytes(bytes[k]);
    return t;
}

bool try_admit(sx_server *s, Request *q) {
    size_t bytes[3];
    request_sizes(q->r, bytes);
    const bool large = (bytes[0] + bytes[1] + bytes[2]) * 16 > s->arena->size();
    if (large && s->large_held >= kMaxLarge) return false;
    size_t off[3] = {0, 0, 0};
    int k = 0;
    for (; k < 3; ++k) {
        if (!bytes[k]) continue;
        if (!s->arena->alloc(bytes[k], &off[k])) break;
    }
    if (k < 3) {
        for (int j = 0; j < k; ++j)
            if (bytes[j]) s->arena->release(off[j], bytes[j]);
        return false;
    }
    for (int j = 0; j < 3; ++j) {
        q->off[j] = off[j];
        q->bytes[j] = bytes[j];
    }
    q->allocated = true;
    if (large) s->large_held++;
    q->state = SX_REQ_ACTIVE;
    q->t_admit = now_seconds();
    q->admit_seq = s->stats.admitted;
    q->phase = 0;
    q->next = 0;
    s->stats.admitted++;
    s->stats.arena_used = s->arena->used();
    s->stats.arena_peak = s->arena->peak();
    return true;
}

// Admission in arrival order with bounded overtaking (sched::admission_pass).
void admit(sx_server *s) {
    if (!s->admit_dirty) return;
    s->admit_dirty = false;
    const double t0 = now_seconds();
    if (sched::admission_pass(s->waiting, s->active, (size_t)s->cfg.max_active,
                              [s](Request *q) { return try_admit(s, q); }))
        s->admit_dirty = true;
    s->stats.host_admit_seconds += now_seconds() - t0;
}

int enqueue_fifo(sx_server *s, Request *q, Step &st) {
    cudaStream_t sm = s->t->stream;
    const sx_request &r = q->r;
    SX_TRY(launch_seed(sm, r.dtype, ptr_of(s, q, 0), r.n, r.seed_x, r.lo, r.hi, 0));
    if (has_y(r.op)) SX_TRY(launch_seed(sm, r.dtype, ptr_of(s, q, 1), r.n, r.seed_y, r.lo, r.hi, 0));
    const sx_launch_cfg c = resolve_cfg(s->t, r.op, r.dtype, r.n, nullptr);
    SX_TRY(validate_cfg(s->t, r.op, c));
    SX_TRY(launch_stream_op(s->t, sm, r.op, r.dtype, ptr_of(s, q, 0), ptr_of(s, q, 1), ptr_of(s, q, 2), r.n, r.q, c));
    if (s->free_events.empty()) {
        cudaEvent_t ev;
        SX_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        s->free_events.push_back(ev);
    }
    st.ev = s->free_events.back();
    s->free_events.pop_back();
    SX_CUDA(cudaEventRecord(st.ev, sm));
    st.finishing.push_back(q);
    st.bytes = (uint64_t)(phase_bytes_per_elem(*q, 0) + phase_bytes_per_elem(*q, 1)) * r.n;
    q->phase = 2;
    return SX_OK;
}

// Build and launch one CONTINUOUS step from the active requests' pending work.
//
// The step's byte budget is shared by cfg.policy (sched::plan_step).
int launch_step(sx_server *s, bool *launched) {
    TraceRange tr("sx_server step");
    *launched = false;
    const uint64_t budget = (uint64_t)(uint32_t)s->cfg.chunk_bytes;
    std::vector<sched::Want> w;
    std::vector<Request *> by_key;
    std::vector<uint8_t> fused;  // construct-then-operate pieces: planned with the bytes of both phases
    const bool split = s->cfg.split_phases != 0;
    for (Request *q : s->active) {
        if (q->phase >= 2) continue;
        const uint64_t p0 = phase_bytes_per_elem(*q, 0), p1 = phase_bytes_per_elem(*q, 1);
        // fused: every piece constructs its range of the inputs and applies the operation to it;
        // split: short requests (whole work at most a quarter of the budget) as one such piece,
        // the others in two phases
        const bool cto = !split || (q->phase == 0 && q->next == 0 && (uint64_t)q->r.n * (p0 + p1) <= budget / 4);
        const uint64_t later = q->phase == 0 && !cto ? (uint64_t)q->r.n * p1 : 0;
        const uint64_t per = cto ? p0 + p1 : phase_bytes_per_elem(*q, q->phase);
        w.push_back({by_key.size(), q->admit_seq, per, q->r.n - q->next, later});
        by_key.push_back(q);
        fused.push_back(cto ? 1 : 0);
    }
    if (w.empty()) return SX_OK;
    // elements of each request's current phase in this step, in the policy's order (sx_sched.h)
    const std::vector<uint64_t> grant = sched::plan_step(s->cfg.policy, budget, w);
    const int slot = s->free_slots.back();
    s->free_slots.pop_back();
    std::vector<StepItem> items;
    Step st;
    st.slot = slot;
    st.seq = s->step_seq + 1;
    std::vector<Request *> watch;  // requests given a completion word in this step
    for (size_t i = 0; i < w.size(); ++i) {
        if (grant[i] == 0) continue;
        Request *q = by_key[w[i].key];
        q->last_step = st.seq;
        const uint64_t elems = grant[i];
        const uint64_t lo = q->next, hi = lo + elems;
        const sx_request &r = q->r;
        const size_t es = dtype_size(r.dtype);
        if (fused[w[i].key] && (!split || elems == r.n)) {
            // construct x (and y) over [lo, hi), then the operation on that range, tile by tile
            StepItem si;
            si.item.op = r.op;
            si.item.dtype = r.dtype;
            si.item.n = elems;
            si.item.x = (char *)ptr_of(s, q, 0) + lo * es;
            si.item.y = has_y(r.op) ? (char *)ptr_of(s, q, 1) + lo * es : nullptr;
            si.item.out = (char *)ptr_of(s, q, 2) + lo * es;
            si.item.q = r.q;
            si.item.q2 = r.lo;
            si.item.seed = r.seed_x;
            si.item.index_base = lo;
            si.flags = kStepConstructThenOp;
            si.seed2 = r.seed_y;
            si.hi = r.hi;
            const bool one_piece = lo == 0 && elems == r.n;
            if (one_piece && !s->free_fin.empty()) {
                // the whole request in this piece: it reports its own completion
                q->fin_word = s->free_fin.back();
                s->free_fin.pop_back();
                ((volatile unsigned long long *)s->fin_host)[q->fin_word] = 0;
                q->fin_step = st.seq;
                si.fin_word = (uint32_t)q->fin_word + 1;
                watch.push_back(q);
            }
            items.push_back(si);
            st.bytes += elems * (phase_bytes_per_elem(*q, 0) + phase_bytes_per_elem(*q, 1));
            q->next = hi;
            if (q->next == r.n) {
                q->next = 0;
                q->phase = 2;
                st.finishing.push_back(q);
            }
            if (one_piece) s->stats.fused++;
            continue;
        }
        const uint64_t per = phase_bytes_per_elem(*q, q->phase);
        if (q->phase == 0) {
            StepItem si;
            si.item.op = SX_OP_SEED;
            si.item.dtype = r.dtype;
            si.item.n = elems;
            si.item.out = (char *)ptr_of(s, q, 0) + lo * es;
            si.item.q = r.lo;
            si.item.q2 = r.hi;
            si.item.seed = r.seed_x;
            si.item.index_base = lo;
            items.push_back(si);
            if (has_y(r.op)) {
                si.item.out = (char *)ptr_of(s, q, 1) + lo * es;
                si.item.seed = r.seed_y;
                items.push_back(si);
            }
        } else {
            StepItem si;
            si.item.op = r.op;
            si.item.dtype = r.dtype;
            si.item.n = elems;
            si.item.x = (const char *)ptr_of(s, q, 0) + lo * es;
            si.item.y = has_y(r.op) ? (const char *)ptr_of(s, q, 1) + lo * es : nullptr;
            si.item.out = (char *)ptr_of(s, q, 2) + lo * es;
            si.item.q = r.q;
            // operation pieces whose inputs come from a step still in flight wait for it
            si.flags = q->inputs_step > s->retired_seq ? kStepDependent : 0u;
            items.push_back(si);
        }
        st.bytes += elems * per;
        q->next = hi;
        if (q->next == r.n) {
            q->next = 0;
            if (q->phase == 0) q->inputs_step = st.seq;
            q->phase++;
            if (q->phase == 2) st.finishing.push_back(q);
        }
    }
    // independent pieces first (in the policy's order), so that blocks reach the ones that must
    // wait as late as possible
    std::stable_sort(items.begin(), items.end(), [](const StepItem &a, const StepItem &b) {
        return (a.flags & kStepDependent) < (b.flags & kStepDependent);
    });
    const StepReport report{st.seq, s->done_dev, s->counters + slot, s->fin_dev, s->fin_count};
    const int rc = step_launch(s->t, s->t->stream, s->slots[slot], items.data(), items.size(), s->kcfg,
                               s->cfg.serialize_steps == 0, &report);
    if (rc != SX_OK) {
        s->free_slots.push_back(slot);
        for (Request *q : watch) {
            s->free_fin.push_back(q->fin_word);
            q->fin_word = -1;
        }
        return rc;
    }
    for (Request *q : watch) s->fin_watch.push_back(q);
    st.t_launch = now_seconds();
    s->step_seq = st.seq;
    s->inflight.push_back(std::move(st));
    s->stats.steps++;
    s->stats.launches++;
    const uint64_t depth = s->slots.size() - s->free_slots.size();
    s->stats.steps_in_flight_peak = std::max<uint64_t>(s->stats.steps_in_flight_peak, depth);
    if (depth > (uint64_t)s->cfg.steps_in_flight) s->stats.backlog_launches++;
    *launched = true;
    return SX_OK;
}

// A cancelled request with no work in flight: arrays freed, CANCELLED.
void finalize_cancel(sx_server *s, Request *q) {
    release_arrays(s, q);
    q->state = SX_REQ_CANCELLED;
    q->t_done = now_seconds();
    s->stats.cancelled++;
    s->admit_dirty = true;
    s->arrivals.fetch_add(1, std::memory_order_release);
}

// Stop watching q's completion word and give the word back.
void unwatch(sx_server *s, Request *q) {
    s->fin_watch.erase(std::find(s->fin_watch.begin(), s->fin_watch.end(), q));
    s->free_fin.push_back(q->fin_word);
    q->fin_word = -1;
}

// True if a watched construct-then-operate piece has reported (server thread, lock not needed).
bool any_fin_reported(const sx_server *s) {
    for (const Request *q : s->fin_watch)
        if (fin_reported(s, q)) return true;
    return false;
}

// Requests whose construct-then-operate piece has reported are DONE (or CANCELLED) at once, while
// the rest of their step may still run: their tiles are all done, and no other piece touches
// their arrays.  Returns true if any completed.
bool collect_reported(sx_server *s) {
    bool any = false;
    for (size_t i = 0; i < s->fin_watch.size();) {
        Request *q = s->fin_watch[i];
        if (!fin_reported(s, q)) {
            ++i;
            continue;
        }
        unwatch(s, q);  // removes s->fin_watch[i]
        for (Step &st : s->inflight) {
            if (st.seq != q->fin_step) continue;
            st.finishing.erase(std::find(st.finishing.begin(), st.finishing.end(), q));
            break;
        }
        s->stats.early_done++;
        s->active.erase(std::find(s->active.begin(), s->active.end(), q));
        if (q->cancel) {
            finalize_cancel(s, q);
        } else {
            q->state = SX_REQ_DONE;
            q->t_done = now_seconds();
            s->stats.completed++;
            if (q->r.flags & SX_REQ_AUTO_RELEASE) release_arrays(s, q);
            s->admit_dirty = true;
        }
        any = true;
    }
    return any;
}

// Retire completed steps from the front of the in-flight queue.  Returns true if any retired
// (or a cancelled request was finalised).
bool retire(sx_server *s) {
    bool any = false;
    while (!s->inflight.empty()) {
        Step &st = s->inflight.front();
        cudaError_t e = cudaSuccess;
        if (st.slot >= 0) {
            if (!step_reported(s, st.seq)) {
                // a failed launch never reports: surface its error instead of waiting forever
                e = cudaStreamQuery(s->t->stream);
                if (e == cudaErrorNotReady || e == cudaSuccess) break;
            }
        } else {
            e = cudaEventQuery(st.ev);
            if (e == cudaErrorNotReady) break;
        }
        if (e != cudaSuccess) {
            s->error = SX_ERR_CUDA;
            s->error_msg = cudaGetErrorString(e);
        }
        const double now = now_seconds();
        for (Request *q : st.finishing) {
            if (q->fin_word >= 0) unwatch(s, q);  // its word was not seen before the step retired
            s->active.erase(std::find(s->active.begin(), s->active.end(), q));
            if (q->cancel) {
                finalize_cancel(s, q);
                continue;
            }
            q->state = SX_REQ_DONE;
            q->t_done = now;
            s->stats.completed++;
            if (q->r.flags & SX_REQ_AUTO_RELEASE) release_arrays(s, q);
            s->admit_dirty = true;
        }
        s->stats.bytes_moved += st.bytes;
        if (st.slot >= 0) s->retired_seq = st.seq;
        if (st.slot >= 0) s->free_slots.push_back(st.slot);
        else s->free_events.push_back(st.ev);
        s->inflight.pop_front();
        any = true;
    }
    for (size_t i = 0; i < s->cancelling.size();) {
        Request *q = s->cancelling[i];
        if (q->last_step <= s->retired_seq) {
            finalize_cancel(s, q);
            s->cancelling.erase(s->cancelling.begin() + i);
            any = true;
        } else {
            ++i;
        }
    }
    return any;
}

// A step may be launched while fewer than steps_in_flight are on the GPU, or fewer than
// steps_in_flight + backlog_steps while requests wait for admission.
bool may_launch_step(const sx_server *s) {
    const int used = (int)s->slots.size() - (int)s->free_slots.size();
    return used < s->cfg.steps_in_flight ||
           (!s->waiting.empty() && used < s->cfg.steps_in_flight + s->cfg.backlog_steps);
}

void server_loop(sx_server *s) {
    DeviceScope ds(s->t->device);
    std::unique_lock<std::mutex> lk(s->mu);
    const bool fifo = s->cfg.mode == SX_SERVE_FIFO;
    for (;;) {
        const bool retired = retire(s) | collect_reported(s);
        if (retired) s->done_cv.notify_all();
        if (!s->stop) admit(s);
        bool launched = false;
        if (s->error == SX_OK) {
            int rc = SX_OK;
            if (fifo) {
                for (Request *q : s->active) {
                    if (q->phase != 0) continue;
                    Step st;
                    rc = enqueue_fifo(s, q, st);
                    if (rc != SX_OK) break;
                    st.t_launch = now_seconds();
                    s->inflight.push_back(std::move(st));
                    s->stats.launches += has_y(q->r.op) ? 3 : 2;
                    launched = true;
                }
            } else if (may_launch_step(s)) {
                const double tl = now_seconds();
                rc = launch_step(s, &launched);
                s->stats.host_step_seconds += now_seconds() - tl;
            }
            if (rc != SX_OK) {
                s->error = rc;
                s->error_msg = sx_last_error();
            }
        }
        const double now = now_seconds();
        if (!s->inflight.empty()) {
            if (s->busy_since < 0) s->busy_since = now;
        } else if (s->busy_since >= 0) {
            s->stats.busy_seconds += now - s->busy_since;
            s->busy_since = -1;
        }
        const bool work_pending = !s->active.empty() || !s->inflight.empty() || !s->cancelling.empty();
        if (s->stop && !work_pending) break;
        if (s->stop && s->error != SX_OK && s->inflight.empty()) break;
        // Between passes the lock goes to any thread that asked for it: the server thread does
        // not take it back while one is announced (an unlock followed at once by a lock would
        // win the race against the woken thread every time and starve submitters).  Each thread
        // announced when the wait starts gets one turn: the wait ends once as many acquisitions
        // have happened (or nobody is left, or after 100 us), so a caller polling in a loop, which
        // announces itself again at once, neither starves nor throttles the server.
        auto give_turns = [s](int c0, uint64_t g0) {
            const double until = now_seconds() + 1e-4;
            while (s->contenders.load(std::memory_order_acquire) &&
                   s->grants.load(std::memory_order_acquire) - g0 < (uint64_t)c0 && now_seconds() < until)
                std::this_thread::yield();
        };
        auto wait_contenders = [s, &give_turns]() {  // lock not held
            const int c0 = s->contenders.load(std::memory_order_acquire);
            if (c0) give_turns(c0, s->grants.load(std::memory_order_acquire));
        };
        auto let_others_in = [s, &lk, &give_turns]() {  // lock held
            const int c0 = s->contenders.load(std::memory_order_acquire);
            if (!c0) return;
            const uint64_t g0 = s->grants.load(std::memory_order_acquire);
            lk.unlock();
            give_turns(c0, g0);
            lk.lock();
        };
        if (launched || retired) {
            let_others_in();
            continue;
        }
        const uint64_t seen = s->arrivals.load(std::memory_order_acquire);
        if (!s->inflight.empty()) {
            // GPU busy: wait for the oldest step without the lock; come back early for arrivals
            // or freed memory (admission), and let callers that want the lock have it.  The first
            // 500 us are spent polling (a step usually takes ~100 us); after that the thread sleeps
            // between polls, so that long steps do not keep a core busy.
            Step &front = s->inflight.front();
            const bool by_word = front.slot >= 0;
            const uint64_t want = front.seq;
            cudaEvent_t ev = front.ev;
            lk.unlock();
            const double spin_until = now_seconds() + 5e-4;
            while (!(by_word ? step_reported(s, want) : cudaEventQuery(ev) != cudaErrorNotReady) &&
                   s->arrivals.load(std::memory_order_acquire) == seen && !any_fin_reported(s)) {
                if (now_seconds() < spin_until) std::this_thread::yield();
                else std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
            wait_contenders();
            lk.lock();
        } else {
            // idle: watch for arrivals for a short while without the lock, then sleep
            lk.unlock();
            const double until = now_seconds() + 2e-4;
            while (s->arrivals.load(std::memory_order_acquire) == seen && now_seconds() < until)
                std::this_thread::yield();
            wait_contenders();
            lk.lock();
            if (s->arrivals.load(std::memory_order_acquire) == seen && !s->stop)
                s->cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
    // reject what never got in
    for (Request *q : s->waiting) {
        q->state = SX_REQ_REJECTED;
        q->status = SX_ERR_STATE;
    }
    s->waiting.clear();
    s->done_cv.notify_all();
}

// The lock as taken by API calls: announced first, so the server thread lets go of it.
struct ApiLock {
    sx_server *s;
    std::unique_lock<std::mutex> lk;
    explicit ApiLock(sx_server *sv) : s(sv) {
        s->contenders.fetch_add(1, std::memory_order_relaxed);
        lk = std::unique_lock<std::mutex>(s->mu);
        s->grants.fetch_add(1, std::memory_order_release);
    }
    ~ApiLock() {
        if (lk.owns_lock()) lk.unlock();
        s->contenders.fetch_sub(1, std::memory_order_relaxed);
    }
};

void fill_status(sx_server *s, const Request *q, sx_request_status *st) {
    st->state = q->state;
    st->status = q->status;
    st->t_submit = q->t_submit;
    st->t_admit = q->t_admit;
    st->t_done = q->t_done;
    const bool live = q->allocated;
    st->x = live ? ptr_of(s, q, 0) : nullptr;
    st->y = live ? ptr_of(s, q, 1) : nullptr;
    st->out = live ? ptr_of(s, q, 2) : nullptr;
}

int check_request(const sx_request *r) {
    if (!r) return fail(SX_ERR_INVALID, "request is NULL");
    if (r->op < SX_OP_COPY || r->op > SX_OP_TRIAD) return fail(SX_ERR_INVALID, "request op %d", r->op);
    if (r->dtype != SX_F32 && r->dtype != SX_F64) return fail(SX_ERR_DTYPE, "request dtype %d", r->dtype);
    if (r->n == 0) return fail(SX_ERR_INVALID, "request of zero elements");
    if (r->n > (1ull << 40)) return fail(SX_ERR_INVALID, "request too large");
    return SX_OK;
}

// Register a request (lock held).  Oversized requests are rejected at once.
void submit_locked(sx_server *s, const sx_request &r, uint64_t id, double t) {
    auto q = std::make_unique<Request>();
    q->id = id;
    q->r = r;
    q->t_submit = t;
    size_t bytes[3];
    request_sizes(r, bytes);
    s->stats.submitted++;
    Request *raw = q.get();
    s->reqs[id] = std::move(q);
    if (rounded_total(bytes) > s->arena->size()) {
        raw->state = SX_REQ_REJECTED;
        raw->status = SX_ERR_OOM;
        s->stats.rejected++;
        s->done_cv.notify_all();
        return;
    }
    s->waiting.push_back(raw);
    s->admit_dirty = true;
    s->arrivals.fetch_add(1, std::memory_order_release);
}

Request *find(sx_server *s, uint64_t id) {
    auto it = s->reqs.find(id);
    return it == s->reqs.end() ? nullptr : it->second.get();
}

}  // namespace
}  // namespace sx

extern "C" {

int sx_server_create(sx_target *t, const sx_server_cfg *cfg, sx_server **out) {
    if (!t || !cfg || !out) return fail(SX_ERR_INVALID, "NULL argument");
    *out = nullptr;
    sx_server_cfg c = *cfg;
    if (c.mode != SX_SERVE_CONTINUOUS && c.mode != SX_SERVE_FIFO) return fail(SX_ERR_INVALID, "mode %d", c.mode);
    if (c.budget_bytes == 0) return fail(SX_ERR_INVALID, "budget_bytes must be positive");
    if (c.max_active == 0) c.max_active = 256;
    // step budget: 1 GiB of STREAM bytes (~110 us of GPU time at saturation); on the served
    // workload, alternating in one process, 768 MiB gave 2-4% lower p99 at 0.8 and 0.95 load but
    // 2.8% less throughput at saturation, 512 MiB a lower and noisier saturation, 2 GiB a higher
    // p50 at 0.95 load
    if (c.chunk_bytes == 0) c.chunk_bytes = 1 << 30;
    if (c.steps_in_flight == 0) c.steps_in_flight = 2;
    if (c.policy != SX_SERVE_POLICY_SHORT_FIRST && c.policy != SX_SERVE_POLICY_FAIR &&
        c.policy != SX_SERVE_POLICY_SRPT)
        return fail(SX_ERR_INVALID, "policy %d", c.policy);
    if (c.serialize_steps != 0 && c.serialize_steps != 1)
        return fail(SX_ERR_INVALID, "serialize_steps %d: 0 or 1", c.serialize_steps);
    if (c.split_phases != 0 && c.split_phases != 1)
        return fail(SX_ERR_INVALID, "split_phases %d: 0 or 1", c.split_phases);
    if (c.max_active < 1 || c.max_active > 65536) return fail(SX_ERR_INVALID, "max_active %d", c.max_active);
    if (c.chunk_bytes < (1 << 20)) return fail(SX_ERR_INVALID, "chunk_bytes %d below 1 MiB", c.chunk_bytes);
    if (c.steps_in_flight < 1 || c.steps_in_flight > 8) return fail(SX_ERR_INVALID, "steps_in_flight %d", c.steps_in_flight);
    // two more steps while requests wait (measured on the served workload: saturation 8.56-9.09
    // TB/s with none, 8.91-9.15 with one, 8.98-9.17 with two; latency at 0.95 load unchanged)
    if (c.backlog_steps == 0) c.backlog_steps = std::min(2, 8 - c.steps_in_flight);
    else if (c.backlog_steps == -1) c.backlog_steps = 0;
    if (c.backlog_steps < 0 || c.steps_in_flight + c.backlog_steps > 8)
        return fail(SX_ERR_INVALID, "backlog_steps %d: -1, 0 or 1..%d with steps_in_flight %d", cfg->backlog_steps,
                    8 - c.steps_in_flight, c.steps_in_flight);
    // default step-kernel shape, measured on the served workload with construct-then-operate
    // pieces: eight blocks of 128 threads per SM (the kernel's 61 registers allow 32 warps) and
    // 256 KiB tiles.  Small blocks at different points of their tiles share each SM: saturation
    // 9.7-9.9 TB/s for 128-thread blocks at 24-32 warps per SM with 256 KiB-1 MiB tiles, 9.0-9.1
    // for four blocks of 256 threads with 128 KiB tiles, 8.4 with 64 KiB; p99 at 0.95 load 1.28
    // ms against 1.51.  (Blocks beyond those an SM holds are not launched: the grid is capped.)
    sx_batch_cfg k{};
    k.chunk_bytes = c.tile_bytes ? c.tile_bytes : 256 * 1024;
    k.threads = c.threads ? c.threads : 128;
    k.blocks_per_sm = c.blocks_per_sm ? c.blocks_per_sm : 8;
    k.vec_bytes = c.vec_bytes ? c.vec_bytes : 32;
    if (k.chunk_bytes < 16384 || k.threads % 32 || k.threads < 64 || k.threads > 1024 ||
        k.blocks_per_sm * k.threads > 2048 || (k.vec_bytes != 16 && k.vec_bytes != 32))
        return fail(SX_ERR_INVALID, "batched-kernel shape (tile %d, threads %d, blocks/SM %d, vec %d)",
                    k.chunk_bytes, k.threads, k.blocks_per_sm, k.vec_bytes);
    // the arena is charged to the target's budget like any allocation
    size_t used = t->used.load();
    do {
        if (used + c.budget_bytes > t->budget)
            return fail(SX_ERR_OOM, "server arena of %llu bytes exceeds the target budget",
                        (unsigned long long)c.budget_bytes);
    } while (!t->used.compare_exchange_weak(used, used + c.budget_bytes));
    DeviceScope ds(t->device);
    sx_server *s = new (std::nothrow) sx_server();
    if (!s) {
        t->used -= c.budget_bytes;
        return fail(SX_ERR_OOM, "host allocation failed");
    }
    s->t = t;
    s->cfg = c;
    s->kcfg = k;
    cudaError_t e = cudaMalloc(&s->base, c.budget_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->read_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (s->base) cudaFree(s->base);
        t->used -= c.budget_bytes;
        delete s;
        cudaGetLastError();
        if (e == cudaErrorMemoryAllocation) return fail(SX_ERR_OOM, "arena allocation failed");
        return cuda_fail(e, "server setup");
    }
    s->arena.reset(new Arena(c.budget_bytes));
    s->stats.arena_bytes = c.budget_bytes;
    if (c.mode == SX_SERVE_CONTINUOUS) {
        const int nslots = c.steps_in_flight + c.backlog_steps;
        s->slots.resize(nslots);
        for (int i = nslots - 1; i >= 0; --i) s->free_slots.push_back(i);
        auto undo = [s, t, &c]() {
            if (s->done_host) cudaFreeHost(s->done_host);
            if (s->counters) cudaFree(s->counters);
            if (s->fin_host) cudaFreeHost(s->fin_host);
            if (s->fin_count) cudaFree(s->fin_count);
            cudaStreamDestroy(s->read_stream);
            cudaFree(s->base);
            t->used -= c.budget_bytes;
            delete s;
        };
        cudaError_t e2 = cudaHostAlloc((void **)&s->done_host, sizeof(unsigned long long), cudaHostAllocMapped);
        if (e2 == cudaSuccess) e2 = cudaHostGetDevicePointer((void **)&s->done_dev, s->done_host, 0);
        if (e2 == cudaSuccess) e2 = cudaMalloc(&s->counters, nslots * sizeof(unsigned int));
        if (e2 == cudaSuccess) e2 = cudaMemset(s->counters, 0, nslots * sizeof(unsigned int));
        if (e2 == cudaSuccess)
            e2 = cudaHostAlloc((void **)&s->fin_host, kFinWords * sizeof(unsigned long long), cudaHostAllocMapped);
        if (e2 == cudaSuccess) e2 = cudaHostGetDevicePointer((void **)&s->fin_dev, s->fin_host, 0);
        if (e2 == cudaSuccess) e2 = cudaMalloc(&s->fin_count, kFinWords * sizeof(unsigned int));
        if (e2 == cudaSuccess) e2 = cudaMemset(s->fin_count, 0, kFinWords * sizeof(unsigned int));
        if (e2 != cudaSuccess) {
            undo();
            return cuda_fail(e2, "server step reports");
        }
        *(volatile unsigned long long *)s->done_host = 0;
        for (int i = kFinWords - 1; i >= 0; --i) {
            ((volatile unsigned long long *)s->fin_host)[i] = 0;
            s->free_fin.push_back(i);
        }
        const int rc = step_warm(t->stream);
        if (rc != SX_OK) {
            undo();
            return rc;
        }
    }
    s->th = std::thread(server_loop, s);
    *out = s;
    return SX_OK;
}

int sx_server_submit(sx_server *s, const sx_request *r, uint64_t *id) {
    if (!s || !id) return fail(SX_ERR_INVALID, "NULL argument");
    SX_TRY(check_request(r));
    const double t = now_seconds();  // the arrival, before any wait for the lock
    {
        ApiLock g(s);
        if (s->stop) return fail(SX_ERR_STATE, "server is stopping");
        *id = s->next_id++;
        submit_locked(s, *r, *id, t);
    }
    s->cv.notify_one();
    return SX_OK;
}

int sx_server_replay(sx_server *s, const sx_request *reqs, const double *t_arrival, size_t count,
                     uint64_t *ids) {
    if (!s || (count && (!reqs || !t_arrival || !ids))) return fail(SX_ERR_INVALID, "NULL argument");
    for (size_t k = 0; k < count; ++k) {
        SX_TRY(check_request(&reqs[k]));
        if (k && t_arrival[k] < t_arrival[k - 1]) return fail(SX_ERR_INVALID, "arrival times must not decrease");
    }
    uint64_t first;
    {
        ApiLock g(s);
        if (s->stop) return fail(SX_ERR_STATE, "server is stopping");
        first = s->next_id;
        s->next_id += count;
    }
    for (size_t k = 0; k < count; ++k) ids[k] = first + k;
    std::vector<sx_request> rs(reqs, reqs + count);
    std::vector<double> ts(t_arrival, t_arrival + count);
    const double t0 = now_seconds();
    ApiLock g(s);
    s->replayers.emplace_back([s, rs = std::move(rs), ts = std::move(ts), first, t0]() {
        for (size_t k = 0; k < rs.size(); ++k) {
            const double due = t0 + ts[k];
            for (;;) {
                const double now = now_seconds();
                if (now >= due) break;
                if (due - now > 2e-4)
                    std::this_thread::sleep_for(std::chrono::duration<double>(due - now - 1e-4));
                else
                    std::this_thread::yield();
            }
            {
                // the scheduled arrival time is the request's arrival, whatever the wait after it
                ApiLock g2(s);
                submit_locked(s, rs[k], first + k, due);
            }
            s->cv.notify_one();
        }
    });
    return SX_OK;
}

int sx_server_poll(sx_server *s, uint64_t id, sx_request_status *st) {
    if (!s || !st) return fail(SX_ERR_INVALID, "NULL argument");
    ApiLock g(s);
    Request *q = find(s, id);
    if (!q) return fail(SX_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
    fill_status(s, q, st);
    return SX_OK;
}

int sx_server_wait(sx_server *s, uint64_t id, int64_t timeout_ms, sx_request_status *st) {
    if (!s) return fail(SX_ERR_INVALID, "NULL argument");
    ApiLock al(s);
    std::unique_lock<std::mutex> &lk = al.lk;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        Request *q = find(s, id);
        if (!q) {
            // a replayed request may not be registered yet
            if (id >= s->next_id) return fail(SX_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
        } else if (q->state == SX_REQ_DONE || q->state == SX_REQ_REJECTED || q->state == SX_REQ_RELEASED ||
                   q->state == SX_REQ_CANCELLED) {
            if (st) fill_status(s, q, st);
            return SX_OK;
        }
        if (s->error != SX_OK) return fail(s->error, "server failed: %s", s->error_msg.c_str());
        if (timeout_ms < 0) {
            s->contenders.fetch_sub(1, std::memory_order_relaxed);  // asleep, not contending
            s->done_cv.wait_for(lk, std::chrono::milliseconds(50));
            s->contenders.fetch_add(1, std::memory_order_relaxed);
        } else {
            if (std::chrono::steady_clock::now() >= deadline)
                return fail(SX_ERR_TIMEOUT, "request %llu not done after %lld ms", (unsigned long long)id,
                            (long long)timeout_ms);
            s->contenders.fetch_sub(1, std::memory_order_relaxed);
            s->done_cv.wait_until(lk, std::min(deadline, std::chrono::steady_clock::now() + std::chrono::milliseconds(50)));
            s->contenders.fetch_add(1, std::memory_order_relaxed);
        }
    }
}

int sx_server_read(sx_server *s, uint64_t id, int which, void *host, size_t n) {
    if (!s || (!host && n)) return fail(SX_ERR_INVALID, "NULL argument");
    if (which < 0 || which > 2) return fail(SX_ERR_INVALID, "which=%d: 0 = x, 1 = y, 2 = out", which);
    const void *src;
    size_t bytes;
    Request *q;
    {
        ApiLock g(s);
        q = find(s, id);
        if (!q) return fail(SX_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
        if (q->state != SX_REQ_DONE || !q->allocated) return fail(SX_ERR_STATE, "request %llu has no resident result", (unsigned long long)id);
        if (!q->bytes[which]) return fail(SX_ERR_INVALID, "request %llu has no array %d", (unsigned long long)id, which);
        if (n > q->r.n) return fail(SX_ERR_INVALID, "n=%zu exceeds the request length", n);
        src = ptr_of(s, q, which);
        bytes = n * dtype_size(q->r.dtype);
        q->readers++;  // the arrays stay allocated until the copy is done (see sx_server_release)
    }
    cudaError_t e;
    {
        DeviceScope ds(s->t->device);
        e = cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, s->read_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->read_stream);
    }
    bool freed = false;
    {
        ApiLock g(s);
        if (--q->readers == 0 && q->free_deferred) {
            q->free_deferred = false;
            release_arrays(s, q);
            s->admit_dirty = true;
            s->arrivals.fetch_add(1, std::memory_order_release);
            freed = true;
        }
    }
    if (freed) s->cv.notify_one();
    if (e != cudaSuccess) return cuda_fail(e, "server read");
    return SX_OK;
}

int sx_server_release(sx_server *s, uint64_t id) {
    if (!s) return fail(SX_ERR_INVALID, "NULL argument");
    {
        ApiLock g(s);
        Request *q = find(s, id);
        if (!q) return fail(SX_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
        if (q->state == SX_REQ_CANCELLED) return SX_OK;  // its arrays were freed when it was cancelled
        if (q->state != SX_REQ_DONE && q->state != SX_REQ_REJECTED)
            return fail(SX_ERR_STATE, "request %llu is not finished", (unsigned long long)id);
        if (q->state == SX_REQ_DONE) q->state = SX_REQ_RELEASED;  // no new reads from here on
        if (q->readers > 0) {
            q->free_deferred = true;  // a read in progress frees the arrays when it ends
            return SX_OK;
        }
        release_arrays(s, q);
        s->admit_dirty = true;
        s->arrivals.fetch_add(1, std::memory_order_release);
    }
    s->cv.notify_one();  // memory freed: admission may proceed
    return SX_OK;
}

int sx_server_cancel(sx_server *s, uint64_t id) {
    if (!s) return fail(SX_ERR_INVALID, "NULL argument");
    {
        ApiLock g(s);
        Request *q = find(s, id);
        if (!q) {
            if (id < s->next_id) return fail(SX_ERR_STATE, "request %llu is not registered yet (replayed)",
                                              (unsigned long long)id);
            return fail(SX_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
        }
        if (q->state == SX_REQ_QUEUED) {
            s->waiting.erase(std::find(s->waiting.begin(), s->waiting.end(), q));
            finalize_cancel(s, q);
        } else if (q->state == SX_REQ_ACTIVE) {
            if (q->cancel) return SX_OK;  // already on its way out
            q->cancel = true;
            // pieces not all launched: no more are; the arrays are freed once the steps holding
            // the launched ones have completed (at once if none was launched)
            if (q->phase < 2) {
                s->active.erase(std::find(s->active.begin(), s->active.end(), q));
                const bool fifo = s->cfg.mode == SX_SERVE_FIFO;
                if (fifo || q->last_step <= s->retired_seq) finalize_cancel(s, q);
                else s->cancelling.push_back(q);
            }
            // otherwise it is in a step's finishing list: retire makes it CANCELLED
        } else {
            return fail(SX_ERR_STATE, "request %llu is finished (release it instead)", (unsigned long long)id);
        }
        s->arrivals.fetch_add(1, std::memory_order_release);
    }
    s->cv.notify_one();
    s->done_cv.notify_all();
    return SX_OK;
}

int sx_server_stats_get(sx_server *s, sx_server_stats *st) {
    if (!s || !st) return fail(SX_ERR_INVALID, "NULL argument");
    ApiLock g(s);
    *st = s->stats;
    st->arena_used = s->arena->used();
    st->arena_peak = s->arena->peak();
    if (s->busy_since >= 0) st->busy_seconds += now_seconds() - s->busy_since;
    return SX_OK;
}

int sx_server_destroy(sx_server *s) {
    if (!s) return fail(SX_ERR_INVALID, "NULL argument");
    std::vector<std::thread> reps;
    {
        ApiLock g(s);
        reps.swap(s->replayers);
    }
    for (auto &r : reps) r.join();  // every replayed request is submitted
    {
        ApiLock g(s);
        s->stop = true;
        s->arrivals.fetch_add(1, std::memory_order_release);
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    const int err = s->error;
    const std::string msg = s->error_msg;
    {
        DeviceScope ds(s->t->device);
        cudaStreamSynchronize(s->t->stream);
        for (auto &sl : s->slots) step_slot_free(sl);
        if (s->done_host) cudaFreeHost(s->done_host);
        if (s->counters) cudaFree(s->counters);
        if (s->fin_host) cudaFreeHost(s->fin_host);
        if (s->fin_count) cudaFree(s->fin_count);
        for (auto ev : s->free_events) cudaEventDestroy(ev);
        if (s->read_stream) cudaStreamDestroy(s->read_stream);
        cudaFree(s->base);
    }
    s->t->used -= s->cfg.budget_bytes;
    delete s;
    if (err != SX_OK) return fail(err, "server stopped after an error: %s", msg.c_str());
    return SX_OK;
}

}  // extern "C"
