// sx_runtime.cpp -- targets, the allocator, executors, futures and the algorithm entry points
// of libsx (Sections 3.1-3.4 and 4.2 of Heller et al.; Listing 4 for sx_stream_iter).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sx_internal.h"

namespace sx {

namespace {
thread_local std::string g_last_error;
}

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

int cuda_fail(cudaError_t e, const char *what) {
    return fail(SX_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

double now_seconds() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int check_device_error(const sx_target *t) {
    int code = 0;
    SX_CUDA(cudaMemcpy(&code, t->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (code != 0) {
        const int zero = 0;
        SX_CUDA(cudaMemcpy(t->d_err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        return fail(SX_ERR_DEVICE, "a device-side bounded wait expired (code %d); outputs of the "
                                   "work since the last check are invalid", code);
    }
    return SX_OK;
}

namespace {

int sync_target(sx_target *t) {
    DeviceScope ds(t->device);
    SX_CUDA(cudaStreamSynchronize(t->stream));
    return check_device_error(t);
}

bool overlaps_partially(const sx_array *in, const sx_array *out) {
    if (!in || !out) return false;
    const uintptr_t a = (uintptr_t)in->ptr, b = (uintptr_t)out->ptr;
    const size_t la = in->n * dtype_size(in->dtype), lb = out->n * dtype_size(out->dtype);
    if (la == 0 || lb == 0) return false;
    if (a == b) return false;  // exact aliasing is allowed (element i read before written)
    return a < b + lb && b < a + la;
}

int check_operands(const sx_executor *e, int op, const sx_array *x, const sx_array *y, const sx_array *out) {
    if (!e) return fail(SX_ERR_INVALID, "executor is NULL");
    if (op < SX_OP_COPY || op > SX_OP_TRIAD) return fail(SX_ERR_INVALID, "op %d is not COPY..TRIAD", op);
    const bool has_y = (op == SX_OP_ADD || op == SX_OP_TRIAD);
    if (!x || !out || (has_y && !y)) return fail(SX_ERR_INVALID, "array argument is NULL");
    if (x->t != e->t || out->t != e->t || (has_y && y->t != e->t))
        return fail(SX_ERR_INVALID, "arrays must be placed on the executor's target");
    if (x->dtype != out->dtype || (has_y && y->dtype != x->dtype))
        return fail(SX_ERR_DTYPE, "operands have different element types");
    if (x->dtype != SX_F32 && x->dtype != SX_F64)
        return fail(SX_ERR_DTYPE, "STREAM kernels take F32 or F64 arrays");
    if (x->n != out->n || (has_y && y->n != x->n))
        return fail(SX_ERR_INVALID, "operand lengths differ (%zu, %zu, %zu)", x->n,
                    has_y ? y->n : x->n, out->n);
    if (overlaps_partially(x, out) || (has_y && overlaps_partially(y, out)))
        return fail(SX_ERR_OVERLAP, "output partially overlaps an input");
    return SX_OK;
}

int enqueue_op(sx_executor *e, int op, const sx_array *x, const sx_array *y, sx_array *out, double q) {
    const sx_launch_cfg c = resolve_cfg(e->t, op, x->dtype, x->n, e->fixed_cfg ? &e->cfg : nullptr);
    SX_TRY(validate_cfg(e->t, op, c));
    const bool has_y = (op == SX_OP_ADD || op == SX_OP_TRIAD);
    return launch_stream_op(e->t, e->t->stream, op, x->dtype, x->ptr, has_y ? y->ptr : nullptr,
                            out->ptr, x->n, q, c);
}

int finish_call(sx_executor *e) {
    if (e->policy == SX_PAR) return sync_target(e->t);
    return SX_OK;
}

}  // namespace

int new_future(sx_target *t, sx_future **out) {
    sx_future *f = new (std::nothrow) sx_future();
    if (!f) return fail(SX_ERR_OOM, "host allocation failed");
    f->t = t;
    cudaError_t err = cudaEventCreate(&f->start);
    if (err == cudaSuccess) err = cudaEventCreate(&f->end);
    if (err != cudaSuccess) {
        if (f->start) cudaEventDestroy(f->start);
        delete f;
        return cuda_fail(err, "cudaEventCreate");
    }
    *out = f;
    return SX_OK;
}

}  // namespace sx

using namespace sx;

extern "C" {

const char *sx_last_error(void) {
    return sx::g_last_error.c_str();
}

const char *sx_status_string(int s) {
    switch (s) {
        case SX_OK: return "SX_OK";
        case SX_ERR_INVALID: return "SX_ERR_INVALID";
        case SX_ERR_OOM: return "SX_ERR_OOM";
        case SX_ERR_DTYPE: return "SX_ERR_DTYPE";
        case SX_ERR_OVERLAP: return "SX_ERR_OVERLAP";
        case SX_ERR_TIMEOUT: return "SX_ERR_TIMEOUT";
        case SX_ERR_CUDA: return "SX_ERR_CUDA";
        case SX_ERR_NOT_READY: return "SX_ERR_NOT_READY";
        case SX_ERR_DEVICE: return "SX_ERR_DEVICE";
        case SX_ERR_STATE: return "SX_ERR_STATE";
        default: return "SX_ERR_UNKNOWN";
    }
}

int sx_version(void) { return 10000; }

// ---- targets ---------------------------------------------------------------------------------
int sx_target_count(int *count) {
    if (!count) return fail(SX_ERR_INVALID, "count is NULL");
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) {
        cudaGetLastError();
        *count = 0;
        return SX_OK;
    }
    SX_CUDA(e);
    *count = n;
    return SX_OK;
}

int sx_target_create_ext(int device, void *stream, size_t budget_bytes, sx_target **out) {
    if (!out) return fail(SX_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int count = 0;
    SX_TRY(sx_target_count(&count));
    if (device < 0 || device >= count)
        return fail(SX_ERR_INVALID, "device %d not present (%d visible)", device, count);
    DeviceScope ds(device);
    cudaDeviceProp p;
    SX_CUDA(cudaGetDeviceProperties(&p, device));
    sx_target *t = new (std::nothrow) sx_target();
    if (!t) return fail(SX_ERR_OOM, "host allocation failed");
    t->device = device;
    t->sm_count = p.multiProcessorCount;
    t->cc_major = p.major;
    t->cc_minor = p.minor;
    t->l2_bytes = (size_t)p.l2CacheSize;
    t->hbm_total = p.totalGlobalMem;
    t->max_smem_block = (int)p.sharedMemPerBlockOptin;
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);
    t->sm_clock_khz = clk;
    t->name = p.name;
    t->budget = budget_bytes ? budget_bytes : p.totalGlobalMem;
    cudaError_t e = cudaSuccess;
    if (stream) {
        t->stream = (cudaStream_t)stream;
        t->owns_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking);
        t->owns_stream = true;
    }
    if (e == cudaSuccess) e = cudaMalloc(&t->d_err, 256);
    if (e == cudaSuccess) e = cudaMemset(t->d_err, 0, 256);
    if (e != cudaSuccess) {
        if (t->owns_stream && t->stream) cudaStreamDestroy(t->stream);
        if (t->d_err) cudaFree(t->d_err);
        delete t;
        return cuda_fail(e, "target setup");
    }
    *out = t;
    return SX_OK;
}

int sx_target_create(int device, sx_target **out) { return sx_target_create_ext(device, nullptr, 0, out); }

int sx_target_destroy(sx_target *t) {
    if (!t) return fail(SX_ERR_INVALID, "target is NULL");
    {
        DeviceScope ds(t->device);
        cudaStreamSynchronize(t->stream);
        if (t->d_err) cudaFree(t->d_err);
        for (auto &ps : t->pipe)
            if (ps) cudaStreamDestroy(ps);
        for (auto &pe : t->pipe_ev)
            if (pe) cudaEventDestroy(pe);
        if (t->owns_stream) cudaStreamDestroy(t->stream);
    }
    delete t;
    return SX_OK;
}

int sx_target_info_get(const sx_target *t, sx_target_info *o) {
    if (!t || !o) return fail(SX_ERR_INVALID, "NULL argument");
    DeviceScope ds(t->device);
    memset(o, 0, sizeof *o);
    o->device = t->device;
    o->sm_count = t->sm_count;
    o->cc_major = t->cc_major;
    o->cc_minor = t->cc_minor;
    o->l2_bytes = (int64_t)t->l2_bytes;
    o->hbm_total = (int64_t)t->hbm_total;
    size_t fr = 0, tot = 0;
    SX_CUDA(cudaMemGetInfo(&fr, &tot));
    o->hbm_free = (int64_t)fr;
    o->budget = (int64_t)t->budget;
    o->used = (int64_t)t->used.load();
    o->max_smem_block = t->max_smem_block;
    o->sm_clock_khz = t->sm_clock_khz;
    snprintf(o->name, sizeof o->name, "%s", t->name.c_str());
    return SX_OK;
}

int sx_target_stream(const sx_target *t, void **stream) {
    if (!t || !stream) return fail(SX_ERR_INVALID, "NULL argument");
    *stream = (void *)t->stream;
    return SX_OK;
}

int sx_target_synchronize(sx_target *t) {
    if (!t) return fail(SX_ERR_INVALID, "target is NULL");
    return sync_target(t);
}

int sx_target_selftest(sx_target *t, int64_t limit_us) {
    if (!t) return fail(SX_ERR_INVALID, "target is NULL");
    if (limit_us < 1 || limit_us > 1000000) return fail(SX_ERR_INVALID, "limit_us=%lld out of [1, 1e6]", (long long)limit_us);
    DeviceScope ds(t->device);
    return launch_selftest(t, t->stream, limit_us);
}

// ---- arrays / allocator ----------------------------------------------------------------------
int sx_alloc(sx_target *t, sx_dtype dtype, size_t n, sx_array **out) {
    if (!t || !out) return fail(SX_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const size_t es = dtype_size(dtype);
    if (es == 0) return fail(SX_ERR_DTYPE, "unknown dtype %d", (int)dtype);
    if (n > (SIZE_MAX - 4 * kGuardBytes) / es) return fail(SX_ERR_INVALID, "n=%zu overflows", n);
    const size_t data = n * es;
    const size_t bytes = ((data + 255) / 256) * 256 + kGuardBytes;
    // host-side budget accounting: never relies on the CUDA allocator failing
    size_t used = t->used.load();
    do {
        if (used + bytes > t->budget)
            return fail(SX_ERR_OOM, "allocation of %zu bytes exceeds the target budget (%zu of %zu used)",
                        bytes, used, t->budget);
    } while (!t->used.compare_exchange_weak(used, used + bytes));
    DeviceScope ds(t->device);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        t->used -= bytes;
        cudaGetLastError();
        if (e == cudaErrorMemoryAllocation) return fail(SX_ERR_OOM, "device allocation of %zu bytes failed", bytes);
        return cuda_fail(e, "cudaMalloc");
    }
    e = cudaMemsetAsync((char *)p + data, kGuardByte, bytes - data, t->stream);
    if (e != cudaSuccess) {
        cudaFree(p);
        t->used -= bytes;
        return cuda_fail(e, "guard fill");
    }
    sx_array *a = new (std::nothrow) sx_array();
    if (!a) {
        cudaFree(p);
        t->used -= bytes;
        return fail(SX_ERR_OOM, "host allocation failed");
    }
    a->t = t;
    a->dtype = dtype;
    a->n = n;
    a->ptr = p;
    a->owned = true;
    a->alloc_bytes = bytes;
    a->data_bytes = data;
    *out = a;
    return SX_OK;
}

int sx_array_wrap(sx_target *t, sx_dtype dtype, void *ptr, size_t n, sx_array **out) {
    if (!t || !out) return fail(SX_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const size_t es = dtype_size(dtype);
    if (es == 0) return fail(SX_ERR_DTYPE, "unknown dtype %d", (int)dtype);
    if (!ptr && n) return fail(SX_ERR_INVALID, "device pointer is NULL");
    if ((uintptr_t)ptr % es) return fail(SX_ERR_INVALID, "pointer not aligned to its element type");
    if (n > SIZE_MAX / es) return fail(SX_ERR_INVALID, "n=%zu overflows", n);
    sx_array *a = new (std::nothrow) sx_array();
    if (!a) return fail(SX_ERR_OOM, "host allocation failed");
    a->t = t;
    a->dtype = dtype;
    a->n = n;
    a->ptr = ptr;
    a->owned = false;
    a->data_bytes = n * es;
    *out = a;
    return SX_OK;
}

int sx_free(sx_array *a) {
    if (!a) return fail(SX_ERR_INVALID, "array is NULL");
    if (a->owned) {
        DeviceScope ds(a->t->device);
        // work on the stream may still use the memory
        cudaStreamSynchronize(a->t->stream);
        cudaFree(a->ptr);
        a->t->used -= a->alloc_bytes;
    }
    delete a;
    return SX_OK;
}

int sx_array_data(const sx_array *a, void **ptr, size_t *n, int *dtype) {
    if (!a) return fail(SX_ERR_INVALID, "array is NULL");
    if (ptr) *ptr = a->ptr;
    if (n) *n = a->n;
    if (dtype) *dtype = a->dtype;
    return SX_OK;
}

int sx_array_guard_ok(const sx_array *a, int *ok) {
    if (!a || !ok) return fail(SX_ERR_INVALID, "NULL argument");
    *ok = 1;
    if (!a->owned) return SX_OK;
    DeviceScope ds(a->t->device);
    SX_CUDA(cudaStreamSynchronize(a->t->stream));
    const size_t gb = a->alloc_bytes - a->data_bytes;
    std::vector<unsigned char> h(gb);
    SX_CUDA(cudaMemcpy(h.data(), (char *)a->ptr + a->data_bytes, gb, cudaMemcpyDeviceToHost));
    for (unsigned char c : h)
        if (c != kGuardByte) {
            *ok = 0;
            break;
        }
    return SX_OK;
}

int sx_bulk_construct(sx_array *a, double value) {
    if (!a) return fail(SX_ERR_INVALID, "array is NULL");
    DeviceScope ds(a->t->device);
    return launch_fill(a->t->stream, a->dtype, a->ptr, a->n, value);
}

int sx_bulk_destroy(sx_array *a) {
    if (!a) return fail(SX_ERR_INVALID, "array is NULL");
    return SX_OK;  // trivially destructible elements: no destructor to run
}

int sx_seed_uniform(sx_array *a, uint64_t seed, double lo, double hi) {
    if (!a) return fail(SX_ERR_INVALID, "array is NULL");
    DeviceScope ds(a->t->device);
    return launch_seed(a->t->stream, a->dtype, a->ptr, a->n, seed, lo, hi, 0);
}

int sx_seed_uniform_at(sx_array *a, uint64_t seed, double lo, double hi, uint64_t index_base) {
    if (!a) return fail(SX_ERR_INVALID, "array is NULL");
    if (a->n && index_base > UINT64_MAX - (a->n - 1))
        return fail(SX_ERR_INVALID, "index_base + n - 1 exceeds the generator's 64-bit index");
    DeviceScope ds(a->t->device);
    return launch_seed(a->t->stream, a->dtype, a->ptr, a->n, seed, lo, hi, index_base);
}

// ---- block partition of one logical array over several targets (Section 4.1) ----------------
int sx_block_partition(uint64_t n, int parts, int part, uint64_t *offset, uint64_t *count) {
    if (!offset || !count) return fail(SX_ERR_INVALID, "NULL argument");
    if (parts < 1) return fail(SX_ERR_INVALID, "parts=%d: need at least 1", parts);
    if (part < 0 || part >= parts) return fail(SX_ERR_INVALID, "part=%d out of [0, %d)", part, parts);
    if (n > (UINT64_MAX >> 1)) return fail(SX_ERR_INVALID, "n too large");
    const uint64_t block = n / (uint64_t)parts + (n % (uint64_t)parts != 0);  // ceil(n / parts)
    const uint64_t lo = std::min<uint64_t>(n, (uint64_t)part * block);
    const uint64_t hi = std::min<uint64_t>(n, lo + block);
    *offset = lo;
    *count = hi - lo;
    return SX_OK;
}

// ---- host <-> device copies (Section 4.2) ------------------------------------------------------
static int copy_common(sx_array *dev, const void *host, size_t n, bool h2d, bool async) {
    if (!dev || (!host && n)) return fail(SX_ERR_INVALID, "NULL argument");
    if (n > dev->n) return fail(SX_ERR_INVALID, "n=%zu exceeds the array length %zu", n, dev->n);
    if (n == 0) return SX_OK;
    DeviceScope ds(dev->t->device);
    const size_t bytes = n * dtype_size(dev->dtype);
    if (h2d)
        SX_CUDA(cudaMemcpyAsync(dev->ptr, host, bytes, cudaMemcpyHostToDevice, dev->t->stream));
    else
        SX_CUDA(cudaMemcpyAsync((void *)host, dev->ptr, bytes, cudaMemcpyDeviceToHost, dev->t->stream));
    if (!async) SX_CUDA(cudaStreamSynchronize(dev->t->stream));
    return SX_OK;
}

int sx_copy_h2d(sx_array *dst, const void *host, size_t n) { return copy_common(dst, host, n, true, false); }
int sx_copy_d2h(void *host, const sx_array *src, size_t n) {
    return copy_common(const_cast<sx_array *>(src), host, n, false, false);
}
int sx_copy_h2d_async(sx_array *dst, const void *host, size_t n) { return copy_common(dst, host, n, true, true); }
int sx_copy_d2h_async(void *host, const sx_array *src, size_t n) {
    return copy_common(const_cast<sx_array *>(src), host, n, false, true);
}

// ---- executors -------------------------------------------------------------------------------
int sx_executor_create(sx_target *t, sx_policy policy, const sx_launch_cfg *cfg, sx_executor **out) {
    if (!t || !out) return fail(SX_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (policy != SX_PAR && policy != SX_PAR_TASK) return fail(SX_ERR_INVALID, "unknown policy %d", (int)policy);
    sx_executor *e = new (std::nothrow) sx_executor();
    if (!e) return fail(SX_ERR_OOM, "host allocation failed");
    e->t = t;
    e->policy = policy;
    if (cfg && cfg->variant != SX_VARIANT_AUTO) {
        e->fixed_cfg = true;
        e->cfg = *cfg;
        // the shape is checked here as for a one-input call; calls with two inputs check again
        // (BULK and TMA stage twice the shared memory for them)
        const sx_launch_cfg full = resolve_cfg(t, SX_OP_SCALE, SX_F64, 1, &e->cfg);
        int s = validate_cfg(t, SX_OP_SCALE, full);
        if (s != SX_OK) {
            delete e;
            return s;
        }
    }
    *out = e;
    return SX_OK;
}

int sx_executor_destroy(sx_executor *e) {
    if (!e) return fail(SX_ERR_INVALID, "executor is NULL");
    {
        DeviceScope ds(e->t->device);
        for (auto &g : e->graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (e->capture) cudaStreamDestroy(e->capture);
    }
    delete e;
    return SX_OK;
}

int sx_executor_wait(sx_executor *e) {
    if (!e) return fail(SX_ERR_INVALID, "executor is NULL");
    return sync_target(e->t);
}

int sx_executor_resolve(const sx_executor *e, sx_op op, sx_dtype dtype, size_t n, sx_launch_cfg *out) {
    if (!e || !out) return fail(SX_ERR_INVALID, "NULL argument");
    *out = resolve_cfg(e->t, op, dtype, n, e->fixed_cfg ? &e->cfg : nullptr);
    return SX_OK;
}

// ---- futures -----------------------------------------------------------------------------------
int sx_future_wait(sx_future *f, int64_t timeout_ms) {
    if (!f) return fail(SX_ERR_INVALID, "future is NULL");
    DeviceScope ds(f->t->device);
    if (timeout_ms < 0) {
        SX_CUDA(cudaEventSynchronize(f->end));
    } else {
        const double deadline = now_seconds() + timeout_ms * 1e-3;
        for (;;) {
            cudaError_t e = cudaEventQuery(f->end);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
            if (now_seconds() > deadline) return fail(SX_ERR_TIMEOUT, "future not complete after %lld ms", (long long)timeout_ms);
            std::this_thread::yield();
        }
    }
    return check_device_error(f->t);
}

int sx_future_test(sx_future *f) {
    if (!f) return fail(SX_ERR_INVALID, "future is NULL");
    DeviceScope ds(f->t->device);
    cudaError_t e = cudaEventQuery(f->end);
    if (e == cudaSuccess) return SX_OK;
    if (e == cudaErrorNotReady) return SX_ERR_NOT_READY;
    return cuda_fail(e, "cudaEventQuery");
}

int sx_future_elapsed_ms(sx_future *f, float *ms) {
    if (!f || !ms) return fail(SX_ERR_INVALID, "NULL argument");
    DeviceScope ds(f->t->device);
    cudaError_t e = cudaEventQuery(f->end);
    if (e == cudaErrorNotReady) return fail(SX_ERR_NOT_READY, "future not complete");
    SX_CUDA(e);
    SX_CUDA(cudaEventElapsedTime(ms, f->start, f->end));
    return SX_OK;
}

int sx_future_destroy(sx_future *f) {
    if (!f) return fail(SX_ERR_INVALID, "future is NULL");
    DeviceScope ds(f->t->device);
    cudaEventDestroy(f->start);
    cudaEventDestroy(f->end);
    delete f;
    return SX_OK;
}

// ---- algorithms ----------------------------------------------------------------------------
int sx_execute(sx_executor *e, sx_op op, const sx_array *x, const sx_array *y, sx_array *out, double q) {
    TraceRange tr("sx_execute");
    SX_TRY(check_operands(e, op, x, y, out));
    DeviceScope ds(e->t->device);
    SX_TRY(enqueue_op(e, op, x, y, out, q));
    return finish_call(e);
}

int sx_execute_async(sx_executor *e, sx_op op, const sx_array *x, const sx_array *y, sx_array *out,
                     double q, sx_future **fut) {
    TraceRange tr("sx_execute_async");
    if (fut) *fut = nullptr;
    SX_TRY(check_operands(e, op, x, y, out));
    DeviceScope ds(e->t->device);
    sx_future *f = nullptr;
    if (fut) {
        SX_TRY(new_future(e->t, &f));
        cudaEventRecord(f->start, e->t->stream);
    }
    int s = enqueue_op(e, op, x, y, out, q);
    if (s != SX_OK) {
        if (f) sx_future_destroy(f);
        return s;
    }
    if (f) {
        cudaError_t err = cudaEventRecord(f->end, e->t->stream);
        if (err != cudaSuccess) {
            sx_future_destroy(f);
            return cuda_fail(err, "cudaEventRecord");
        }
        *fut = f;
    }
    return SX_OK;
}

int sx_copy(sx_executor *e, const sx_array *src, sx_array *dst) {
    return sx_execute(e, SX_OP_COPY, src, nullptr, dst, 0.0);
}

int sx_transform_scale(sx_executor *e, const sx_array *in, sx_array *out, double q) {
    return sx_execute(e, SX_OP_SCALE, in, nullptr, out, q);
}

int sx_transform_add(sx_executor *e, const sx_array *x, const sx_array *y, sx_array *out) {
    return sx_execute(e, SX_OP_ADD, x, y, out, 0.0);
}

int sx_transform_triad(sx_executor *e, const sx_array *x, const sx_array *y, sx_array *out, double q) {
    return sx_execute(e, SX_OP_TRIAD, x, y, out, q);
}

static int check_stream_arrays(sx_executor *e, sx_array *a, sx_array *b, sx_array *c, int iters) {
    if (!e || !a || !b || !c) return fail(SX_ERR_INVALID, "NULL argument");
    if (iters < 0) return fail(SX_ERR_INVALID, "iters=%d is negative", iters);
    if (a->t != e->t || b->t != e->t || c->t != e->t)
        return fail(SX_ERR_INVALID, "arrays must be placed on the executor's target");
    if (a->dtype != b->dtype || a->dtype != c->dtype) return fail(SX_ERR_DTYPE, "a, b, c differ in type");
    if (a->dtype != SX_F32 && a->dtype != SX_F64) return fail(SX_ERR_DTYPE, "STREAM takes F32 or F64");
    if (a->n != b->n || a->n != c->n) return fail(SX_ERR_INVALID, "a, b, c differ in length");
    const size_t bytes = a->n * dtype_size(a->dtype);
    const uintptr_t pa = (uintptr_t)a->ptr, pb = (uintptr_t)b->ptr, pc = (uintptr_t)c->ptr;
    auto ov = [bytes](uintptr_t u, uintptr_t v) { return bytes && u < v + bytes && v < u + bytes; };
    if (ov(pa, pb) || ov(pa, pc) || ov(pb, pc)) return fail(SX_ERR_OVERLAP, "a, b, c must not overlap");
    return SX_OK;
}

// One pass of Listing 4 (four launches in stream order) on stream `s`.
static int enqueue_pass(sx_executor *e, cudaStream_t s, sx_array *a, sx_array *b, sx_array *c, double q,
                        const sx_launch_cfg (&cfg)[4]) {
    const int dt = a->dtype;
    const size_t n = a->n;
    SX_TRY(launch_stream_op(e->t, s, SX_OP_COPY, dt, a->ptr, nullptr, c->ptr, n, q, cfg[0]));  // c = a
    SX_TRY(launch_stream_op(e->t, s, SX_OP_SCALE, dt, c->ptr, nullptr, b->ptr, n, q, cfg[1])); // b = c*q
    SX_TRY(launch_stream_op(e->t, s, SX_OP_ADD, dt, a->ptr, b->ptr, c->ptr, n, q, cfg[2]));    // c = a+b
    SX_TRY(launch_stream_op(e->t, s, SX_OP_TRIAD, dt, b->ptr, c->ptr, a->ptr, n, q, cfg[3]));  // a = b+c*q
    return SX_OK;
}

// A graph of `key.passes` passes for this executor, captured on its private stream the first
// time and kept (up to kMaxGraphs, oldest dropped).  Nothing is launched on failure; the caller
// then launches directly, and the failure is kept too (a null entry), so it is not retried.
static cudaGraphExec_t pass_graph(sx_executor *e, sx_array *a, sx_array *b, sx_array *c, double q,
                                  const sx_pass_graph_key &key) {
    for (size_t i = 0; i < e->graphs.size(); ++i) {
        if (std::memcmp(&e->graphs[i].key, &key, sizeof key) == 0) {
            auto g = e->graphs[i];
            e->graphs.erase(e->graphs.begin() + i);
            e->graphs.push_back(g);
            return g.exec;
        }
    }
    if (!e->capture && cudaStreamCreateWithFlags(&e->capture, cudaStreamNonBlocking) != cudaSuccess) {
        e->capture = nullptr;
        cudaGetLastError();
        return nullptr;
    }
    if (cudaStreamBeginCapture(e->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int rc = SX_OK;
    for (int k = 0; k < key.passes && rc == SX_OK; ++k) rc = enqueue_pass(e, e->capture, a, b, c, q, key.cfg);
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(e->capture, &graph);  // always ends the capture
    cudaGraphExec_t exec = nullptr;
    if (rc == SX_OK && end == cudaSuccess && graph &&
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (!exec) clear_error();
    if (e->graphs.size() >= sx_executor::kMaxGraphs) {
        if (e->graphs.front().exec) cudaGraphExecDestroy(e->graphs.front().exec);
        e->graphs.erase(e->graphs.begin());
    }
    e->graphs.push_back({key, exec});
    return exec;
}

// Passes run from CUDA graphs of up to kGraphPasses passes (4 kernel nodes each) when there
// are at least two: one graph launch replaces up to 64 kernel launches, which dominate the
// time of small arrays.  Same kernels in the same order, so the same bits.  Direct launches
// are used for a single pass, while the target's stream is itself being captured, or if a
// graph cannot be made.
constexpr int kGraphPasses = 16;

int sx_stream_iter(sx_executor *e, sx_array *a, sx_array *b, sx_array *c, double q, int iters) {
    TraceRange tr("sx_stream_iter");
    SX_TRY(check_stream_arrays(e, a, b, c, iters));
    DeviceScope ds(e->t->device);
    sx_launch_cfg cfg[4];
    const int ops[4] = {SX_OP_COPY, SX_OP_SCALE, SX_OP_ADD, SX_OP_TRIAD};
    for (int k = 0; k < 4; ++k) {
        cfg[k] = resolve_cfg(e->t, ops[k], a->dtype, a->n, e->fixed_cfg ? &e->cfg : nullptr);
        SX_TRY(validate_cfg(e->t, ops[k], cfg[k]));
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool graphs = iters >= 2 && a->n > 0 &&
                        cudaStreamIsCapturing(e->t->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    int done = 0;
    while (graphs && iters - done >= 2) {
        sx_pass_graph_key key;
        std::memset(&key, 0, sizeof key);
        key.a = a->ptr;
        key.b = b->ptr;
        key.c = c->ptr;
        key.n = a->n;
        key.dtype = a->dtype;
        key.passes = std::min(kGraphPasses, iters - done);
        std::memcpy(&key.q_bits, &q, sizeof q);
        std::memcpy(key.cfg, cfg, sizeof cfg);
        cudaGraphExec_t g = pass_graph(e, a, b, c, q, key);
        if (!g) break;
        const int reps = (iters - done) / key.passes;
        for (int r = 0; r < reps; ++r) SX_CUDA(cudaGraphLaunch(g, e->t->stream));
        done += reps * key.passes;
    }
    for (; done < iters; ++done) SX_TRY(enqueue_pass(e, e->t->stream, a, b, c, q, cfg));
    return finish_call(e);
}

int sx_stream_fused(sx_executor *e, sx_array *a, sx_array *b, sx_array *c, double q, int iters) {
    TraceRange tr("sx_stream_fused");
    SX_TRY(check_stream_arrays(e, a, b, c, iters));
    DeviceScope ds(e->t->device);
    // the chain is four binary64 operations per pass, two of them products: unless the executor
    // fixes fp64_mul, the launch picks the unit (FP64 pipe for few elements per SM, the integer
    // units otherwise; bit-identical either way)
    const int mm = e->fixed_cfg ? e->cfg.fp64_mul : -1;
    SX_TRY(launch_stream_fused(e->t, e->t->stream, a->dtype, a->ptr, b->ptr, c->ptr, a->n, q, iters, mm));
    return finish_call(e);
}

// Every element's chain of passes depends only on its own start values, so the work is cut into
// chunks of elements, each copied in, run through `iters` passes and copied out on one of three
// pipeline streams: host-to-device and device-to-host copies of different chunks then share the
// two directions of the host link, and the kernels overlap both.  Results are the same bits as one
// copy, `iters` whole-array passes and one copy back.
int sx_stream_host(sx_executor *e, void *ha, void *hb, void *hc, sx_array *a, sx_array *b, sx_array *c,
                   double q, int iters) {
    TraceRange tr("sx_stream_host");
    SX_TRY(check_stream_arrays(e, a, b, c, iters));
    if (!ha || !hb || !hc) return fail(SX_ERR_INVALID, "host pointer is NULL");
    sx_target *t = e->t;
    DeviceScope ds(t->device);
    for (int i = 0; i < sx_target::kPipe; ++i)
        if (!t->pipe[i]) SX_CUDA(cudaStreamCreateWithFlags(&t->pipe[i], cudaStreamNonBlocking));
    for (auto &pe : t->pipe_ev)
        if (!pe) SX_CUDA(cudaEventCreateWithFlags(&pe, cudaEventDisableTiming));
    const size_t es = dtype_size(a->dtype);
    const size_t n = a->n;
    size_t chunk = ((size_t)32 << 20) / es;  // 32 MiB per array
    chunk = std::max<size_t>(64, chunk / 64 * 64);
    // the pipeline starts after the work already on the target's stream
    SX_CUDA(cudaEventRecord(t->pipe_ev[sx_target::kPipe], t->stream));
    for (int i = 0; i < sx_target::kPipe; ++i) SX_CUDA(cudaStreamWaitEvent(t->pipe[i], t->pipe_ev[sx_target::kPipe], 0));
    char *pa = (char *)a->ptr, *pb = (char *)b->ptr, *pc = (char *)c->ptr;
    char *qa = (char *)ha, *qb = (char *)hb, *qc = (char *)hc;
    const sx_launch_cfg *fixed = e->fixed_cfg ? &e->cfg : nullptr;
    size_t k = 0;
    for (size_t off = 0; off < n; off += chunk, ++k) {
        const size_t m = std::min(chunk, n - off);
        const size_t ob = off * es, mb = m * es;
        cudaStream_t s = t->pipe[k % sx_target::kPipe];
        SX_CUDA(cudaMemcpyAsync(pa + ob, qa + ob, mb, cudaMemcpyHostToDevice, s));
        if (iters == 0) {
            // a pass writes c (Copy) and b (Scale) before it reads them, so their start values
            // only matter when no pass runs
            SX_CUDA(cudaMemcpyAsync(pb + ob, qb + ob, mb, cudaMemcpyHostToDevice, s));
            SX_CUDA(cudaMemcpyAsync(pc + ob, qc + ob, mb, cudaMemcpyHostToDevice, s));
        }
        const int ops[4] = {SX_OP_COPY, SX_OP_SCALE, SX_OP_ADD, SX_OP_TRIAD};
        for (int it = 0; it < iters; ++it) {
            for (int op : ops) {
                const sx_launch_cfg cfg = resolve_cfg(t, op, a->dtype, m, fixed);
                SX_TRY(validate_cfg(t, op, cfg));
                // Listing 4's roles: copy a->c, scale c->b, add a,b->c, triad b,c->a
                const void *x = op == SX_OP_COPY ? pa + ob : op == SX_OP_SCALE ? pc + ob : op == SX_OP_ADD ? pa + ob : pb + ob;
                const void *y = op == SX_OP_ADD ? pb + ob : op == SX_OP_TRIAD ? pc + ob : nullptr;
                void *o = op == SX_OP_COPY ? pc + ob : op == SX_OP_SCALE ? pb + ob : op == SX_OP_ADD ? pc + ob : pa + ob;
                SX_TRY(launch_stream_op(t, s, op, a->dtype, x, y, o, m, q, cfg));
            }
        }
        SX_CUDA(cudaMemcpyAsync(qa + ob, pa + ob, mb, cudaMemcpyDeviceToHost, s));
        SX_CUDA(cudaMemcpyAsync(qb + ob, pb + ob, mb, cudaMemcpyDeviceToHost, s));
        SX_CUDA(cudaMemcpyAsync(qc + ob, pc + ob, mb, cudaMemcpyDeviceToHost, s));
    }
    // the target's stream continues after the whole pipeline
    for (int i = 0; i < sx_target::kPipe; ++i) {
        SX_CUDA(cudaEventRecord(t->pipe_ev[i], t->pipe[i]));
        SX_CUDA(cudaStreamWaitEvent(t->stream, t->pipe_ev[i], 0));
    }
    return sync_target(t);
}

int sx_transform_u8(sx_executor *e, int fn, const sx_array *in, sx_array *out) {
    if (!e || !in || !out) return fail(SX_ERR_INVALID, "NULL argument");
    if (in->t != e->t || out->t != e->t) return fail(SX_ERR_INVALID, "arrays must be placed on the executor's target");
    if (in->dtype != SX_U8 || out->dtype != SX_U8) return fail(SX_ERR_DTYPE, "byte transform takes U8 arrays");
    if (in->n != out->n) return fail(SX_ERR_INVALID, "lengths differ");
    if (overlaps_partially(in, out)) return fail(SX_ERR_OVERLAP, "output partially overlaps the input");
    DeviceScope ds(e->t->device);
    SX_TRY(launch_u8_transform(e->t, e->t->stream, fn, in->ptr, out->ptr, in->n));
    return finish_call(e);
}

}  // extern "C"
