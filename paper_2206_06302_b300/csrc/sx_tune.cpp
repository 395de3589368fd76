// sx_tune.cpp -- the launch-shape autotuner and its table, and the resolution of a call's launch
// shape (the tuner's table or the caller's shape, with defaults filled in, then checked).
//
// For one (op, dtype, n) the tuner times candidate launch shapes of the kernel families on
// scratch arrays and keeps the fastest; the pass tuner then times the four kernels together in
// a STREAM pass and picks the VECTOR kernels' cache hints for that context.  The table is keyed by (device name, op, dtype,
// floor(log2 n)) so that one measurement covers a size octave; executors with an AUTO
// configuration look it up on every call.  Batch shapes are keyed by (device name,
// floor(log2 mean item bytes)).  The table persists as a small JSON file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "sx_internal.h"

namespace sx {
namespace {

struct OpKey {
    std::string dev;
    int op, dtype, bucket;
    bool operator<(const OpKey &o) const {
        return std::tie(dev, op, dtype, bucket) < std::tie(o.dev, o.op, o.dtype, o.bucket);
    }
};
struct BatchKey {
    std::string dev;
    int bucket;
    bool operator<(const BatchKey &o) const { return std::tie(dev, bucket) < std::tie(o.dev, o.bucket); }
};

std::mutex g_mu;
std::map<OpKey, sx_launch_cfg> g_ops;
std::map<BatchKey, sx_batch_cfg> g_batch;

int log2_bucket(double v) { return v < 1 ? 0 : (int)std::floor(std::log2(v)); }

// ---- a minimal JSON reader for the table's own format --------------------------------------
struct JsonReader {
    const std::string &s;
    size_t i = 0;
    bool ok = true;
    explicit JsonReader(const std::string &str) : s(str) {}
    void ws() {
        while (i < s.size() && std::isspace((unsigned char)s[i])) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < s.size() && s[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    std::string str() {
        ws();
        std::string out;
        if (i >= s.size() || s[i] != '"') {
            ok = false;
            return out;
        }
        ++i;
        while (i < s.size() && s[i] != '"') {
            if (s[i] == '\\' && i + 1 < s.size()) ++i;
            out += s[i++];
        }
        if (i < s.size()) ++i;
        else ok = false;
        return out;
    }
    double num() {
        ws();
        const char *b = s.c_str() + i;
        char *e = nullptr;
        double v = std::strtod(b, &e);
        if (e == b) ok = false;
        i += (size_t)(e - b);
        return v;
    }
    // {"k": number-or-string, ...}
    bool object(std::map<std::string, std::string> &kv) {
        if (!eat('{')) return false;
        if (eat('}')) return true;
        do {
            std::string k = str();
            if (!eat(':')) return false;
            ws();
            if (i < s.size() && s[i] == '"') kv[k] = str();
            else {
                double v = num();
                char buf[64];
                snprintf(buf, sizeof buf, "%.17g", v);
                kv[k] = buf;
            }
            if (!ok) return false;
        } while (eat(','));
        return eat('}');
    }
};

int geti(const std::map<std::string, std::string> &kv, const char *k) {
    auto it = kv.find(k);
    return it == kv.end() ? 0 : std::atoi(it->second.c_str());
}

std::string esc(const std::string &v) {
    std::string o;
    for (char c : v) {
        if (c == '"' || c == '\\') o += '\\';
        o += c;
    }
    return o;
}

// ---- timing ---------------------------------------------------------------------------------
// Device time of `reps` back-to-back launches after `warm` untimed ones, best of `trials`.
template <class F>
int time_launches(cudaStream_t s, F &&launch, int warm, int reps, int trials, float *ms_per) {
    cudaEvent_t a, b;
    SX_CUDA(cudaEventCreate(&a));
    SX_CUDA(cudaEventCreate(&b));
    int st = SX_OK;
    float best = 1e30f;
    for (int w = 0; w < warm && st == SX_OK; ++w) st = launch();
    for (int t = 0; t < trials && st == SX_OK; ++t) {
        cudaEventRecord(a, s);
        for (int r = 0; r < reps && st == SX_OK; ++r) st = launch();
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "tuner timing");
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms / reps);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms_per = best;
    return st;
}

}  // namespace

// The entry of the nearest tuned log2(n) bucket for (device, op, dtype); on a tie the larger.
bool tune_table_lookup(const sx_target *t, int op, int dtype, size_t n, sx_launch_cfg *cfg) {
    std::lock_guard<std::mutex> g(g_mu);
    if (g_ops.empty()) return false;
    const int b = log2_bucket((double)n);
    auto same = [&](const std::map<OpKey, sx_launch_cfg>::const_iterator &i) {
        return i != g_ops.end() && i->first.dev == t->name && i->first.op == op && i->first.dtype == dtype;
    };
    auto hi = g_ops.lower_bound(OpKey{t->name, op, dtype, b});  // first bucket >= b
    auto lo = hi;
    const bool has_lo = hi != g_ops.begin() && same(--lo);
    const bool has_hi = same(hi);
    if (!has_lo && !has_hi) return false;
    const bool take_hi = has_hi && (!has_lo || hi->first.bucket - b <= b - lo->first.bucket);
    *cfg = take_hi ? hi->second : lo->second;
    return true;
}

bool tune_batch_lookup(const sx_target *t, double mean_item_bytes, sx_batch_cfg *cfg) {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_batch.find(BatchKey{t->name, log2_bucket(mean_item_bytes)});
    if (it == g_batch.end()) return false;
    *cfg = it->second;
    return true;
}

void tune_batch_store(const sx_target *t, double mean_item_bytes, const sx_batch_cfg &cfg) {
    std::lock_guard<std::mutex> g(g_mu);
    g_batch[BatchKey{t->name, log2_bucket(mean_item_bytes)}] = cfg;
}

// ---- launch shapes: the tuner's table or the caller's shape, defaults filled in, then checked ----
sx_launch_cfg resolve_cfg(const sx_target *t, int op, int dtype, size_t n, const sx_launch_cfg *req) {
    sx_launch_cfg c{};
    if (req && req->variant != SX_VARIANT_AUTO) {
        c = *req;
    } else if (!tune_table_lookup(t, op, dtype, n, &c)) {
        c = sx_launch_cfg{};
        c.variant = SX_VARIANT_VECTOR;
    }
    if (c.variant == SX_VARIANT_VECTOR) {
        if (c.threads == 0) c.threads = 256;
        if (c.vec_bytes == 0) c.vec_bytes = 32;
        if (c.unroll == 0) c.unroll = 2;
    } else if (c.variant == SX_VARIANT_BULK || c.variant == SX_VARIANT_TMA || c.variant == SX_VARIANT_TMA_TENSOR) {
        // each family's fastest shape per kernel at n = 2^27 (binary64, measured on B300 over the
        // tuner's candidates): threads, blocks per SM, tile bytes, stages
        static const int kShape[3][4][4] = {
            // copy                scale                 add                  triad
            {{128, 1, 32768, 2}, {512, 1, 32768, 3}, {256, 1, 16384, 3}, {128, 4, 8192, 2}},  // BULK
            {{96, 3, 8192, 3}, {512, 2, 32768, 4}, {512, 2, 8192, 4}, {256, 4, 8192, 3}},     // TMA
            {{96, 1, 32768, 3}, {512, 3, 32768, 4}, {512, 2, 8192, 4}, {256, 4, 8192, 3}}};   // TMA_TENSOR
        const int *d = kShape[c.variant - SX_VARIANT_BULK][(op >= SX_OP_COPY && op <= SX_OP_TRIAD) ? op : SX_OP_TRIAD];
        if (c.threads == 0) c.threads = d[0];
        if (c.blocks_per_sm == 0) c.blocks_per_sm = d[1];
        if (c.tile_bytes == 0) c.tile_bytes = d[2];
        if (c.stages == 0) c.stages = d[3];
    }
    return c;
}

int validate_cfg(const sx_target *t, int op, const sx_launch_cfg &c) {
    if (c.variant == SX_VARIANT_VECTOR) {
        if (c.threads < 32 || c.threads > 1024 || c.threads % 32)
            return fail(SX_ERR_INVALID, "threads=%d: need a multiple of 32 in [32, 1024]", c.threads);
        if (c.vec_bytes != 16 && c.vec_bytes != 32)
            return fail(SX_ERR_INVALID, "vec_bytes=%d: need 16 or 32", c.vec_bytes);
        if (c.unroll != 1 && c.unroll != 2 && c.unroll != 4)
            return fail(SX_ERR_INVALID, "unroll=%d: need 1, 2 or 4", c.unroll);
        if (c.blocks_per_sm < 0 || c.blocks_per_sm > 64)
            return fail(SX_ERR_INVALID, "blocks_per_sm=%d out of [0, 64]", c.blocks_per_sm);
        if (c.cache_hint < 0 || c.cache_hint > 1)
            return fail(SX_ERR_INVALID, "cache_hint=%d: need 0 or 1", c.cache_hint);
        if (c.fp64_mul < 0 || c.fp64_mul > 2)
            return fail(SX_ERR_INVALID, "fp64_mul=%d: need 0, 1 or 2", c.fp64_mul);
        return SX_OK;
    }
    if (c.variant == SX_VARIANT_BULK || c.variant == SX_VARIANT_TMA || c.variant == SX_VARIANT_TMA_TENSOR)
        return validate_bulk_cfg(t, op, c);
    return fail(SX_ERR_INVALID, "variant=%d: need VECTOR (1), BULK (2), TMA (3) or TMA_TENSOR (4)", c.variant);
}

// Candidate shapes: a first pass over the per-thread access pattern (vector width, unroll,
// cache hint) at a fixed block shape, then a pass over the block shape (threads, blocks per
// SM or one tile per block) for the best access pattern, then the BULK and TMA families.
static bool mul64(int op, int dtype) { return dtype == SX_F64 && (op == SX_OP_SCALE || op == SX_OP_TRIAD); }

static std::vector<sx_launch_cfg> vector_pass1(int op, int dtype) {
    std::vector<sx_launch_cfg> v;
    const int nmm = mul64(op, dtype) ? 3 : 1;
    for (int vb : {16, 32})
        for (int u : {1, 2, 4})
            for (int h : {0, 1})
                for (int mm = 0; mm < nmm; ++mm) {
                    sx_launch_cfg c{};
                    c.variant = SX_VARIANT_VECTOR;
                    c.threads = 256;
                    c.blocks_per_sm = 0;
                    c.vec_bytes = vb;
                    c.unroll = u;
                    c.cache_hint = h;
                    c.fp64_mul = mm;
                    v.push_back(c);
                }
    return v;
}

static std::vector<sx_launch_cfg> vector_pass2(const sx_launch_cfg &best) {
    std::vector<sx_launch_cfg> v;
    for (int th : {128, 256, 512, 1024})
        for (int bps : {0, 1, 2, 4, 8, 16}) {
            if (th * bps > 2048) continue;
            sx_launch_cfg c = best;
            c.threads = th;
            c.blocks_per_sm = bps;
            v.push_back(c);
        }
    return v;
}

static std::vector<sx_launch_cfg> bulk_candidates(int op, int dtype) {
    std::vector<sx_launch_cfg> v;
    const int mm = mul64(op, dtype) ? 2 : 0;  // half of the FP64 products on the integer units
    for (int tile : {8192, 16384, 32768})
        for (int st : {2, 3, 4, 6})
            for (int th : {128, 256, 512, 1024})
                for (int bps : {1, 2}) {
                    sx_launch_cfg c{};
                    c.variant = SX_VARIANT_BULK;
                    c.threads = th;
                    c.blocks_per_sm = bps;
                    c.tile_bytes = tile;
                    c.stages = st;
                    c.fp64_mul = mm;
                    v.push_back(c);
                }
    return v;
}

static std::vector<sx_launch_cfg> tma_candidates(int op, int dtype) {
    std::vector<sx_launch_cfg> v;
    const int mm = mul64(op, dtype) ? 2 : 0;
    const std::vector<int> threads = op == SX_OP_COPY ? std::vector<int>{96} : std::vector<int>{128, 256, 512};
    for (int tile : {8192, 16384, 32768})
        for (int st : {3, 4})
            for (int th : threads)
                for (int bps : {1, 2, 4}) {
                    sx_launch_cfg c{};
                    c.variant = SX_VARIANT_TMA;
                    c.threads = th;
                    c.blocks_per_sm = bps;
                    c.tile_bytes = tile;
                    c.stages = st;
                    c.fp64_mul = mm;
                    v.push_back(c);
                }
    return v;
}

}  // namespace sx

using namespace sx;

extern "C" {

int sx_tune(sx_target *t, sx_op op, sx_dtype dtype, size_t n, sx_launch_cfg *best_out, float *gbs) {
    TraceRange tr("sx_tune");
    if (!t) return fail(SX_ERR_INVALID, "target is NULL");
    if (op < SX_OP_COPY || op > SX_OP_TRIAD) return fail(SX_ERR_INVALID, "op %d is not COPY..TRIAD", (int)op);
    if (dtype != SX_F32 && dtype != SX_F64) return fail(SX_ERR_DTYPE, "tuner takes F32 or F64");
    if (n == 0) return fail(SX_ERR_INVALID, "n must be positive");
    DeviceScope ds(t->device);
    sx_array *x = nullptr, *y = nullptr, *o = nullptr;
    int st = sx_alloc(t, dtype, n, &x);
    if (st == SX_OK) st = sx_alloc(t, dtype, n, &y);
    if (st == SX_OK) st = sx_alloc(t, dtype, n, &o);
    if (st == SX_OK) st = sx_seed_uniform(x, 1, -1.0, 1.0);
    if (st == SX_OK) st = sx_seed_uniform(y, 2, -1.0, 1.0);
    const double bytes = (double)op_arrays(op) * (double)n * (double)dtype_size(dtype);
    // enough launches per trial that a trial lasts about 2 ms (capped)
    const double est_ms = std::max(1e-3, bytes / 6.0e9);
    const int reps = (int)std::min(200.0, std::max(3.0, 2.0 / est_ms));
    sx_launch_cfg best{};
    float best_ms = 1e30f;
    auto try_cfg = [&](const sx_launch_cfg &c) {
        if (validate_cfg(t, op, c) != SX_OK) return;
        float ms = 0;
        auto launch = [&]() {
            return launch_stream_op(t, t->stream, op, dtype, x->ptr, y->ptr, o->ptr, n, 3.0, c);
        };
        if (time_launches(t->stream, launch, 2, reps, 3, &ms) != SX_OK) {
            clear_error();
            cudaGetLastError();
            return;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    if (st == SX_OK) {
        for (const auto &c : vector_pass1(op, dtype)) try_cfg(c);
        const sx_launch_cfg b1 = best;
        for (const auto &c : vector_pass2(b1)) try_cfg(c);
        for (const auto &c : bulk_candidates(op, dtype)) try_cfg(c);
        for (const auto &c : tma_candidates(op, dtype)) try_cfg(c);
        clear_error();
        if (best.variant == 0) st = fail(SX_ERR_CUDA, "no candidate launch shape ran");
        else st = check_device_error(t);
    }
    if (x) sx_free(x);
    if (y) sx_free(y);
    if (o) sx_free(o);
    if (st != SX_OK) return st;
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_ops[OpKey{t->name, op, dtype, log2_bucket((double)n)}] = best;
    }
    if (best_out) *best_out = best;
    if (gbs) *gbs = (float)(bytes / (best_ms * 1e-3) / 1e9);
    return SX_OK;
}

int sx_tune_pass(sx_target *t, sx_dtype dtype, size_t n, sx_launch_cfg *best_out, float *gbs) {
    TraceRange tr("sx_tune_pass");
    if (!t) return fail(SX_ERR_INVALID, "target is NULL");
    if (dtype != SX_F32 && dtype != SX_F64) return fail(SX_ERR_DTYPE, "tuner takes F32 or F64");
    if (n == 0) return fail(SX_ERR_INVALID, "n must be positive");
    DeviceScope ds(t->device);
    static const int kOps[4] = {SX_OP_COPY, SX_OP_SCALE, SX_OP_ADD, SX_OP_TRIAD};
    sx_launch_cfg base[4];
    for (int k = 0; k < 4; ++k) {
        base[k] = resolve_cfg(t, kOps[k], dtype, n, nullptr);
        SX_TRY(validate_cfg(t, kOps[k], base[k]));
    }
    sx_array *a = nullptr, *b = nullptr, *c = nullptr;
    int st = sx_alloc(t, dtype, n, &a);
    if (st == SX_OK) st = sx_alloc(t, dtype, n, &b);
    if (st == SX_OK) st = sx_alloc(t, dtype, n, &c);
    const double bytes = 10.0 * (double)n * (double)dtype_size(dtype);
    // passes per trial: about 8 ms of work, 2..50 (values grow 15-fold a pass; 51 FP64 passes
    // stay finite, so the integer-unit products never meet their special-value path)
    const double est_ms = std::max(1e-3, bytes / 6.0e9);
    const int reps = (int)std::min(50.0, std::max(2.0, 8.0 / est_ms));
    auto seed_all = [&]() {
        int r = sx_seed_uniform(a, 1, -1.0, 1.0);
        if (r == SX_OK) r = sx_seed_uniform(b, 2, -1.0, 1.0);
        if (r == SX_OK) r = sx_seed_uniform(c, 3, -1.0, 1.0);
        return r;
    };
    // one pass in Listing 4's order, as sx_stream_iter launches it
    auto pass = [&](const sx_launch_cfg *cf) {
        cudaStream_t s = t->stream;
        SX_TRY(launch_stream_op(t, s, SX_OP_COPY, dtype, a->ptr, nullptr, c->ptr, n, 3.0, cf[0]));
        SX_TRY(launch_stream_op(t, s, SX_OP_SCALE, dtype, c->ptr, nullptr, b->ptr, n, 3.0, cf[1]));
        SX_TRY(launch_stream_op(t, s, SX_OP_ADD, dtype, a->ptr, b->ptr, c->ptr, n, 3.0, cf[2]));
        return launch_stream_op(t, s, SX_OP_TRIAD, dtype, b->ptr, c->ptr, a->ptr, n, 3.0, cf[3]);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == SX_OK && cudaEventCreate(&e0) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "event");
    if (st == SX_OK && cudaEventCreate(&e1) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "event");
    sx_launch_cfg best[4];
    std::copy(base, base + 4, best);
    float best_ms = 1e30f;
    for (int mask = 0; mask < 16 && st == SX_OK; ++mask) {
        sx_launch_cfg cf[4];
        bool dup = false;
        for (int k = 0; k < 4; ++k) {
            cf[k] = base[k];
            const int h = (mask >> k) & 1;
            if (cf[k].variant == SX_VARIANT_VECTOR) cf[k].cache_hint = h;
            else if (h) dup = true;  // the bulk-copy families take no hint: one combination each
        }
        if (dup) continue;
        float ms = 1e30f;
        for (int trial = 0; trial < 3 && st == SX_OK; ++trial) {
            st = seed_all();
            if (st == SX_OK) st = pass(cf);  // warm-up, untimed
            if (st == SX_OK && cudaEventRecord(e0, t->stream) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "event");
            for (int r = 0; r < reps && st == SX_OK; ++r) st = pass(cf);
            if (st == SX_OK && cudaEventRecord(e1, t->stream) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "event");
            if (st == SX_OK && cudaEventSynchronize(e1) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "pass tuner timing");
            float tr_ms = 0;
            if (st == SX_OK) {
                cudaEventElapsedTime(&tr_ms, e0, e1);
                ms = std::min(ms, tr_ms / reps);
            }
        }
        if (st == SX_OK && ms < best_ms) {
            best_ms = ms;
            std::copy(cf, cf + 4, best);
        }
    }
    if (st == SX_OK) st = check_device_error(t);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (a) sx_free(a);
    if (b) sx_free(b);
    if (c) sx_free(c);
    if (st != SX_OK) return st;
    {
        std::lock_guard<std::mutex> g(g_mu);
        for (int k = 0; k < 4; ++k) g_ops[OpKey{t->name, kOps[k], dtype, log2_bucket((double)n)}] = best[k];
    }
    if (best_out) std::copy(best, best + 4, best_out);
    if (gbs) *gbs = (float)(bytes / (best_ms * 1e-3) / 1e9);
    return SX_OK;
}

int sx_tune_lookup(const sx_target *t, sx_op op, sx_dtype dtype, size_t n, sx_launch_cfg *cfg) {
    if (!t || !cfg) return fail(SX_ERR_INVALID, "NULL argument");
    if (!tune_table_lookup(t, op, dtype, n, cfg)) return SX_ERR_NOT_READY;
    return SX_OK;
}

int sx_tune_clear(void) {
    std::lock_guard<std::mutex> g(g_mu);
    g_ops.clear();
    g_batch.clear();
    return SX_OK;
}

int sx_tune_save(const char *path) {
    if (!path) return fail(SX_ERR_INVALID, "path is NULL");
    std::ostringstream os;
    {
        std::lock_guard<std::mutex> g(g_mu);
        os << "{\n  \"ops\": [";
        bool first = true;
        for (const auto &kv : g_ops) {
            const auto &k = kv.first;
            const auto &c = kv.second;
            os << (first ? "\n" : ",\n") << "    {\"device\": \"" << esc(k.dev) << "\", \"op\": " << k.op
               << ", \"dtype\": " << k.dtype << ", \"bucket\": " << k.bucket << ", \"variant\": " << c.variant
               << ", \"threads\": " << c.threads << ", \"blocks_per_sm\": " << c.blocks_per_sm
               << ", \"vec_bytes\": " << c.vec_bytes << ", \"unroll\": " << c.unroll
               << ", \"cache_hint\": " << c.cache_hint << ", \"tile_bytes\": " << c.tile_bytes
               << ", \"stages\": " << c.stages << ", \"fp64_mul\": " << c.fp64_mul << "}";
            first = false;
        }
        os << "\n  ],\n  \"batch\": [";
        first = true;
        for (const auto &kv : g_batch) {
            const auto &c = kv.second;
            os << (first ? "\n" : ",\n") << "    {\"device\": \"" << esc(kv.first.dev)
               << "\", \"bucket\": " << kv.first.bucket << ", \"chunk_bytes\": " << c.chunk_bytes
               << ", \"threads\": " << c.threads << ", \"blocks_per_sm\": " << c.blocks_per_sm
               << ", \"vec_bytes\": " << c.vec_bytes << "}";
            first = false;
        }
        os << "\n  ]\n}\n";
    }
    std::ofstream f(path);
    if (!f) return fail(SX_ERR_INVALID, "cannot write %s", path);
    f << os.str();
    return f.good() ? SX_OK : fail(SX_ERR_INVALID, "write to %s failed", path);
}

int sx_tune_load(const char *path) {
    if (!path) return fail(SX_ERR_INVALID, "path is NULL");
    std::ifstream f(path);
    if (!f) return fail(SX_ERR_INVALID, "cannot read %s", path);
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    JsonReader r(s);
    std::map<OpKey, sx_launch_cfg> ops;
    std::map<BatchKey, sx_batch_cfg> batch;
    if (!r.eat('{')) return fail(SX_ERR_INVALID, "%s: not a tuner table", path);
    do {
        const std::string section = r.str();
        if (!r.eat(':') || !r.eat('[')) return fail(SX_ERR_INVALID, "%s: malformed", path);
        if (!r.eat(']')) {
            do {
                std::map<std::string, std::string> kv;
                if (!r.object(kv)) return fail(SX_ERR_INVALID, "%s: malformed entry", path);
                if (section == "ops") {
                    sx_launch_cfg c{};
                    c.variant = geti(kv, "variant");
                    c.threads = geti(kv, "threads");
                    c.blocks_per_sm = geti(kv, "blocks_per_sm");
                    c.vec_bytes = geti(kv, "vec_bytes");
                    c.unroll = geti(kv, "unroll");
                    c.cache_hint = geti(kv, "cache_hint");
                    c.tile_bytes = geti(kv, "tile_bytes");
                    c.stages = geti(kv, "stages");
                    c.fp64_mul = geti(kv, "fp64_mul");
                    ops[OpKey{kv["device"], geti(kv, "op"), geti(kv, "dtype"), geti(kv, "bucket")}] = c;
                } else if (section == "batch") {
                    sx_batch_cfg c{};
                    c.chunk_bytes = geti(kv, "chunk_bytes");
                    c.threads = geti(kv, "threads");
                    c.blocks_per_sm = geti(kv, "blocks_per_sm");
                    c.vec_bytes = geti(kv, "vec_bytes");
                    batch[BatchKey{kv["device"], geti(kv, "bucket")}] = c;
                }
            } while (r.eat(','));
            if (!r.eat(']')) return fail(SX_ERR_INVALID, "%s: malformed list", path);
        }
    } while (r.eat(','));
    if (!r.eat('}')) return fail(SX_ERR_INVALID, "%s: malformed table", path);
    std::lock_guard<std::mutex> g(g_mu);
    for (auto &kv : ops) g_ops[kv.first] = kv.second;
    for (auto &kv : batch) g_batch[kv.first] = kv.second;
    return SX_OK;
}

}  // extern "C"
