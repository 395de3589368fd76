/*
 * sx.hpp -- header-only C++17 layer over the C ABI (sx.h), in the shape of the paper's programming
 * model: a target (Section 3.1), an allocator that places arrays on a target and constructs them
 * there in bulk (Section 3.2, Listing 1), an executor with async_execute returning a future and a
 * bulk executor with bulk_async_execute (Section 3.3, Listing 2), and copy/transform algorithms
 * taking a parallel policy bound to an executor, par.on(exec) (Section 3.4, Listing 3), enough to
 * write STREAM as Section 5 does.  Every call goes to libsx; failures throw sx::error.  Handles are
 * move-only and released in their destructors.
 */
#ifndef SX_HPP_
#define SX_HPP_

#include <cstddef>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <utility>

#include "sx.h"

namespace sx {

// A failed call: the status code and sx_last_error()'s message.
class error : public std::runtime_error {
  public:
    error(int status, const std::string &what) : std::runtime_error(what), status_(status) {}
    int status() const noexcept { return status_; }

  private:
    int status_;
};

inline void check(int status, const char *call) {
    if (status != SX_OK)
        throw error(status, std::string(call) + ": " + sx_status_string(status) + ": " + sx_last_error());
}

// Element types the library computes in.
template <class T> struct dtype_of;
template <> struct dtype_of<float> { static constexpr sx_dtype value = SX_F32; };
template <> struct dtype_of<double> { static constexpr sx_dtype value = SX_F64; };
template <> struct dtype_of<unsigned char> { static constexpr sx_dtype value = SX_U8; };

// A place to allocate and run: a GPU and a stream (owned, or borrowed from the caller).
class target {
  public:
    explicit target(int device = 0) { check(sx_target_create(device, &t_), "sx_target_create"); }
    target(int device, void *stream, size_t budget_bytes = 0) {
        check(sx_target_create_ext(device, stream, budget_bytes, &t_), "sx_target_create_ext");
    }
    ~target() {
        if (t_) sx_target_destroy(t_);
    }
    target(target &&o) noexcept : t_(std::exchange(o.t_, nullptr)) {}
    target &operator=(target &&o) noexcept {
        std::swap(t_, o.t_);
        return *this;
    }
    target(const target &) = delete;
    target &operator=(const target &) = delete;

    static int count() {
        int n = 0;
        check(sx_target_count(&n), "sx_target_count");
        return n;
    }
    void synchronize() { check(sx_target_synchronize(t_), "sx_target_synchronize"); }
    sx_target *get() const noexcept { return t_; }

  private:
    sx_target *t_ = nullptr;
};

// Allocates arrays of T on its target and constructs or destroys their elements there in bulk.
template <class T>
class allocator {
  public:
    using value_type = T;
    explicit allocator(target &t) noexcept : t_(&t) {}
    target &get_target() const noexcept { return *t_; }  // allocator_traits' target()
    sx_array *allocate(size_t n) const {
        sx_array *a = nullptr;
        check(sx_alloc(t_->get(), dtype_of<T>::value, n, &a), "sx_alloc");
        return a;
    }
    void deallocate(sx_array *a) const noexcept { sx_free(a); }
    void bulk_construct(sx_array *a, T value) const { check(sx_bulk_construct(a, (double)value), "sx_bulk_construct"); }
    void bulk_destroy(sx_array *a) const noexcept { sx_bulk_destroy(a); }

  private:
    target *t_;
};

// n elements of T placed on a target by an allocator; construction runs on the device.
template <class T>
class vector {
  public:
    vector(size_t n, T value, allocator<T> alloc) : alloc_(alloc), a_(alloc.allocate(n)), n_(n) {
        try {
            alloc_.bulk_construct(a_, value);
        } catch (...) {
            alloc_.deallocate(a_);
            throw;
        }
    }
    vector(size_t n, allocator<T> alloc) : vector(n, T(), alloc) {}
    ~vector() {
        if (a_) {
            alloc_.bulk_destroy(a_);
            alloc_.deallocate(a_);
        }
    }
    vector(vector &&o) noexcept : alloc_(o.alloc_), a_(std::exchange(o.a_, nullptr)), n_(o.n_) {}
    vector(const vector &) = delete;
    vector &operator=(const vector &) = delete;

    size_t size() const noexcept { return n_; }
    sx_array *get() const noexcept { return a_; }
    // The elements' device address (for batch items and interoperation).
    T *data() const {
        void *p = nullptr;
        check(sx_array_data(a_, &p, nullptr, nullptr), "sx_array_data");
        return static_cast<T *>(p);
    }
    const allocator<T> &get_allocator() const noexcept { return alloc_; }
    // Seeded uniform values in [lo, hi) (sx_seed_uniform), constructed on the device.
    void seed_uniform(uint64_t seed, double lo = -1.0, double hi = 1.0) {
        check(sx_seed_uniform(a_, seed, lo, hi), "sx_seed_uniform");
    }
    void copy_to_host(T *host) const { check(sx_copy_d2h(host, a_, n_), "sx_copy_d2h"); }
    void copy_from_host(const T *host) { check(sx_copy_h2d(a_, host, n_), "sx_copy_h2d"); }

  private:
    allocator<T> alloc_;
    sx_array *a_;
    size_t n_;
};

// Runs work on a target; SX_PAR returns after the work is done, SX_PAR_TASK once it is enqueued.
class executor {
  public:
    explicit executor(target &t, sx_policy policy = SX_PAR, const sx_launch_cfg *cfg = nullptr) {
        check(sx_executor_create(t.get(), policy, cfg, &e_), "sx_executor_create");
    }
    ~executor() {
        if (e_) sx_executor_destroy(e_);
    }
    executor(executor &&o) noexcept : e_(std::exchange(o.e_, nullptr)) {}
    executor(const executor &) = delete;
    executor &operator=(const executor &) = delete;
    void wait() { check(sx_executor_wait(e_), "sx_executor_wait"); }
    sx_executor *get() const noexcept { return e_; }

  private:
    sx_executor *e_ = nullptr;
};

// The result of asynchronous work (Listing 2's future): wait() blocks until the work is done and
// rethrows its failure; elapsed_ms() is its device time.
class future {
  public:
    future() = default;
    explicit future(sx_future *f) noexcept : f_(f) {}
    ~future() {
        if (f_) sx_future_destroy(f_);
    }
    future(future &&o) noexcept : f_(std::exchange(o.f_, nullptr)) {}
    future &operator=(future &&o) noexcept {
        std::swap(f_, o.f_);
        return *this;
    }
    future(const future &) = delete;
    future &operator=(const future &) = delete;

    bool valid() const noexcept { return f_ != nullptr; }
    void wait() const { check(sx_future_wait(f_, -1), "sx_future_wait"); }
    bool ready() const {
        const int st = sx_future_test(f_);
        if (st == SX_ERR_NOT_READY) return false;
        check(st, "sx_future_test");
        return true;
    }
    float elapsed_ms() const {
        float ms = 0;
        check(sx_future_elapsed_ms(f_, &ms), "sx_future_elapsed_ms");
        return ms;
    }

  private:
    sx_future *f_ = nullptr;
};

// Keeps a parameter out of template argument deduction (so that y may be nullptr).
template <class U>
struct same_type {
    using type = U;
};

// async_execute (Listing 2) of one of the four STREAM operations: returns once the work is
// enqueued on the executor's target, with a future for it (y: the second input of add and
// triad, nullptr otherwise).
template <class T>
future async_execute(executor &e, sx_op op, const vector<T> &x, const typename same_type<vector<T>>::type *y,
                     vector<T> &out, double q = 0.0) {
    sx_future *f = nullptr;
    check(sx_execute_async(e.get(), op, x.get(), y ? y->get() : nullptr, out.get(), q, &f), "sx_execute_async");
    return future(f);
}

// execute (Listing 2): the work has completed when it returns.
template <class T>
void execute(executor &e, sx_op op, const vector<T> &x, const typename same_type<vector<T>>::type *y,
             vector<T> &out, double q = 0.0) {
    async_execute(e, op, x, y, out, q).wait();
}

// apply_execute (Listing 2): enqueued on the executor's target, no future (completion is seen
// through a later future, executor::wait or target::synchronize).
template <class T>
void apply_execute(executor &e, sx_op op, const vector<T> &x, const typename same_type<vector<T>>::type *y,
                   vector<T> &out, double q = 0.0) {
    check(sx_execute_async(e.get(), op, x.get(), y ? y->get() : nullptr, out.get(), q, nullptr), "sx_execute_async");
}

// A bulk executor over a fixed shape of work items (Listing 2's bulk_async_execute): the items
// run in one persistent launch of the batched kernel, captured once into a CUDA graph.
class bulk_executor {
  public:
    bulk_executor(target &t, const sx_batch_item *items, size_t count, const sx_batch_cfg *cfg = nullptr) {
        check(sx_batch_create(t.get(), items, count, cfg, &b_), "sx_batch_create");
    }
    ~bulk_executor() {
        if (b_) sx_batch_destroy(b_);
    }
    bulk_executor(bulk_executor &&o) noexcept : b_(std::exchange(o.b_, nullptr)) {}
    bulk_executor(const bulk_executor &) = delete;
    bulk_executor &operator=(const bulk_executor &) = delete;

    future bulk_async_execute() {
        sx_future *f = nullptr;
        check(sx_batch_launch_async(b_, &f), "sx_batch_launch_async");
        return future(f);
    }
    void bulk_execute() { bulk_async_execute().wait(); }
    sx_batch *get() const noexcept { return b_; }

  private:
    sx_batch *b_ = nullptr;
};

// A parallel policy bound to an executor: par.on(exec).
struct bound_policy {
    executor *exec;
};
struct parallel_policy {
    bound_policy on(executor &e) const noexcept { return bound_policy{&e}; }
};
inline constexpr parallel_policy par{};

// The element operations of STREAM's transforms.
struct scale_by {
    double q;
};
struct plus {};
struct plus_scaled {  // x + y * q
    double q;
};

template <class T>
void copy(bound_policy p, const vector<T> &src, vector<T> &dst) {
    check(sx_copy(p.exec->get(), src.get(), dst.get()), "sx_copy");
}
template <class T>
void transform(bound_policy p, const vector<T> &in, vector<T> &out, scale_by f) {
    check(sx_transform_scale(p.exec->get(), in.get(), out.get(), f.q), "sx_transform_scale");
}
template <class T>
void transform(bound_policy p, const vector<T> &x, const vector<T> &y, vector<T> &out, plus) {
    check(sx_transform_add(p.exec->get(), x.get(), y.get(), out.get()), "sx_transform_add");
}
template <class T>
void transform(bound_policy p, const vector<T> &x, const vector<T> &y, vector<T> &out, plus_scaled f) {
    check(sx_transform_triad(p.exec->get(), x.get(), y.get(), out.get(), f.q), "sx_transform_triad");
}
// Any device callable given as source: out[i] = sx_fn(in[i]) (sx_transform_src).
template <class T>
void transform(bound_policy p, const vector<T> &in, vector<T> &out, const char *callable_source) {
    check(sx_transform_src(p.exec->get(), callable_source, in.get(), out.get()), "sx_transform_src");
}

// `iters` STREAM passes in the library (graph-replayed kernels), the same result as issuing the
// four algorithm calls per pass.
template <class T>
void stream_passes(executor &e, vector<T> &a, vector<T> &b, vector<T> &c, double q, int iters) {
    check(sx_stream_iter(e.get(), a.get(), b.get(), c.get(), q, iters), "sx_stream_iter");
}

}  // namespace sx

#endif  // SX_HPP_
