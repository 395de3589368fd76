// A C++17 client of the header-only layer sx.hpp (test program): STREAM written with the
// algorithms of Section 3.4 on vectors placed on a target, checked against the closed form; then
// async_execute with a future and bulk_async_execute over a bulk executor (Listing 2).
//
// a = 1, b = 2, c = 0 (bulk construction on the device), q = 3; five passes issued as algorithm
// calls under par.on(exec), five more through the library's pass loop; then a = 15^10,
// b = 3 * 15^9, c = 4 * 15^9 exactly in binary64.  Exit status: 0 when the check passes, 1 on a
// wrong value or an error, 2 when no device is present.
#include <cstdio>
#include <vector>

#include "sx.hpp"

int main() {
    try {
        if (sx::target::count() < 1) {
            std::fprintf(stderr, "no device\n");
            return 2;
        }
    } catch (const sx::error &e) {
        std::fprintf(stderr, "no device: %s\n", e.what());
        return 2;
    }
    try {
        const size_t n = 1 << 20;
        const double q = 3.0;
        sx::target gpu(0);
        sx::allocator<double> alloc(gpu);
        sx::vector<double> a(n, 1.0, alloc), b(n, 2.0, alloc), c(n, 0.0, alloc);
        sx::executor exec(gpu);
        for (int pass = 0; pass < 5; ++pass) {
            sx::copy(sx::par.on(exec), a, c);                                  // c = a
            sx::transform(sx::par.on(exec), c, b, sx::scale_by{q});           // b = c q
            sx::transform(sx::par.on(exec), a, b, c, sx::plus{});             // c = a + b
            sx::transform(sx::par.on(exec), b, c, a, sx::plus_scaled{q});     // a = b + c q
        }
        sx::stream_passes(exec, a, b, c, q, 5);
        const double want[3] = {576650390625.0, 115330078125.0, 153773437500.0};
        const sx::vector<double> *arr[3] = {&a, &b, &c};
        std::vector<double> host(n);
        for (int k = 0; k < 3; ++k) {
            arr[k]->copy_to_host(host.data());
            for (size_t i = 0; i < n; ++i)
                if (host[i] != want[k]) {
                    std::fprintf(stderr, "array %d element %zu: %.17g, want %.17g\n", k, i, host[i], want[k]);
                    return 1;
                }
        }
        // a failed call throws sx::error with the library's status
        sx::vector<double> shorter(n - 1, alloc);
        try {
            sx::copy(sx::par.on(exec), a, shorter);
            std::fprintf(stderr, "copy between lengths %zu and %zu did not throw\n", n, n - 1);
            return 1;
        } catch (const sx::error &e) {
            if (e.status() != SX_ERR_INVALID) {
                std::fprintf(stderr, "unexpected status %d: %s\n", e.status(), e.what());
                return 1;
            }
        }
        // async_execute with a future, and bulk_async_execute over two items (Listing 2)
        const size_t m = 100003;
        sx::vector<double> x(m, 1.0, alloc), y(m, 2.0, alloc), o1(m, 0.0, alloc), o2(m, 0.0, alloc);
        sx::apply_execute(exec, SX_OP_COPY, y, nullptr, o2);                 // o2 = 2 (no future)
        sx::execute(exec, SX_OP_SCALE, o2, nullptr, o2, q);                  // o2 = 6, done on return
        std::vector<double> h0(m);
        o2.copy_to_host(h0.data());
        for (size_t i = 0; i < m; ++i)
            if (h0[i] != 6.0) {
                std::fprintf(stderr, "apply_execute/execute element %zu: %.17g, want 6\n", i, h0[i]);
                return 1;
            }
        sx::future f = sx::async_execute(exec, SX_OP_TRIAD, x, &y, o1, q);  // o1 = 1 + 2*3
        f.wait();
        if (!f.ready() || f.elapsed_ms() < 0.0f) {
            std::fprintf(stderr, "future not complete after wait\n");
            return 1;
        }
        sx_batch_item items[2] = {};
        items[0].op = SX_OP_TRIAD;
        items[0].dtype = SX_F64;
        items[0].n = m;
        items[0].x = x.data();
        items[0].y = y.data();
        items[0].out = o2.data();
        items[0].q = -0.5;  // o2 = 1 + 2*(-0.5) = 0
        items[1] = items[0];
        items[1].op = SX_OP_ADD;
        items[1].n = m / 2;
        items[1].out = o1.data();  // first half of o1 = 1 + 2 = 3
        // the first item reads x and y and writes o2; the second reads them and writes o1: disjoint
        sx::bulk_executor bulk(gpu, items, 2);
        sx::future fb = bulk.bulk_async_execute();
        fb.wait();
        std::vector<double> h1(m), h2(m);
        o1.copy_to_host(h1.data());
        o2.copy_to_host(h2.data());
        for (size_t i = 0; i < m; ++i) {
            const double w1 = i < m / 2 ? 3.0 : 7.0;
            if (h1[i] != w1 || h2[i] != 0.0) {
                std::fprintf(stderr, "async/bulk element %zu: %.17g %.17g, want %.17g 0\n", i, h1[i], h2[i], w1);
                return 1;
            }
        }
        std::printf("closed form ok through sx.hpp: a = %.0f after 10 passes; async and bulk ok\n", want[0]);
        return 0;
    } catch (const sx::error &e) {
        std::fprintf(stderr, "%s\n", e.what());
        return 1;
    }
}
