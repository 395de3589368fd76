// A C++17 client of the header-only layer sx.hpp (test program): STREAM written with the
// algorithms of Section 3.4 on vectors placed on a target, checked against the closed form.
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
        std::printf("closed form ok through sx.hpp: a = %.0f after 10 passes\n", want[0]);
        return 0;
    } catch (const sx::error &e) {
        std::fprintf(stderr, "%s\n", e.what());
        return 1;
    }
}
