/*
 * stream_oracle.c -- plain, serial CPU oracle of the STREAM hot path.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the tests, the package's smoke()
 * check and bench.py's CPU-baseline leg may load this library.  It shares no source, header,
 * table or helper with the CUDA library; the two meet only on the seeded inputs that the
 * tests hand to both.
 *
 * What it computes (Heller et al., "Closing the Performance Gap with Modern C++",
 * Section 5, Listing 4, the generic stream(): one STREAM pass is four parallel-algorithm
 * calls over three equally long arrays a, b, c with scalar q = 3.0, each call finishing over
 * all elements before the next starts):
 *
 *     Copy   c[i] = a[i]                       (copy(e, a, c))
 *     Scale  b[i] = c[i] * q                   (unary transform c -> b)
 *     Add    c[i] = a[i] + b[i]                (binary transform a, b -> c)
 *     Triad  a[i] = b[i] + c[i] * q            (binary transform b, c -> a)
 *
 * Every operation is one IEEE-754 binary64 (or binary32) operation rounded to nearest-even;
 * Triad is two roundings, the product first.  This file must be compiled with
 * -ffp-contract=off and without -ffast-math so that no multiply-add is fused and no
 * flush-to-zero mode is set; it is then the plain definition written out.
 *
 * Array roles follow the paper's listing.  out may equal an input (as std::transform allows):
 * each loop reads element i before writing element i.
 *
 * Pins (the tests under tests/ that do not need a GPU): STREAM's closed form after k passes
 * from a=1, b=2, c=0, q=3; an error bound after 100 passes; hand-derived IEEE rounding cases
 * (ties to even, no fused multiply-add, signed zeros, subnormals, overflow) stored under
 * tests/golden/; agreement with numpy's elementwise ufuncs on seeded inputs; the pass
 * invariant c == 4*a_prev.
 */
#include <stddef.h>
#include <stdint.h>

/* ---- binary64 ------------------------------------------------------------------------ */

/* Section 5, Listing 4, Copy: c = a. */
void oracle_copy_f64(const double *a, double *c, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        c[i] = a[i];
}

/* Section 5, Listing 4, Scale: b = c * q. */
void oracle_scale_f64(const double *c, double *b, size_t n, double q)
{
    for (size_t i = 0; i < n; ++i)
        b[i] = c[i] * q;
}

/* Section 5, Listing 4, Add: c = a + b. */
void oracle_add_f64(const double *a, const double *b, double *c, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        c[i] = a[i] + b[i];
}

/* Section 5, Listing 4, Triad: a = b + c * q (product rounded, then the sum). */
void oracle_triad_f64(const double *b, const double *c, double *a, size_t n, double q)
{
    for (size_t i = 0; i < n; ++i) {
        double t = c[i] * q;
        a[i] = b[i] + t;
    }
}

/* Section 5, Listing 4: `iters` STREAM passes, in the listing's order. */
void oracle_stream_f64(double *a, double *b, double *c, size_t n, double q, int iters)
{
    for (int k = 0; k < iters; ++k) {
        oracle_copy_f64(a, c, n);
        oracle_scale_f64(c, b, n, q);
        oracle_add_f64(a, b, c, n);
        oracle_triad_f64(b, c, a, n, q);
    }
}

/* ---- binary32 ------------------------------------------------------------------------ */

void oracle_copy_f32(const float *a, float *c, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        c[i] = a[i];
}

/* q arrives as a double and is rounded to binary32 once. */
void oracle_scale_f32(const float *c, float *b, size_t n, double q)
{
    const float qf = (float)q;
    for (size_t i = 0; i < n; ++i)
        b[i] = c[i] * qf;
}

void oracle_add_f32(const float *a, const float *b, float *c, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        c[i] = a[i] + b[i];
}

void oracle_triad_f32(const float *b, const float *c, float *a, size_t n, double q)
{
    const float qf = (float)q;
    for (size_t i = 0; i < n; ++i) {
        float t = c[i] * qf;
        a[i] = b[i] + t;
    }
}

void oracle_stream_f32(float *a, float *b, float *c, size_t n, double q, int iters)
{
    for (int k = 0; k < iters; ++k) {
        oracle_copy_f32(a, c, n);
        oracle_scale_f32(c, b, n, q);
        oracle_add_f32(a, b, c, n);
        oracle_triad_f32(b, c, a, n, q);
    }
}

/* ---- generic element transform (Section 3.4, Listing 3: transform over a placed
 *      vector of char with an upper-casing callable) -------------------------------------- */

/* ASCII upper-casing: 'a'..'z' map to 'A'..'Z', every other byte is unchanged. */
void oracle_to_upper_u8(const uint8_t *s, uint8_t *out, size_t n)
{
    for (size_t i = 0; i < n; ++i) {
        uint8_t ch = s[i];
        out[i] = (ch >= 'a' && ch <= 'z') ? (uint8_t)(ch - ('a' - 'A')) : ch;
    }
}
