/* A plain C11 client of libsx (test program): STREAM's closed form through the C ABI alone.
 *
 * a = 1, b = 2, c = 0 (bulk construction on the device, Section 3.2), q = 3, ten passes of
 * Listing 4 (sx_stream_iter), then the arrays are copied back and checked against the exact
 * values a = 15^10, b = 3 * 15^9, c = 4 * 15^9 (exact in binary64).  Before any device call it
 * checks the block partition of Section 4.1 (host arithmetic): the blocks of n elements over
 * 1..8 parts tile [0, n) in order.  Exit status: 0 when the checks pass, 1 on a wrong value or a
 * failed call, 2 when no device is present (the message of the failing call is printed). */
#include <stdio.h>
#include <stdlib.h>

#include "sx.h"

#define N (1u << 20)

static int check(int status, const char *what) {
    if (status != SX_OK) fprintf(stderr, "%s: %s (%s)\n", what, sx_status_string(status), sx_last_error());
    return status;
}

static int check_partition(void) {
    const uint64_t sizes[4] = {0, 7, 1000003, ((uint64_t)1 << 33) + 5};
    for (int i = 0; i < 4; ++i)
        for (int parts = 1; parts <= 8; ++parts) {
            uint64_t at = 0;
            for (int part = 0; part < parts; ++part) {
                uint64_t off = 0, cnt = 0;
                if (check(sx_block_partition(sizes[i], parts, part, &off, &cnt), "sx_block_partition")) return 1;
                if (off != at) {
                    fprintf(stderr, "block %d of %d: offset %llu, want %llu\n", part, parts,
                            (unsigned long long)off, (unsigned long long)at);
                    return 1;
                }
                at += cnt;
            }
            if (at != sizes[i]) return 1;
        }
    return 0;
}

int main(void) {
    if (check_partition()) return 1;
    int count = 0;
    if (sx_target_count(&count) != SX_OK || count < 1) {
        fprintf(stderr, "no device: %s\n", sx_last_error());
        return 2;
    }
    sx_target *t = NULL;
    if (check(sx_target_create(0, &t), "sx_target_create")) return 2;
    sx_array *a = NULL, *b = NULL, *c = NULL;
    sx_executor *e = NULL;
    double *host = malloc(sizeof(double) * N);
    int rc = 1;
    if (!host) goto done;
    if (check(sx_alloc(t, SX_F64, N, &a), "sx_alloc") || check(sx_alloc(t, SX_F64, N, &b), "sx_alloc") ||
        check(sx_alloc(t, SX_F64, N, &c), "sx_alloc"))
        goto done;
    if (check(sx_bulk_construct(a, 1.0), "sx_bulk_construct") || check(sx_bulk_construct(b, 2.0), "sx_bulk_construct") ||
        check(sx_bulk_construct(c, 0.0), "sx_bulk_construct"))
        goto done;
    if (check(sx_executor_create(t, SX_PAR, NULL, &e), "sx_executor_create")) goto done;
    if (check(sx_stream_iter(e, a, b, c, 3.0, 10), "sx_stream_iter")) goto done;
    {
        const double want[3] = {576650390625.0, 115330078125.0, 153773437500.0};
        sx_array *arr[3] = {a, b, c};
        for (int k = 0; k < 3; ++k) {
            if (check(sx_copy_d2h(host, arr[k], N), "sx_copy_d2h")) goto done;
            for (size_t i = 0; i < N; ++i)
                if (host[i] != want[k]) {
                    fprintf(stderr, "array %d element %zu: %.17g, want %.17g\n", k, i, host[i], want[k]);
                    goto done;
                }
        }
    }
    printf("closed form ok: a = %.0f after 10 passes of %u elements\n", 576650390625.0, N);
    rc = 0;
done:
    if (e) sx_executor_destroy(e);
    {
        sx_array *arr[3] = {a, b, c};
        for (int k = 0; k < 3; ++k) {
            if (!arr[k]) continue;
            sx_bulk_destroy(arr[k]);  /* Listing 1: bulk_destroy before the memory goes */
            sx_free(arr[k]);
        }
    }
    sx_target_destroy(t);
    free(host);
    return rc;
}
