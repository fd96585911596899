/* A plain C99 client of the C ABI (include/dte.h): builds, commits and
 * queries types on the host and checks the results against closed forms
 * (§3.2's example layout in small, MPI's vector extent rule), the iov
 * queries of §3.1 and the error codes.  Needs no GPU: commit defers the
 * device upload when no device exists.  Prints "ok" and exits 0 on success;
 * on failure it prints the failing check and exits 1. */
#include <stdio.h>
#include <string.h>

#include "dte.h"

static int failures = 0;

#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            printf("FAILED line %d: %s\n", __LINE__, #cond);          \
            failures++;                                               \
        }                                                             \
    } while (0)

int main(void)
{
    dte_type f64, f32, byte, face, vec, val, cube, bad = NULL;
    int64_t size, lb, ext, tlb, text, n, bytes, got;
    dte_iov iov[4];

    CHECK(dte_type_basic(DTE_FLOAT64, &f64) == DTE_SUCCESS);
    CHECK(dte_type_basic(DTE_FLOAT32, &f32) == DTE_SUCCESS);
    CHECK(dte_type_basic(DTE_BYTE, &byte) == DTE_SUCCESS);
    CHECK(dte_type_basic(DTE_NBASIC, &bad) == DTE_ERR_ARG);

    /* a face normal to the fastest axis of a 16^3 float64 grid: one 16-byte
     * segment per grid row (the YZ-surface rule of §3) */
    {
        int64_t sizes[3] = {16, 16, 16}, sub[3] = {16, 16, 2}, start[3] = {0, 0, 2};
        CHECK(dte_type_subarray(3, sizes, sub, start, DTE_ORDER_C, f64, &face) == DTE_SUCCESS);
    }
    CHECK(dte_type_iov_len(face, -1, &n, &bytes) == DTE_ERR_TYPE); /* not committed yet */
    CHECK(dte_type_commit(&face) == DTE_SUCCESS);
    CHECK(dte_type_size(face, &size) == DTE_SUCCESS && size == 16 * 16 * 2 * 8);
    CHECK(dte_type_get_extent(face, &lb, &ext) == DTE_SUCCESS && lb == 0 && ext == 16 * 16 * 16 * 8);
    CHECK(dte_type_get_true_extent(face, &tlb, &text) == DTE_SUCCESS && tlb == 16 &&
          text == (15 * 256 + 15 * 16 + 3) * 8 - 16 + 8);
    CHECK(dte_type_num_segments(face, &n) == DTE_SUCCESS && n == 256);
    CHECK(dte_type_iov_len(face, -1, &n, &bytes) == DTE_SUCCESS && n == 256 && bytes == size);
    CHECK(dte_type_iov_len(face, 40, &n, &bytes) == DTE_SUCCESS && n == 2 && bytes == 32);
    CHECK(dte_type_iov_len(face, -2, &n, &bytes) == DTE_ERR_ARG);
    CHECK(dte_type_iov(face, 17, iov, 4, &got) == DTE_SUCCESS && got == 4);
    CHECK((int64_t)iov[0].iov_base == 17 * 128 + 16 && iov[0].iov_len == 16);
    CHECK((int64_t)iov[3].iov_base == 20 * 128 + 16 && iov[3].iov_len == 16);
    CHECK(dte_type_iov(face, 255, iov, 4, &got) == DTE_SUCCESS && got == 1);
    CHECK(dte_type_iov(face, 256, iov, 4, &got) == DTE_SUCCESS && got == 0);
    CHECK(dte_pack_size(3, face, &size) == DTE_SUCCESS && size == 3 * 16 * 16 * 2 * 8);

    /* vector(count, bl, stride): size c*bl*s, extent ((c-1)*stride + bl)*ext(old) */
    CHECK(dte_type_vector(1024, 4, 16, f32, &vec) == DTE_SUCCESS);
    CHECK(dte_type_commit(&vec) == DTE_SUCCESS);
    CHECK(dte_type_size(vec, &size) == DTE_SUCCESS && size == 16384);
    CHECK(dte_type_get_extent(vec, &lb, &ext) == DTE_SUCCESS && lb == 0 && ext == (1023 * 16 + 4) * 4);
    CHECK(dte_type_vector(-1, 4, 16, f32, &bad) == DTE_ERR_ARG);

    /* §3.2's layout in small: 16 bytes per value, a 4x4x4 block of a 10^3
     * array starting at (3, 3, 3): one 64-byte segment per row of the block */
    CHECK(dte_type_contiguous(16, byte, &val) == DTE_SUCCESS);
    {
        int64_t sizes[3] = {10, 10, 10}, sub[3] = {4, 4, 4}, start[3] = {3, 3, 3};
        CHECK(dte_type_subarray(3, sizes, sub, start, DTE_ORDER_C, val, &cube) == DTE_SUCCESS);
    }
    CHECK(dte_type_commit(&cube) == DTE_SUCCESS);
    CHECK(dte_type_size(cube, &size) == DTE_SUCCESS && size == 64 * 16);
    CHECK(dte_type_iov_len(cube, 1L << 30, &n, &bytes) == DTE_SUCCESS && n == 16 && bytes == 1024);
    CHECK(dte_type_iov(cube, 0, iov, 2, &got) == DTE_SUCCESS && got == 2);
    CHECK((int64_t)iov[0].iov_base == 16 * ((3 * 10 + 3) * 10 + 3) && iov[0].iov_len == 64);
    CHECK((int64_t)iov[1].iov_base == 16 * ((3 * 10 + 4) * 10 + 3) && iov[1].iov_len == 64);

    /* error strings, freeing */
    CHECK(strlen(dte_error_string(DTE_ERR_OVERLAP)) > 0 && strlen(dte_error_string(12345)) > 0);
    CHECK(dte_type_free(&f64) == DTE_ERR_TYPE); /* predefined */
    CHECK(dte_type_free(&face) == DTE_SUCCESS && face == NULL);
    CHECK(dte_type_free(&vec) == DTE_SUCCESS && dte_type_free(&cube) == DTE_SUCCESS);
    CHECK(dte_type_free(&val) == DTE_SUCCESS);
    CHECK(dte_type_size(face, &size) == DTE_ERR_TYPE);

    if (failures) return 1;
    printf("ok\n");
    return 0;
}
