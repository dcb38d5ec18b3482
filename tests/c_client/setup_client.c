/* A plain C client of the library's host-only set-up calls (include/rlsq.h):
 * reads a CSR matrix, runs the row-selecting ILUP set-up (Algorithms 4-6,
 * Sec. 4) through rlsq_setup_*, and prints what it returns as text, floats
 * in C99 hexadecimal so that nothing is rounded on the way.  Used by
 * tests/test_c_abi_client.py; it needs no GPU.
 *
 * usage: setup_client <matrix file> <host threads>
 * matrix file: int64 m, n, nnz; int64 rowptr[m+1]; int32 colidx[nnz]; double vals[nnz]
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "rlsq.h"

static void *read_n(FILE *f, size_t size, size_t count) {
    void *p = malloc(size * (count ? count : 1));
    if (!p || fread(p, size, count, f) != count) {
        fprintf(stderr, "short read\n");
        exit(2);
    }
    return p;
}

static void print_csr(rlsq_setup s, int32_t part, const char *name, int64_t rows, int64_t nnz) {
    int64_t *ptr = malloc(sizeof(int64_t) * (size_t)(rows + 1));
    int32_t *idx = malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    double *val = malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    if (rlsq_setup_factor(s, part, ptr, idx, val) != RLSQ_OK) {
        fprintf(stderr, "rlsq_setup_factor: %s\n", rlsq_last_error());
        exit(3);
    }
    printf("%s", name);
    for (int64_t i = 0; i <= rows; ++i) printf(" %lld", (long long)ptr[i]);
    printf("\n%s.idx", name);
    for (int64_t e = 0; e < nnz; ++e) printf(" %d", idx[e]);
    printf("\n%s.val", name);
    for (int64_t e = 0; e < nnz; ++e) printf(" %a", val[e]);
    printf("\n");
    free(ptr);
    free(idx);
    free(val);
}

int main(int argc, char **argv) {
    if (argc != 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t *hdr = read_n(f, sizeof(int64_t), 3);
    const int64_t m = hdr[0], n = hdr[1], nnz = hdr[2];
    int64_t *rowptr = read_n(f, sizeof(int64_t), (size_t)(m + 1));
    int32_t *colidx = read_n(f, sizeof(int32_t), (size_t)nnz);
    double *vals = read_n(f, sizeof(double), (size_t)nnz);
    fclose(f);

    rlsq_factor_opts o;
    rlsq_factor_opts_default(&o);
    o.mu = 1.0;
    o.host_threads = atoi(argv[2]);

    /* an error first: m <= n is refused with a status and a message */
    rlsq_setup bad = NULL;
    const int code = rlsq_setup_create(n, n, rowptr, colidx, vals, &o, &bad);
    printf("bad_shape %d %d\n", code, rlsq_last_error()[0] != '\0');

    rlsq_setup s = NULL;
    if (rlsq_setup_create(m, n, rowptr, colidx, vals, &o, &s) != RLSQ_OK) {
        fprintf(stderr, "rlsq_setup_create: %s\n", rlsq_last_error());
        return 3;
    }
    printf("threads %d\n", rlsq_setup_threads(o.host_threads, m, n));
    int64_t sizes[8];
    rlsq_setup_sizes(s, sizes);
    printf("sizes");
    for (int k = 0; k < 8; ++k) printf(" %lld", (long long)sizes[k]);
    printf("\n");

    int32_t *prow = malloc(sizeof(int32_t) * (size_t)n);
    int32_t *a2 = malloc(sizeof(int32_t) * (size_t)(m - n));
    double *d = malloc(sizeof(double) * (size_t)n);
    double *ud = malloc(sizeof(double) * (size_t)n);
    rlsq_setup_split(s, prow, a2, d, ud);
    printf("prow");
    for (int64_t k = 0; k < n; ++k) printf(" %d", prow[k]);
    printf("\na2");
    for (int64_t k = 0; k < m - n; ++k) printf(" %d", a2[k]);
    printf("\nd");
    for (int64_t k = 0; k < n; ++k) printf(" %a", d[k]);
    printf("\nudiag");
    for (int64_t k = 0; k < n; ++k) printf(" %a", ud[k]);
    printf("\n");
    print_csr(s, RLSQ_PART_L1, "L1", n, sizes[0]);
    print_csr(s, RLSQ_PART_L2, "L2", m - n, sizes[1]);
    print_csr(s, RLSQ_PART_U, "U", n, sizes[2]);

    /* error statuses of the update and S^{-1} calls (nothing changes on error) */
    int64_t one_ptr[2] = {0, 1};
    int32_t bad_col[1] = {(int32_t)n};
    double one_val[1] = {1.0};
    printf("errors %d %d %d %d\n",
           rlsq_setup_schur_inverse(s, 0, NULL),                 /* ARG: no output */
           rlsq_setup_remove_rows(s, m - n, a2),                 /* SHAPE: no row of A2 would remain */
           rlsq_setup_remove_rows(s, 1, prow),                   /* ARG: a pivot row */
           rlsq_setup_add_rows(s, 1, one_ptr, bad_col, one_val)); /* CSR: column out of range */
    double *sinv = malloc(sizeof(double) * (size_t)((m - n) * (m - n)));
    if (rlsq_setup_schur_inverse(s, 0, sinv) != RLSQ_OK) {
        fprintf(stderr, "rlsq_setup_schur_inverse: %s\n", rlsq_last_error());
        return 3;
    }
    printf("sinv");
    for (int64_t k = 0; k < (m - n) * (m - n); ++k) printf(" %a", sinv[k]);
    printf("\n");
    free(sinv);

    rlsq_setup_destroy(s);
    free(prow);
    free(a2);
    free(d);
    free(ud);
    free(hdr);
    free(rowptr);
    free(colidx);
    free(vals);
    return 0;
}
