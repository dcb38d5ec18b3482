/* A plain C client of the library's GPU calls (include/rlsq.h): reads a CSR
 * matrix and a right-hand side, then, through the C ABI alone,
 *   - rlsq_create + rlsq_factor (ILUP(10, 1e-2), mu = 1, CG(2) correction),
 *   - rlsq_solve (preconditioned LSMR to ||A^T r|| / (||A|| ||r||) < 1e-8),
 *   - rlsq_batch_solve of two handles of the same matrix (b and 2 b),
 *   - a server: rlsq_server_create / register / submit / poll / get_stats /
 *     destroy, one request,
 * and prints each x in C99 hexadecimal with its status and iteration count.
 * Used by tests/test_c_abi_client.py (GPU test).
 *
 * usage: solve_client <matrix file>
 * matrix file: int64 m, n, nnz; int64 rowptr[m+1]; int32 colidx[nnz];
 *              double vals[nnz]; double b[m]
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <time.h>

#include "rlsq.h"

static void *read_n(FILE *f, size_t size, size_t count) {
    void *p = malloc(size * (count ? count : 1));
    if (!p || fread(p, size, count, f) != count) {
        fprintf(stderr, "short read\n");
        exit(2);
    }
    return p;
}

static void check(int code, const char *what) {
    if (code != RLSQ_OK) {
        fprintf(stderr, "%s: %d %s\n", what, code, rlsq_last_error());
        exit(3);
    }
}

static void print_x(const char *name, const double *x, int64_t n, const rlsq_info *info) {
    printf("%s %d %d %a", name, info->status, info->iterations, info->ratio);
    for (int64_t j = 0; j < n; ++j) printf(" %a", x[j]);
    printf("\n");
}

int main(int argc, char **argv) {
    if (argc != 2) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t *hdr = read_n(f, sizeof(int64_t), 3);
    const int64_t m = hdr[0], n = hdr[1], nnz = hdr[2];
    int64_t *rowptr = read_n(f, sizeof(int64_t), (size_t)(m + 1));
    int32_t *colidx = read_n(f, sizeof(int32_t), (size_t)nnz);
    double *vals = read_n(f, sizeof(double), (size_t)nnz);
    double *b = read_n(f, sizeof(double), (size_t)m);
    fclose(f);

    rlsq_problem P = NULL;
    check(rlsq_create(m, n, rowptr, colidx, vals, RLSQ_HOST_PTRS, NULL, &P), "rlsq_create");
    rlsq_factor_opts fo;
    rlsq_factor_opts_default(&fo);
    fo.mu = 1.0;
    fo.correction = RLSQ_CORR_CG;
    fo.cg_steps = 2;
    check(rlsq_factor(P, &fo), "rlsq_factor");

    rlsq_solve_opts so;
    rlsq_solve_opts_default(&so);
    double *x = malloc(sizeof(double) * (size_t)n);
    rlsq_info info;
    check(rlsq_solve(P, b, x, &so, &info), "rlsq_solve");
    print_x("solve", x, n, &info);

    /* two handles of the same matrix in one batch (a handle holds its own
       Krylov state, so it may appear once), with b and 2 b */
    rlsq_problem P2 = NULL;
    check(rlsq_create(m, n, rowptr, colidx, vals, RLSQ_HOST_PTRS, NULL, &P2), "rlsq_create");
    check(rlsq_factor(P2, &fo), "rlsq_factor");
    double *b2 = malloc(sizeof(double) * (size_t)m);
    for (int64_t i = 0; i < m; ++i) b2[i] = 2.0 * b[i];
    double *x0 = malloc(sizeof(double) * (size_t)n), *x1 = malloc(sizeof(double) * (size_t)n);
    rlsq_problem hs[2] = {P, P2};
    const double *bs[2] = {b, b2};
    double *xs[2] = {x0, x1};
    rlsq_info infos[2];
    check(rlsq_batch_solve(hs, bs, xs, 2, &so, infos), "rlsq_batch_solve");
    print_x("batch0", x0, n, &infos[0]);
    print_x("batch1", x1, n, &infos[1]);

    /* one request through the continuous-batching server */
    rlsq_server_opts sv = {(int64_t)1 << 30, 4, 1e-8, 2000};
    rlsq_server S = NULL;
    check(rlsq_server_create(&sv, &S), "rlsq_server_create");
    int32_t id = -1;
    check(rlsq_server_register(S, P, &id), "rlsq_server_register");
    int64_t ticket = 0;
    check(rlsq_server_submit(S, id, b, &ticket), "rlsq_server_submit");
    double *xs_srv = malloc(sizeof(double) * (size_t)n);
    rlsq_info sinfo;
    int code = RLSQ_PENDING;
    for (int spin = 0; spin < 60000 && code == RLSQ_PENDING; ++spin) {
        code = rlsq_server_poll(S, ticket, xs_srv, &sinfo);
        if (code == RLSQ_PENDING) {
            struct timespec ts = {0, 1000000}; /* 1 ms */
            nanosleep(&ts, NULL);
        }
    }
    check(code, "rlsq_server_poll");
    print_x("server", xs_srv, n, &sinfo);
    rlsq_server_stats st;
    check(rlsq_server_get_stats(S, &st), "rlsq_server_get_stats");
    printf("stats %lld %lld\n", (long long)st.submitted, (long long)st.completed);
    rlsq_server_destroy(S);

    /* errors reach C: solving an unfactored problem */
    rlsq_problem Q = NULL;
    check(rlsq_create(m, n, rowptr, colidx, vals, RLSQ_HOST_PTRS, NULL, &Q), "rlsq_create");
    printf("unfactored %d\n", rlsq_solve(Q, b, x, &so, NULL));
    rlsq_destroy(Q);
    rlsq_destroy(P2);
    rlsq_destroy(P);
    free(x);
    free(b2);
    free(x0);
    free(x1);
    free(xs_srv);
    free(hdr);
    free(rowptr);
    free(colidx);
    free(vals);
    free(b);
    return 0;
}
