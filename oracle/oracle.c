/*
 * Reference oracle for the row-splitting ILU preconditioned least-squares
 * method of Scott & Tuma, "Row-Splitting ILU Preconditioners for Sparse
 * Least-Squares Problems" (arXiv 2603.28642).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * FP64 restatement of the method that the GPU library is checked against.
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header or table with the library.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math: every sum
 * is evaluated in the order written, in IEEE double).
 *
 * What is computed, and where it comes from:
 *   orc_factor_create   column scaling (Sec. 5.1: unit 2-norm columns) and the
 *                       column-wise rectangular ILUP(p,tau) of Algorithm 4
 *                       with the pivot choice of Algorithm 5 and the pivot
 *                       modification of Algorithm 6; then the split
 *                       P A D ~ [L1; L2] U of eq. (3.8).
 *   orc_levels          level sets of a triangular matrix (longest path in
 *                       its dependency graph).
 *   orc_correction      the auxiliary system S = I + Y Y^T, Y = L2 L1^{-1}
 *                       (eq. 3.9): identity (S^ = I), k CG steps on the
 *                       implicit S (Sec. 3.2), or the dense S factorised by
 *                       Cholesky (Table 2 variant).
 *   orc_cg_tolerance    the CG steps on S stopped adaptively (Sec. 3.2
 *                       leaves their number open and Table 3 varies it):
 *                       after the step that brings ||r_j|| to at most
 *                       tol ||r_0||, or after k steps.
 *   orc_apply           t = M^{-1} s, with
 *                       M^{-1} = D U^{-1} L1^{-1} K L1^{-T} U^{-T} D,
 *                       K = I - Y^T S^-1 Y: Algorithm 3 (steps 1-4) applied to
 *                       the x-space vector, whose exact-S form is the Woodbury
 *                       identity of Lemma 3.1 (eq. 3.1-3.2).
 *   orc_lsmr            LSMR (Fong & Saunders 2011, the solver cited in
 *                       Sec. 1) run on A R^{-1} with R^T R = M, carried out in
 *                       x-space so only M^{-1} is needed; stops when
 *                       ||A^T r|| / (||A||_2 ||r||) < atol with r = b - A x
 *                       recomputed explicitly, ||A||_2 from the power method
 *                       (Sec. 5.1).
 *   orc_norm2           power method on A^T A.
 *   orc_apply_residual  Algorithm 3 as printed, on a residual r (the paper's
 *                       left preconditioner): r1 = the pivot rows of r in
 *                       pivot order, r2 = the A2 rows; u = r2 - Y r1,
 *                       S^ w = u, y = r1 + Y^T w, L1 v = y, U h = v, and the
 *                       column scaling D back to x-space.
 *   orc_cgls            Algorithm 1 (left preconditioned CGLS) with
 *                       h = orc_apply_residual(r) in place of M^{-1} A^T r.
 *   orc_factor_add_rows / orc_factor_remove_rows
 *                       Sec. 3.4: rows appended to A2 get an L2 row l
 *                       solving U^T l = (a D)^T with L1, U, D and the pivots
 *                       kept; removed A2 rows lose their L2 row.
 *
 * Readings of points the paper leaves open (all also listed in the design
 * notes):
 *   - rc(i) at step j counts the nonzeros of the ORIGINAL scaled matrix in row
 *     i and columns j..n (Algorithm 4, first and last steps).
 *   - Algorithm 5 ties: smallest rc, then largest |L_qj|, then smallest
 *     original row id.  R(j) uses >= .
 *   - Empty column (Algorithm 4, "no nonzero entries"): pivot on the
 *     unpivoted row with the smallest rc (then smallest id) with value
 *     max(beta ||A_:,j||_inf, small).
 *   - Small pivot: |piv| < small -> sign(piv) * max(beta ||A_:,j||_inf, small).
 *     beta = 10^(-2 (1 - j/n)) with 1-based j.  ||A_:,j||_inf is taken on the
 *     scaled original column.
 *   - Dropping (Algorithm 4): tau is absolute; keep |.| >= tau, then at most p
 *     of the largest; ties keep the smaller pivot position (U) or the smaller
 *     original row id (L).  The U drop happens after the L part is computed,
 *     so the L part uses the undropped U values.  Exact zeros are not stored.
 *   - The triangular solve of Algorithm 4 step 6 visits pivot positions in
 *     ascending order (a min-heap here).
 *   - L2 rows are the unpivoted rows in ascending original id.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static void *xmalloc(size_t bytes) {
    void *p = malloc(bytes ? bytes : 1);
    if (!p) abort();
    return p;
}

static void *xcalloc(size_t count, size_t size) {
    void *p = calloc(count ? count : 1, size ? size : 1);
    if (!p) abort();
    return p;
}

/* growable list of (index, value) pairs */
typedef struct {
    int32_t *idx;
    double *val;
    int64_t len, cap;
} pairlist;

static void pl_push(pairlist *l, int32_t i, double v) {
    if (l->len == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 1024;
        l->idx = (int32_t *)realloc(l->idx, (size_t)l->cap * sizeof(int32_t));
        l->val = (double *)realloc(l->val, (size_t)l->cap * sizeof(double));
        if (!l->idx || !l->val) abort();
    }
    l->idx[l->len] = i;
    l->val[l->len] = v;
    l->len++;
}

/* binary min-heap of int32 */
typedef struct {
    int32_t *a;
    int64_t len;
} minheap;

static void heap_push(minheap *h, int32_t v) {
    int64_t i = h->len++;
    h->a[i] = v;
    while (i > 0) {
        int64_t parent = (i - 1) / 2;
        if (h->a[parent] <= h->a[i]) break;
        int32_t t = h->a[parent];
        h->a[parent] = h->a[i];
        h->a[i] = t;
        i = parent;
    }
}

static int32_t heap_pop(minheap *h) {
    int32_t top = h->a[0];
    h->a[0] = h->a[--h->len];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < h->len && h->a[l] < h->a[s]) s = l;
        if (r < h->len && h->a[r] < h->a[s]) s = r;
        if (s == i) break;
        int32_t t = h->a[s];
        h->a[s] = h->a[i];
        h->a[i] = t;
        i = s;
    }
    return top;
}

/* candidate for the "keep the p largest" rule */
typedef struct {
    double mag;
    int32_t key;
    double val;
} cand;

/* larger magnitude first; equal magnitude -> smaller key first */
static int cand_cmp(const void *pa, const void *pb) {
    const cand *a = (const cand *)pa, *b = (const cand *)pb;
    if (a->mag > b->mag) return -1;
    if (a->mag < b->mag) return 1;
    return (a->key < b->key) ? -1 : (a->key > b->key);
}

static int cand_key_cmp(const void *pa, const void *pb) {
    const cand *a = (const cand *)pa, *b = (const cand *)pb;
    return (a->key < b->key) ? -1 : (a->key > b->key);
}

/* Dual dropping of Algorithm 4: drop |v| < tau, then keep at most p of the
 * largest.  Returns the kept count; c[0..kept) ends sorted by key. */
static int64_t drop_keep(cand *c, int64_t len, int p, double tau) {
    int64_t w = 0;
    for (int64_t i = 0; i < len; i++)
        if (c[i].mag >= tau && c[i].val != 0.0) c[w++] = c[i];
    if (p >= 0 && w > p) {
        qsort(c, (size_t)w, sizeof(cand), cand_cmp);
        w = p;
    }
    qsort(c, (size_t)w, sizeof(cand), cand_key_cmp);
    return w;
}

/* ------------------------------------------------------------------ */
/* factor object                                                       */
/* ------------------------------------------------------------------ */

typedef struct orc_factor {
    int64_t m, n;
    double *d;        /* column scaling, length n */
    int32_t *prow;    /* prow[k] = original row pivoted at position k */
    int32_t *pivpos;  /* pivpos[i] = position of row i, or -1 */
    int32_t *a2rows;  /* unpivoted rows, ascending, length m-n */
    int32_t *a2idx;   /* a2idx[i] = index of row i within A2, or -1 */
    int64_t nmod;
    /* L columns: entries (original row, multiplier), column k at
       Lptr[k]..Lptr[k+1], ascending original row */
    int64_t *Lptr;
    int32_t *Lrow;
    double *Lval;
    /* U columns: entries (pivot position k < j, U_kj), ascending k */
    int64_t *Uptr;
    int32_t *Upos;
    double *Uval;
    double *Udiag;
    /* CSR forms used by the apply */
    int64_t *L1p; int32_t *L1i; double *L1v;   /* n x n strictly lower, rows by pivot position */
    int64_t *L1tp; int32_t *L1ti; double *L1tv; /* its transpose (strictly upper) */
    int64_t *L2p; int32_t *L2i; double *L2v;   /* (m-n) x n */
    int64_t *L2tp; int32_t *L2ti; double *L2tv; /* n x (m-n) */
    int64_t *Up; int32_t *Ui; double *Uv;      /* n x n strictly upper */
    int64_t *Utp; int32_t *Uti; double *Utv;   /* its transpose (strictly lower) */
    /* correction */
    int mode;       /* 0 NONE, 1 SI, 2 CG, 3 DENSE */
    int cg_steps;   /* CG: the number of steps, or their maximum when cg_tol > 0 */
    double cg_tol;  /* CG: stop once ||r_j|| <= cg_tol ||r_0|| (0: always cg_steps steps) */
    int cg_last;    /* CG: steps the last S solve took */
    double *G;      /* DENSE: Cholesky factor of S (row-major, lower), (m-n)^2 */
} orc_factor;

/* plain CSR transpose: rows x cols -> cols x rows, entries of each output row
   in ascending column (= input row) order */
static void csr_transpose(int64_t rows, int64_t cols, const int64_t *p, const int32_t *ix,
                          const double *v, int64_t **tp, int32_t **ti, double **tv) {
    int64_t nnz = p[rows];
    int64_t *cp = (int64_t *)xcalloc((size_t)cols + 1, sizeof(int64_t));
    int32_t *ci = (int32_t *)xmalloc((size_t)nnz * sizeof(int32_t));
    double *cv = (double *)xmalloc((size_t)nnz * sizeof(double));
    for (int64_t e = 0; e < nnz; e++) cp[ix[e] + 1]++;
    for (int64_t c = 0; c < cols; c++) cp[c + 1] += cp[c];
    int64_t *fill = (int64_t *)xmalloc((size_t)(cols + 1) * sizeof(int64_t));
    memcpy(fill, cp, (size_t)(cols + 1) * sizeof(int64_t));
    for (int64_t r = 0; r < rows; r++)
        for (int64_t e = p[r]; e < p[r + 1]; e++) {
            int64_t dst = fill[ix[e]]++;
            ci[dst] = (int32_t)r;
            cv[dst] = v[e];
        }
    free(fill);
    *tp = cp;
    *ti = ci;
    *tv = cv;
}

void orc_factor_free(orc_factor *f) {
    if (!f) return;
    free(f->d); free(f->prow); free(f->pivpos); free(f->a2rows); free(f->a2idx);
    free(f->Lptr); free(f->Lrow); free(f->Lval);
    free(f->Uptr); free(f->Upos); free(f->Uval); free(f->Udiag);
    free(f->L1p); free(f->L1i); free(f->L1v); free(f->L1tp); free(f->L1ti); free(f->L1tv);
    free(f->L2p); free(f->L2i); free(f->L2v); free(f->L2tp); free(f->L2ti); free(f->L2tv);
    free(f->Up); free(f->Ui); free(f->Uv); free(f->Utp); free(f->Uti); free(f->Utv);
    free(f->G);
    free(f);
}

/*
 * Column scaling (Sec. 5.1, "prescaled so that the 2-norm of each column ...
 * is equal to 1"): d_j = 1 / sqrt(sum_i a_ij^2), the sum taken in ascending
 * row order.  Returns -1 if a column is empty (the paper removes null
 * columns before solving).
 */
int orc_column_scaling(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                       const double *vals, double *d) {
    double *ss = (double *)xcalloc((size_t)n, sizeof(double));
    for (int64_t i = 0; i < m; i++)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            double a = vals[e];
            ss[colidx[e]] = ss[colidx[e]] + a * a;
        }
    int bad = 0;
    for (int64_t j = 0; j < n; j++) {
        if (!(ss[j] > 0.0)) bad = 1;
        d[j] = 1.0 / sqrt(ss[j]);
    }
    free(ss);
    return bad ? -1 : 0;
}

/*
 * Algorithm 4 (column-wise ILUP(p, tau) with threshold partial pivoting),
 * Algorithm 5 (pivot choice) and Algorithm 6 (pivot modification) on the
 * column-scaled matrix A D.  p < 0 means "no limit".
 * scale == 0 uses D = I.
 */
orc_factor *orc_factor_create(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                              const double *vals, int p, double tau, double mu, double small,
                              int scale) {
    if (!(m > n && n > 0)) return NULL;
    orc_factor *f = (orc_factor *)xcalloc(1, sizeof(orc_factor));
    f->m = m;
    f->n = n;
    f->d = (double *)xmalloc((size_t)n * sizeof(double));
    if (scale) {
        if (orc_column_scaling(m, n, rowptr, colidx, vals, f->d) != 0) {
            orc_factor_free(f);
            return NULL;
        }
    } else {
        for (int64_t j = 0; j < n; j++) f->d[j] = 1.0;
    }

    /* column access to the scaled matrix: CSC, rows ascending per column */
    int64_t nnz = rowptr[m];
    int64_t *cp; int32_t *ci; double *cv;
    csr_transpose(m, n, rowptr, colidx, vals, &cp, &ci, &cv);
    for (int64_t j = 0; j < n; j++) {
        if (cp[j + 1] == cp[j]) { free(cp); free(ci); free(cv); orc_factor_free(f); return NULL; }
        for (int64_t e = cp[j]; e < cp[j + 1]; e++) cv[e] = cv[e] * f->d[j];
    }
    (void)nnz;

    /* Algorithm 4, step 1: row counts of the (scaled) original matrix */
    int64_t *rc = (int64_t *)xcalloc((size_t)m, sizeof(int64_t));
    for (int64_t i = 0; i < m; i++) rc[i] = rowptr[i + 1] - rowptr[i];

    f->pivpos = (int32_t *)xmalloc((size_t)m * sizeof(int32_t));
    for (int64_t i = 0; i < m; i++) f->pivpos[i] = -1;
    f->prow = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
    f->Udiag = (double *)xmalloc((size_t)n * sizeof(double));
    f->Lptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    f->Uptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    pairlist Lcols = {0}, Ucols = {0};

    double *x = (double *)xmalloc((size_t)m * sizeof(double));
    int64_t *stamp = (int64_t *)xmalloc((size_t)m * sizeof(int64_t));
    for (int64_t i = 0; i < m; i++) stamp[i] = -1;
    int32_t *touched = (int32_t *)xmalloc((size_t)m * sizeof(int32_t));
    minheap heap;
    heap.a = (int32_t *)xmalloc((size_t)n * sizeof(int32_t));
    cand *cbuf = (cand *)xmalloc((size_t)(m > n ? m : n) * sizeof(cand));

    for (int64_t j = 0; j < n; j++) {
        int64_t nt = 0;
        heap.len = 0;
        /* x := scaled column j, scattered by original row id */
        double colinf = 0.0;
        for (int64_t e = cp[j]; e < cp[j + 1]; e++) {
            int32_t i = ci[e];
            x[i] = cv[e];
            stamp[i] = j;
            touched[nt++] = i;
            if (f->pivpos[i] >= 0) heap_push(&heap, f->pivpos[i]);
            if (fabs(cv[e]) > colinf) colinf = fabs(cv[e]);
        }
        /* Algorithm 4 steps 6-7: sparse triangular solve with the unit lower
           L(1:j-1,1:j-1) in ascending pivot position, eliminating into the
           not-yet-pivoted rows at the same time. */
        int64_t ucount = 0;
        while (heap.len > 0) {
            int32_t k = heap_pop(&heap);
            double ukj = x[f->prow[k]];
            if (ukj == 0.0) continue;
            cbuf[ucount].mag = fabs(ukj);
            cbuf[ucount].key = k;
            cbuf[ucount].val = ukj;
            ucount++;
            for (int64_t e = f->Lptr[k]; e < f->Lptr[k + 1]; e++) {
                int32_t i = Lcols.idx[e];
                if (stamp[i] != j) {
                    stamp[i] = j;
                    x[i] = 0.0;
                    touched[nt++] = i;
                    if (f->pivpos[i] >= 0) heap_push(&heap, f->pivpos[i]);
                }
                x[i] = x[i] - Lcols.val[e] * ukj;
            }
        }
        /* Algorithm 4 step 8: drop in the U part */
        int64_t ukeep = drop_keep(cbuf, ucount, p, tau);
        for (int64_t t = 0; t < ukeep; t++) pl_push(&Ucols, cbuf[t].key, cbuf[t].val);
        f->Uptr[j + 1] = Ucols.len;

        /* pivot candidates: unpivoted rows with a nonzero */
        double beta = pow(10.0, -2.0 * (1.0 - (double)(j + 1) / (double)n));
        double modval = beta * colinf;
        if (modval < small) modval = small;
        double maxabs = 0.0;
        int64_t ncand = 0;
        for (int64_t t = 0; t < nt; t++) {
            int32_t i = touched[t];
            if (f->pivpos[i] < 0 && x[i] != 0.0) {
                ncand++;
                if (fabs(x[i]) > maxabs) maxabs = fabs(x[i]);
            }
        }
        int32_t r = -1;
        double piv;
        if (ncand == 0) {
            /* empty column: pivot on the unpivoted row with smallest rc */
            for (int64_t i = 0; i < m; i++)
                if (f->pivpos[i] < 0 && (r < 0 || rc[i] < rc[r])) r = (int32_t)i;
            piv = modval;
            f->nmod++;
        } else {
            /* Algorithm 5 */
            double thr = mu * maxabs;
            for (int64_t t = 0; t < nt; t++) {
                int32_t i = touched[t];
                if (f->pivpos[i] >= 0 || x[i] == 0.0) continue;
                if (!(fabs(x[i]) >= thr)) continue;
                if (r < 0 || rc[i] < rc[r] ||
                    (rc[i] == rc[r] && (fabs(x[i]) > fabs(x[r]) ||
                                        (fabs(x[i]) == fabs(x[r]) && i < r))))
                    r = i;
            }
            piv = x[r];
            if (fabs(piv) < small) {
                /* Algorithm 6 */
                piv = (piv < 0.0) ? -modval : modval;
                f->nmod++;
            }
        }
        f->Udiag[j] = piv;
        f->pivpos[r] = (int32_t)j;
        f->prow[j] = r;

        /* Algorithm 4: scale the L part by the pivot, then drop */
        int64_t lcount = 0;
        for (int64_t t = 0; t < nt; t++) {
            int32_t i = touched[t];
            if (f->pivpos[i] >= 0 || x[i] == 0.0) continue;
            double l = x[i] / piv;
            cbuf[lcount].mag = fabs(l);
            cbuf[lcount].key = i;
            cbuf[lcount].val = l;
            lcount++;
        }
        int64_t lkeep = drop_keep(cbuf, lcount, p, tau);
        for (int64_t t = 0; t < lkeep; t++) pl_push(&Lcols, cbuf[t].key, cbuf[t].val);
        f->Lptr[j + 1] = Lcols.len;

        /* Algorithm 4 last step: row counts now cover columns j+1..n */
        for (int64_t e = cp[j]; e < cp[j + 1]; e++) rc[ci[e]]--;
    }
    f->Lrow = Lcols.idx;
    f->Lval = Lcols.val;
    f->Upos = Ucols.idx;
    f->Uval = Ucols.val;
    free(x); free(stamp); free(touched); free(heap.a); free(cbuf); free(rc);
    free(cp); free(ci); free(cv);

    /* split (eq. 3.8): L1 = pivoted rows in pivot order, L2 = the rest in
       ascending original id */
    int64_t m2 = m - n;
    f->a2rows = (int32_t *)xmalloc((size_t)(m2 > 0 ? m2 : 1) * sizeof(int32_t));
    f->a2idx = (int32_t *)xmalloc((size_t)m * sizeof(int32_t));
    {
        int64_t c = 0;
        for (int64_t i = 0; i < m; i++) {
            if (f->pivpos[i] < 0) { f->a2idx[i] = (int32_t)c; f->a2rows[c++] = (int32_t)i; }
            else f->a2idx[i] = -1;
        }
    }
    /* CSR of L1 (rows = pivot positions) and L2, built column by column so
       each row's column indices ascend */
    f->L1p = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    f->L2p = (int64_t *)xcalloc((size_t)m2 + 1, sizeof(int64_t));
    int64_t nL = f->Lptr[n];
    for (int64_t e = 0; e < nL; e++) {
        int32_t i = f->Lrow[e];
        if (f->pivpos[i] >= 0) f->L1p[f->pivpos[i] + 1]++;
        else f->L2p[f->a2idx[i] + 1]++;
    }
    for (int64_t k = 0; k < n; k++) f->L1p[k + 1] += f->L1p[k];
    for (int64_t k = 0; k < m2; k++) f->L2p[k + 1] += f->L2p[k];
    f->L1i = (int32_t *)xmalloc((size_t)f->L1p[n] * sizeof(int32_t) + 4);
    f->L1v = (double *)xmalloc((size_t)f->L1p[n] * sizeof(double) + 8);
    f->L2i = (int32_t *)xmalloc((size_t)f->L2p[m2] * sizeof(int32_t) + 4);
    f->L2v = (double *)xmalloc((size_t)f->L2p[m2] * sizeof(double) + 8);
    {
        int64_t *f1 = (int64_t *)xmalloc((size_t)(n + 1) * sizeof(int64_t));
        int64_t *f2 = (int64_t *)xmalloc((size_t)(m2 + 1) * sizeof(int64_t));
        memcpy(f1, f->L1p, (size_t)(n + 1) * sizeof(int64_t));
        memcpy(f2, f->L2p, (size_t)(m2 + 1) * sizeof(int64_t));
        for (int64_t k = 0; k < n; k++)
            for (int64_t e = f->Lptr[k]; e < f->Lptr[k + 1]; e++) {
                int32_t i = f->Lrow[e];
                if (f->pivpos[i] >= 0) {
                    int64_t dst = f1[f->pivpos[i]]++;
                    f->L1i[dst] = (int32_t)k;
                    f->L1v[dst] = f->Lval[e];
                } else {
                    int64_t dst = f2[f->a2idx[i]]++;
                    f->L2i[dst] = (int32_t)k;
                    f->L2v[dst] = f->Lval[e];
                }
            }
        free(f1);
        free(f2);
    }
    /* CSR of U (strictly upper): entry (k, j) from column j */
    f->Up = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    int64_t nU = f->Uptr[n];
    for (int64_t e = 0; e < nU; e++) f->Up[f->Upos[e] + 1]++;
    for (int64_t k = 0; k < n; k++) f->Up[k + 1] += f->Up[k];
    f->Ui = (int32_t *)xmalloc((size_t)nU * sizeof(int32_t) + 4);
    f->Uv = (double *)xmalloc((size_t)nU * sizeof(double) + 8);
    {
        int64_t *fu = (int64_t *)xmalloc((size_t)(n + 1) * sizeof(int64_t));
        memcpy(fu, f->Up, (size_t)(n + 1) * sizeof(int64_t));
        for (int64_t j = 0; j < n; j++)
            for (int64_t e = f->Uptr[j]; e < f->Uptr[j + 1]; e++) {
                int64_t dst = fu[f->Upos[e]]++;
                f->Ui[dst] = (int32_t)j;
                f->Uv[dst] = f->Uval[e];
            }
        free(fu);
    }
    csr_transpose(n, n, f->L1p, f->L1i, f->L1v, &f->L1tp, &f->L1ti, &f->L1tv);
    csr_transpose(m2, n, f->L2p, f->L2i, f->L2v, &f->L2tp, &f->L2ti, &f->L2tv);
    csr_transpose(n, n, f->Up, f->Ui, f->Uv, &f->Utp, &f->Uti, &f->Utv);
    f->mode = 0;
    return f;
}

/* sizes: [nnz(L1 strict), nnz(L2), nnz(U strict), nmod] */
void orc_factor_sizes(const orc_factor *f, int64_t *out) {
    out[0] = f->L1p[f->n];
    out[1] = f->L2p[f->m - f->n];
    out[2] = f->Up[f->n];
    out[3] = f->nmod;
}

void orc_factor_perm(const orc_factor *f, int32_t *prow, int32_t *a2rows) {
    memcpy(prow, f->prow, (size_t)f->n * sizeof(int32_t));
    if (f->m - f->n > 0) memcpy(a2rows, f->a2rows, (size_t)(f->m - f->n) * sizeof(int32_t));
}

void orc_factor_scaling(const orc_factor *f, double *d) {
    memcpy(d, f->d, (size_t)f->n * sizeof(double));
}

static void copy_csr(int64_t rows, const int64_t *p, const int32_t *i, const double *v,
                     int64_t *po, int32_t *io, double *vo) {
    memcpy(po, p, (size_t)(rows + 1) * sizeof(int64_t));
    memcpy(io, i, (size_t)p[rows] * sizeof(int32_t));
    memcpy(vo, v, (size_t)p[rows] * sizeof(double));
}

void orc_factor_L1(const orc_factor *f, int64_t *p, int32_t *i, double *v) {
    copy_csr(f->n, f->L1p, f->L1i, f->L1v, p, i, v);
}
void orc_factor_L2(const orc_factor *f, int64_t *p, int32_t *i, double *v) {
    copy_csr(f->m - f->n, f->L2p, f->L2i, f->L2v, p, i, v);
}
void orc_factor_U(const orc_factor *f, int64_t *p, int32_t *i, double *v, double *diag) {
    copy_csr(f->n, f->Up, f->Ui, f->Uv, p, i, v);
    memcpy(diag, f->Udiag, (size_t)f->n * sizeof(double));
}

/*
 * Level sets of a triangular matrix given by the CSR of its strictly
 * triangular part.  lower != 0: row i depends on columns k < i,
 * lev(i) = 1 + max lev(k) (0 if none), evaluated for i ascending.
 * lower == 0: mirror image, row i depends on k > i, i descending.
 * Returns the number of levels.
 */
int64_t orc_levels(int64_t n, const int64_t *p, const int32_t *idx, int lower, int32_t *lev) {
    int64_t nlev = 0;
    for (int64_t t = 0; t < n; t++) {
        int64_t i = lower ? t : n - 1 - t;
        int32_t L = 0;
        for (int64_t e = p[i]; e < p[i + 1]; e++) {
            int32_t k = idx[e];
            if (lev[k] + 1 > L) L = lev[k] + 1;
        }
        lev[i] = L;
        if (L + 1 > nlev) nlev = L + 1;
    }
    return nlev;
}

/* ------------------------------------------------------------------ */
/* triangular solves and products (textbook row forms)                 */
/* ------------------------------------------------------------------ */

/* lower triangular, strictly-lower CSR T plus diagonal (NULL = unit):
   x_i = (b_i - sum_{k<i} T_ik x_k) / T_ii, i ascending */
static void solve_lower(int64_t n, const int64_t *p, const int32_t *idx, const double *v,
                        const double *diag, const double *b, double *x) {
    for (int64_t i = 0; i < n; i++) {
        double s = b[i];
        for (int64_t e = p[i]; e < p[i + 1]; e++) s = s - v[e] * x[idx[e]];
        x[i] = diag ? s / diag[i] : s;
    }
}

/* upper triangular, strictly-upper CSR T plus diagonal (NULL = unit):
   x_i = (b_i - sum_{k>i} T_ik x_k) / T_ii, i descending */
static void solve_upper(int64_t n, const int64_t *p, const int32_t *idx, const double *v,
                        const double *diag, const double *b, double *x) {
    for (int64_t i = n - 1; i >= 0; i--) {
        double s = b[i];
        for (int64_t e = p[i]; e < p[i + 1]; e++) s = s - v[e] * x[idx[e]];
        x[i] = diag ? s / diag[i] : s;
    }
}

/* y = T x for a CSR matrix */
static void csr_mv(int64_t rows, const int64_t *p, const int32_t *idx, const double *v,
                   const double *x, double *y) {
    for (int64_t i = 0; i < rows; i++) {
        double s = 0.0;
        for (int64_t e = p[i]; e < p[i + 1]; e++) s = s + v[e] * x[idx[e]];
        y[i] = s;
    }
}

/* y = T^T x for a CSR matrix (rows x cols), y has length cols; contributions
   to each y_j are added in ascending row order */
static void csr_mtv(int64_t rows, int64_t cols, const int64_t *p, const int32_t *idx,
                    const double *v, const double *x, double *y) {
    for (int64_t j = 0; j < cols; j++) y[j] = 0.0;
    for (int64_t i = 0; i < rows; i++)
        for (int64_t e = p[i]; e < p[i + 1]; e++) y[idx[e]] = y[idx[e]] + v[e] * x[i];
}

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s = s + a[i] * b[i];
    return s;
}

/* v -> S v with S = I + L2 L1^{-1} L1^{-T} L2^T (implicit, Sec. 3.2) */
static void s_matvec(const orc_factor *f, const double *v, double *out, double *wn1, double *wn2) {
    int64_t n = f->n, m2 = f->m - f->n;
    csr_mv(n, f->L2tp, f->L2ti, f->L2tv, v, wn1);                 /* L2^T v */
    solve_upper(n, f->L1tp, f->L1ti, f->L1tv, NULL, wn1, wn2);    /* L1^{-T} */
    solve_lower(n, f->L1p, f->L1i, f->L1v, NULL, wn2, wn1);       /* L1^{-1} */
    csr_mv(m2, f->L2p, f->L2i, f->L2v, wn1, out);                  /* L2 */
    for (int64_t i = 0; i < m2; i++) out[i] = v[i] + out[i];
}

/*
 * Correction set-up (Algorithm 3 step 2 variants, Sec. 3.2):
 * mode 0 NONE  -> K = I (the A1-only preconditioner, no correction),
 * mode 1 SI    -> S^ = I,
 * mode 2 CG    -> cg_steps CG iterations from zero on the implicit S,
 * mode 3 DENSE -> S = I + Z^T Z, Z = L1^{-T} L2^T, assembled densely and
 *                 factorised S = G G^T (Cholesky).
 * Returns 0, or -1 if DENSE meets a non-positive pivot.
 */
int orc_correction(orc_factor *f, int mode, int cg_steps) {
    f->mode = mode;
    f->cg_steps = cg_steps;
    free(f->G);
    f->G = NULL;
    if (mode != 3) return 0;
    int64_t n = f->n, m2 = f->m - f->n;
    double *Z = (double *)xcalloc((size_t)(n * m2), sizeof(double)); /* column c at Z[c*n] */
    double *rhs = (double *)xcalloc((size_t)n, sizeof(double));
    for (int64_t c = 0; c < m2; c++) {
        for (int64_t i = 0; i < n; i++) rhs[i] = 0.0;
        for (int64_t e = f->L2p[c]; e < f->L2p[c + 1]; e++) rhs[f->L2i[e]] = f->L2v[e];
        solve_upper(n, f->L1tp, f->L1ti, f->L1tv, NULL, rhs, Z + c * n);
    }
    double *G = (double *)xcalloc((size_t)(m2 * m2), sizeof(double));
    for (int64_t a = 0; a < m2; a++)
        for (int64_t b = 0; b <= a; b++) {
            double s = dot(n, Z + a * n, Z + b * n);
            if (a == b) s = 1.0 + s;
            G[a * m2 + b] = s;
        }
    free(Z);
    free(rhs);
    /* in-place Cholesky of the lower triangle, textbook column order */
    for (int64_t j = 0; j < m2; j++) {
        double s = G[j * m2 + j];
        for (int64_t k = 0; k < j; k++) s = s - G[j * m2 + k] * G[j * m2 + k];
        if (!(s > 0.0)) { free(G); return -1; }
        double gjj = sqrt(s);
        G[j * m2 + j] = gjj;
        for (int64_t i = j + 1; i < m2; i++) {
            double t = G[i * m2 + j];
            for (int64_t k = 0; k < j; k++) t = t - G[i * m2 + k] * G[j * m2 + k];
            G[i * m2 + j] = t / gjj;
        }
    }
    for (int64_t a = 0; a < m2; a++)
        for (int64_t b = a + 1; b < m2; b++) G[a * m2 + b] = 0.0;
    f->G = G;
    return 0;
}

/* Adaptive CG steps on S (mode 2): stop after the step that makes
 * ||r_j||^2 <= tol^2 ||r_0||^2, at most cg_steps steps; tol = 0 restores the
 * fixed count. */
void orc_cg_tolerance(orc_factor *f, double tol) { f->cg_tol = tol; }
int orc_cg_last_steps(const orc_factor *f) { return f->cg_last; }

/* Export the dense Cholesky factor (row-major lower, (m-n)^2); 0 if none. */
int orc_correction_dense(const orc_factor *f, double *out) {
    if (!f->G) return 0;
    int64_t m2 = f->m - f->n;
    memcpy(out, f->G, (size_t)(m2 * m2) * sizeof(double));
    return 1;
}

/* w = S^ ^{-1} e per the correction mode (e, w of length m - n) */
static void s_solve(const orc_factor *f, const double *e, double *w) {
    int64_t n = f->n, m2 = f->m - f->n;
    if (f->mode == 1) {
        for (int64_t i = 0; i < m2; i++) w[i] = e[i];
        return;
    }
    if (f->mode == 3) {
        double *y = (double *)xmalloc((size_t)m2 * sizeof(double));
        for (int64_t i = 0; i < m2; i++) {
            double s = e[i];
            for (int64_t k = 0; k < i; k++) s = s - f->G[i * m2 + k] * y[k];
            y[i] = s / f->G[i * m2 + i];
        }
        for (int64_t i = m2 - 1; i >= 0; i--) {
            double s = y[i];
            for (int64_t k = i + 1; k < m2; k++) s = s - f->G[k * m2 + i] * w[k];
            w[i] = s / f->G[i * m2 + i];
        }
        free(y);
        return;
    }
    /* mode 2: conjugate gradients from w = 0: cg_steps steps, or fewer when
     * cg_tol > 0 and the residual has dropped to cg_tol times its start */
    double *r = (double *)xmalloc((size_t)m2 * sizeof(double));
    double *pv = (double *)xmalloc((size_t)m2 * sizeof(double));
    double *sp = (double *)xmalloc((size_t)m2 * sizeof(double));
    double *wn1 = (double *)xmalloc((size_t)n * sizeof(double));
    double *wn2 = (double *)xmalloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < m2; i++) { w[i] = 0.0; r[i] = e[i]; pv[i] = e[i]; }
    double rr = dot(m2, r, r);
    const double rr0 = rr;
    int steps = 0;
    for (int it = 0; it < f->cg_steps; it++) {
        if (rr == 0.0) break;
        s_matvec(f, pv, sp, wn1, wn2);
        double psp = dot(m2, pv, sp);
        double a = rr / psp;
        for (int64_t i = 0; i < m2; i++) {
            w[i] = w[i] + a * pv[i];
            r[i] = r[i] - a * sp[i];
        }
        steps = it + 1;
        double rrn = dot(m2, r, r);
        if (f->cg_tol > 0.0 && rrn <= f->cg_tol * f->cg_tol * rr0) break;
        double bcg = rrn / rr;
        for (int64_t i = 0; i < m2; i++) pv[i] = r[i] + bcg * pv[i];
        rr = rrn;
    }
    ((orc_factor *)f)->cg_last = steps; /* a record for the tests, not part of the arithmetic */
    free(r); free(pv); free(sp); free(wn1); free(wn2);
}

/*
 * t = M^{-1} s, M^{-1} = D U^{-1} L1^{-1} K L1^{-T} U^{-T} D with
 * K g = g - L1^{-T} L2^T S^-1 L2 L1^{-1} g (Algorithm 3 steps 1-4 with the
 * implicit Y of Sec. 3.2; mode 0 skips the correction).
 */
void orc_apply(const orc_factor *f, const double *s, double *t) {
    int64_t n = f->n, m2 = f->m - f->n;
    double *a = (double *)xmalloc((size_t)n * sizeof(double));
    double *g1 = (double *)xmalloc((size_t)n * sizeof(double));
    double *g2 = (double *)xmalloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; i++) a[i] = f->d[i] * s[i];
    solve_lower(n, f->Utp, f->Uti, f->Utv, f->Udiag, a, g1);   /* U^{-T} */
    solve_upper(n, f->L1tp, f->L1ti, f->L1tv, NULL, g1, g2);   /* L1^{-T} */
    if (f->mode != 0 && m2 > 0) {
        double *q1 = (double *)xmalloc((size_t)n * sizeof(double));
        double *ev = (double *)xmalloc((size_t)m2 * sizeof(double));
        double *wv = (double *)xmalloc((size_t)m2 * sizeof(double));
        double *fv = (double *)xmalloc((size_t)n * sizeof(double));
        double *yv = (double *)xmalloc((size_t)n * sizeof(double));
        solve_lower(n, f->L1p, f->L1i, f->L1v, NULL, g2, q1);    /* Algorithm 3 step 1: */
        csr_mv(m2, f->L2p, f->L2i, f->L2v, q1, ev);              /*   e = Y g2          */
        s_solve(f, ev, wv);                                      /* step 2              */
        csr_mv(n, f->L2tp, f->L2ti, f->L2tv, wv, fv);            /* step 3: Y^T w       */
        solve_upper(n, f->L1tp, f->L1ti, f->L1tv, NULL, fv, yv);
        for (int64_t i = 0; i < n; i++) g2[i] = g2[i] - yv[i];
        free(q1); free(ev); free(wv); free(fv); free(yv);
    }
    solve_lower(n, f->L1p, f->L1i, f->L1v, NULL, g2, g1);      /* step 4: L1^{-1} */
    solve_upper(n, f->Up, f->Ui, f->Uv, f->Udiag, g1, a);      /*         U^{-1}  */
    for (int64_t i = 0; i < n; i++) t[i] = f->d[i] * a[i];
    free(a); free(g1); free(g2);
}

/* the individual solves, exported for adjointness and per-step checks */
void orc_solve_L1(const orc_factor *f, const double *b, double *x) {
    solve_lower(f->n, f->L1p, f->L1i, f->L1v, NULL, b, x);
}
void orc_solve_L1t(const orc_factor *f, const double *b, double *x) {
    solve_upper(f->n, f->L1tp, f->L1ti, f->L1tv, NULL, b, x);
}
void orc_solve_U(const orc_factor *f, const double *b, double *x) {
    solve_upper(f->n, f->Up, f->Ui, f->Uv, f->Udiag, b, x);
}
void orc_solve_Ut(const orc_factor *f, const double *b, double *x) {
    solve_lower(f->n, f->Utp, f->Uti, f->Utv, f->Udiag, b, x);
}
void orc_s_solve(const orc_factor *f, const double *e, double *w) { s_solve(f, e, w); }

/* ------------------------------------------------------------------ */
/* norms and LSMR                                                      */
/* ------------------------------------------------------------------ */

void orc_spmv(int64_t m, const int64_t *rowptr, const int32_t *colidx, const double *vals,
              const double *x, double *y) {
    csr_mv(m, rowptr, colidx, vals, x, y);
}

void orc_spmv_t(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                const double *vals, const double *x, double *y) {
    csr_mtv(m, n, rowptr, colidx, vals, x, y);
}

/* ||A||_2 by the power method on A^T A from v = 1/sqrt(n): iters steps of
   w = A^T A v, lambda = ||w||, v = w / lambda; returns sqrt(lambda). */
double orc_norm2(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                 const double *vals, int iters) {
    double *v = (double *)xmalloc((size_t)n * sizeof(double));
    double *y = (double *)xmalloc((size_t)m * sizeof(double));
    double *w = (double *)xmalloc((size_t)n * sizeof(double));
    double v0 = 1.0 / sqrt((double)n);
    for (int64_t j = 0; j < n; j++) v[j] = v0;
    double lambda = 0.0;
    for (int it = 0; it < iters; it++) {
        csr_mv(m, rowptr, colidx, vals, v, y);
        csr_mtv(m, n, rowptr, colidx, vals, y, w);
        lambda = sqrt(dot(n, w, w));
        if (lambda == 0.0) break;
        for (int64_t j = 0; j < n; j++) v[j] = w[j] / lambda;
    }
    free(v); free(y); free(w);
    return sqrt(lambda);
}

/*
 * Preconditioned LSMR in x-space.  With R^T R = M, LSMR on B = A R^{-1}
 * needs only t = M^{-1} s: with v^ = R^{-1} v and w = R^T v the Golub-Kahan
 * step alpha v = B^T u - beta v becomes s = A^T u - beta w, t = M^{-1} s,
 * alpha = sqrt(<t, s>), v^ = t / alpha, w = s / alpha, and every x-space
 * update of LSMR uses v^ in place of v.
 *
 * f == NULL runs unpreconditioned LSMR (M = I).
 * Stopping: for k = 0, 1, ...: r_k = b - A x_k and A^T r_k are recomputed
 * from scratch; stop when ||A^T r_k|| / (anorm ||r_k||) < atol (or r_k = 0),
 * or when k = maxit.
 * Returns 0 converged, 1 iteration limit, -2 breakdown (<t, s> <= 0 or not
 * finite).  ratio_hist (optional, length maxit + 1) receives ratio_k.
 */
int orc_lsmr(const orc_factor *f, int64_t m, int64_t n, const int64_t *rowptr,
             const int32_t *colidx, const double *vals, const double *b, double anorm,
             double atol, int maxit, double *x, int *its_out, double *ratio_hist,
             double *final_ratio) {
    double *u = (double *)xmalloc((size_t)m * sizeof(double));
    double *r = (double *)xmalloc((size_t)m * sizeof(double));
    double *ax = (double *)xmalloc((size_t)m * sizeof(double));
    double *s = (double *)xmalloc((size_t)n * sizeof(double));
    double *t = (double *)xmalloc((size_t)n * sizeof(double));
    double *vh = (double *)xmalloc((size_t)n * sizeof(double));
    double *w = (double *)xmalloc((size_t)n * sizeof(double));
    double *h = (double *)xmalloc((size_t)n * sizeof(double));
    double *hb = (double *)xmalloc((size_t)n * sizeof(double));
    double *z = (double *)xmalloc((size_t)n * sizeof(double));
    int status = 1, k = 0;
    double ratio = 0.0;

    for (int64_t j = 0; j < n; j++) { x[j] = 0.0; hb[j] = 0.0; }

    /* Golub-Kahan start: beta_1 u_1 = b, alpha_1 v_1 = B^T u_1 */
    double beta = sqrt(dot(m, b, b));
    double alpha = 0.0;
    if (beta > 0.0)
        for (int64_t i = 0; i < m; i++) u[i] = b[i] / beta;
    else
        for (int64_t i = 0; i < m; i++) u[i] = 0.0;
    csr_mtv(m, n, rowptr, colidx, vals, u, s);
    if (f) orc_apply(f, s, t); else memcpy(t, s, (size_t)n * sizeof(double));
    double a2 = dot(n, t, s);
    if (!(a2 >= 0.0) || !isfinite(a2)) { status = -2; goto done; }
    alpha = sqrt(a2);
    for (int64_t j = 0; j < n; j++) {
        vh[j] = alpha > 0.0 ? t[j] / alpha : 0.0;
        w[j] = alpha > 0.0 ? s[j] / alpha : 0.0;
        h[j] = vh[j];
    }
    double alphabar = alpha, zetabar = alpha * beta;
    double rho = 1.0, rhobar = 1.0, cbar = 1.0, sbar = 0.0;

    for (k = 0;; k++) {
        /* explicit stopping quantities for x_k */
        csr_mv(m, rowptr, colidx, vals, x, ax);
        for (int64_t i = 0; i < m; i++) r[i] = b[i] - ax[i];
        csr_mtv(m, n, rowptr, colidx, vals, r, z);
        double rn = sqrt(dot(m, r, r));
        double zn = sqrt(dot(n, z, z));
        ratio = (rn > 0.0) ? zn / (anorm * rn) : 0.0;
        if (ratio_hist) ratio_hist[k] = ratio;
        if (ratio < atol) { status = 0; break; }
        if (k == maxit) { status = 1; break; }

        /* continue the bidiagonalisation */
        for (int64_t i = 0; i < m; i++) ax[i] = 0.0;
        csr_mv(m, rowptr, colidx, vals, vh, ax);
        for (int64_t i = 0; i < m; i++) u[i] = ax[i] - alpha * u[i];
        beta = sqrt(dot(m, u, u));
        if (beta > 0.0)
            for (int64_t i = 0; i < m; i++) u[i] = u[i] / beta;
        csr_mtv(m, n, rowptr, colidx, vals, u, s);
        for (int64_t j = 0; j < n; j++) s[j] = s[j] - beta * w[j];
        if (f) orc_apply(f, s, t); else memcpy(t, s, (size_t)n * sizeof(double));
        a2 = dot(n, t, s);
        if (!(a2 >= 0.0) || !isfinite(a2)) { status = -2; break; }
        alpha = sqrt(a2);
        for (int64_t j = 0; j < n; j++) {
            vh[j] = alpha > 0.0 ? t[j] / alpha : 0.0;
            w[j] = alpha > 0.0 ? s[j] / alpha : 0.0;
        }

        /* rotation P_k */
        double rhoold = rho;
        rho = sqrt(alphabar * alphabar + beta * beta);
        double c = alphabar / rho, sn = beta / rho;
        double theta = sn * alpha;
        alphabar = c * alpha;
        /* rotation Pbar_k */
        double rhobarold = rhobar;
        double thetabar = sbar * rho;
        double crho = cbar * rho;
        rhobar = sqrt(crho * crho + theta * theta);
        cbar = crho / rhobar;
        sbar = theta / rhobar;
        double zeta = cbar * zetabar;
        zetabar = -sbar * zetabar;

        /* h-bar, x, h updates */
        double chb = thetabar * rho / (rhoold * rhobarold);
        double cx = zeta / (rho * rhobar);
        double ch = theta / rho;
        for (int64_t j = 0; j < n; j++) {
            hb[j] = h[j] - chb * hb[j];
            x[j] = x[j] + cx * hb[j];
            h[j] = vh[j] - ch * h[j];
        }
    }
done:
    if (its_out) *its_out = k;
    if (final_ratio) *final_ratio = ratio;
    free(u); free(r); free(ax); free(s); free(t); free(vh); free(w); free(h); free(hb); free(z);
    return status;
}

/*
 * Algorithm 3 on the residual r (length m, original row order): the
 * factors are those of the scaled matrix A D, so h = D h^ for the user's
 * unknowns.  Mode 0 (NONE) takes w = 0, i.e. h = D U^{-1} L1^{-1} r1.
 */
void orc_apply_residual(const orc_factor *f, const double *r, double *h) {
    int64_t n = f->n, m2 = f->m - f->n;
    double *r1 = (double *)xmalloc((size_t)n * sizeof(double));
    double *q1 = (double *)xmalloc((size_t)n * sizeof(double));
    double *y = (double *)xmalloc((size_t)n * sizeof(double));
    double *v = (double *)xmalloc((size_t)n * sizeof(double));
    for (int64_t k = 0; k < n; k++) r1[k] = r[f->prow[k]];
    for (int64_t k = 0; k < n; k++) y[k] = r1[k];
    if (f->mode != 0 && m2 > 0) {
        double *u = (double *)xmalloc((size_t)m2 * sizeof(double));
        double *w = (double *)xmalloc((size_t)m2 * sizeof(double));
        double *fv = (double *)xmalloc((size_t)n * sizeof(double));
        double *g = (double *)xmalloc((size_t)n * sizeof(double));
        /* step 1: u = r2 - Y r1, Y = L2 L1^{-1} */
        solve_lower(n, f->L1p, f->L1i, f->L1v, NULL, r1, q1);
        csr_mv(m2, f->L2p, f->L2i, f->L2v, q1, u);
        for (int64_t i = 0; i < m2; i++) u[i] = r[f->a2rows[i]] - u[i];
        /* step 2: S^ w = u */
        s_solve(f, u, w);
        /* step 3: y = r1 + Y^T w, Y^T = L1^{-T} L2^T */
        csr_mv(n, f->L2tp, f->L2ti, f->L2tv, w, fv);
        solve_upper(n, f->L1tp, f->L1ti, f->L1tv, NULL, fv, g);
        for (int64_t k = 0; k < n; k++) y[k] = r1[k] + g[k];
        free(u); free(w); free(fv); free(g);
    }
    /* step 4: L1 v = y, then U h = v */
    solve_lower(n, f->L1p, f->L1i, f->L1v, NULL, y, v);
    solve_upper(n, f->Up, f->Ui, f->Uv, f->Udiag, v, q1);
    for (int64_t j = 0; j < n; j++) h[j] = f->d[j] * q1[j];
    free(r1); free(q1); free(y); free(v);
}

/*
 * Algorithm 1 from x0 = 0 (the printed step 3 overwrites z0; read as
 * h0 = M^{-1} z0, rho0 = (z0, h0), p0 = h0).  form 0: h = orc_apply_residual(r)
 * (Algorithm 3 fed the residual split, as the paper combines M^{-1} with A^T);
 * form 1: h = orc_apply(A^T r) (the symmetric x-space operator used with LSMR);
 * f == NULL: M = I (plain CGLS).
 * Stopping: for k = 0, 1, ...: ratio_k = ||z_k|| / (anorm ||r_k||) with the
 * recurrence residual r_k and z_k = A^T r_k (Algorithm 1 step 11); stop when
 * ratio_k < atol (or r_k = 0), or when k = maxit.
 * Returns 0 converged, 1 iteration limit, -2 breakdown (rho <= 0, ||q|| = 0
 * or not finite).  ratio_hist (optional, length maxit + 1).
 */
int orc_cgls(const orc_factor *f, int form, int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
             const double *vals, const double *b, double anorm, double atol, int maxit, double *x,
             int *its_out, double *ratio_hist, double *final_ratio) {
    double *r = (double *)xmalloc((size_t)m * sizeof(double));
    double *q = (double *)xmalloc((size_t)m * sizeof(double));
    double *z = (double *)xmalloc((size_t)n * sizeof(double));
    double *h = (double *)xmalloc((size_t)n * sizeof(double));
    double *p = (double *)xmalloc((size_t)n * sizeof(double));
    int status = 1, k = 0;
    double ratio = 0.0;
    for (int64_t j = 0; j < n; j++) x[j] = 0.0;
    for (int64_t i = 0; i < m; i++) r[i] = b[i];                 /* step 1 */
    csr_mtv(m, n, rowptr, colidx, vals, r, z);                    /* step 2 */
    if (!f) memcpy(h, z, (size_t)n * sizeof(double));               /* M = I */
    else if (form == 0) orc_apply_residual(f, r, h); else orc_apply(f, z, h);   /* step 3 */
    double rho = dot(n, z, h);                                    /* step 4 */
    for (int64_t j = 0; j < n; j++) p[j] = h[j];                  /* step 5 */
    for (k = 0;; k++) {
        double rn = sqrt(dot(m, r, r));
        double zn = sqrt(dot(n, z, z));
        ratio = (rn > 0.0) ? zn / (anorm * rn) : 0.0;
        if (ratio_hist) ratio_hist[k] = ratio;
        if (ratio < atol) { status = 0; break; }
        if (k == maxit) { status = 1; break; }
        if (!(rho > 0.0) || !isfinite(rho)) { status = -2; break; }
        csr_mv(m, rowptr, colidx, vals, p, q);                    /* step 7 */
        double qq = dot(m, q, q);
        if (!(qq > 0.0) || !isfinite(qq)) { status = -2; break; }
        double alpha = rho / qq;                                  /* step 8 */
        for (int64_t j = 0; j < n; j++) x[j] = x[j] + alpha * p[j];   /* step 9 */
        for (int64_t i = 0; i < m; i++) r[i] = r[i] - alpha * q[i];   /* step 10 */
        csr_mtv(m, n, rowptr, colidx, vals, r, z);                /* step 11 */
        if (!f) memcpy(h, z, (size_t)n * sizeof(double));
        else if (form == 0) orc_apply_residual(f, r, h); else orc_apply(f, z, h);   /* step 12 */
        double rhon = dot(n, z, h);                               /* step 13 */
        double beta = rhon / rho;                                 /* step 14 */
        for (int64_t j = 0; j < n; j++) p[j] = h[j] + beta * p[j];    /* step 15 */
        rho = rhon;
    }
    if (its_out) *its_out = k;
    if (final_ratio) *final_ratio = ratio;
    free(r); free(q); free(z); free(h); free(p);
    return status;
}

/*
 * Sec. 3.4, adding rows: each new row a (the user's values, columns of A) is
 * scaled by the existing D and gets the L2 row l with l U = a D, i.e.
 * U^T l^T = (a D)^T (lower solve, position order), dropped by the rule of
 * Algorithm 4 (|l| >= tau, then at most p of the largest, ties to the smaller
 * position).  L1, U, D and the pivots stay; the new rows take ids m .. m+k-1
 * and join A2 at its end (A2 rows stay in ascending id).  With the dense
 * correction the dense S is set up again.  Returns orc_correction's status.
 */
int orc_factor_add_rows(orc_factor *f, int64_t k, const int64_t *rp, const int32_t *ci, const double *v,
                        int p, double tau) {
    int64_t n = f->n, m = f->m, m2 = m - n;
    int64_t old_nnz = f->L2p[m2];
    double *ah = (double *)xcalloc((size_t)n, sizeof(double));
    double *l = (double *)xmalloc((size_t)n * sizeof(double));
    cand *c = (cand *)xmalloc((size_t)n * sizeof(cand));
    /* new rows collected first, then the CSR grown once */
    int64_t cap = old_nnz + k * (p >= 0 ? p : n) + 1;
    int64_t *np = (int64_t *)xmalloc((size_t)(m2 + k + 1) * sizeof(int64_t));
    int32_t *ni = (int32_t *)xmalloc((size_t)cap * sizeof(int32_t));
    double *nv = (double *)xmalloc((size_t)cap * sizeof(double));
    memcpy(np, f->L2p, (size_t)(m2 + 1) * sizeof(int64_t));
    memcpy(ni, f->L2i, (size_t)old_nnz * sizeof(int32_t));
    memcpy(nv, f->L2v, (size_t)old_nnz * sizeof(double));
    int64_t w = old_nnz;
    for (int64_t t = 0; t < k; t++) {
        for (int64_t j = 0; j < n; j++) ah[j] = 0.0;
        for (int64_t e = rp[t]; e < rp[t + 1]; e++) ah[ci[e]] = v[e] * f->d[ci[e]];
        solve_lower(n, f->Utp, f->Uti, f->Utv, f->Udiag, ah, l);
        int64_t len = 0;
        for (int64_t q = 0; q < n; q++)
            if (l[q] != 0.0) { c[len].mag = fabs(l[q]); c[len].key = (int32_t)q; c[len].val = l[q]; len++; }
        int64_t kept = drop_keep(c, len, p, tau);
        for (int64_t q = 0; q < kept; q++) { ni[w] = c[q].key; nv[w] = c[q].val; w++; }
        np[m2 + t + 1] = w;
    }
    free(ah); free(l); free(c);
    free(f->L2p); free(f->L2i); free(f->L2v);
    f->L2p = np; f->L2i = ni; f->L2v = nv;
    free(f->L2tp); free(f->L2ti); free(f->L2tv);
    csr_transpose(m2 + k, n, f->L2p, f->L2i, f->L2v, &f->L2tp, &f->L2ti, &f->L2tv);
    f->a2rows = (int32_t *)realloc(f->a2rows, (size_t)(m2 + k) * sizeof(int32_t));
    f->pivpos = (int32_t *)realloc(f->pivpos, (size_t)(m + k) * sizeof(int32_t));
    f->a2idx = (int32_t *)realloc(f->a2idx, (size_t)(m + k) * sizeof(int32_t));
    for (int64_t t = 0; t < k; t++) {
        f->a2rows[m2 + t] = (int32_t)(m + t);
        f->pivpos[m + t] = -1;
        f->a2idx[m + t] = (int32_t)(m2 + t);
    }
    f->m = m + k;
    if (f->mode == 3) return orc_correction(f, 3, f->cg_steps);
    return 0;
}

/*
 * Sec. 3.4, removing rows of A2 (ids ascending, distinct): their L2 rows go;
 * the remaining rows keep their order and are renumbered (ids above a removed
 * one move down).  A pivot row cannot be removed this way (-1: refactorise).
 * With the dense correction the dense S is set up again.
 */
int orc_factor_remove_rows(orc_factor *f, int64_t k, const int32_t *ids) {
    int64_t n = f->n, m = f->m, m2 = m - n;
    for (int64_t t = 0; t < k; t++) {
        if (ids[t] < 0 || ids[t] >= m || f->pivpos[ids[t]] >= 0) return -1;
        if (t > 0 && ids[t] <= ids[t - 1]) return -1;
    }
    /* new id of every old row (-1: removed) */
    int32_t *nid = (int32_t *)xmalloc((size_t)m * sizeof(int32_t));
    int64_t t = 0, next = 0;
    for (int64_t i = 0; i < m; i++) {
        if (t < k && ids[t] == i) { nid[i] = -1; t++; }
        else nid[i] = (int32_t)next++;
    }
    int64_t *np = (int64_t *)xmalloc((size_t)(m2 - k + 1) * sizeof(int64_t));
    int32_t *ni = (int32_t *)xmalloc((size_t)(f->L2p[m2] + 1) * sizeof(int32_t));
    double *nv = (double *)xmalloc((size_t)(f->L2p[m2] + 1) * sizeof(double));
    int32_t *na2 = (int32_t *)xmalloc((size_t)(m2 - k > 0 ? m2 - k : 1) * sizeof(int32_t));
    np[0] = 0;
    int64_t r = 0, w = 0;
    for (int64_t c = 0; c < m2; c++) {
        int32_t orig = f->a2rows[c];
        if (nid[orig] < 0) continue;
        for (int64_t e = f->L2p[c]; e < f->L2p[c + 1]; e++) { ni[w] = f->L2i[e]; nv[w] = f->L2v[e]; w++; }
        na2[r] = nid[orig];
        np[++r] = w;
    }
    for (int64_t q = 0; q < n; q++) f->prow[q] = nid[f->prow[q]];
    free(f->L2p); free(f->L2i); free(f->L2v); free(f->a2rows);
    f->L2p = np; f->L2i = ni; f->L2v = nv; f->a2rows = na2;
    free(f->L2tp); free(f->L2ti); free(f->L2tv);
    csr_transpose(m2 - k, n, f->L2p, f->L2i, f->L2v, &f->L2tp, &f->L2ti, &f->L2tv);
    int32_t *pp = (int32_t *)xmalloc((size_t)(m - k > 0 ? m - k : 1) * sizeof(int32_t));
    int32_t *ai = (int32_t *)xmalloc((size_t)(m - k > 0 ? m - k : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < m - k; i++) { pp[i] = -1; ai[i] = -1; }
    for (int64_t q = 0; q < n; q++) pp[f->prow[q]] = (int32_t)q;
    for (int64_t c = 0; c < m2 - k; c++) ai[f->a2rows[c]] = (int32_t)c;
    free(f->pivpos); free(f->a2idx); free(nid);
    f->pivpos = pp; f->a2idx = ai;
    f->m = m - k;
    if (f->mode == 3) return orc_correction(f, 3, f->cg_steps);
    return 0;
}
