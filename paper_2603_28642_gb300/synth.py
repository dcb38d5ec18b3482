"""Seeded synthetic least-squares problems shaped like the paper's workloads.

This module only draws inputs: a sparse m x n matrix A in CSR form (int64 row
pointers, int32 sorted column indices, float64 values) and a right-hand side b.
It holds none of the preconditioner's or the solver's arithmetic, so both the
CPU oracle and the GPU library can consume the same arrays.

The paper's own test matrices (SuiteSparse / CUTEst, Table 1) are not
available; these generators stand in for them:

* ``sparse_problem`` -- general sparse rows: every row has ``d`` distinct
  uniform-random columns with N(0,1) values, and n rows (either the first n,
  or a hidden random subset of n rows) carry a +-4 entry in their "own"
  column so that A has full column rank (the paper assumes full rank, Sec. 1).
  Rows are then shuffled.  b = A x_true + 1e-3 * N(0,1).
* ``sparse_dense_problem`` -- the same plus a few fully dense rows with
  N(0,1)/sqrt(n) entries shuffled in: the sparse-dense case of Sec. 3.3.
* ``batch_problems`` / ``serving_matrices`` -- many problems of uneven size.

Random numbers come from numpy's PCG64 generator; the draw order is fixed and
documented per function, so a seed names one matrix exactly.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "Problem",
    "sparse_problem",
    "sparse_dense_problem",
    "config_problem",
    "batch_problem_sizes",
    "batch_problems",
    "serving_matrices",
    "serving_rhs",
    "random_rhs",
    "poisson_arrivals",
]


@dataclass
class Problem:
    """A least-squares instance min ||b - A x|| with A in CSR form."""

    m: int
    n: int
    rowptr: np.ndarray  # int64, length m + 1
    colidx: np.ndarray  # int32, length nnz, strictly increasing within a row
    vals: np.ndarray  # float64, length nnz
    b: np.ndarray  # float64, length m
    x_true: np.ndarray  # float64, length n
    dense_rows: np.ndarray  # int64 ids (after shuffling) of fully dense rows

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.vals, self.colidx, self.rowptr), shape=(self.m, self.n))


def _distinct_columns(rng: np.random.Generator, rows: int, d: int, n: int) -> np.ndarray:
    """rows x d matrix of column ids, distinct within each row, each row sorted.

    Draw order: one integers((rows, d)) block, then, while some rows hold a
    repeated column, one integers((bad, d)) block that replaces those rows
    wholesale (bad rows taken in ascending order)."""
    if d > n:
        raise ValueError("more nonzeros per row than columns")
    cols = rng.integers(0, n, size=(rows, d), dtype=np.int64)
    cols.sort(axis=1)
    while True:
        if d > 1:
            bad = np.nonzero((cols[:, 1:] == cols[:, :-1]).any(axis=1))[0]
        else:
            bad = np.zeros(0, dtype=np.int64)
        if bad.size == 0:
            return cols
        redraw = rng.integers(0, n, size=(bad.size, d), dtype=np.int64)
        redraw.sort(axis=1)
        cols[bad] = redraw


def _assemble(m, n, row_cols, row_vals, diag_rows, diag_vals, perm, extra_dense=None):
    """Build sorted CSR from per-row random entries plus one 'diagonal' entry.

    row_cols/row_vals: (m_sparse, d) arrays.  diag_rows[j] is the (pre-shuffle)
    row that gets diag_vals[j] at column j; on a collision with a random column
    the random value is overwritten.  extra_dense: optional (k, n) block of
    dense rows appended after the sparse rows before shuffling.  perm[r] is the
    pre-shuffle row placed at final position r."""
    ms, d = row_cols.shape
    cols = row_cols.copy()
    vals = row_vals.copy()
    # rows that receive a diagonal entry: overwrite on collision, else append
    has_diag = np.full(ms, -1, dtype=np.int64)
    has_diag[diag_rows] = np.arange(diag_rows.size)
    extra_col = np.full(ms, -1, dtype=np.int64)
    extra_val = np.zeros(ms)
    rr = np.nonzero(has_diag >= 0)[0]
    jj = has_diag[rr]
    hit = cols[rr] == jj[:, None]
    collide = hit.any(axis=1)
    # overwrite
    ci = rr[collide]
    vals[ci] = np.where(hit[collide], diag_vals[jj[collide]][:, None], vals[ci])
    # append
    ai = rr[~collide]
    extra_col[ai] = jj[~collide]
    extra_val[ai] = diag_vals[jj[~collide]]

    counts = np.full(ms, d, dtype=np.int64) + (extra_col >= 0)
    k_dense = 0 if extra_dense is None else extra_dense.shape[0]
    all_counts = np.concatenate([counts, np.full(k_dense, n, dtype=np.int64)])
    # final order
    final_counts = all_counts[perm]
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(final_counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    colidx = np.empty(nnz, dtype=np.int32)
    values = np.empty(nnz, dtype=np.float64)

    # sparse rows: merge the optional extra entry into the sorted list
    full_c = np.concatenate([cols, extra_col[:, None]], axis=1)
    full_v = np.concatenate([vals, extra_val[:, None]], axis=1)
    key = np.where(full_c < 0, np.iinfo(np.int64).max, full_c)
    order = np.argsort(key, axis=1, kind="stable")
    full_c = np.take_along_axis(full_c, order, axis=1)
    full_v = np.take_along_axis(full_v, order, axis=1)
    inv = np.empty(m, dtype=np.int64)
    inv[perm] = np.arange(m)
    # destination start of each pre-shuffle row
    start = rowptr[inv]
    # scatter sparse rows
    width = d + 1
    valid = full_c >= 0
    pos = start[:ms, None] + np.cumsum(valid, axis=1) - 1
    colidx[pos[valid]] = full_c[valid].astype(np.int32)
    values[pos[valid]] = full_v[valid]
    if k_dense:
        for t in range(k_dense):
            s = start[ms + t]
            colidx[s : s + n] = np.arange(n, dtype=np.int32)
            values[s : s + n] = extra_dense[t]
    del width
    dense_final = np.sort(inv[ms:]) if k_dense else np.zeros(0, dtype=np.int64)
    return rowptr, colidx, values, dense_final


def _rhs(rng, rowptr, colidx, vals, m, n, noise=1e-3):
    """x_true ~ N(0,1)^n, then b = A x_true + noise * N(0,1)^m (two draws, in that order)."""
    import scipy.sparse as sp

    x_true = rng.standard_normal(n)
    eps = rng.standard_normal(m)
    A = sp.csr_matrix((vals, colidx, rowptr), shape=(m, n))
    b = A @ x_true + noise * eps
    return x_true, b


def sparse_problem(m: int, n: int, d: int, seed: int, hidden_diag: bool = False,
                   diag_value: float = 4.0) -> Problem:
    """General sparse least-squares problem.

    Draw order from PCG64(seed):
      1. random columns (``_distinct_columns``), 2. values N(0,1) (m x d),
      3. diagonal signs integers(0, 2, n) -> +-diag_value,
      4. if hidden_diag: permutation(m)[:n] picks the rows carrying the
         diagonal, else rows 0..n-1 do,
      5. row shuffle permutation(m),
      6. x_true, 7. noise (see ``_rhs``).
    """
    if not (m > n > 0):
        raise ValueError("need m > n > 0")
    rng = np.random.Generator(np.random.PCG64(seed))
    cols = _distinct_columns(rng, m, d, n)
    vals = rng.standard_normal((m, d))
    signs = rng.integers(0, 2, size=n) * 2 - 1
    diag_vals = diag_value * signs.astype(np.float64)
    if hidden_diag:
        diag_rows = rng.permutation(m)[:n]
    else:
        diag_rows = np.arange(n)
    perm = rng.permutation(m)
    rowptr, colidx, values, dense = _assemble(m, n, cols, vals, diag_rows, diag_vals, perm)
    x_true, b = _rhs(rng, rowptr, colidx, values, m, n)
    return Problem(m, n, rowptr, colidx, values, b, x_true, dense)


def sparse_dense_problem(m_sparse: int, n: int, d: int, n_dense: int, seed: int) -> Problem:
    """Sparse rows as ``sparse_problem(hidden_diag=True)`` plus ``n_dense`` rows
    that are full, with N(0,1)/sqrt(n) entries (Sec. 3.3 sparse-dense case).

    Draw order: columns, values, signs, hidden rows permutation(m_sparse)[:n],
    dense block standard_normal((n_dense, n)), shuffle permutation(m), x_true,
    noise."""
    m = m_sparse + n_dense
    rng = np.random.Generator(np.random.PCG64(seed))
    cols = _distinct_columns(rng, m_sparse, d, n)
    vals = rng.standard_normal((m_sparse, d))
    signs = rng.integers(0, 2, size=n) * 2 - 1
    diag_vals = 4.0 * signs.astype(np.float64)
    diag_rows = rng.permutation(m_sparse)[:n]
    dense = rng.standard_normal((n_dense, n)) / np.sqrt(n)
    perm = rng.permutation(m)
    rowptr, colidx, values, dense_ids = _assemble(m, n, cols, vals, diag_rows, diag_vals, perm,
                                                  extra_dense=dense)
    x_true, b = _rhs(rng, rowptr, colidx, values, m, n)
    return Problem(m, n, rowptr, colidx, values, b, x_true, dense_ids)


def config_problem(which: int, scale: float = 1.0) -> Problem:
    """The single-problem workloads.

    0: m 1500, n 1000, 6 nnz/row + first-n-rows diagonal, seed 0.
    1: m 2,000,000, n 1,000,000, 8 nnz/row + hidden diagonal, seed 1.
    2: n 500,000, 1,000,000 sparse rows (6 nnz + hidden diagonal) and 200
       dense rows, seed 2.
    ``scale`` shrinks m and n (same seed) for quick runs of the same recipe."""
    if which == 0:
        return sparse_problem(int(1500 * scale), int(1000 * scale), 6, seed=0)
    if which == 1:
        return sparse_problem(int(2_000_000 * scale), int(1_000_000 * scale), 8, seed=1,
                              hidden_diag=True)
    if which == 2:
        return sparse_dense_problem(int(1_000_000 * scale), int(500_000 * scale), 6,
                                    200, seed=2)
    raise ValueError(which)


def batch_problem_sizes(count: int = 512, master_seed: int = 3, n_lo: int = 2000,
                        n_hi: int = 50000):
    """(n_k, m_k, d_k) for the batched workload: n log-uniform in [n_lo, n_hi],
    m/n uniform in [1.2, 2.0], d uniform in {4..10}.  Draws from
    PCG64(master_seed): uniform(count) for n, uniform(count) for m/n,
    integers(4, 11, count) for d."""
    rng = np.random.Generator(np.random.PCG64(master_seed))
    n = np.round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count))).astype(np.int64)
    ratio = rng.uniform(1.2, 2.0, size=count)
    m = np.round(n * ratio).astype(np.int64)
    m = np.maximum(m, n + 1)
    d = rng.integers(4, 11, size=count)
    return n, m, d


def batch_problems(count: int = 512, master_seed: int = 3, n_lo: int = 2000,
                   n_hi: int = 50000, seed_base: int = 3000, first: int | None = None):
    """Independent problems of uneven size; problem k uses seed seed_base + k
    with the first-n-rows diagonal rule.  ``first`` keeps only the first
    problems of the ``count``-problem recipe (same sizes and seeds)."""
    n, m, d = batch_problem_sizes(count, master_seed, n_lo, n_hi)
    take = count if first is None else min(first, count)
    return [sparse_problem(int(m[k]), int(n[k]), int(d[k]), seed=seed_base + k)
            for k in range(take)]


def serving_matrices(count: int = 64, master_seed: int = 4, n_lo: int = 1000,
                     n_hi: int = 200000, seed_base: int = 4000):
    """Resident matrices for the serving workload: n log-uniform in
    [n_lo, n_hi] (uniform(count) from PCG64(master_seed)), m = 1.5 n, 6 nnz
    per row, matrix k from seed seed_base + k."""
    rng = np.random.Generator(np.random.PCG64(master_seed))
    n = np.round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count))).astype(np.int64)
    return [sparse_problem(int(round(1.5 * n[k])), int(n[k]), 6, seed=seed_base + k)
            for k in range(count)]


def random_rhs(prob: Problem, seed: int, noise: float = 1e-3) -> np.ndarray:
    """A fresh right-hand side for a resident matrix: b = A x + noise*N(0,1)
    with x ~ N(0,1) drawn from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    _, b = _rhs(rng, prob.rowptr, prob.colidx, prob.vals, prob.m, prob.n, noise)
    return b


def serving_rhs(prob: Problem, request_id: int) -> np.ndarray:
    """Right-hand side of serving request ``request_id`` (seed 10**6 + id)."""
    return random_rhs(prob, 10**6 + request_id)


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate: cumulative
    sums of exponential(1/rate) gaps drawn from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
