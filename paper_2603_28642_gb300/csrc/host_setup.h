// Host-side set-up of the row-splitting ILU preconditioner: column scaling,
// the rectangular threshold-pivoted ILUP(p, tau) factorisation (Algorithms
// 4-6 of Scott & Tuma), the row split P A D ~ [L1; L2] U (eq. 3.8), level
// analysis of the four triangular systems and the dense auxiliary matrix
// S = I + Y Y^T (eq. 3.9) for the dense correction mode.
//
// Everything here runs once per matrix on the CPU.  Floating-point sums are
// evaluated in a fixed order and this translation unit is compiled with
// -ffp-contract=off, so the factor is reproducible bit for bit.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace rlsq {

struct HostCSR {
    int64_t rows = 0, cols = 0;
    std::vector<int64_t> ptr;  // rows + 1
    std::vector<int32_t> idx;  // column ids ascending within each row
    std::vector<double> val;
    int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// Transpose (rows x cols -> cols x rows); entries of each output row keep
// ascending column order.
HostCSR transpose(const HostCSR& a);
// The same on up to `threads` threads (the same arrays for any count).
HostCSR transpose(const HostCSR& a, int threads);

struct IlupParams {
    int p = 10;          // max off-diagonal entries kept per column of L and U (< 0: all)
    double tau = 1e-2;   // absolute drop tolerance
    double mu = 0.1;     // threshold pivoting parameter (Algorithm 5)
    double small = 1e-10;// smallest admissible |U_jj| (Algorithm 6)
    bool scale = true;   // prescale columns to unit 2-norm
    int threads = 1;     // threads of the (pipelined) column loop; the factor is the same for any count
};

// Level structure of one triangular system: level of every row, rows sorted
// by (level, row id), and the start of each level in that order.
struct Levels {
    std::vector<int32_t> level;
    std::vector<int32_t> order;
    std::vector<int32_t> level_ptr;  // nlevels + 1
    int32_t nlevels = 0;
    int32_t max_width = 0;
};

struct IlupResult {
    int64_t m = 0, n = 0;
    std::vector<double> d;          // column scaling
    std::vector<int32_t> prow;      // prow[k]: original row pivoted at position k
    std::vector<int32_t> a2rows;    // rows of A2 (unpivoted), ascending
    HostCSR L1, L1t;                // strictly lower unit factor (rows = pivot positions) and its transpose
    HostCSR L2, L2t;                // (m-n) x n and its transpose
    HostCSR U, Ut;                  // strictly upper part of U and its transpose
    std::vector<double> Udiag;
    int64_t nmod = 0;
    Levels lev_L1, lev_L1t, lev_U, lev_Ut;
};

// Sec. 3.4, adding rows: every row of `rows` (n columns, the user's values)
// joins A2 with the ids m, m+1, ...; its L2 row l solves l U = a D (a lower
// solve with U^T in position order), dropped like an L column of Algorithm 4
// (|l| >= tau, then at most p of the largest).  L1, U, D and the pivots are
// unchanged; L2^T is rebuilt.
void add_rows(IlupResult& F, const HostCSR& rows, const IlupParams& prm);
// Sec. 3.4, removing rows of A2 (ids ascending and distinct): their L2 rows
// go and the remaining rows are renumbered in order.  Throws
// std::invalid_argument for a pivot row or a bad id (a refactorisation is
// needed then) and std::length_error if no row of A2 would remain (m > n).
void remove_rows(IlupResult& F, const std::vector<int32_t>& ids);

// Column scaling d_j = 1 / ||A_:,j||_2.  Returns false if a column is empty.
bool column_scaling(const HostCSR& a, std::vector<double>& d);

// Full set-up.  Throws std::runtime_error with a message on bad input.
IlupResult ilup_factor(const HostCSR& a, const IlupParams& prm);

// Threads for the column loop of an m x n factorisation: `requested` if > 0
// (at most 64), else the CPUs the process may run on (at most 16); fewer where one
// working array per thread (16 bytes per row of A) would pass 2 GiB.  Each
// thread keeps up to 8 columns in flight, as many as such arrays fit in 2 GiB.
int ilup_threads(int requested, int64_t m, int64_t n);

// lower = true: row i depends on k < i; otherwise on k > i.
Levels analyse_levels(const HostCSR& strict, bool lower);

// A triangular system with groups of `k` consecutive levels fused: inside a
// group, a row's dependencies on rows of the same group are substituted, so
// every remaining dependency lies in an earlier group.  Row i then reads
//   x_i = (rhs_i + sum_R c rhs_j - sum_T c x_j) / diag_i
// with R the right-hand-side terms brought in by the substitution.  The
// result is the same solution (up to rounding) with about levels / k levels.
struct MergedTri {
    HostCSR T;       // remaining dependencies (unknown ids), strictly earlier groups
    HostCSR R;       // extra right-hand-side terms (unknown ids, coefficients)
    Levels lev;      // levels of T
    int k = 1;       // levels per group (adaptive: the largest group)
    bool adaptive = false;
};
// Cost model of a fused solve, fitted to the measured solves of a 2M x 1M
// problem on GB300 (every schedule, k = 1..4): about kLevelCost seconds per
// level plus kEntryCost seconds per stored float64 entry of T and R (an
// entry's cost is a random gather, not its bytes; float32 entries scale by
// width).  Groups grown level by level hold at most kMaxFusedGroup levels.
constexpr double kLevelCost = 3.0e-6;
constexpr double kEntryCost = 13.7e-12;
constexpr int kMaxFusedGroup = 16;

// max_nnz > 0: give up (k = 0 in the result) once T and R hold more entries.
MergedTri merge_levels(const HostCSR& strict, const double* diag, const Levels& lev, int k, int64_t max_nnz = 0);
// Groups of consecutive levels chosen greedily: a level joins the current
// group (of at most max_group levels) when the entries its substitution adds
// are at most level_entries (the cost of one level expressed in entries),
// otherwise it opens a new group.
MergedTri merge_levels_adaptive(const HostCSR& strict, const double* diag, const Levels& lev,
                                double level_entries, int max_group);

// Dense inverse of S = I + Z^T Z, Z = L1^{-T} L2^T, through its Cholesky
// factor; row-major (m-n)^2.  Returns false if S is not numerically SPD.
// keep_z (if not null) receives Z, column-major n x (m-n).
bool dense_schur_inverse(const IlupResult& f, std::vector<double>& sinv, int threads,
                         std::vector<double>* keep_z = nullptr);

// Sec. 3.4 for the dense correction: a row joining A2 borders S with one row
// and column, and a row leaving A2 takes its row and column away, so S^{-1}
// follows by block inversion through the Schur complement instead of being
// formed again: O(n (m-n) + (m-n)^2) per added row (the border is z_a . z
// with the columns of Z, which the caller keeps beside S^{-1}, and z
// = L1^{-T} l^T; exactly the entries a new formation would compute), O((m-n)^2)
// per removed row.  S's eigenvalues are >= 1, so every Schur complement is
// >= 1; both updates throw std::runtime_error (the caller then forms the
// inverse again) where their subtractions would cancel more than 4 digits.
// schur_inverse_add: F already holds the k added rows as the last rows of L2;
// sinv and Z belong to the first m-n-k rows on entry, to all rows on return.
void schur_inverse_add(const IlupResult& F, int64_t k, std::vector<double>& sinv, std::vector<double>& Z);
// schur_inverse_remove: `pos` are the removed rows' positions in A2 (before the
// removal, ascending); sinv and Z belong to all m2 rows on entry.
void schur_inverse_remove(const std::vector<int64_t>& pos, int64_t m2, std::vector<double>& sinv,
                          std::vector<double>& Z);

}  // namespace rlsq
