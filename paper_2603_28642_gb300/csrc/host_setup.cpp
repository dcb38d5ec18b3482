// Host set-up of the row-splitting ILU preconditioner (see host_setup.h).
//
// The factorisation follows the column-wise ILUP(p, tau) of Algorithm 4 with
// the pivot rule of Algorithm 5 and the pivot modification of Algorithm 6
// (Scott & Tuma, Sec. 4).  Column j is computed left-looking, in the
// Gilbert-Peierls manner the paper describes: a graph search over the
// already computed columns of L finds the pivot positions reached from the
// nonzeros of A(:, j) (the pattern of U(1:j-1, j)), the positions are sorted
// ascending (a topological order because L is unit lower triangular in pivot
// order), and the sparse triangular solve then updates the not-yet-pivoted
// rows at the same time, which yields the L part of step 7.  With more than
// one thread the column loop is pipelined over consecutive columns
// (columns_pipelined below); the factor is the same bit for bit.
//
// Readings of points the paper leaves open:
//  * rc(i) at step j counts the nonzeros of the original scaled matrix in row
//    i and columns j..n.
//  * Algorithm 5 ties: smallest rc, then largest |L_qj|, then smallest row id.
//  * empty column: pivot on the unpivoted row with the smallest rc (then id),
//    value max(beta ||A_:,j||_inf, small); small pivot: the same magnitude
//    with the pivot's sign.  beta = 10^(-2 (1 - j/n)), 1-based j.
//  * dropping: |.| >= tau kept, then the p largest; ties keep the smaller
//    pivot position (U) or the smaller row id (L); the U part is dropped
//    after the L part has been computed from the undropped values.
#include "host_setup.h"

#include <algorithm>
#include <atomic>
#if defined(__linux__)
#include <sched.h>
#endif
#include <cmath>
#include <exception>
#include <functional>
#include <memory>
#include <stdexcept>
#include <system_error>
#include <thread>

namespace rlsq {

HostCSR transpose(const HostCSR& a) {
    HostCSR t;
    t.rows = a.cols;
    t.cols = a.rows;
    t.ptr.assign(static_cast<size_t>(a.cols) + 1, 0);
    const int64_t nnz = a.nnz();
    t.idx.resize(static_cast<size_t>(nnz));
    t.val.resize(static_cast<size_t>(nnz));
    for (int64_t e = 0; e < nnz; ++e) t.ptr[a.idx[e] + 1]++;
    for (int64_t c = 0; c < a.cols; ++c) t.ptr[c + 1] += t.ptr[c];
    std::vector<int64_t> pos(t.ptr.begin(), t.ptr.end() - 1);
    for (int64_t r = 0; r < a.rows; ++r)
        for (int64_t e = a.ptr[r]; e < a.ptr[r + 1]; ++e) {
            const int64_t dst = pos[a.idx[e]]++;
            t.idx[dst] = static_cast<int32_t>(r);
            t.val[dst] = a.val[e];
        }
    return t;
}

namespace {

// The transpose of a CSR structure (rows x cols) on up to `threads` threads:
// output row relabel[c] (c itself without a relabelling, which must then be a
// permutation onto 0..cols-1) holds the entries of column c in ascending
// source row, exactly as transpose() orders them.  Each thread counts and
// then scatters one block of source rows; per-block offsets keep the order.
void transpose_into(int64_t rows, int64_t cols, const int64_t* ptr, const int32_t* idx, const double* val,
                    const int32_t* relabel, int threads, HostCSR& out) {
    const int64_t nnz = ptr[rows];
    const int64_t T = std::max<int64_t>(1, std::min<int64_t>(threads, nnz / (int64_t(1) << 18) + 1));
    out.rows = cols;
    out.cols = rows;
    out.ptr.assign(static_cast<size_t>(cols) + 1, 0);
    out.idx.resize(static_cast<size_t>(nnz));
    out.val.resize(static_cast<size_t>(nnz));
    // blocks of source rows with about nnz / T entries each
    std::vector<int64_t> start(static_cast<size_t>(T) + 1, rows);
    start[0] = 0;
    for (int64_t b = 1; b < T; ++b)
        start[b] = std::lower_bound(ptr, ptr + rows + 1, b * nnz / T) - ptr;
    for (int64_t b = 1; b <= T; ++b) start[b] = std::max(start[b], start[b - 1]);
    std::vector<std::vector<int64_t>> off(static_cast<size_t>(T));
    auto parallel = [&](auto&& body) {
        std::vector<std::thread> ts;
        std::vector<std::exception_ptr> errs(static_cast<size_t>(T));
        auto guarded_body = [&](int64_t b) {
            try {
                body(b);
            } catch (...) {
                errs[static_cast<size_t>(b)] = std::current_exception();
            }
        };
        for (int64_t b = 1; b < T; ++b) ts.emplace_back(guarded_body, b);
        guarded_body(0);
        for (auto& t : ts) t.join();
        for (const auto& e : errs)
            if (e) std::rethrow_exception(e);
    };
    auto row_of = [&](int32_t c) -> int64_t { return relabel ? relabel[c] : c; };
    parallel([&](int64_t b) {
        std::vector<int64_t>& cnt = off[static_cast<size_t>(b)];
        cnt.assign(static_cast<size_t>(cols), 0);
        for (int64_t e = ptr[start[b]]; e < ptr[start[b + 1]]; ++e) cnt[row_of(idx[e])]++;
    });
    // output row r starts after all earlier rows; block b after blocks < b
    for (int64_t r = 0; r < cols; ++r) {
        int64_t run = out.ptr[r];
        for (int64_t b = 0; b < T; ++b) {
            const int64_t c = off[static_cast<size_t>(b)][r];
            off[static_cast<size_t>(b)][r] = run;
            run += c;
        }
        out.ptr[r + 1] = run;
    }
    parallel([&](int64_t b) {
        std::vector<int64_t>& at = off[static_cast<size_t>(b)];
        for (int64_t r = start[b]; r < start[b + 1]; ++r)
            for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) {
                const int64_t dst = at[row_of(idx[e])]++;
                out.idx[dst] = static_cast<int32_t>(r);
                out.val[dst] = val[e];
            }
    });
}

}  // namespace

HostCSR transpose(const HostCSR& a, int threads) {
    HostCSR t;
    transpose_into(a.rows, a.cols, a.ptr.data(), a.idx.data(), a.val.data(), nullptr, threads, t);
    return t;
}

bool column_scaling(const HostCSR& a, std::vector<double>& d) {
    std::vector<double> ss(static_cast<size_t>(a.cols), 0.0);
    for (int64_t r = 0; r < a.rows; ++r)
        for (int64_t e = a.ptr[r]; e < a.ptr[r + 1]; ++e) {
            const double v = a.val[e];
            ss[a.idx[e]] = ss[a.idx[e]] + v * v;
        }
    d.resize(static_cast<size_t>(a.cols));
    bool ok = true;
    for (int64_t j = 0; j < a.cols; ++j) {
        if (!(ss[j] > 0.0)) ok = false;
        d[j] = 1.0 / std::sqrt(ss[j]);
    }
    return ok;
}

namespace {

struct Entry {
    double mag;
    int32_t key;
    double val;
};

// keep |v| >= tau, then the p largest (ties: smaller key); result sorted by key
void dual_drop(std::vector<Entry>& c, int p, double tau) {
    size_t w = 0;
    for (size_t i = 0; i < c.size(); ++i)
        if (c[i].mag >= tau && c[i].val != 0.0) c[w++] = c[i];
    c.resize(w);
    if (p >= 0 && c.size() > static_cast<size_t>(p)) {
        auto better = [](const Entry& a, const Entry& b) {
            return a.mag > b.mag || (a.mag == b.mag && a.key < b.key);
        };
        std::nth_element(c.begin(), c.begin() + p, c.end(), better);
        c.resize(static_cast<size_t>(p));
    }
    std::sort(c.begin(), c.end(), [](const Entry& a, const Entry& b) { return a.key < b.key; });
}

}  // namespace

Levels analyse_levels(const HostCSR& s, bool lower) {
    Levels L;
    const int64_t n = s.rows;
    L.level.assign(static_cast<size_t>(n), 0);
    int32_t nlev = 0;
    for (int64_t t = 0; t < n; ++t) {
        const int64_t i = lower ? t : n - 1 - t;
        int32_t lv = 0;
        for (int64_t e = s.ptr[i]; e < s.ptr[i + 1]; ++e) lv = std::max(lv, L.level[s.idx[e]] + 1);
        L.level[i] = lv;
        nlev = std::max(nlev, lv + 1);
    }
    if (n == 0) nlev = 0;
    L.nlevels = nlev;
    L.level_ptr.assign(static_cast<size_t>(nlev) + 1, 0);
    for (int64_t i = 0; i < n; ++i) L.level_ptr[L.level[i] + 1]++;
    for (int32_t l = 0; l < nlev; ++l) {
        L.max_width = std::max(L.max_width, L.level_ptr[l + 1]);
        L.level_ptr[l + 1] += L.level_ptr[l];
    }
    L.order.resize(static_cast<size_t>(n));
    std::vector<int32_t> pos(L.level_ptr.begin(), L.level_ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) L.order[pos[L.level[i]]++] = static_cast<int32_t>(i);
    return L;
}

namespace {

// Columns of L (original row ids, multipliers) and of U (pivot positions,
// values) in the order Algorithm 4 produces them, and the pivot position of
// every row (-1: a row of A2).
struct ColumnFactor {
    std::vector<int64_t> Lp, Up;
    std::vector<int32_t> Li, Ui;
    std::vector<double> Lv, Uv;
    std::vector<int32_t> pivpos;
};

// Algorithm 6: the magnitude a modified pivot of column j (0-based) gets.
double modified_pivot(double colinf, int64_t j, int64_t n, double small) {
    const double beta = std::pow(10.0, -2.0 * (1.0 - static_cast<double>(j + 1) / static_cast<double>(n)));
    double modval = beta * colinf;
    if (modval < small) modval = small;
    return modval;
}

// Column by column on one thread.
void columns_serial(const HostCSR& a, const HostCSR& ac, const IlupParams& prm, IlupResult& R, ColumnFactor& C) {
    const int64_t m = a.rows, n = a.cols;
    std::vector<int32_t> rc(static_cast<size_t>(m));
    for (int64_t i = 0; i < m; ++i) rc[i] = static_cast<int32_t>(a.ptr[i + 1] - a.ptr[i]);

    // Per-row state touched together by the solve: working value, "touched in
    // column j" mark and pivot position, one 16-byte record per row so a
    // random row access costs one cache line.
    struct RowState {
        double x;
        int32_t mark;
        int32_t piv;
    };
    std::vector<RowState> rows(static_cast<size_t>(m), RowState{0.0, -1, -1});

    std::vector<int64_t>& Lp = C.Lp;
    std::vector<int64_t>& Up = C.Up;
    std::vector<int32_t>& Li = C.Li;
    std::vector<int32_t>& Ui = C.Ui;
    std::vector<double>& Lv = C.Lv;
    std::vector<double>& Uv = C.Uv;
    Lp.assign(static_cast<size_t>(n) + 1, 0);
    Up.assign(static_cast<size_t>(n) + 1, 0);
    const size_t guess = std::min<size_t>(size_t(1) << 27,
                                          static_cast<size_t>(n) * static_cast<size_t>(prm.p >= 0 ? prm.p : 16));
    Li.reserve(guess);
    Lv.reserve(guess);
    Ui.reserve(guess);
    Uv.reserve(guess);

    std::vector<int32_t> vmark(static_cast<size_t>(n), -1);
    std::vector<int32_t> touched, reach, stack;
    std::vector<Entry> cand;

    for (int64_t jj = 0; jj < n; ++jj) {
        const int32_t j = static_cast<int32_t>(jj);
        touched.clear();
        reach.clear();
        stack.clear();
        double colinf = 0.0;
        // scatter the scaled column and seed the graph search
        for (int64_t e = ac.ptr[j]; e < ac.ptr[j + 1]; ++e) {
            const int32_t i = ac.idx[e];
            RowState& ri = rows[i];
            ri.x = ac.val[e];
            ri.mark = j;
            touched.push_back(i);
            colinf = std::max(colinf, std::fabs(ac.val[e]));
            const int32_t k = ri.piv;
            if (k >= 0 && vmark[k] != j) {
                vmark[k] = j;
                stack.push_back(k);
            }
        }
        // symbolic: every pivot position reachable through the columns of L
        while (!stack.empty()) {
            const int32_t k = stack.back();
            stack.pop_back();
            reach.push_back(k);
            for (int64_t e = Lp[k]; e < Lp[k + 1]; ++e) {
                const int32_t q = rows[Li[e]].piv;
                if (q >= 0 && vmark[q] != j) {
                    vmark[q] = j;
                    stack.push_back(q);
                }
            }
        }
        std::sort(reach.begin(), reach.end());
        // numeric: unit lower solve in ascending pivot position
        cand.clear();
        // two-stage prefetch: the L column arrays kFar positions ahead, the
        // rows they name kNear positions ahead
        constexpr size_t kNear = 4, kFar = 8;
        for (size_t t = 0; t < std::min(kFar, reach.size()); ++t) {
            __builtin_prefetch(&Li[Lp[reach[t]]]);
            __builtin_prefetch(&Lv[Lp[reach[t]]]);
        }
        for (size_t t = 0; t < std::min(kNear, reach.size()); ++t)
            for (int64_t e = Lp[reach[t]]; e < Lp[reach[t] + 1]; ++e) __builtin_prefetch(&rows[Li[e]], 1);
        for (size_t t = 0; t < reach.size(); ++t) {
            if (t + kFar < reach.size()) {
                const int32_t kf = reach[t + kFar];
                __builtin_prefetch(&Li[Lp[kf]]);
                __builtin_prefetch(&Lv[Lp[kf]]);
                __builtin_prefetch(&rows[R.prow[kf]]);
            }
            if (t + kNear < reach.size()) {
                const int32_t kp = reach[t + kNear];
                for (int64_t e = Lp[kp]; e < Lp[kp + 1]; ++e) __builtin_prefetch(&rows[Li[e]], 1);
            }
            const int32_t k = reach[t];
            const RowState& rp = rows[R.prow[k]];
            const double ukj = (rp.mark == j) ? rp.x : 0.0;
            if (ukj == 0.0) continue;
            cand.push_back({std::fabs(ukj), k, ukj});
            for (int64_t e = Lp[k]; e < Lp[k + 1]; ++e) {
                RowState& ri = rows[Li[e]];
                if (ri.mark != j) {
                    ri.mark = j;
                    ri.x = 0.0;
                    touched.push_back(Li[e]);
                }
                ri.x = ri.x - Lv[e] * ukj;
            }
        }
        dual_drop(cand, prm.p, prm.tau);
        for (const Entry& c : cand) {
            Ui.push_back(c.key);
            Uv.push_back(c.val);
        }
        Up[j + 1] = static_cast<int64_t>(Ui.size());

        // pivot choice
        const double beta = std::pow(10.0, -2.0 * (1.0 - static_cast<double>(jj + 1) / static_cast<double>(n)));
        double modval = beta * colinf;
        if (modval < prm.small) modval = prm.small;
        double maxabs = 0.0;
        bool any = false;
        for (const int32_t i : touched)
            if (rows[i].piv < 0 && rows[i].x != 0.0) {
                any = true;
                maxabs = std::max(maxabs, std::fabs(rows[i].x));
            }
        int32_t r = -1;
        double piv;
        if (!any) {
            for (int64_t i = 0; i < m; ++i)
                if (rows[i].piv < 0 && (r < 0 || rc[i] < rc[r])) r = static_cast<int32_t>(i);
            piv = modval;
            R.nmod++;
        } else {
            const double thr = prm.mu * maxabs;
            double rmag = 0.0;
            for (const int32_t i : touched) {
                if (rows[i].piv >= 0 || rows[i].x == 0.0) continue;
                const double mag = std::fabs(rows[i].x);
                if (!(mag >= thr)) continue;
                bool take = r < 0;
                if (!take) {
                    if (rc[i] != rc[r]) take = rc[i] < rc[r];
                    else if (mag != rmag) take = mag > rmag;
                    else take = i < r;
                }
                if (take) {
                    r = i;
                    rmag = mag;
                }
            }
            piv = rows[r].x;
            if (std::fabs(piv) < prm.small) {
                piv = (piv < 0.0) ? -modval : modval;
                R.nmod++;
            }
        }
        R.Udiag[j] = piv;
        rows[r].piv = j;
        R.prow[j] = r;

        // L part: scale by the pivot, then drop
        cand.clear();
        for (const int32_t i : touched) {
            if (rows[i].piv >= 0 || rows[i].x == 0.0) continue;
            const double l = rows[i].x / piv;
            cand.push_back({std::fabs(l), i, l});
        }
        dual_drop(cand, prm.p, prm.tau);
        for (const Entry& c : cand) {
            Li.push_back(c.key);
            Lv.push_back(c.val);
        }
        Lp[j + 1] = static_cast<int64_t>(Li.size());

        for (int64_t e = ac.ptr[j]; e < ac.ptr[j + 1]; ++e) rc[ac.idx[e]]--;
    }

    C.pivpos.resize(static_cast<size_t>(m));
    for (int64_t i = 0; i < m; ++i) C.pivpos[i] = rows[i].piv;
}

// ---------------------------------------------------------------------------
// Pipelined columns.  Column c's triangular solve over the pivot positions
// k < h uses only columns 0 .. h-1 and their pivots, so once h columns are
// final that part can run while columns h .. c-1 are still being finished.
// W threads take every W-th column each and keep up to D of their columns in
// flight, each in working arrays (a slot) of its own: a thread starts a
// column's solve with h = the number of final columns, and finishes its
// oldest column once column c - 1 is final (checking for that between steps
// of a long solve): the positions h .. c-1 (in ascending order, after all
// smaller ones, as the serial solve takes them), the U drop, the pivot
// choice and the L part.  Every floating-point operation happens on the same
// operands in the same order as in the serial loop, so the factor is the same
// bit for bit.  Solve times are very uneven (a few columns reach thousands of
// pivot positions), which is what the D columns of look-ahead absorb.

struct Touched {
    double x;         // value of the row in this column
    int32_t row;      // original row id
    uint8_t out;      // pivoted (at a position above the horizon, or here)
    uint8_t changed;  // flagged, updated or added while the column is finished
};

// A worker's view of one row, one 16-byte record so a random row access
// costs one cache line.  During the worker's solve `x` is the row's working
// value; afterwards, for a row listed in `act`, it holds the row's index
// there.  `piv` is the row's pivot position if it is below the worker's
// horizon, else -1.
struct WorkerRow {
    double x;
    int32_t mark;  // column that last touched the row
    int32_t piv;
};

// The p + 1 largest magnitudes seen, largest first (a multiset).
struct TopMags {
    std::vector<double> v;
    size_t cap = 0;
    void reset(size_t k) {
        v.clear();
        cap = k;
    }
    void add(double g) {
        if (cap == 0) return;
        if (v.size() == cap) {
            if (!(g > v.back())) return;
            v.pop_back();
        }
        size_t i = v.size();
        v.push_back(g);
        for (; i > 0 && v[i - 1] < g; --i) v[i] = v[i - 1];
        v[i] = g;
    }
};

// Working state of one column in flight.
struct Slot {
    std::vector<WorkerRow> rows;
    std::vector<int32_t> heap;
    std::vector<Touched> act;    // touched rows not pivoted below the horizon
    std::vector<Entry> cand;     // U part, ascending position
    std::vector<Entry> lc;       // L part
    TopMags top;
    int64_t applied = 0;         // pivot positions copied into rows[].piv
    int64_t horizon = 0;         // columns final when the column's solve began
    // The rows the finish is likely to need, listed by the solve: every
    // nonzero with |x| >= big_lo; big_hi (>= big_lo) is at most the
    // (p + 9)-th largest |x| and mu times the largest (0 with fewer than
    // p + 9 nonzeros).  Rows left out are below big_lo.
    std::vector<int32_t> big;
    double big_lo = 0.0, big_hi = 0.0;
    std::vector<int32_t> chg;    // rows changed while finishing
    std::vector<int32_t> sel;    // rows the finish examines
};

struct alignas(64) PaddedCounter {
    std::atomic<int64_t> v{0};
};

class Aborted {};

template <class Ready>
void wait_for(Ready ready, const std::atomic<bool>& abort) {
    for (int spin = 0; !ready(); ++spin) {
        if (abort.load(std::memory_order_relaxed)) throw Aborted();
        if (spin > 64) std::this_thread::yield();
    }
}

// Keep the entries of `c` (those not out and nonzero) that dual_drop keeps
// when each becomes {|x / pv|, row, x / pv}, dividing only the candidates
// that can be kept.  `xp` is the p-th largest |x| among them (0 if there are
// at most p).  x -> fl(x / pv) is monotone in |x|, so an entry clearly
// smaller in |x| than the p-th largest is clearly smaller after the division.
// `sel` (if not null) names the entries of `c` to consider; the others are
// known to be out, zero or below the p-th largest by more than the margin.
void drop_scaled(const std::vector<Touched>& c, const std::vector<int32_t>* sel, double pv, double xp, int p,
                 double tau, std::vector<Entry>& out) {
    out.clear();
    if (p == 0 || c.empty()) return;
    double lo = 0.0;
    // the margin is far above the quotients' rounding; it is not used where a
    // quotient could be subnormal
    if (xp > 0.0 && xp / std::fabs(pv) > 1e-290) lo = xp * (1.0 - 0x1p-40);
    auto take = [&](const Touched& t) {
        if (!t.out && t.x != 0.0 && std::fabs(t.x) >= lo) {
            const double l = t.x / pv;
            out.push_back({std::fabs(l), t.row, l});
        }
    };
    if (sel)
        for (const int32_t s : *sel) take(c[static_cast<size_t>(s)]);
    else
        for (const Touched& t : c) take(t);
    dual_drop(out, p, tau);
}

void columns_pipelined(const HostCSR& a, const HostCSR& ac, const IlupParams& prm, int nthreads, int depth,
                       IlupResult& R, ColumnFactor& C) {
    const int64_t m = a.rows, n = a.cols;
    const int64_t W = nthreads, D = depth;
    const size_t cap = static_cast<size_t>(n) * static_cast<size_t>(prm.p);
    // L storage is appended to while other threads read finished columns,
    // so it never moves: each column keeps at most p entries.
    std::unique_ptr<int32_t[]> Li(new int32_t[cap > 0 ? cap : 1]);
    std::unique_ptr<double[]> Lv(new double[cap > 0 ? cap : 1]);
    std::vector<int64_t>& Lp = C.Lp;
    std::vector<int64_t>& Up = C.Up;
    Lp.assign(static_cast<size_t>(n) + 1, 0);
    Up.assign(static_cast<size_t>(n) + 1, 0);
    C.Ui.reserve(cap);
    C.Uv.reserve(cap);
    std::vector<int32_t>& piv = C.pivpos;  // touched only while finishing a column
    piv.assign(static_cast<size_t>(m), -1);
    std::vector<int32_t> rc(static_cast<size_t>(m));
    for (int64_t i = 0; i < m; ++i) rc[i] = static_cast<int32_t>(a.ptr[i + 1] - a.ptr[i]);

    PaddedCounter done;  // columns final
    std::atomic<bool> abort{false};
    const int32_t* prow = R.prow.data();
    const auto heap_after = std::greater<int32_t>();

    // column c's solve over the positions below the horizon, ascending;
    // poll() is called now and then to finish an older column
    auto solve_below_horizon = [&](Slot& K, int64_t cc, auto&& poll) {
        const int32_t c = static_cast<int32_t>(cc);
        const int64_t horizon = done.v.load(std::memory_order_acquire);
        K.horizon = horizon;
        WorkerRow* rw = K.rows.data();
        for (; K.applied < horizon; ++K.applied) rw[prow[K.applied]].piv = static_cast<int32_t>(K.applied);
        K.act.clear();
        K.cand.clear();
        K.heap.clear();
        for (int64_t e = ac.ptr[c]; e < ac.ptr[c + 1]; ++e) {
            const int32_t i = ac.idx[e];
            WorkerRow& r = rw[i];
            r.x = ac.val[e];
            r.mark = c;
            // a pivot position is queued when its pivot row is first touched
            // in this column, so at most once
            if (r.piv >= 0) {
                K.heap.push_back(r.piv);
            } else {
                K.act.push_back({0.0, i, 0, 0});
            }
        }
        std::make_heap(K.heap.begin(), K.heap.end(), heap_after);
        for (uint32_t step = 1; !K.heap.empty(); ++step) {
            if ((step & 31u) == 0) poll();
            std::pop_heap(K.heap.begin(), K.heap.end(), heap_after);
            const int32_t k = K.heap.back();
            K.heap.pop_back();
            // the rows the next position will update, while this one's are updated
            if (!K.heap.empty()) {
                const int32_t nk = K.heap.front();
                for (int64_t e = Lp[nk]; e < Lp[nk + 1]; ++e) __builtin_prefetch(&rw[Li[e]]);
            }
            const double ukj = rw[prow[k]].x;
            if (ukj == 0.0) continue;
            K.cand.push_back({std::fabs(ukj), k, ukj});
            const int64_t e1 = Lp[k + 1];
            for (int64_t e = Lp[k]; e < e1; ++e) {
                const int32_t i = Li[e];
                WorkerRow& r = rw[i];
                if (r.mark != c) {
                    r.mark = c;
                    r.x = 0.0;
                    const int32_t q = r.piv;
                    if (q >= 0) {
                        K.heap.push_back(q);
                        std::push_heap(K.heap.begin(), K.heap.end(), heap_after);
                        __builtin_prefetch(&Li[Lp[q]]);
                        __builtin_prefetch(&Lv[Lp[q]]);
                    } else {
                        K.act.push_back({0.0, i, 0, 0});
                    }
                }
                r.x = r.x - Lv[e] * ukj;
            }
        }
        for (size_t s = 0; s < K.act.size(); ++s) {
            WorkerRow& r = rw[K.act[s].row];
            K.act[s].x = r.x;
            r.x = static_cast<double>(s);
        }
        // the U drop of these positions now (off the ordered chain): an entry
        // outside their p best is beaten by p entries of the column anyway,
        // so dropping again with the later positions keeps the same ones
        dual_drop(K.cand, prm.p, prm.tau);
        // the rows the finish is likely to need (off the ordered chain)
        K.big.clear();
        const size_t want = static_cast<size_t>(prm.p) + 9;
        K.top.reset(want);
        double mw = 0.0, gate = -1.0;
        for (const Touched& t : K.act)
            if (t.x != 0.0) {
                const double g = std::fabs(t.x);
                mw = std::max(mw, g);
                if (g > gate) {
                    K.top.add(g);
                    if (K.top.v.size() == want) gate = K.top.v.back();
                }
            }
        K.big_hi = K.big_lo = 0.0;
        if (K.top.v.size() == want) {
            K.big_hi = std::min(K.top.v.back(), prm.mu * mw * (1.0 - 0x1p-30));
            K.big_lo = K.big_hi * (1.0 - 0x1p-30);
        }
        for (size_t s = 0; s < K.act.size(); ++s)
            if (K.act[s].x != 0.0 && std::fabs(K.act[s].x) >= K.big_lo) K.big.push_back(static_cast<int32_t>(s));
    };

    // the rest of column j, once columns 0 .. j-1 are final
    auto finish_column = [&](Slot& K, int64_t jj) {
        const int32_t j = static_cast<int32_t>(jj);
        WorkerRow* rw = K.rows.data();
        // the positions from the horizon on, ascending
        for (int64_t k = K.horizon; k < jj; ++k) __builtin_prefetch(&rw[prow[k]]);
        K.chg.clear();
        auto changed = [&](size_t s) {
            if (!K.act[s].changed) {
                K.act[s].changed = 1;
                K.chg.push_back(static_cast<int32_t>(s));
            }
        };
        for (int64_t k = K.horizon; k < jj; ++k) {
            const WorkerRow& pr = rw[prow[k]];
            if (pr.mark != j) continue;
            const size_t ps = static_cast<size_t>(pr.x);
            K.act[ps].out = 1;
            changed(ps);
            const double ukj = K.act[ps].x;
            if (ukj == 0.0) continue;
            K.cand.push_back({std::fabs(ukj), static_cast<int32_t>(k), ukj});
            for (int64_t e = Lp[k]; e < Lp[k + 1]; ++e) {
                const int32_t i = Li[e];
                WorkerRow& r = rw[i];
                if (r.mark != j) {
                    r.mark = j;
                    r.x = static_cast<double>(K.act.size());
                    K.act.push_back({0.0, i, 0, 0});
                }
                const size_t ts = static_cast<size_t>(r.x);
                changed(ts);
                Touched& t = K.act[ts];
                t.x = t.x - Lv[e] * ukj;
            }
        }
        dual_drop(K.cand, prm.p, prm.tau);
        for (const Entry& c : K.cand) {
            C.Ui.push_back(c.key);
            C.Uv.push_back(c.val);
        }
        Up[j + 1] = static_cast<int64_t>(C.Ui.size());

        // Pivot choice (Algorithms 5 and 6) among the unpivoted nonzeros.  The
        // rows examined first are the solve's list (unchanged ones) and the
        // changed ones; every other row is below big_lo, so they decide alone
        // when the largest and the threshold are at least big_lo.  Otherwise
        // all rows are examined.
        K.sel.clear();
        for (const int32_t s : K.big)
            if (!K.act[static_cast<size_t>(s)].changed) K.sel.push_back(s);
        for (const int32_t s : K.chg) K.sel.push_back(s);
        double maxabs = 0.0;
        size_t neligible = 0;
        for (const int32_t s : K.sel) {
            const Touched& t = K.act[static_cast<size_t>(s)];
            if (!t.out && t.x != 0.0) {
                ++neligible;
                maxabs = std::max(maxabs, std::fabs(t.x));
            }
        }
        bool listed = neligible > 0 && maxabs >= K.big_lo && prm.mu * maxabs >= K.big_lo;
        if (!listed) {
            maxabs = 0.0;
            neligible = 0;
            for (const Touched& t : K.act)
                if (!t.out && t.x != 0.0) {
                    ++neligible;
                    maxabs = std::max(maxabs, std::fabs(t.x));
                }
        }
        double colinf = 0.0;
        for (int64_t e = ac.ptr[j]; e < ac.ptr[j + 1]; ++e) colinf = std::max(colinf, std::fabs(ac.val[e]));
        const double modval = modified_pivot(colinf, jj, n, prm.small);
        int32_t r = -1;
        double pv;
        if (neligible == 0) {
            for (int64_t i = 0; i < m; ++i)
                if (piv[i] < 0 && (r < 0 || rc[i] < rc[r])) r = static_cast<int32_t>(i);
            pv = modval;
            R.nmod++;
        } else {
            const double thr = prm.mu * maxabs;
            double rmag = 0.0;
            size_t rslot = 0;
            auto consider = [&](size_t s) {
                const Touched& t = K.act[s];
                const double mag = std::fabs(t.x);
                if (t.out || t.x == 0.0 || !(mag >= thr)) return;
                const int32_t i = t.row;
                bool take = r < 0;
                if (!take) {
                    if (rc[i] != rc[r]) take = rc[i] < rc[r];
                    else if (mag != rmag) take = mag > rmag;
                    else take = i < r;
                }
                if (take) {
                    r = i;
                    rmag = mag;
                    rslot = s;
                }
            };
            if (listed)
                for (const int32_t s : K.sel) consider(static_cast<size_t>(s));
            else
                for (size_t s = 0; s < K.act.size(); ++s) consider(s);
            pv = K.act[rslot].x;
            if (std::fabs(pv) < prm.small) {
                pv = (pv < 0.0) ? -modval : modval;
                R.nmod++;
            }
            K.act[rslot].out = 1;
        }
        R.Udiag[j] = pv;
        R.prow[j] = r;
        piv[r] = j;

        // L part: scale by the pivot, then drop.  The p-th largest |x| among
        // the remaining rows comes from the examined rows when at least p of
        // them reach big_hi (every other row is then below it by more than
        // the margin drop_scaled uses); otherwise from all rows.
        const size_t pp = static_cast<size_t>(prm.p);
        K.top.reset(pp + 1);
        size_t nhi = 0;
        if (listed && pp > 0) {
            for (const int32_t s : K.sel) {
                const Touched& t = K.act[static_cast<size_t>(s)];
                if (t.out || t.x == 0.0) continue;
                const double g = std::fabs(t.x);
                if (g >= K.big_hi) ++nhi;
                K.top.add(g);
            }
        }
        if (pp > 0 && listed && nhi >= pp) {
            drop_scaled(K.act, &K.sel, pv, K.top.v[pp - 1], prm.p, prm.tau, K.lc);
        } else {
            K.top.reset(pp + 1);
            double gate = -1.0;
            size_t nrest = 0;
            for (const Touched& t : K.act)
                if (!t.out && t.x != 0.0) {
                    ++nrest;
                    const double g = std::fabs(t.x);
                    if (g > gate) {
                        K.top.add(g);
                        if (K.top.v.size() == K.top.cap) gate = K.top.v.back();
                    }
                }
            const double xp = (pp > 0 && nrest > pp) ? K.top.v[pp - 1] : 0.0;
            drop_scaled(K.act, nullptr, pv, xp, prm.p, prm.tau, K.lc);
        }
        int64_t at = Lp[j];
        for (const Entry& c : K.lc) {
            Li[at] = c.key;
            Lv[at] = c.val;
            ++at;
        }
        Lp[j + 1] = at;

        for (int64_t e = ac.ptr[j]; e < ac.ptr[j + 1]; ++e) rc[ac.idx[e]]--;
    };

    std::vector<std::exception_ptr> errs(static_cast<size_t>(W));
    auto run = [&](int64_t w) {
        try {
            // this thread's slots, allocated (and first touched) here
            std::vector<std::unique_ptr<Slot>> slots;
            for (int64_t d = 0; d < D && w + d * W < n; ++d) {
                std::unique_ptr<Slot> k(new Slot());
                k->rows.assign(static_cast<size_t>(m), WorkerRow{0.0, -1, -1});
                slots.push_back(std::move(k));
            }
            auto slot_of = [&](int64_t c) -> Slot& { return *slots[static_cast<size_t>((c / W) % D)]; };
            // this thread's columns whose solve is done, oldest first
            std::vector<int64_t> pending;
            size_t head = 0;
            auto finish_ready = [&]() {
                while (head < pending.size() && done.v.load(std::memory_order_acquire) == pending[head]) {
                    const int64_t c = pending[head++];
                    finish_column(slot_of(c), c);
                    done.v.store(c + 1, std::memory_order_release);
                }
            };
            for (int64_t next = w; next < n || head < pending.size();) {
                if (next < n && pending.size() - head < static_cast<size_t>(D)) {
                    solve_below_horizon(slot_of(next), next, finish_ready);
                    pending.push_back(next);
                    next += W;
                } else {
                    const int64_t c = pending[head];
                    wait_for([&]() { return done.v.load(std::memory_order_acquire) >= c; }, abort);
                }
                finish_ready();
            }
        } catch (const Aborted&) {
        } catch (...) {
            errs[static_cast<size_t>(w)] = std::current_exception();
            abort.store(true);
        }
    };
    std::vector<std::thread> threads;
    try {
        for (int64_t w = 1; w < W; ++w) threads.emplace_back(run, w);
    } catch (...) {
        abort.store(true);
        for (auto& t : threads) t.join();
        throw;
    }
    run(0);
    for (auto& t : threads) t.join();
    for (const auto& e : errs)
        if (e) std::rethrow_exception(e);

    C.Li.assign(Li.get(), Li.get() + Lp[n]);
    C.Lv.assign(Lv.get(), Lv.get() + Lp[n]);
}

// The split (pivot rows in pivot order form L1, the rest in ascending id L2),
// U by rows, the transposes and the level sets.
void split_and_analyse(IlupResult& R, const ColumnFactor& C, int threads) {
    const int64_t m = R.m, n = R.n;
    const int64_t m2 = m - n;
    const std::vector<int32_t>& pivpos = C.pivpos;
    const std::vector<int64_t>& Lp = C.Lp;
    const std::vector<int64_t>& Up = C.Up;
    const std::vector<int32_t>& Li = C.Li;
    const std::vector<int32_t>& Ui = C.Ui;
    const std::vector<double>& Lv = C.Lv;
    const std::vector<double>& Uv = C.Uv;
    std::vector<int32_t> a2idx(static_cast<size_t>(m), -1);
    R.a2rows.reserve(static_cast<size_t>(m2));
    for (int64_t i = 0; i < m; ++i)
        if (pivpos[i] < 0) {
            a2idx[i] = static_cast<int32_t>(R.a2rows.size());
            R.a2rows.push_back(static_cast<int32_t>(i));
        }
    // L by rows: row label(i) holds original row i's multipliers in ascending
    // position, with the pivot rows first (in pivot order) and the rows of A2
    // after them (ascending id)
    {
        std::vector<int32_t> label(static_cast<size_t>(m));
        for (int64_t i = 0; i < m; ++i)
            label[i] = pivpos[i] >= 0 ? pivpos[i] : static_cast<int32_t>(n + a2idx[i]);
        HostCSR LL;
        transpose_into(n, m, Lp.data(), Li.data(), Lv.data(), label.data(), threads, LL);
        const int64_t cut = LL.ptr[n];
        R.L1.rows = n; R.L1.cols = n;
        R.L1.ptr.assign(LL.ptr.begin(), LL.ptr.begin() + n + 1);
        R.L1.idx.assign(LL.idx.begin(), LL.idx.begin() + cut);
        R.L1.val.assign(LL.val.begin(), LL.val.begin() + cut);
        R.L2.rows = m2; R.L2.cols = n;
        R.L2.ptr.resize(static_cast<size_t>(m2) + 1);
        for (int64_t r = 0; r <= m2; ++r) R.L2.ptr[r] = LL.ptr[n + r] - cut;
        R.L2.idx.assign(LL.idx.begin() + cut, LL.idx.end());
        R.L2.val.assign(LL.val.begin() + cut, LL.val.end());
    }
    transpose_into(n, n, Up.data(), Ui.data(), Uv.data(), nullptr, threads, R.U);
    // transposes and level sets: independent of each other, built on three
    // threads (each result is deterministic)
    {
        std::exception_ptr e1, e2;
        std::thread t1([&R, &e1]() {
            try {
                R.L1t = transpose(R.L1);
                R.lev_L1 = analyse_levels(R.L1, true);
                R.lev_L1t = analyse_levels(R.L1t, false);
            } catch (...) {
                e1 = std::current_exception();
            }
        });
        std::thread t2([&R, &e2]() {
            try {
                R.Ut = transpose(R.U);
                R.lev_U = analyse_levels(R.U, false);
                R.lev_Ut = analyse_levels(R.Ut, true);
            } catch (...) {
                e2 = std::current_exception();
            }
        });
        std::exception_ptr e0;
        try {
            R.L2t = transpose(R.L2);
        } catch (...) {
            e0 = std::current_exception();
        }
        t1.join();
        t2.join();
        for (const auto& e : {e0, e1, e2})
            if (e) std::rethrow_exception(e);
    }
}

}  // namespace

namespace {

// Working arrays of one column in flight: 16 bytes per row of A.
int64_t slot_bytes(int64_t m) {
    return 16 * std::max<int64_t>(m, 1);
}

// Columns in flight per thread: up to 8 while all slots fit in 2 GiB; one
// for a single thread, which never waits for another.
int ilup_depth(int threads, int64_t m) {
    if (threads <= 1) return 1;
    const int64_t fit = (int64_t(1) << 31) / (slot_bytes(m) * std::max(threads, 1));
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(8, fit)));
}

}  // namespace

// CPUs this process may run on (its affinity mask; the whole machine where
// that cannot be read).
int usable_cpus() {
#if defined(__linux__)
    cpu_set_t set;
    CPU_ZERO(&set);
    if (sched_getaffinity(0, sizeof(set), &set) == 0) return std::max(1, CPU_COUNT(&set));
#endif
    return static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
}

int ilup_threads(int requested, int64_t m, int64_t n) {
    (void)n;
    int64_t t = requested > 0 ? std::min(requested, 64) : std::min(16, usable_cpus());
    t = std::min<int64_t>(t, std::max<int64_t>(1, (int64_t(1) << 31) / slot_bytes(m)));
    return static_cast<int>(t);
}

IlupResult ilup_factor(const HostCSR& a, const IlupParams& prm) {
    const int64_t m = a.rows, n = a.cols;
    if (!(m > n && n > 0)) throw std::runtime_error("need m > n > 0");
    IlupResult R;
    R.m = m;
    R.n = n;
    if (prm.scale) {
        if (!column_scaling(a, R.d)) throw std::runtime_error("A has an empty column");
    } else {
        R.d.assign(static_cast<size_t>(n), 1.0);
    }

    // scaled matrix by columns, rows ascending in each column
    HostCSR ac;
    transpose_into(a.rows, a.cols, a.ptr.data(), a.idx.data(), a.val.data(), nullptr, prm.threads, ac);
    for (int64_t j = 0; j < n; ++j) {
        if (ac.ptr[j + 1] == ac.ptr[j]) throw std::runtime_error("A has an empty column");
        for (int64_t e = ac.ptr[j]; e < ac.ptr[j + 1]; ++e) ac.val[e] = ac.val[e] * R.d[j];
    }
    R.prow.assign(static_cast<size_t>(n), -1);
    R.Udiag.assign(static_cast<size_t>(n), 0.0);

    ColumnFactor C;
    // The pipelined loop (also on one thread, where it is the faster of the
    // two) stores L in place, so it needs a bound on the entries of an L column
    // (p >= 0) that keeps n p entries to a sensible size (2^27).  If the system
    // refuses a thread, the serial loop does the work instead.
    bool serial = !(prm.p >= 0 && prm.threads >= 1 &&
                    static_cast<double>(n) * static_cast<double>(prm.p) <= static_cast<double>(int64_t(1) << 27));
    if (!serial) {
        try {
            columns_pipelined(a, ac, prm, prm.threads, ilup_depth(prm.threads, m), R, C);
        } catch (const std::system_error&) {
            R.prow.assign(static_cast<size_t>(n), -1);
            R.Udiag.assign(static_cast<size_t>(n), 0.0);
            R.nmod = 0;
            C = ColumnFactor();
            serial = true;
        }
    }
    if (serial) columns_serial(a, ac, prm, R, C);
    split_and_analyse(R, C, prm.threads);
    return R;
}

namespace {

// Rows of a fused system, built in level order.  group_of(level) names the
// group of every level already processed; a row's dependencies on rows of its
// own group are substituted (x_j = (rhs_j + sum_Rj c rhs - sum_Tj c x) / d_j,
// so the rows those come from must already be final), the others stay.
struct Fuser {
    const HostCSR& strict;
    const double* diag;
    const Levels& lev;
    // the rows built so far, appended to one arena each for T and R (a row
    // built again is appended again; its newest copy counts)
    struct Span {
        int64_t at = 0;
        int32_t len = 0;
    };
    std::vector<Span> Tspan, Rspan;
    std::vector<int32_t> Tcol, Rcol;
    std::vector<double> Tval, Rval;
    std::vector<double> accT, accR;
    std::vector<int64_t> markT, markR;  // stamp of the build that last touched a column
    std::vector<int32_t> listT, listR;
    int64_t stamp = 0;
    Fuser(const HostCSR& s, const double* d, const Levels& l)
        : strict(s), diag(d), lev(l), Tspan(static_cast<size_t>(s.rows)), Rspan(static_cast<size_t>(s.rows)),
          accT(static_cast<size_t>(s.rows), 0.0), accR(static_cast<size_t>(s.rows), 0.0),
          markT(static_cast<size_t>(s.rows), -1), markR(static_cast<size_t>(s.rows), -1) {
        Tcol.reserve(static_cast<size_t>(s.nnz()));
        Tval.reserve(static_cast<size_t>(s.nnz()));
    }

    // builds (or rebuilds) row i for group g of its level; returns its stored entries
    template <class GroupOf>
    int64_t build(int32_t i, int32_t g, const GroupOf& group_of) {
        const int64_t b = stamp++;
        listT.clear();
        listR.clear();
        auto addT = [&](int32_t c, double v) {
            if (markT[c] != b) { markT[c] = b; accT[c] = 0.0; listT.push_back(c); }
            accT[c] += v;
        };
        auto addR = [&](int32_t c, double v) {
            if (markR[c] != b) { markR[c] = b; accR[c] = 0.0; listR.push_back(c); }
            accR[c] += v;
        };
        for (int64_t e = strict.ptr[i]; e < strict.ptr[i + 1]; ++e) {
            const int32_t j = strict.idx[e];
            const double a = strict.val[e];
            if (group_of(lev.level[j]) != g) {
                addT(j, a);
                continue;
            }
            const double f = diag ? a / diag[j] : a;
            addR(j, -f);
            const Span rj = Rspan[j], tj = Tspan[j];
            for (int32_t q = 0; q < rj.len; ++q) addR(Rcol[rj.at + q], -f * Rval[rj.at + q]);
            for (int32_t q = 0; q < tj.len; ++q) addT(Tcol[tj.at + q], -f * Tval[tj.at + q]);
        }
        std::sort(listT.begin(), listT.end());
        std::sort(listR.begin(), listR.end());
        Tspan[i] = Span{static_cast<int64_t>(Tcol.size()), static_cast<int32_t>(listT.size())};
        for (int32_t c : listT) {
            Tcol.push_back(c);
            Tval.push_back(accT[c]);
        }
        Rspan[i] = Span{static_cast<int64_t>(Rcol.size()), static_cast<int32_t>(listR.size())};
        for (int32_t c : listR) {
            Rcol.push_back(c);
            Rval.push_back(accR[c]);
        }
        return static_cast<int64_t>(listT.size() + listR.size());
    }

    void finish(MergedTri& M) {
        const int64_t n = strict.rows;
        auto to_csr = [&](const std::vector<Span>& span, const std::vector<int32_t>& col,
                          const std::vector<double>& val, HostCSR& out) {
            out.rows = n;
            out.cols = n;
            out.ptr.assign(static_cast<size_t>(n) + 1, 0);
            for (int64_t i = 0; i < n; ++i) out.ptr[i + 1] = out.ptr[i] + span[i].len;
            out.idx.resize(static_cast<size_t>(out.ptr[n]));
            out.val.resize(static_cast<size_t>(out.ptr[n]));
            for (int64_t i = 0; i < n; ++i) {
                std::copy(col.begin() + span[i].at, col.begin() + span[i].at + span[i].len, out.idx.begin() + out.ptr[i]);
                std::copy(val.begin() + span[i].at, val.begin() + span[i].at + span[i].len, out.val.begin() + out.ptr[i]);
            }
        };
        to_csr(Tspan, Tcol, Tval, M.T);
        to_csr(Rspan, Rcol, Rval, M.R);
        // lower systems depend on smaller ids, upper ones on larger ids; the
        // merged dependencies keep that direction
        bool lower = true;
        for (int64_t i = 0; i < n && lower; ++i)
            for (int64_t e = strict.ptr[i]; e < strict.ptr[i + 1]; ++e)
                if (strict.idx[e] > i) { lower = false; break; }
        M.lev = analyse_levels(M.T, lower);
    }
};

MergedTri unmerged(const HostCSR& strict, const Levels& lev) {
    MergedTri M;
    M.k = 1;
    M.T = strict;
    M.R.rows = strict.rows;
    M.R.cols = strict.rows;
    M.R.ptr.assign(static_cast<size_t>(strict.rows) + 1, 0);
    M.lev = lev;
    return M;
}

}  // namespace

MergedTri merge_levels(const HostCSR& strict, const double* diag, const Levels& lev, int k, int64_t max_nnz) {
    if (k <= 1) return unmerged(strict, lev);
    MergedTri M;
    M.k = k;
    Fuser fz(strict, diag, lev);
    auto group_of = [k](int32_t l) { return l / k; };
    int64_t total = 0;
    for (int64_t t = 0; t < strict.rows; ++t) {
        const int32_t i = lev.order[t];
        total += fz.build(i, group_of(lev.level[i]), group_of);
        if (max_nnz > 0 && total > max_nnz) {
            M.k = 0;  // too much fill: rejected
            return M;
        }
    }
    fz.finish(M);
    return M;
}

MergedTri merge_levels_adaptive(const HostCSR& strict, const double* diag, const Levels& lev,
                                double level_entries, int max_group) {
    if (lev.nlevels <= 1 || max_group <= 1) return unmerged(strict, lev);
    MergedTri M;
    Fuser fz(strict, diag, lev);
    std::vector<int32_t> gid(static_cast<size_t>(lev.nlevels), 0);
    auto group_of = [&gid](int32_t l) { return gid[static_cast<size_t>(l)]; };
    int32_t cur = 0, start = 0, widest = 1;
    for (int32_t l = 0; l < lev.nlevels; ++l) {
        const int32_t lo = lev.level_ptr[l], hi = lev.level_ptr[l + 1];
        bool joined = false;
        if (l > 0 && l - start < max_group) {
            // tentatively in the current group: the fill it adds against the
            // cost of one more level
            gid[l] = cur;
            int64_t grown = 0;
            for (int32_t t = lo; t < hi; ++t) {
                const int32_t i = lev.order[t];
                grown += fz.build(i, cur, group_of) - (strict.ptr[i + 1] - strict.ptr[i]);
            }
            joined = static_cast<double>(grown) <= level_entries;
        }
        if (!joined) {
            if (l > 0) ++cur;
            start = l;
            gid[l] = cur;
            for (int32_t t = lo; t < hi; ++t) fz.build(lev.order[t], cur, group_of);
        }
        widest = std::max(widest, l - start + 1);
    }
    M.k = widest;
    M.adaptive = true;
    fz.finish(M);
    return M;
}

void add_rows(IlupResult& F, const HostCSR& rows, const IlupParams& prm) {
    const int64_t n = F.n, k = rows.rows;
    if (rows.cols != n) throw std::invalid_argument("added rows must have n columns");
    std::vector<double> rhs(static_cast<size_t>(n)), l(static_cast<size_t>(n));
    std::vector<Entry> cand;
    HostCSR& L2 = F.L2;
    for (int64_t t = 0; t < k; ++t) {
        std::fill(rhs.begin(), rhs.end(), 0.0);
        for (int64_t e = rows.ptr[t]; e < rows.ptr[t + 1]; ++e) {
            const int32_t j = rows.idx[e];
            if (j < 0 || j >= n) throw std::invalid_argument("column index out of range");
            rhs[j] = rows.val[e] * F.d[j];
        }
        // U^T l = rhs: rows of Ut are positions, entries ascending, then the pivot
        for (int64_t i = 0; i < n; ++i) {
            double s = rhs[i];
            for (int64_t e = F.Ut.ptr[i]; e < F.Ut.ptr[i + 1]; ++e) s = s - F.Ut.val[e] * l[F.Ut.idx[e]];
            l[i] = s / F.Udiag[i];
        }
        cand.clear();
        for (int64_t q = 0; q < n; ++q)
            if (l[q] != 0.0) cand.push_back({std::fabs(l[q]), static_cast<int32_t>(q), l[q]});
        dual_drop(cand, prm.p, prm.tau);
        for (const Entry& c : cand) {
            L2.idx.push_back(c.key);
            L2.val.push_back(c.val);
        }
        L2.ptr.push_back(static_cast<int64_t>(L2.idx.size()));
        F.a2rows.push_back(static_cast<int32_t>(F.m + t));
    }
    L2.rows += k;
    F.m += k;
    F.L2t = transpose(L2);
}

void remove_rows(IlupResult& F, const std::vector<int32_t>& ids) {
    const int64_t m = F.m;
    if (static_cast<int64_t>(ids.size()) >= m - F.n)
        throw std::length_error("at least one row of A2 must remain (m > n)");
    std::vector<char> gone(static_cast<size_t>(m), 0);
    std::vector<char> pivot(static_cast<size_t>(m), 0);
    for (const int32_t r : F.prow) pivot[static_cast<size_t>(r)] = 1;
    for (size_t t = 0; t < ids.size(); ++t) {
        const int32_t r = ids[t];
        if (r < 0 || r >= m || (t > 0 && r <= ids[t - 1]))
            throw std::invalid_argument("row ids must be ascending, distinct and in range");
        if (pivot[static_cast<size_t>(r)]) throw std::invalid_argument("a pivot row cannot be removed without refactorising");
        gone[static_cast<size_t>(r)] = 1;
    }
    std::vector<int32_t> newid(static_cast<size_t>(m), -1);
    int32_t next = 0;
    for (int64_t i = 0; i < m; ++i)
        if (!gone[static_cast<size_t>(i)]) newid[static_cast<size_t>(i)] = next++;
    HostCSR L2;
    L2.cols = F.L2.cols;
    L2.ptr.push_back(0);
    std::vector<int32_t> a2;
    for (size_t c = 0; c < F.a2rows.size(); ++c) {
        const int32_t orig = F.a2rows[c];
        if (gone[static_cast<size_t>(orig)]) continue;
        for (int64_t e = F.L2.ptr[c]; e < F.L2.ptr[c + 1]; ++e) {
            L2.idx.push_back(F.L2.idx[e]);
            L2.val.push_back(F.L2.val[e]);
        }
        L2.ptr.push_back(static_cast<int64_t>(L2.idx.size()));
        a2.push_back(newid[static_cast<size_t>(orig)]);
    }
    L2.rows = static_cast<int64_t>(a2.size());
    for (auto& r : F.prow) r = newid[static_cast<size_t>(r)];
    F.L2 = std::move(L2);
    F.L2t = transpose(F.L2);
    F.a2rows = std::move(a2);
    F.m = m - static_cast<int64_t>(ids.size());
}

bool dense_schur_inverse(const IlupResult& f, std::vector<double>& sinv, int threads, std::vector<double>* keep_z) {
    const int64_t n = f.n, m2 = f.m - f.n;
    if (m2 <= 0) {
        sinv.clear();
        return true;
    }
    if (threads < 1) threads = 1;
    // Z(:, c) = L1^{-T} L2(c, :)^T, stored column-major (n x m2)
    std::vector<double> Z(static_cast<size_t>(n * m2), 0.0);
    auto zcols = [&](int64_t c0, int64_t c1) {
        for (int64_t c = c0; c < c1; ++c) {
            double* z = Z.data() + c * n;
            for (int64_t e = f.L2.ptr[c]; e < f.L2.ptr[c + 1]; ++e) z[f.L2.idx[e]] = f.L2.val[e];
            // unit upper solve with L1^T: z_i -= sum_{k > i} L1t(i, k) z_k, i descending
            for (int64_t i = n - 1; i >= 0; --i) {
                double s = z[i];
                for (int64_t e = f.L1t.ptr[i]; e < f.L1t.ptr[i + 1]; ++e) s -= f.L1t.val[e] * z[f.L1t.idx[e]];
                z[i] = s;
            }
        }
    };
    auto par = [&](int64_t count, auto&& body) {
        std::vector<std::thread> th;
        const int64_t chunk = (count + threads - 1) / threads;
        for (int t = 0; t < threads; ++t) {
            const int64_t lo = t * chunk, hi = std::min(count, lo + chunk);
            if (lo < hi) th.emplace_back(body, lo, hi);
        }
        for (auto& x : th) x.join();
    };
    par(m2, zcols);
    // S = I + Z^T Z (lower triangle, row-major).  Each entry is one running
    // sum over the rows in ascending order, kept in S between chunks of rows
    // so that a chunk of every column stays in cache while all pairs use it;
    // 4 x 4 tiles of column pairs (each owned by one thread) keep 16
    // independent sums going.
    std::vector<double> S(static_cast<size_t>(m2 * m2), 0.0);
    const int64_t nt = (m2 + 3) / 4;
    constexpr int64_t kChunk = 512;
    par(threads, [&](int64_t t0, int64_t t1) {
        for (int64_t i0 = 0; i0 < n; i0 += kChunk) {
            const int64_t i1 = std::min(n, i0 + kChunk);
            int64_t tile = 0;
            for (int64_t ta = 0; ta < nt; ++ta)
                for (int64_t tb = 0; tb <= ta; ++tb, ++tile) {
                    if (tile % threads < t0 || tile % threads >= t1) continue;
                    const int64_t a0 = 4 * ta, b0 = 4 * tb;
                    if (a0 + 4 <= m2 && b0 + 4 <= m2) {
                        double acc[4][4];
                        for (int x = 0; x < 4; ++x)
                            for (int y = 0; y < 4; ++y) acc[x][y] = S[(a0 + x) * m2 + b0 + y];
                        const double* za = Z.data() + a0 * n;
                        const double* zb = Z.data() + b0 * n;
                        for (int64_t i = i0; i < i1; ++i) {
                            const double u0 = za[i], u1 = za[n + i], u2 = za[2 * n + i], u3 = za[3 * n + i];
                            const double v0 = zb[i], v1 = zb[n + i], v2 = zb[2 * n + i], v3 = zb[3 * n + i];
                            acc[0][0] += u0 * v0; acc[0][1] += u0 * v1; acc[0][2] += u0 * v2; acc[0][3] += u0 * v3;
                            acc[1][0] += u1 * v0; acc[1][1] += u1 * v1; acc[1][2] += u1 * v2; acc[1][3] += u1 * v3;
                            acc[2][0] += u2 * v0; acc[2][1] += u2 * v1; acc[2][2] += u2 * v2; acc[2][3] += u2 * v3;
                            acc[3][0] += u3 * v0; acc[3][1] += u3 * v1; acc[3][2] += u3 * v2; acc[3][3] += u3 * v3;
                        }
                        for (int x = 0; x < 4; ++x)
                            for (int y = 0; y < 4; ++y) S[(a0 + x) * m2 + b0 + y] = acc[x][y];
                    } else {
                        for (int64_t a = a0; a < std::min(m2, a0 + 4); ++a)
                            for (int64_t b = b0; b < std::min(m2, b0 + 4); ++b) {
                                const double* za = Z.data() + a * n;
                                const double* zb = Z.data() + b * n;
                                double acc = S[a * m2 + b];
                                for (int64_t i = i0; i < i1; ++i) acc += za[i] * zb[i];
                                S[a * m2 + b] = acc;
                            }
                    }
                }
        }
    });
    for (int64_t a = 0; a < m2; ++a) S[a * m2 + a] = 1.0 + S[a * m2 + a];
    if (keep_z)
        keep_z->swap(Z);
    Z.clear();
    Z.shrink_to_fit();
    // Cholesky S = G G^T in place (lower)
    for (int64_t j = 0; j < m2; ++j) {
        double s = S[j * m2 + j];
        for (int64_t k = 0; k < j; ++k) s -= S[j * m2 + k] * S[j * m2 + k];
        if (!(s > 0.0)) return false;
        const double g = std::sqrt(s);
        S[j * m2 + j] = g;
        for (int64_t i = j + 1; i < m2; ++i) {
            double t = S[i * m2 + j];
            for (int64_t k = 0; k < j; ++k) t -= S[i * m2 + k] * S[j * m2 + k];
            S[i * m2 + j] = t / g;
        }
    }
    // W = G^{-1} (lower), then S^{-1} = W^T W
    std::vector<double> W(static_cast<size_t>(m2 * m2), 0.0);
    par(m2, [&](int64_t c0, int64_t c1) {
        for (int64_t c = c0; c < c1; ++c) {
            // column c of G^{-1}: forward substitution with e_c
            for (int64_t i = c; i < m2; ++i) {
                double s = (i == c) ? 1.0 : 0.0;
                for (int64_t k = c; k < i; ++k) s -= S[i * m2 + k] * W[k * m2 + c];
                W[i * m2 + c] = s / S[i * m2 + i];
            }
        }
    });
    sinv.assign(static_cast<size_t>(m2 * m2), 0.0);
    par(m2, [&](int64_t a0, int64_t a1) {
        for (int64_t a = a0; a < a1; ++a)
            for (int64_t b = 0; b < m2; ++b) {
                double s = 0.0;
                for (int64_t k = std::max(a, b); k < m2; ++k) s += W[k * m2 + a] * W[k * m2 + b];
                sinv[a * m2 + b] = s;
            }
    });
    return true;
}

void schur_inverse_add(const IlupResult& F, int64_t k, std::vector<double>& sinv, std::vector<double>& Z) {
    const int64_t n = F.n, m2 = F.m - F.n, s0 = m2 - k;
    if (k < 0 || s0 < 0 || static_cast<int64_t>(sinv.size()) != s0 * s0 ||
        static_cast<int64_t>(Z.size()) != s0 * n)
        throw std::invalid_argument("the inverse does not match the rows of A2");
    std::vector<double> X(sinv), ZZ(Z), b, u, Y;
    ZZ.resize(static_cast<size_t>(m2 * n), 0.0);
    for (int64_t r = s0; r < m2; ++r) {
        const int64_t sz = r;  // the inverse held is sz x sz
        // z = L1^{-T} l_r^T (column r of Z): unit upper solve with L1^T, i descending
        double* z = ZZ.data() + r * n;
        for (int64_t e = F.L2.ptr[r]; e < F.L2.ptr[r + 1]; ++e) z[F.L2.idx[e]] = F.L2.val[e];
        for (int64_t i = n - 1; i >= 0; --i) {
            double t = z[i];
            for (int64_t e = F.L1t.ptr[i]; e < F.L1t.ptr[i + 1]; ++e) t -= F.L1t.val[e] * z[F.L1t.idx[e]];
            z[i] = t;
        }
        // the border b_a = z_a . z and the corner 1 + z . z: the entries the
        // formation of S would compute, summed in the same order
        b.assign(static_cast<size_t>(sz), 0.0);
        for (int64_t a = 0; a < sz; ++a) {
            const double* za = ZZ.data() + a * n;
            double t = 0.0;
            for (int64_t i = 0; i < n; ++i) t += z[i] * za[i];
            b[a] = t;
        }
        double zz = 0.0;
        for (int64_t i = 0; i < n; ++i) zz += z[i] * z[i];
        const double c = 1.0 + zz;
        // u = S^{-1} b, sigma = c - b . u; the new inverse is
        // [X + u u^T / sigma, -u / sigma; -u^T / sigma, 1 / sigma]
        u.assign(static_cast<size_t>(sz), 0.0);
        for (int64_t a = 0; a < sz; ++a) {
            double t = 0.0;
            for (int64_t q = 0; q < sz; ++q) t += X[a * sz + q] * b[q];
            u[a] = t;
        }
        double sigma = c;
        for (int64_t a = 0; a < sz; ++a) sigma -= b[a] * u[a];
        // sigma >= 1 in exact arithmetic; computed as c - b.u it keeps about
        // log10(c / sigma) fewer digits, so past 4 the inverse is formed again
        if (!(sigma > 0.0) || c > 1e4 * sigma) throw std::runtime_error("the bordered S loses too many digits");
        const int64_t nz = sz + 1;
        Y.assign(static_cast<size_t>(nz * nz), 0.0);
        for (int64_t a = 0; a < sz; ++a) {
            for (int64_t q = 0; q < sz; ++q) Y[a * nz + q] = X[a * sz + q] + u[a] * u[q] / sigma;
            Y[a * nz + sz] = -u[a] / sigma;
            Y[sz * nz + a] = -u[a] / sigma;
        }
        Y[sz * nz + sz] = 1.0 / sigma;
        X.swap(Y);
    }
    sinv.swap(X);
    Z.swap(ZZ);
}

void schur_inverse_remove(const std::vector<int64_t>& pos, int64_t m2, std::vector<double>& sinv,
                          std::vector<double>& Z) {
    if (static_cast<int64_t>(sinv.size()) != m2 * m2 || (m2 > 0 && Z.size() % static_cast<size_t>(m2) != 0))
        throw std::invalid_argument("the inverse does not match");
    const int64_t n = m2 > 0 ? static_cast<int64_t>(Z.size()) / m2 : 0;
    for (size_t t = 0; t < pos.size(); ++t)
        if (pos[t] < 0 || pos[t] >= m2 || (t > 0 && pos[t] <= pos[t - 1]))
            throw std::invalid_argument("positions must be ascending, distinct and in range");
    std::vector<double> X(sinv), Y;
    int64_t sz = m2;
    // the inverse of S without row and column i is X - X(:, i) X(i, :) / X(i, i)
    // with row and column i dropped; the last position first keeps the others
    for (size_t t = pos.size(); t-- > 0;) {
        const int64_t i = pos[t];
        const double g = X[i * sz + i];
        if (!(g > 0.0)) throw std::runtime_error("the inverse of S is not positive definite");
        // a diagonal entry that shrinks by more than 10^4 has lost that many
        // digits: the inverse is formed again instead
        for (int64_t a = 0; a < sz; ++a) {
            if (a == i) continue;
            const double keep = X[a * sz + a] - X[a * sz + i] * X[a * sz + i] / g;
            if (!(keep > 1e-4 * X[a * sz + a])) throw std::runtime_error("the reduced S loses too many digits");
        }
        const int64_t nz = sz - 1;
        Y.assign(static_cast<size_t>(nz * nz), 0.0);
        for (int64_t a = 0, ya = 0; a < sz; ++a) {
            if (a == i) continue;
            const double f = X[a * sz + i] / g;
            for (int64_t q = 0, yq = 0; q < sz; ++q) {
                if (q == i) continue;
                Y[ya * nz + yq] = X[a * sz + q] - f * X[i * sz + q];
                ++yq;
            }
            ++ya;
        }
        X.swap(Y);
        sz = nz;
    }
    // Z loses the same columns
    std::vector<double> ZZ;
    ZZ.reserve(static_cast<size_t>(sz * n));
    for (int64_t c = 0, t = 0; c < m2; ++c) {
        if (t < static_cast<int64_t>(pos.size()) && pos[static_cast<size_t>(t)] == c) {
            ++t;
            continue;
        }
        ZZ.insert(ZZ.end(), Z.begin() + c * n, Z.begin() + (c + 1) * n);
    }
    sinv.swap(X);
    Z.swap(ZZ);
}

}  // namespace rlsq
