// Single-problem path of the rlsq C ABI: create / factor / solve / apply.
//
// One LSMR iteration is the kernel sequence
//   k_spmv_lsmr   q = A v^ - alpha u (norm -> beta), r = b - A x (norm)
//   k_spmvt_lsmr  s = A^T u - beta w, ||A^T r|| -> stopping test on x_k
//   apply         t = M^{-1} s  (triangular solves, L2 products, S^ solve)
//   k_finish      alpha = sqrt(<t, s>), LSMR rotations
//   k_lsmr_update h-bar, x, h
// captured once in a CUDA graph (check_every iterations per graph) and
// replayed; the host only reads the `done` word between graphs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <exception>
#include <thread>
#include <type_traits>

#include "common.h"

namespace rlsq {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

void throw_cuda(cudaError_t e, const char* what, int line) {
    const int code = (e == cudaErrorMemoryAllocation) ? RLSQ_ERR_OOM : RLSQ_ERR_CUDA;
    throw ApiError(code, std::string("CUDA error ") + cudaGetErrorString(e) + " in " + what +
                             " (line " + std::to_string(line) + ")");
}

template <typename T>
void DevCsr<T>::upload(const HostCSR& h, cudaStream_t s, bool sliced) {
    rows = static_cast<int32_t>(h.rows);
    cols = static_cast<int32_t>(h.cols);
    nnz = h.nnz();
    if (nnz >= (int64_t(1) << 31)) throw ApiError(RLSQ_ERR_SHAPE, "more than 2^31 - 1 nonzeros");
    std::vector<int32_t> p32(h.ptr.begin(), h.ptr.end());
    ptr.upload(p32.data(), p32.size(), s);
    idx.upload(h.idx.data(), h.idx.size(), s);
    if constexpr (std::is_same<T, double>::value) {
        val.upload(reinterpret_cast<const T*>(h.val.data()), h.val.size(), s);
    } else {
        std::vector<T> v(h.val.begin(), h.val.end());
        val.upload(v.data(), v.size(), s);
    }
    sperm.release();
    sbase.release();
    sidx.release();
    sval.release();
    snpos = 0;
    sentries = 0;
    std::vector<int32_t> perm, base, si;
    std::vector<T> sv;
    if (sliced && h.rows > 0) {
        // positions: rows by decreasing length (ties: lower row first) within
        // windows of kSliceWindow rows, so that the 32 rows of a slice have
        // about the same length; -1 pads the last slice
        const int64_t R = h.rows, nsl = (R + 31) / 32;
        auto len = [&](int64_t r) { return h.ptr[r + 1] - h.ptr[r]; };
        perm.assign(static_cast<size_t>(nsl * 32), -1);
        for (int64_t r = 0; r < R; ++r) perm[r] = static_cast<int32_t>(r);
        for (int64_t w0 = 0; w0 < R; w0 += kSliceWindow) {
            const int64_t w1 = std::min<int64_t>(R, w0 + kSliceWindow);
            std::stable_sort(perm.begin() + w0, perm.begin() + w1,
                             [&](int32_t a, int32_t b) { return len(a) > len(b); });
        }
        std::vector<int64_t> b64(static_cast<size_t>(nsl) + 1, 0);
        for (int64_t q = 0; q < nsl; ++q) {
            int64_t w = 0;
            for (int64_t t = 32 * q; t < 32 * q + 32; ++t)
                if (perm[t] >= 0) w = std::max(w, len(perm[t]));
            b64[q + 1] = b64[q] + 32 * w;
        }
        if (b64[nsl] < (int64_t(1) << 31)) {
            base.assign(b64.begin(), b64.end());
            si.assign(static_cast<size_t>(b64[nsl]), -1);
            sv.assign(static_cast<size_t>(b64[nsl]), (T)0);
            for (int64_t t = 0; t < nsl * 32; ++t) {
                const int32_t r = perm[t];
                if (r < 0) continue;
                const int64_t e0 = b64[t >> 5] + (t & 31);
                for (int64_t k = 0; k < len(r); ++k) {
                    si[e0 + 32 * k] = h.idx[h.ptr[r] + k];
                    sv[e0 + 32 * k] = (T)h.val[h.ptr[r] + k];
                }
            }
            sperm.upload(perm.data(), perm.size(), s);
            sbase.upload(base.data(), base.size(), s);
            sidx.upload(si.data(), si.size(), s);
            sval.upload(sv.data(), sv.size(), s);
            snpos = static_cast<int32_t>(nsl * 32);
            sentries = b64[nsl];
        }
    }
    // host vectors die at return: make the copies complete first
    RLSQ_CUDA(cudaStreamSynchronize(s));
}

template <typename T>
static void upload_vec(DevArray<T>& dst, const std::vector<double>& src, cudaStream_t s) {
    std::vector<T> v(src.begin(), src.end());
    dst.upload(v.data(), v.size(), s);
    RLSQ_CUDA(cudaStreamSynchronize(s));
}

// Lanes per row of the binned solve: enough that every lane gathers at most
// four entries in one round (32 lanes for rows longer than 64 entries).
static int binned_lanes(int64_t entries) {
    int g = 1;
    while (g < 32 && 4 * g < entries) g *= 2;
    return g;
}

// The binned form of one fused system (see BinTri): within each level group
// the rows are ordered by lanes per row and slot size, most first (ties:
// solve position); a row's entries are its own right-hand side (-1), its
// right-hand-side terms (-c) and its dependencies (c), in a slot of the
// segment's size (padding: index -1, value 0).
template <typename T>
static void upload_binned(DevFactor<T>& D, int w, const IlupResult& F, const MergedTri& M, cudaStream_t s) {
    const std::vector<int32_t>& ord = M.lev.order;
    const std::vector<int32_t>& lp = M.lev.level_ptr;
    const int64_t n = static_cast<int64_t>(ord.size());
    const int ng = static_cast<int>(lp.size()) - 1;
    const bool fused = M.R.nnz() > 0;
    auto count = [&](int32_t r) {
        return (M.T.ptr[r + 1] - M.T.ptr[r]) + (fused ? M.R.ptr[r + 1] - M.R.ptr[r] : 0) + 1;
    };
    std::vector<int32_t> bord(ord.size());
    std::vector<BinSeg> seg;
    std::vector<int32_t> gseg(static_cast<size_t>(ng) + 1, 0), gitems(static_cast<size_t>(std::max(ng, 1)), 0),
        gpos(static_cast<size_t>(ng) + 1, 0), gentry(static_cast<size_t>(ng) + 1, 0);
    int64_t base = 0;
    for (int g = 0; g < ng; ++g) {
        const int32_t p0 = lp[g], p1 = lp[g + 1];
        gpos[g] = p0;
        gseg[g] = static_cast<int32_t>(seg.size());
        gentry[g] = static_cast<int32_t>(base);
        // rows ordered by lanes (32, 16, ..., 1), then by slot size (the entry
        // count rounded up to the lanes; most first), then by solve position;
        // every (lanes, slot size) run is one segment, so a slot pads its row
        // by fewer than G entries
        std::vector<std::pair<int64_t, int32_t>> key;
        key.reserve(static_cast<size_t>(p1 - p0));
        for (int32_t t = p0; t < p1; ++t) {
            const int64_t c = count(ord[t]);
            const int G = binned_lanes(c);
            const int64_t cap = ((c + G - 1) / G) * G;
            key.emplace_back((static_cast<int64_t>(G) << 40) | cap, t);
        }
        std::stable_sort(key.begin(), key.end(),
                         [](const std::pair<int64_t, int32_t>& a, const std::pair<int64_t, int32_t>& b) {
                             return a.first > b.first;
                         });
        int32_t item = 0;
        for (size_t q = 0; q < key.size();) {
            size_t r = q;
            while (r < key.size() && key[r].first == key[q].first) ++r;
            const int G = static_cast<int>(key[q].first >> 40);
            const int64_t cap = key[q].first & ((int64_t(1) << 40) - 1);
            const int32_t s0 = p0 + static_cast<int32_t>(q), s1 = p0 + static_cast<int32_t>(r);
            for (size_t u = q; u < r; ++u) bord[p0 + u] = ord[key[u].second];
            if (base + cap * (s1 - s0) >= (int64_t(1) << 31))
                throw ApiError(RLSQ_ERR_SHAPE, "binned solve: more than 2^31 - 1 entries");
            seg.push_back(BinSeg{s0, s1, G, item, static_cast<int32_t>(cap), static_cast<int32_t>(base)});
            item += (s1 - s0 + (32 / G) - 1) / (32 / G);
            base += cap * (s1 - s0);
            q = r;
        }
        gitems[g] = item;
    }
    gseg[ng] = static_cast<int32_t>(seg.size());
    gpos[ng] = static_cast<int32_t>(n);
    gentry[ng] = static_cast<int32_t>(base);
    std::vector<int32_t> bi(static_cast<size_t>(std::max<int64_t>(base, 1)), -1);
    std::vector<T> bv(bi.size(), (T)0);
    const int32_t flag = static_cast<int32_t>(0x80000000u);
    for (const BinSeg& sg : seg) {
        for (int32_t t = sg.p0; t < sg.p1; ++t) {
            const int32_t r = bord[t];
            int64_t e = sg.base + static_cast<int64_t>(t - sg.p0) * sg.cap;
            bi[e] = r | flag;
            bv[e++] = (T)-1.0;
            if (fused)
                for (int64_t q = M.R.ptr[r]; q < M.R.ptr[r + 1]; ++q) {
                    bi[e] = M.R.idx[q] | flag;
                    bv[e++] = (T)(-M.R.val[q]);
                }
            for (int64_t q = M.T.ptr[r]; q < M.T.ptr[r + 1]; ++q) {
                bi[e] = M.T.idx[q];
                bv[e++] = (T)M.T.val[q];
            }
        }
    }
    D.bidx[w].upload(bi.data(), bi.size(), s);
    D.bval[w].upload(bv.data(), bv.size(), s);
    D.border[w].upload(bord.data(), bord.size(), s);
    if (w >= 2) {
        std::vector<T> dl(static_cast<size_t>(n));
        for (int64_t t = 0; t < n; ++t) dl[t] = (T)(1.0 / F.Udiag[bord[t]]);
        D.bdiag[w].upload(dl.data(), dl.size(), s);
        RLSQ_CUDA(cudaStreamSynchronize(s));
    }
    D.bseg[w].upload(seg.data(), seg.size(), s);
    D.bgseg[w].upload(gseg.data(), gseg.size(), s);
    D.bgitems[w].upload(gitems.data(), gitems.size(), s);
    D.bgpos[w].upload(gpos.data(), gpos.size(), s);
    D.bgentry[w].upload(gentry.data(), gentry.size(), s);
    D.bngroups[w] = ng;
    D.bentries[w] = base;
    // the host vectors die at return
    RLSQ_CUDA(cudaStreamSynchronize(s));
}

template <typename T>
void DevFactor<T>::upload(const IlupResult& F, const MergedTri* merged, const std::vector<double>& sinv_h,
                          cudaStream_t s, bool sliced) {
    for (int w = 0; w < 4; ++w) {
        upload_binned<T>(*this, w, F, merged[w], s);
        // rows permuted into solve order so each level is contiguous
        const MergedTri& M = merged[w];
        const std::vector<int32_t>& ord = M.lev.order;
        auto permute = [&](const HostCSR& a) {
            HostCSR lo;
            lo.rows = a.rows;
            lo.cols = a.cols;
            lo.ptr.assign(static_cast<size_t>(a.rows) + 1, 0);
            lo.idx.reserve(a.idx.size());
            lo.val.reserve(a.val.size());
            for (int64_t t = 0; t < a.rows; ++t) {
                const int32_t r = ord[t];
                for (int64_t e = a.ptr[r]; e < a.ptr[r + 1]; ++e) {
                    lo.idx.push_back(a.idx[e]);
                    lo.val.push_back(a.val[e]);
                }
                lo.ptr[t + 1] = static_cast<int64_t>(lo.idx.size());
            }
            return lo;
        };
        const HostCSR T_pos = permute(M.T);
        tri[w].upload(T_pos, s);
        {
            const size_t nn = static_cast<size_t>(T_pos.rows);
            const int kp = (static_cast<double>(T_pos.nnz()) <= 4.5 * static_cast<double>(std::max<size_t>(nn, 1))) ? 4 : 8;
            std::vector<int32_t> ei(static_cast<size_t>(kp) * std::max<size_t>(nn, 1), -1);
            std::vector<double> ev(ei.size(), 0.0);
            for (size_t t = 0; t < nn; ++t) {
                const int64_t e0 = T_pos.ptr[t], e1 = std::min<int64_t>(T_pos.ptr[t + 1], e0 + kp);
                for (int64_t e = e0; e < e1; ++e) {
                    ei[static_cast<size_t>(e - e0) * nn + t] = T_pos.idx[e];
                    ev[static_cast<size_t>(e - e0) * nn + t] = T_pos.val[e];
                }
            }
            ell_kp[w] = kp;
            ell_idx[w].upload(ei.data(), ei.size(), s);
            upload_vec(ell_val[w], ev, s);
        }
        if (M.R.nnz() > 0) rtri[w].upload(permute(M.R), s);
        else { rtri[w].ptr.release(); rtri[w].idx.release(); rtri[w].val.release(); rtri[w].nnz = 0; }
        order[w].upload(ord.data(), ord.size(), s);
        level_ptr[w] = M.lev.level_ptr;
        level_ptr_d[w].upload(level_ptr[w].data(), level_ptr[w].size(), s);
        if (w >= 2) {
            std::vector<double> dl(ord.size());
            // the solves multiply by the inverse diagonal (a float64 division is
            // a long instruction sequence on this GPU)
            for (size_t t = 0; t < ord.size(); ++t) dl[t] = 1.0 / F.Udiag[ord[t]];
            upload_vec(diag[w], dl, s);
        }
    }
    L2.upload(F.L2, s, sliced);
    L2t.upload(F.L2t, s, sliced);
    upload_vec(d, F.d, s);
    prow.upload(F.prow.data(), F.prow.size(), s);
    if (!F.a2rows.empty()) a2rows.upload(F.a2rows.data(), F.a2rows.size(), s);
    else a2rows.release();
    if (!sinv_h.empty()) upload_vec(sinv, sinv_h, s);
    else sinv.release();
    const size_t n = static_cast<size_t>(F.n), m2 = static_cast<size_t>(F.m - F.n);
    for (auto& v : vn) v.alloc(n);
    for (auto& v : vm) v.alloc(std::max<size_t>(m2, 1));
    RLSQ_CUDA(cudaStreamSynchronize(s));
}

void copy_half(double* dst, const double2* pairs, int64_t n, int half, bool dev, double* staging,
               cudaStream_t st) {
    if (n <= 0) return;
    double* out = dev ? dst : staging;
    const int grid = static_cast<int>(std::min<int64_t>((n + kBlock - 1) / kBlock, 4096));
    if (half) k_half<1><<<grid, kBlock, 0, st>>>(static_cast<int>(n), pairs, out);
    else k_half<0><<<grid, kBlock, 0, st>>>(static_cast<int>(n), pairs, out);
    RLSQ_CUDA(cudaGetLastError());
    if (!dev) RLSQ_CUDA(cudaMemcpyAsync(dst, staging, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
}

template struct DevCsr<double>;
template struct DevCsr<float>;
template struct DevFactor<double>;
template struct DevFactor<float>;

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
template <class F>
static void with_G(int G, F&& f) {
    switch (G) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 16: f(std::integral_constant<int, 16>{}); break;
        default: f(std::integral_constant<int, 32>{}); break;
    }
}
// the same with 0: the sliced layout (products only)
template <class F>
static void with_Gp(int G, F&& f) {
    if (G == 0) f(std::integral_constant<int, 0>{});
    else with_G(G, f);
}

// Lanes of a product over M: 0 (sliced) when chosen and built, else the CSR
// lanes G; and the threads it is launched for (rows x lanes, or the padded
// positions of the slices).
template <typename T>
static int prod_G(int G, int sliced, const DevCsr<T>& M) {
    return (sliced && M.snpos > 0) ? 0 : G;
}
template <typename T>
static int64_t prod_threads(int G, const DevCsr<T>& M) {
    return G == 0 ? static_cast<int64_t>(M.snpos) : static_cast<int64_t>(M.rows) * G;
}

template <class F>
static void with_rhs(int k, F&& f) {
    switch (k) {
        case RHS_SCALED: f(std::integral_constant<int, RHS_SCALED>{}); break;
        case RHS_SUB: f(std::integral_constant<int, RHS_SUB>{}); break;
        default: f(std::integral_constant<int, RHS_VEC>{}); break;
    }
}

static int max_grid(const rlsq_problem_s* P) { return std::max(1, P->num_sms * kGridBlocksPerSm); }

// kernels without a grid-wide reduction keep a wide grid (32 blocks per SM)
static int grid_rows_wide(const rlsq_problem_s* P, int64_t rows, int G) {
    const int64_t g = (rows * G + kBlock - 1) / kBlock;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, std::max(1, P->num_sms * 32))));
}

static int grid_rows(const rlsq_problem_s* P, int64_t rows, int G) {
    const int64_t g = (rows * G + kBlock - 1) / kBlock;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, max_grid(P))));
}

static LsmrState* state_ptr(rlsq_problem_s* P, int which) { return P->S.p + which; }

// dense-row block products (defined with the A layout below)
template <bool PAIR>
static void enqueue_dense_av(rlsq_problem_s* P, const void* v, const LsmrState* S, cudaStream_t st);
template <bool PAIR>
static void enqueue_dense_atv(rlsq_problem_s* P, const void* u, const LsmrState* S, cudaStream_t st);
static int* error_word(LsmrState* S) {
    return reinterpret_cast<int*>(reinterpret_cast<char*>(S) + offsetof(LsmrState, error));
}

// Brackets the launches of its lifetime with an event pair when profiling.
struct RecScope {
    rlsq_problem_s* P;
    cudaStream_t st;
    size_t slot = 0;
    RecScope(rlsq_problem_s* p, int cls, double bytes, cudaStream_t s) : P(p), st(s) {
        if (!P->rec) return;
        Recorder::Entry e{cls, bytes, nullptr, nullptr, 1};
        RLSQ_CUDA(cudaEventCreate(&e.a));
        RLSQ_CUDA(cudaEventCreate(&e.b));
        // external record: becomes an event-record node when captured
        RLSQ_CUDA(cudaEventRecordWithFlags(e.a, st, cudaEventRecordExternal));
        P->rec->entries.push_back(e);
        slot = P->rec->entries.size();
    }
    ~RecScope() {
        if (P->rec && slot) cudaEventRecordWithFlags(P->rec->entries[slot - 1].b, st, cudaEventRecordExternal);
    }
};

// Algorithmic bytes of one solve with system `which` of the factor (not of
// its fused form): every stored entry once (value + int32 index), the row
// pointers, the right-hand side in and the solution out.  Entries that level
// fusion adds are the schedule's overhead and are not counted here.
template <typename T>
static double trsv_bytes(const rlsq_problem_s* P, int which) {
    const double n = static_cast<double>(P->n), v = sizeof(T);
    double nnz = 0.0;
    if (P->F) {
        const IlupResult& F = *P->F;
        nnz = (which < 2) ? static_cast<double>(F.L1.nnz()) : static_cast<double>(F.U.nnz()) + n;  // U: + diagonal
    }
    return (v + 4.0) * nnz + 4.0 * n + 2.0 * v * n;
}
// A sparse product y = M x: every stored entry once, the row pointers, x read
// and y written once each.
template <typename T>
static double mv_bytes(const DevCsr<T>& M, double in_bytes_per_col, double out_bytes_per_row) {
    return (sizeof(T) + 4.0) * static_cast<double>(M.nnz) + 4.0 * M.rows +
           in_bytes_per_col * M.cols + out_bytes_per_row * M.rows;
}

// Opt-in shared memory of the persistent solve (more than the default 48 KB
// for 8 entries in float64); set outside any stream capture.
template <typename T>
static void coop_attributes() {
    auto set = [](auto kern, int kp) {
        RLSQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(coop_smem_bytes<T>(kp))));
    };
    set(k_trsv_coop<T, RHS_VEC, 4>, 4);
    set(k_trsv_coop<T, RHS_VEC, 8>, 8);
    set(k_trsv_coop<T, RHS_SUB, 4>, 4);
    set(k_trsv_coop<T, RHS_SUB, 8>, 8);
    set(k_trsv_coop<T, RHS_SCALED, 4>, 4);
    set(k_trsv_coop<T, RHS_SCALED, 8>, 8);
}

// `gate` (optional): the state whose done word the kernels check instead of
// S's (the CG steps' gate when their number is adaptive); errors still go to
// S's error word.
template <typename T>
static void launch_trsv(rlsq_problem_s* P, DevFactor<T>& F, int which, int rk, Rhs<T> rhs, T* x,
                        int slot, LsmrState* S, cudaStream_t st, const LsmrState* gate = nullptr) {
    const Tri<T> tri = F.tview(which);
    int* const err = error_word(S);
    const LsmrState* const G8 = gate ? gate : S;
    const int n = tri.n;
    const int G = P->map.G_tri[which];
    RecScope rs(P, RLSQ_KCLASS_TRSV_L1 + which, trsv_bytes<T>(P, which), st);
    if (P->map.sched[which] == RLSQ_TRSV_LEVEL) {
        const auto& lp = F.level_ptr[which];
        for (size_t l = 0; l + 1 < lp.size(); ++l) {
            const int lo = lp[l], hi = lp[l + 1];
            const int grid = grid_rows(P, hi - lo, G);
            with_G(G, [&](auto g) {
                with_rhs(rk, [&](auto k) {
                    k_trsv_level<T, decltype(g)::value, decltype(k)::value>
                        <<<grid, kBlock, 0, st>>>(tri, rhs, x, lo, hi, G8);
                });
            });
        }
        if (P->rec && !P->rec->entries.empty()) P->rec->entries.back().launches = static_cast<int>(lp.size()) - 1;
    } else if (P->map.sched[which] == RLSQ_TRSV_COOP) {
        if (slot >= kMaxSlots) throw ApiError(RLSQ_ERR_ARG, "too many triangular solves in one apply");
        // leading levels wider than the persistent grid go to full-occupancy
        // level launches (each row of such a level would otherwise wait for
        // the one before it on the same thread); the persistent kernel takes
        // over at the first narrower level
        const auto& lp = F.level_ptr[which];
        const int nall = static_cast<int>(lp.size()) - 1;
        const int64_t resident = static_cast<int64_t>(P->coop_blocks) * kCoopBlock;
        int lead = 0;
        while (lead < nall && lp[lead + 1] - lp[lead] > resident) ++lead;
        for (int l = 0; l < lead; ++l) {
            const int grid = grid_rows(P, lp[l + 1] - lp[l], 1);
            with_rhs(rk, [&](auto k) {
                k_trsv_level<T, 1, decltype(k)::value><<<grid, kBlock, 0, st>>>(tri, rhs, x, lp[l], lp[l + 1], G8);
            });
        }
        const int nlev = nall - lead;
        if (P->rec && !P->rec->entries.empty()) P->rec->entries.back().launches = lead + (nlev > 0 ? 1 : 0);
        if (nlev > 0) with_rhs(rk, [&](auto k) {
            const int kp = F.ell_kp[which] >= 8 ? 8 : 4;
            auto kern = kp == 8 ? k_trsv_coop<T, decltype(k)::value, 8> : k_trsv_coop<T, decltype(k)::value, 4>;
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(static_cast<unsigned>(P->coop_blocks));
            cfg.blockDim = dim3(kCoopBlock);
            cfg.dynamicSmemBytes = coop_smem_bytes<T>(kp);
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            RLSQ_CUDA(cudaLaunchKernelEx(&cfg, kern, tri, rhs, x, F.level_ptr_d[which].p + lead, nlev,
                                         P->barriers.p + slot, G8, err));
        });
    } else if (P->map.sched[which] == RLSQ_TRSV_BINNED) {
        if (slot >= kMaxSlots) throw ApiError(RLSQ_ERR_ARG, "too many triangular solves in one apply");
        const BinTri<T> bt = F.bview(which);
        with_rhs(rk, [&](auto k) {
            auto kern = k_trsv_binned<T, decltype(k)::value>;
            int occ = 0;
            RLSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBinBlock, 0));
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(static_cast<unsigned>(std::max(1, occ) * P->num_sms));
            cfg.blockDim = dim3(kBinBlock);
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            RLSQ_CUDA(cudaLaunchKernelEx(&cfg, kern, bt, rhs, x, P->barriers.p + slot, G8, err));
        });
    } else if (P->map.sched[which] == RLSQ_TRSV_WAVE) {
        // all-one bytes mark "not yet solved" (see k_trsv_wave)
        RLSQ_CUDA(cudaMemsetAsync(x, 0xff, sizeof(T) * static_cast<size_t>(n), st));
        const int kp = P->map.wave_kp[which];
        with_rhs(rk, [&](auto k) {
            auto run = [&](auto kern) {
                int occ = 0;
                RLSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWaveBlock, 0));
                const int need = (n + kWaveBlock - 1) / kWaveBlock;
                const int grid = std::max(1, std::min(need, std::max(1, occ) * P->num_sms));
                cudaLaunchConfig_t cfg{};
                cfg.gridDim = dim3(static_cast<unsigned>(grid));
                cfg.blockDim = dim3(kWaveBlock);
                cfg.stream = st;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeCooperative;
                attr[0].val.cooperative = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                RLSQ_CUDA(cudaLaunchKernelEx(&cfg, kern, tri, rhs, x, G8, err));
            };
            if (kp >= 8) run(k_trsv_wave<T, decltype(k)::value, 8>);
            else run(k_trsv_wave<T, decltype(k)::value, 4>);
        });
    } else {
        if (slot >= kMaxSlots) throw ApiError(RLSQ_ERR_ARG, "too many triangular solves in one apply");
        // all-one bytes mark "not yet solved" (see k_trsv_sentinel)
        RLSQ_CUDA(cudaMemsetAsync(x, 0xff, sizeof(T) * static_cast<size_t>(n), st));
        const int R = P->map.sf_rows[which];
        with_G(G, [&](auto g) {
            constexpr int GG = decltype(g)::value;
            with_rhs(rk, [&](auto k) {
                constexpr int KK = decltype(k)::value;
                // rows in flight = grid * kBlock / G (times R); every one of them
                // polls, so the window is kept to a few levels rather than the
                // whole GPU
                auto run = [&](auto kern, int chunk_rows) {
                    int occ = 0;
                    RLSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlock, 0));
                    occ = std::max(1, std::min(occ, P->map.sf_blocks[which]));
                    const int chunks = (n + chunk_rows - 1) / chunk_rows;
                    const int blocks_needed = (chunks + kBlock / 32 - 1) / (kBlock / 32);
                    const int grid = std::max(1, std::min(R > 0 ? blocks_needed : chunks, occ * P->num_sms));
                    kern<<<grid, kBlock, 0, st>>>(tri, rhs, x, slot, P->tickets.p, G8, err);
                };
                if (R >= 4) run(k_trsv_warp<T, GG, KK, 4>, (32 / GG) * 4);
                else if (R == 2) run(k_trsv_warp<T, GG, KK, 2>, (32 / GG) * 2);
                else if (R == 1) run(k_trsv_warp<T, GG, KK, 1>, 32 / GG);
                else run(k_trsv_sentinel<T, GG, KK, 1>, kBlock / GG);
            });
        });
    }
}

// t = M^{-1} s for the float64 vector s, result in P->t; advances the LSMR
// scalars (INIT: the first alpha), or the CGLS ones (CGLS), or only the apply
// count (standalone).
//
// With split_r (an m-vector r, entries split_stride doubles apart) the apply
// is Algorithm 3 fed the residual split instead: r1 = r[prow], r2 =
// r[a2rows], u = r2 - L2 L1^{-1} r1, S^ w = u, y = r1 + L1^{-T} L2^T w,
// t = D U^{-1} L1^{-1} y.  The correction runs on -u (the same steps as the
// x-space form, whose right-hand side is +L2 q1), so it yields -w and
// y = r1 - L1^{-T} L2^T (-w); negation is exact, so this is the same
// arithmetic.  s then only enters the scalar step (<t, s>, s = A^T r).
template <typename T, bool INIT, bool CGLS = false>
static void enqueue_apply(rlsq_problem_s* P, DevFactor<T>& F, const double* s, LsmrState* S,
                          cudaStream_t st, const double* split_r = nullptr, int split_stride = 1) {
    const int n = static_cast<int>(P->n);
    const int m2 = static_cast<int>(P->m - P->n);
    RLSQ_CUDA(cudaMemsetAsync(P->tickets.p, 0, sizeof(unsigned) * kMaxSlots, st));
    RLSQ_CUDA(cudaMemsetAsync(P->barriers.p, 0, sizeof(unsigned) * kMaxSlots, st));
    int slot = 0;
    T* g2 = F.vn[1].p;       // x-space: L1^{-T} U^{-T} D s; split: r1
    const T* sub = nullptr;  // split: r2, subtracted from L2 q1
    if (split_r) {
        T* r2 = F.vm[2].p;
        RecScope rs(P, RLSQ_KCLASS_VEC, (12.0 + sizeof(T)) * (static_cast<double>(n) + m2), st);
        k_split_gather<T><<<grid_rows_wide(P, std::max(n, m2), 1), kBlock, 0, st>>>(
            n, m2, F.prow.p, m2 > 0 ? F.a2rows.p : nullptr, split_r, split_stride, g2, r2, S);
        sub = r2;
    } else {
        T* g1 = F.vn[0].p;
        launch_trsv<T>(P, F, 3, RHS_SCALED, Rhs<T>{F.d.p, nullptr, s}, g1, slot++, S, st);  // U^{-T} D s
        launch_trsv<T>(P, F, 1, RHS_VEC, Rhs<T>{g1, nullptr, nullptr}, g2, slot++, S, st);  // L1^{-T}
    }
    T* g4 = F.vn[0].p;
    if (P->correction != RLSQ_CORR_NONE) {
        T* q1 = F.vn[2].p;
        launch_trsv<T>(P, F, 0, RHS_VEC, Rhs<T>{g2, nullptr, nullptr}, q1, slot++, S, st);  // L1^{-1}
        const Csr<T> L2 = F.L2.view(), L2t = F.L2t.view();
        // lanes of the L2 / L2^T products (0: sliced layout) and their grids
        const int GL2 = prod_G(P->map.G_L2, P->map.sl_L2, F.L2), GL2t = prod_G(P->map.G_L2t, P->map.sl_L2t, F.L2t);
        const int gl2 = grid_rows(P, prod_threads(GL2, F.L2), 1);
        const int gl2t = grid_rows_wide(P, prod_threads(GL2t, F.L2t), 1);
        const int gl2w = grid_rows_wide(P, prod_threads(GL2, F.L2), 1);
        const int gv = grid_rows(P, std::max(m2, n), 1);
        T* wv = nullptr;
        if (P->correction == RLSQ_CORR_CG) {
            // CG(k) on S^ w = e.  Each step carries its direction p through L2^T,
            // L1^{-T} and L1^{-1} (c3); z = sum_j a_j c3_j is then L1^{-1}
            // L1^{-T} L2^T w, so L1^{-1}(g2 - L1^{-T} L2^T w) = q1 - z and the
            // apply ends with U^{-1}(q1 - z): Algorithm 3's steps 3-4 without
            // their L2^T product and two solves (linearity in w; w is not formed).
            T *rv = F.vm[0].p, *pv = F.vm[1].p, *sp = F.vm[2].p;
            T *c1 = F.vn[3].p, *c2 = F.vn[4].p, *c3 = F.vn[5].p, *z = F.vn[0].p;
            // adaptive number of CG steps: a gate the remaining steps check
            LsmrState* gate = P->opts.cg_tol > 0.0 ? state_ptr(P, 2) : nullptr;
            const double tol2 = P->opts.cg_tol * P->opts.cg_tol;
            {
                RecScope rs(P, RLSQ_KCLASS_L2, mv_bytes(F.L2, sizeof(T), sizeof(T)), st);
                with_Gp(GL2, [&](auto g) {
                    k_l2_start<T, decltype(g)::value><<<gl2, kBlock, 0, st>>>(L2, q1, rv, S, P->part.p,
                                                                              P->counter.p, gate, sub);
                });
            }
            for (int it = 0; it < P->opts.cg_steps; ++it) {
                const bool first = (it == 0);
                {
                    RecScope rs(P, RLSQ_KCLASS_L2T, mv_bytes(F.L2t, sizeof(T), sizeof(T)), st);
                    with_Gp(GL2t, [&](auto g) {
                        constexpr int GG = decltype(g)::value;
                        if (first) k_l2t_cg<T, GG, true><<<gl2t, kBlock, 0, st>>>(L2t, rv, pv, c1, S, gate);
                        else k_l2t_cg<T, GG, false><<<gl2t, kBlock, 0, st>>>(L2t, rv, pv, c1, S, gate);
                    });
                }
                launch_trsv<T>(P, F, 1, RHS_VEC, Rhs<T>{c1, nullptr, nullptr}, c2, slot++, S, st, gate);
                launch_trsv<T>(P, F, 0, RHS_VEC, Rhs<T>{c2, nullptr, nullptr}, c3, slot++, S, st, gate);
                RecScope rs2(P, RLSQ_KCLASS_L2, mv_bytes(F.L2, sizeof(T), sizeof(T)), st);
                with_Gp(GL2, [&](auto g) {
                    constexpr int GG = decltype(g)::value;
                    if (first)
                        k_l2_sp<T, GG, true><<<gl2, kBlock, 0, st>>>(L2, c3, rv, pv, sp, S, P->part.p,
                                                                     P->counter.p, gate);
                    else
                        k_l2_sp<T, GG, false><<<gl2, kBlock, 0, st>>>(L2, c3, rv, pv, sp, S, P->part.p,
                                                                      P->counter.p, gate);
                });
                RecScope rs3(P, RLSQ_KCLASS_VEC, sizeof(T) * (4.0 * m2 + (first ? 2.0 : 3.0) * n), st);
                if (first)
                    k_cg_update<T, true><<<gv, kBlock, 0, st>>>(m2, pv, sp, rv, nullptr, S, P->part.p,
                                                                P->counter.p, gate, tol2, n, c3, z);
                else
                    k_cg_update<T, false><<<gv, kBlock, 0, st>>>(m2, pv, sp, rv, nullptr, S, P->part.p,
                                                                 P->counter.p, gate, tol2, n, c3, z);
            }
            // U^{-1}(q1 - z), then t = D g5
            T* g5 = F.vn[1].p;
            launch_trsv<T>(P, F, 2, RHS_SUB, Rhs<T>{q1, z, nullptr}, g5, slot++, S, st);
            RecScope rs(P, RLSQ_KCLASS_FINISH, (2.0 * sizeof(T) + 16.0) * n, st);
            k_finish_apply<T, INIT, false, CGLS><<<grid_rows(P, n, 1), kBlock, 0, st>>>(n, F.d.p, g5, s, P->tx.p,
                                                                                        S, P->part.p, P->counter.p);
            return;
        } else {
            T* e = F.vm[0].p;
            {
                RecScope rs(P, RLSQ_KCLASS_L2, mv_bytes(F.L2, sizeof(T), sizeof(T)), st);
                with_Gp(GL2, [&](auto g) {
                    k_csr_mv<T, decltype(g)::value><<<gl2w, kBlock, 0, st>>>(L2, q1, e, S, sub);
                });
            }
            wv = e;
            if (P->correction == RLSQ_CORR_DENSE) {
                T* w = F.vm[3].p;
                RecScope rs(P, RLSQ_KCLASS_VEC, sizeof(T) * (double)m2 * (m2 + 2), st);
                k_dense_gemv<T><<<grid_rows(P, m2, 32), kBlock, 0, st>>>(m2, F.sinv.p, e, w, S);
                wv = w;
            }
        }
        T* f = F.vn[3].p;
        T* y = F.vn[4].p;
        {
            RecScope rs(P, RLSQ_KCLASS_L2T, mv_bytes(F.L2t, sizeof(T), sizeof(T)), st);
            with_Gp(GL2t, [&](auto g) {
                k_csr_mv<T, decltype(g)::value><<<gl2t, kBlock, 0, st>>>(L2t, wv, f, S);
            });
        }
        launch_trsv<T>(P, F, 1, RHS_VEC, Rhs<T>{f, nullptr, nullptr}, y, slot++, S, st);   // L1^{-T} Y^T w
        launch_trsv<T>(P, F, 0, RHS_SUB, Rhs<T>{g2, y, nullptr}, g4, slot++, S, st);       // L1^{-1}(g2 - .)
    } else {
        launch_trsv<T>(P, F, 0, RHS_VEC, Rhs<T>{g2, nullptr, nullptr}, g4, slot++, S, st);
    }
    T* g5 = F.vn[2].p;
    launch_trsv<T>(P, F, 2, RHS_VEC, Rhs<T>{g4, nullptr, nullptr}, g5, slot++, S, st);    // U^{-1}
    RecScope rs(P, RLSQ_KCLASS_FINISH, (2.0 * sizeof(T) + 16.0) * n, st);
    k_finish_apply<T, INIT, false, CGLS><<<grid_rows(P, n, 1), kBlock, 0, st>>>(n, F.d.p, g5, s, P->tx.p, S,
                                                                                P->part.p, P->counter.p);
}

template <bool INIT, bool CGLS = false>
static void enqueue_identity_apply(rlsq_problem_s* P, const double* s, LsmrState* S, cudaStream_t st) {
    // M = I: t = s (the unpreconditioned baseline)
    const int n = static_cast<int>(P->n);
    RecScope rs(P, RLSQ_KCLASS_FINISH, 24.0 * n, st);
    k_finish_apply<double, INIT, true, CGLS><<<grid_rows(P, n, 1), kBlock, 0, st>>>(n, nullptr, s, s, P->tx.p,
                                                                                    S, P->part.p, P->counter.p);
}

// split_r: Algorithm 3 on the residual split of split_r (see enqueue_apply);
// with plain (M = I) it is ignored.
template <bool INIT, bool CGLS = false>
static void enqueue_apply_any(rlsq_problem_s* P, const double* s, LsmrState* S, cudaStream_t st,
                              bool plain, const double* split_r = nullptr, int split_stride = 1) {
    if (plain) {
        enqueue_identity_apply<INIT, CGLS>(P, s, S, st);
    } else if (P->precision == RLSQ_PREC_FP32) {
        enqueue_apply<float, INIT, CGLS>(P, P->f32, s, S, st, split_r, split_stride);
    } else {
        enqueue_apply<double, INIT, CGLS>(P, P->f64, s, S, st, split_r, split_stride);
    }
}

static void enqueue_iteration(rlsq_problem_s* P, LsmrState* S, cudaStream_t st, bool plain) {
    const int m = static_cast<int>(P->m), n = static_cast<int>(P->n);
    const bool dense = P->md > 0;
    const double dense_bytes = 8.0 * static_cast<double>(P->md) * static_cast<double>(P->n) + 16.0 * P->n;
    if (dense) {
        RecScope rs(P, RLSQ_KCLASS_DENSE, dense_bytes, st);
        enqueue_dense_av<true>(P, P->tx.p, S, st);
    }
    {
        RecScope rs(P, RLSQ_KCLASS_SPMV, mv_bytes(P->dA, 8.0, 8.0), st);
        const int GA = prod_G(P->map.G_A, P->map.sl_A, P->dA);
        with_Gp(GA, [&](auto g) {
            k_spmv_lsmr<decltype(g)::value><<<grid_rows(P, prod_threads(GA, P->dA), 1), kBlock, 0, st>>>(
                P->dA.view(), P->tx.p, P->qr.p, P->b.p, S, P->part.p, P->counter.p, static_cast<int>(P->ms),
                dense ? P->dense_av.p : nullptr);
        });
    }
    if (dense) {
        RecScope rs(P, RLSQ_KCLASS_DENSE, dense_bytes, st);
        enqueue_dense_atv<true>(P, P->qr.p + P->ms, S, st);
    }
    {
        RecScope rs(P, RLSQ_KCLASS_SPMVT, mv_bytes(P->dAt, 8.0, 8.0), st);
        const int GAt = prod_G(P->map.G_At, P->map.sl_At, P->dAt);
        with_Gp(GAt, [&](auto g) {
            k_spmvt_lsmr<decltype(g)::value, false>
                <<<grid_rows(P, prod_threads(GAt, P->dAt), 1), kBlock, 0, st>>>(P->dAt.view(), P->qr.p, P->s.p,
                                                                               S, P->part.p, P->counter.p,
                                                                               dense ? P->dense_atv.p : nullptr);
        });
    }
    enqueue_apply_any<false>(P, P->s.p, S, st, plain);
    RecScope rs(P, RLSQ_KCLASS_UPDATE, 56.0 * n, st);
    k_lsmr_update<false><<<grid_rows_wide(P, n, 1), kBlock, 0, st>>>(n, P->tx.p, P->h.p, P->hb.p, S);
}

static void enqueue_start(rlsq_problem_s* P, LsmrState* S, cudaStream_t st, bool plain) {
    const int m = static_cast<int>(P->m), n = static_cast<int>(P->n);
    k_start_b<0><<<grid_rows(P, m, 1), kBlock, 0, st>>>(m, P->b.p, P->qr.p, S, P->part.p, P->counter.p);
    const bool dense = P->md > 0;
    if (dense) enqueue_dense_atv<true>(P, P->qr.p + P->ms, S, st);
    const int GAt = prod_G(P->map.G_At, P->map.sl_At, P->dAt);
    with_Gp(GAt, [&](auto g) {
        k_spmvt_lsmr<decltype(g)::value, true>
            <<<grid_rows(P, prod_threads(GAt, P->dAt), 1), kBlock, 0, st>>>(P->dAt.view(), P->qr.p, P->s.p, S,
                                                                           P->part.p, P->counter.p,
                                                                           dense ? P->dense_atv.p : nullptr);
    });
    enqueue_apply_any<true>(P, P->s.p, S, st, plain);
    k_lsmr_update<true><<<grid_rows(P, n, 1), kBlock, 0, st>>>(n, P->tx.p, P->h.p, P->hb.p, S);
}

// Preconditioned CGLS (Algorithm 1) with h = M^{-1} A^T r, M^{-1} the same
// x-space operator LSMR uses, or (split) h = Algorithm 3 applied to the
// residual split of r, as the paper combines the preconditioner with A^T.
// Vectors: (q, r) in qr, (h, x) in tx, z in s, p in h.  No dense-row block.
static void enqueue_cgls_z(rlsq_problem_s* P, LsmrState* S, cudaStream_t st) {
    const int n = static_cast<int>(P->n);
    RecScope rs(P, RLSQ_KCLASS_SPMVT, mv_bytes(P->dAt, 8.0, 8.0), st);
    with_G(P->map.G_At, [&](auto g) {
        k_cgls_z<decltype(g)::value><<<grid_rows(P, n, decltype(g)::value), kBlock, 0, st>>>(
            P->dAt.view(), P->qr.p, P->s.p, S, P->part.p, P->counter.p);
    });
}

// the residual r_i at r[2 i] of the interleaved (q, r) pairs
static const double* cgls_residual(const rlsq_problem_s* P) {
    return reinterpret_cast<const double*>(P->qr.p) + 1;
}

static void enqueue_start_cgls(rlsq_problem_s* P, LsmrState* S, cudaStream_t st, bool plain, bool split) {
    const int m = static_cast<int>(P->m), n = static_cast<int>(P->n);
    k_cgls_begin<<<grid_rows(P, std::max(m, n), 1), kBlock, 0, st>>>(m, n, P->b.p, P->qr.p, P->tx.p, S, P->part.p,
                                                                     P->counter.p);
    enqueue_cgls_z(P, S, st);                                      // z0 = A^T r0, ratio_0
    // h0 = M^{-1} z0 (or Algorithm 3 on r0), rho0
    enqueue_apply_any<true, true>(P, P->s.p, S, st, plain, split ? cgls_residual(P) : nullptr, 2);
    k_cgls_p<true><<<grid_rows(P, n, 1), kBlock, 0, st>>>(n, P->tx.p, P->h.p, S);  // p0 = h0
}

static void enqueue_iteration_cgls(rlsq_problem_s* P, LsmrState* S, cudaStream_t st, bool plain, bool split) {
    const int m = static_cast<int>(P->m), n = static_cast<int>(P->n);
    {
        RecScope rs(P, RLSQ_KCLASS_SPMV, mv_bytes(P->dA, 8.0, 16.0), st);
        with_G(P->map.G_A, [&](auto g) {
            k_cgls_q<decltype(g)::value><<<grid_rows(P, m, decltype(g)::value), kBlock, 0, st>>>(
                P->dA.view(), P->h.p, P->qr.p, S, P->part.p, P->counter.p);
        });
    }
    {
        RecScope rs(P, RLSQ_KCLASS_UPDATE, 32.0 * m + 24.0 * n, st);
        k_cgls_xr<<<grid_rows(P, std::max(m, n), 1), kBlock, 0, st>>>(m, n, P->h.p, P->qr.p, P->tx.p, S,
                                                                       P->part.p, P->counter.p);
    }
    enqueue_cgls_z(P, S, st);
    enqueue_apply_any<false, true>(P, P->s.p, S, st, plain, split ? cgls_residual(P) : nullptr, 2);
    RecScope rs(P, RLSQ_KCLASS_VEC, 24.0 * n, st);
    k_cgls_p<false><<<grid_rows(P, n, 1), kBlock, 0, st>>>(n, P->tx.p, P->h.p, S);
}

static LsmrState initial_state(const rlsq_problem_s* P, double atol, int maxit) {
    LsmrState s;
    std::memset(&s, 0, sizeof(s));
    s.anorm = P->anorm;
    s.atol = atol;
    s.maxit = maxit;
    s.rho = s.rhobar = s.cbar = 1.0;
    s.check = 1;
    return s;
}

static void put_state(rlsq_problem_s* P, LsmrState* S, const LsmrState& h, cudaStream_t st) {
    *P->pinned_state = h;
    RLSQ_CUDA(cudaMemcpyAsync(S, P->pinned_state, sizeof(LsmrState), cudaMemcpyHostToDevice, st));
    RLSQ_CUDA(cudaStreamSynchronize(st));
}

static void drop_graphs(rlsq_problem_s* P) {
    for (int i = 0; i < 5; ++i) {
        if (P->graph[i]) cudaGraphExecDestroy(P->graph[i]);
        P->graph[i] = nullptr;
        P->graph_iters[i] = 0;
    }
}

static cudaGraphExec_t iteration_graph(rlsq_problem_s* P, int iters, bool plain, bool cgls = false,
                                       bool split = false) {
    const int gi = (cgls && split && !plain) ? 4 : (plain ? 1 : 0) + (cgls ? 2 : 0);
    if (P->graph[gi] && P->graph_iters[gi] == iters) return P->graph[gi];
    if (P->graph[gi]) cudaGraphExecDestroy(P->graph[gi]);
    P->graph[gi] = nullptr;
    cudaStream_t st = P->stream;
    LsmrState* S = state_ptr(P, 0);
    RLSQ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        for (int i = 0; i < iters; ++i) {
            if (cgls) enqueue_iteration_cgls(P, S, st, plain, split);
            else enqueue_iteration(P, S, st, plain);
        }
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    cudaGraph_t g = nullptr;
    RLSQ_CUDA(cudaStreamEndCapture(st, &g));
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) throw_cuda(e, "cudaGraphInstantiate", __LINE__);
    P->graph[gi] = ex;
    P->graph_iters[gi] = iters;
    return ex;
}

// Algorithmic HBM bytes of one LSMR iteration: every stored entry of A, A^T
// and of each factor system once per use (value + int32 index), row
// pointers, each product's and solve's input and output vector once, and
// the LSMR vector passes (12 n-vectors and 6 m-vectors of float64).  Work
// the schedule adds -- fused level groups' extra entries, the explicit
// residual A x_k and A^T r_k the stopping test uses -- is not counted.
static double algorithmic_bytes(const rlsq_problem_s* P, bool plain) {
    const double m = static_cast<double>(P->m), n = static_cast<double>(P->n);
    const double dnnz = static_cast<double>(P->md) * n;
    double bytes = 2.0 * 12.0 * (static_cast<double>(P->nnz) - dnnz) + 2.0 * 8.0 * dnnz;  // A, A^T; dense block
    bytes += 4.0 * (m + n) + 16.0 * (m + n);  // row pointers of A and A^T; v^ -> q and u -> s
    bytes += 12.0 * 8.0 * n + 6.0 * 8.0 * m;  // LSMR vector passes
    if (plain || !P->F) return bytes;
    const IlupResult& F = *P->F;
    const double wv = (P->precision == RLSQ_PREC_FP32) ? 4.0 : 8.0;
    const double wf = wv + 4.0;
    const double m2 = m - n;
    const double tri_l1 = wf * F.L1.nnz() + 4.0 * n + 2.0 * wv * n;
    const double tri_u = wf * (F.U.nnz() + n) + 4.0 * n + 2.0 * wv * n;
    const double l2 = wf * F.L2.nnz() + 4.0 * (m2 + n) / 2.0 + wv * m;  // mean of L2 (m2 rows) and L2^T (n rows)
    const int k = P->opts.cg_steps;
    int c_l1 = 2, c_l2 = 0;
    double dense = 0.0;
    if (P->correction == RLSQ_CORR_SI || P->correction == RLSQ_CORR_DENSE) {
        c_l1 = 4;
        c_l2 = 2;
        if (P->correction == RLSQ_CORR_DENSE) dense = wv * m2 * m2;
    } else if (P->correction == RLSQ_CORR_CG) {
        // L1^{-T}, L1^{-1} before the correction and two per CG step; L2 once,
        // then L2^T and L2 per step (the apply ends with U^{-1}(q1 - z))
        c_l1 = 2 + 2 * k;
        c_l2 = 1 + 2 * k;
    }
    return bytes + 2.0 * tri_u + c_l1 * tri_l1 + c_l2 * l2 + dense;
}

static void fill_factor_info(const rlsq_problem_s* P, rlsq_info* info) {
    info->m = P->m;
    info->n = P->n;
    info->nnz_A = P->nnz;
    info->n_dense_rows = P->md;
    info->anorm = P->anorm;
    info->correction = P->correction;
    info->precision = P->precision;
    info->factor_seconds = P->factor_seconds;
    info->ilup_seconds = P->ilup_seconds;
    info->ilup_threads = P->ilup_threads;
    if (P->F) {
        const IlupResult& F = *P->F;
        info->nnz_L1 = F.L1.nnz();
        info->nnz_L2 = F.L2.nnz();
        info->nnz_U = F.U.nnz() + F.n;
        info->nmod = F.nmod;
        info->levels_L1 = F.lev_L1.nlevels;
        info->levels_L1t = F.lev_L1t.nlevels;
        info->levels_U = F.lev_U.nlevels;
        info->levels_Ut = F.lev_Ut.nlevels;
    }
    for (size_t w = 0; w < P->merged.size() && w < 4; ++w) {
        info->solve_levels[w] = P->merged[w].lev.nlevels;
        info->level_merge[w] = P->merged[w].k;
        info->trsv_schedule[w] = P->map.sched[w];
        info->solve_entries[w] = P->merged[w].T.nnz() + P->merged[w].R.nnz() + (w >= 2 ? P->n : 0);
    }
    info->bytes_per_iter = algorithmic_bytes(P, !P->factored);
    int sl = 0;
    if (prod_G(1, P->map.sl_A, P->dA) == 0) sl |= 1;
    if (prod_G(1, P->map.sl_At, P->dAt) == 0) sl |= 2;
    if (P->factored) {
        const bool f32 = P->precision == RLSQ_PREC_FP32;
        const int32_t np2 = f32 ? P->f32.L2.snpos : P->f64.L2.snpos, np2t = f32 ? P->f32.L2t.snpos : P->f64.L2t.snpos;
        if (P->map.sl_L2 && np2 > 0) sl |= 4;
        if (P->map.sl_L2t && np2t > 0) sl |= 8;
    }
    info->sliced_products = sl;
}

// b (user row order) -> P->b (internal row order: dense rows last)
static void upload_b(rlsq_problem_s* P, const double* b, bool dev, cudaStream_t st) {
    const auto kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (P->md == 0) {
        RLSQ_CUDA(cudaMemcpyAsync(P->b.p, b, sizeof(double) * P->m, kind, st));
        return;
    }
    double* tmp = reinterpret_cast<double*>(P->qr.p);  // 2m doubles, free before the solve starts
    RLSQ_CUDA(cudaMemcpyAsync(tmp, b, sizeof(double) * P->m, kind, st));
    k_gather<<<grid_rows(P, P->m, 1), kBlock, 0, st>>>(static_cast<int>(P->m), P->row_perm_d.p, tmp, P->b.p);
}

// Moves b in, runs LSMR, moves x out.
static int run_solve(rlsq_problem_s* P, const double* b, double* x, const rlsq_solve_opts* o,
                     rlsq_info* info, bool plain) {
    const auto t0 = std::chrono::steady_clock::now();
    rlsq_solve_opts opts;
    rlsq_solve_opts_default(&opts);
    if (o) opts = *o;
    if (!b || !x) throw ApiError(RLSQ_ERR_ARG, "null b or x");
    if (!(opts.atol >= 0.0) || opts.maxit < 0) throw ApiError(RLSQ_ERR_ARG, "bad atol or maxit");
    if (!plain && !P->factored) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
    if (opts.solver != RLSQ_SOLVER_LSMR && opts.solver != RLSQ_SOLVER_CGLS && opts.solver != RLSQ_SOLVER_CGLS_SPLIT)
        throw ApiError(RLSQ_ERR_ARG, "bad solver");
    const bool cgls = opts.solver != RLSQ_SOLVER_LSMR;
    const bool split = opts.solver == RLSQ_SOLVER_CGLS_SPLIT;
    if (cgls && P->md > 0) throw ApiError(RLSQ_ERR_ARG, "the CGLS solver does not take dense-row problems");
    const int iters = std::max(1, opts.check_every);
    cudaStream_t st = P->stream;
    cudaStream_t user = static_cast<cudaStream_t>(opts.stream);
    const bool dev = opts.ptr_mode == RLSQ_DEVICE_PTRS;
    if (dev) {
        RLSQ_CUDA(cudaEventRecord(P->ev[0], user));
        RLSQ_CUDA(cudaStreamWaitEvent(st, P->ev[0], 0));
    }
    upload_b(P, b, dev, st);
    LsmrState* S = state_ptr(P, 0);
    put_state(P, S, initial_state(P, opts.atol, opts.maxit), st);
    if (cgls) enqueue_start_cgls(P, S, st, plain, split);
    else enqueue_start(P, S, st, plain);
    cudaGraphExec_t g = iteration_graph(P, iters, plain, cgls, split);
    const int64_t max_launches = static_cast<int64_t>(opts.maxit) / iters + 4;
    int64_t launches = 0;
    // two graphs in flight; read `done` of the older one
    int* done = P->pinned_done;
    done[0] = done[1] = 0;
    RLSQ_CUDA(cudaGraphLaunch(g, st));
    RLSQ_CUDA(cudaMemcpyAsync(&done[0], reinterpret_cast<char*>(S) + offsetof(LsmrState, done), sizeof(int),
                              cudaMemcpyDeviceToHost, st));
    RLSQ_CUDA(cudaEventRecord(P->ev[0], st));
    ++launches;
    int cur = 0;
    for (;;) {
        const int nxt = cur ^ 1;
        RLSQ_CUDA(cudaGraphLaunch(g, st));
        RLSQ_CUDA(cudaMemcpyAsync(&done[nxt], reinterpret_cast<char*>(S) + offsetof(LsmrState, done),
                                  sizeof(int), cudaMemcpyDeviceToHost, st));
        RLSQ_CUDA(cudaEventRecord(P->ev[nxt], st));
        ++launches;
        RLSQ_CUDA(cudaEventSynchronize(P->ev[cur]));
        if (done[cur]) break;
        if (launches > max_launches) break;
        cur = nxt;
    }
    RLSQ_CUDA(cudaStreamSynchronize(st));
    LsmrState hs;
    RLSQ_CUDA(cudaMemcpy(&hs, S, sizeof(LsmrState), cudaMemcpyDeviceToHost));
    if (!hs.done) throw ApiError(RLSQ_ERR_CUDA, "solver did not reach a stopping point");
    // x_j lives at tx[j].y; s is free once the solve has stopped
    copy_half(x, P->tx.p, P->n, 1, dev, P->s.p, st);
    RLSQ_CUDA(cudaStreamSynchronize(st));
    if (dev) {
        RLSQ_CUDA(cudaEventRecord(P->ev[0], st));
        RLSQ_CUDA(cudaStreamWaitEvent(user, P->ev[0], 0));
    }
    int status = hs.status;
    if (hs.error != 0) status = RLSQ_ERR_DEVICE_TIMEOUT;
    if (info) {
        std::memset(info, 0, sizeof(*info));
        fill_factor_info(P, info);
        if (plain) {
            info->correction = -1;
            info->bytes_per_iter = algorithmic_bytes(P, true);
        }
        info->status = status;
        info->iterations = hs.k;
        info->ratio = hs.ratio;
        info->rnorm = hs.rnorm;
        info->arnorm = hs.arnorm;
        info->solve_seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status == RLSQ_ERR_BREAKDOWN) set_last_error("<s, M^{-1} s> <= 0: preconditioner not positive");
    else if (status == RLSQ_ERR_MAXIT) set_last_error("iteration limit reached");
    else if (status == RLSQ_ERR_DEVICE_TIMEOUT) set_last_error("a sync-free triangular solve timed out");
    return status;
}

// Splits A into sparse rows (CSR + CSC, internal order: sparse rows first in
// user order, dense rows last and empty) and a dense row-major block.  A row
// is dense when it has at least `threshold` nonzeros (threshold <= 0: no
// dense rows); at most kMaxDenseRows rows are taken, densest first.
constexpr int64_t kMaxDenseRows = 3000;  // the A^T kernel keeps them in 48 KB of shared memory

static int64_t auto_dense_threshold(const HostCSR& A) {
    std::vector<int64_t> len(static_cast<size_t>(A.rows));
    for (int64_t i = 0; i < A.rows; ++i) len[i] = A.ptr[i + 1] - A.ptr[i];
    std::nth_element(len.begin(), len.begin() + len.size() / 2, len.end());
    const int64_t med = len[len.size() / 2];
    return std::max<int64_t>(64, 16 * std::max<int64_t>(med, 1));
}

// sliced: also the sliced layout of A and A^T (the products may run on it)
static void layout_A(rlsq_problem_s* P, int64_t threshold, bool sliced = false) {
    P->layout_threshold = threshold;
    const HostCSR& A = P->A;
    const int64_t m = A.rows, n = A.cols;
    std::vector<int32_t> dense;
    if (threshold > 0)
        for (int64_t i = 0; i < m; ++i)
            if (A.ptr[i + 1] - A.ptr[i] >= threshold) dense.push_back(static_cast<int32_t>(i));
    if (static_cast<int64_t>(dense.size()) > kMaxDenseRows) {
        std::stable_sort(dense.begin(), dense.end(), [&](int32_t a, int32_t b) {
            return A.ptr[a + 1] - A.ptr[a] > A.ptr[b + 1] - A.ptr[b];
        });
        dense.resize(kMaxDenseRows);
        std::sort(dense.begin(), dense.end());
    }
    cudaStream_t st = P->stream;
    P->md = static_cast<int64_t>(dense.size());
    P->ms = m - P->md;
    if (P->md == 0) {
        P->row_perm.clear();
        P->row_perm_d.release();
        P->Ad.release();
        P->dA.upload(A, st, sliced);
        P->dAt.upload(transpose(A, ilup_threads(0, A.rows, A.cols)), st, sliced);
        return;
    }
    std::vector<char> is_dense(static_cast<size_t>(m), 0);
    for (int32_t r : dense) is_dense[r] = 1;
    P->row_perm.clear();
    for (int64_t i = 0; i < m; ++i)
        if (!is_dense[i]) P->row_perm.push_back(static_cast<int32_t>(i));
    for (int32_t r : dense) P->row_perm.push_back(r);
    HostCSR S;
    S.rows = m;
    S.cols = n;
    S.ptr.assign(static_cast<size_t>(m) + 1, 0);
    for (int64_t i = 0; i < P->ms; ++i) {
        const int32_t r = P->row_perm[i];
        for (int64_t e = A.ptr[r]; e < A.ptr[r + 1]; ++e) {
            S.idx.push_back(A.idx[e]);
            S.val.push_back(A.val[e]);
        }
        S.ptr[i + 1] = static_cast<int64_t>(S.idx.size());
    }
    for (int64_t i = P->ms; i < m; ++i) S.ptr[i + 1] = S.ptr[i];
    P->dA.upload(S, st, sliced);
    P->dAt.upload(transpose(S, ilup_threads(0, S.rows, S.cols)), st, sliced);
    std::vector<double> ad(static_cast<size_t>(P->md * n), 0.0);
    for (int64_t q = 0; q < P->md; ++q) {
        const int32_t r = dense[q];
        for (int64_t e = A.ptr[r]; e < A.ptr[r + 1]; ++e) ad[q * n + A.idx[e]] = A.val[e];
    }
    P->Ad.upload(ad.data(), ad.size(), st);
    P->row_perm_d.upload(P->row_perm.data(), P->row_perm.size(), st);
    P->dense_chunks = static_cast<int>((n + kDenseChunk - 1) / kDenseChunk);
    P->dense_part.alloc(static_cast<size_t>(P->md * P->dense_chunks));
    P->dense_av.alloc(static_cast<size_t>(P->md));
    P->dense_atv.alloc(static_cast<size_t>(n));
    RLSQ_CUDA(cudaStreamSynchronize(st));
}

// A_d (v1, v2) -> dense_av; PAIR reads interleaved pairs, else (v, 0).
template <bool PAIR>
static void enqueue_dense_av(rlsq_problem_s* P, const void* v, const LsmrState* S, cudaStream_t st) {
    const int md = static_cast<int>(P->md), n = static_cast<int>(P->n);
    dim3 grid(static_cast<unsigned>(P->dense_chunks), static_cast<unsigned>((md + kDenseRowsPerBlock - 1) / kDenseRowsPerBlock));
    k_dense_av<PAIR><<<grid, kBlock, 0, st>>>(P->Ad.p, md, n, v, P->dense_part.p, S);
    k_dense_av_finish<<<(md + kBlock - 1) / kBlock, kBlock, 0, st>>>(md, P->dense_chunks, P->dense_part.p,
                                                                    P->dense_av.p, S);
}
// A_d^T (u1, u2) -> dense_atv; u points at the dense rows' entries
template <bool PAIR>
static void enqueue_dense_atv(rlsq_problem_s* P, const void* u, const LsmrState* S, cudaStream_t st) {
    const int md = static_cast<int>(P->md), n = static_cast<int>(P->n);
    const int grid = static_cast<int>(std::min<int64_t>((n + kBlock - 1) / kBlock, max_grid(P)));
    k_dense_atv<PAIR><<<grid, kBlock, sizeof(double2) * md, st>>>(P->Ad.p, md, n, u, P->dense_atv.p, S);
}

// ||A||_2 by 50 power iterations on A^T A from v = 1/sqrt(n) (Sec. 5.1)
static double power_norm(rlsq_problem_s* P, int iters) {
    cudaStream_t st = P->stream;
    const int m = static_cast<int>(P->m), n = static_cast<int>(P->n);
    DevArray<double> v, y;
    DevArray<PowerState> ps;
    v.alloc(n);
    y.alloc(m);
    ps.alloc(1);
    std::vector<double> v0(static_cast<size_t>(n), 1.0 / std::sqrt(static_cast<double>(n)));
    RLSQ_CUDA(cudaMemcpyAsync(v.p, v0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    PowerState p0{0.0, 1.0};
    RLSQ_CUDA(cudaMemcpyAsync(ps.p, &p0, sizeof(p0), cudaMemcpyHostToDevice, st));
    const bool dense = P->md > 0;
    for (int it = 0; it < iters; ++it) {
        with_G(P->map.G_A, [&](auto g) {
            k_power_av<decltype(g)::value><<<grid_rows(P, m, decltype(g)::value), kBlock, 0, st>>>(
                P->dA.view(), v.p, y.p, ps.p);
        });
        if (dense) {
            enqueue_dense_av<false>(P, v.p, nullptr, st);
            k_put_dense<<<static_cast<int>((P->md + kBlock - 1) / kBlock), kBlock, 0, st>>>(
                static_cast<int>(P->md), static_cast<int>(P->ms), P->dense_av.p, y.p, ps.p);
            enqueue_dense_atv<false>(P, y.p + P->ms, nullptr, st);
        }
        with_G(P->map.G_At, [&](auto g) {
            k_power_atv<decltype(g)::value><<<grid_rows(P, n, decltype(g)::value), kBlock, 0, st>>>(
                P->dAt.view(), y.p, v.p, ps.p, P->part.p, P->counter.p, dense ? P->dense_atv.p : nullptr);
        });
    }
    PowerState out;
    RLSQ_CUDA(cudaMemcpyAsync(&out, ps.p, sizeof(out), cudaMemcpyDeviceToHost, st));
    RLSQ_CUDA(cudaStreamSynchronize(st));
    return std::sqrt(out.lambda);
}

static int pow2_lanes(double avg, int lo, int hi) {
    int g = lo;
    while (g < hi && g < avg) g *= 2;
    return g;
}

void default_mapping(rlsq_problem_s* P) {
    const double m = static_cast<double>(P->m), n = static_cast<double>(P->n);
    // about four entries per lane; the autotuner refines this
    P->map.G_A = pow2_lanes(P->nnz / m / 4.0, 1, 32);
    P->map.G_At = pow2_lanes(P->nnz / n / 4.0, 1, 32);
    if (P->F) {
        const IlupResult& F = *P->F;
        const HostCSR* parts[4] = {&F.L1, &F.L1t, &F.U, &F.Ut};
        for (int w = 0; w < 4; ++w) {
            // one thread per row unless rows are long
            const double nz = P->merged.size() == 4 ? static_cast<double>(P->merged[w].T.nnz())
                                                    : static_cast<double>(parts[w]->nnz());
            const double avg = nz / std::max(1.0, n);
            P->map.G_tri[w] = avg <= 12.0 ? 1 : pow2_lanes(avg / 4.0, 1, 32);
            P->map.sched[w] = RLSQ_TRSV_SYNCFREE;
            P->map.sf_blocks[w] = 2;
            P->map.sf_rows[w] = 0;
            P->map.wave_kp[w] = 4;
        }
        P->map.G_L2 = pow2_lanes(F.L2.nnz() / std::max(1.0, m - n) / 4.0, 1, 32);
        P->map.G_L2t = pow2_lanes(F.L2t.nnz() / std::max(1.0, n) / 4.0, 1, 32);
    }
}

void autotune(rlsq_problem_s* P, int mode);  // autotune.cu
void device_schur_inverse(const IlupResult& F, DevArray<double>& out, cudaStream_t st, int num_sms);  // schur.cu

// Times one standalone solve of system `which` with the current mapping
// (used by the autotuner); inputs in vn[3], output in vn[4].
int rlsq_trsv_time(rlsq_problem_s* P, int which, float* ms) {
    cudaStream_t st = P->stream;
    LsmrState* S = state_ptr(P, 1);
    put_state(P, S, initial_state(P, 0.0, 0), st);
    cudaEvent_t a, b;
    RLSQ_CUDA(cudaEventCreate(&a));
    RLSQ_CUDA(cudaEventCreate(&b));
    auto body = [&]() {
        RLSQ_CUDA(cudaMemsetAsync(P->tickets.p, 0, sizeof(unsigned) * kMaxSlots, st));
        RLSQ_CUDA(cudaMemsetAsync(P->barriers.p, 0, sizeof(unsigned) * kMaxSlots, st));
        if (P->precision == RLSQ_PREC_FP32)
            launch_trsv<float>(P, P->f32, which, RHS_VEC, Rhs<float>{P->f32.vn[3].p, nullptr, nullptr},
                               P->f32.vn[4].p, 0, S, st);
        else
            launch_trsv<double>(P, P->f64, which, RHS_VEC, Rhs<double>{P->f64.vn[3].p, nullptr, nullptr},
                                P->f64.vn[4].p, 0, S, st);
        RLSQ_CUDA(cudaGetLastError());
    };
    body();
    std::vector<float> ts;
    for (int i = 0; i < 5; ++i) {
        RLSQ_CUDA(cudaEventRecord(a, st));
        body();
        RLSQ_CUDA(cudaEventRecord(b, st));
        RLSQ_CUDA(cudaEventSynchronize(b));
        float t = 0.f;
        RLSQ_CUDA(cudaEventElapsedTime(&t, a, b));
        ts.push_back(t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    RLSQ_CUDA(cudaMemcpy(P->pinned_state, S, sizeof(LsmrState), cudaMemcpyDeviceToHost));
    if (P->pinned_state->error) return RLSQ_ERR_DEVICE_TIMEOUT;
    std::sort(ts.begin(), ts.end());
    *ms = ts[ts.size() / 2];
    return RLSQ_OK;
}


}  // namespace rlsq

using namespace rlsq;

rlsq_problem_s::~rlsq_problem_s() {
    drop_graphs(this);
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (pinned_state) cudaFreeHost(pinned_state);
    if (pinned_done) cudaFreeHost(pinned_done);
    if (stream) cudaStreamDestroy(stream);
}

extern "C" {

void rlsq_factor_opts_default(rlsq_factor_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->p = 10;
    o->tau = 1e-2;
    o->mu = 0.1;
    o->small = 1e-10;
    o->scale_columns = 1;
    o->correction = RLSQ_CORR_AUTO;
    o->cg_steps = 2;
    o->dense_cap = 1024;
    o->precision = RLSQ_PREC_FP64;
    o->trsv_schedule = RLSQ_TRSV_AUTO;
    o->autotune = 0;
    o->dense_row_min = 0;
    o->host_threads = 0;
    o->level_merge = 0;
    o->sliced = -1;
}

void rlsq_solve_opts_default(rlsq_solve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->atol = 1e-8;
    o->maxit = 2000;
    o->ptr_mode = RLSQ_HOST_PTRS;
    o->stream = nullptr;
    o->check_every = 8;
    o->solver = RLSQ_SOLVER_LSMR;
}

const char* rlsq_last_error(void) { return g_last_error.c_str(); }

int rlsq_create(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* vals,
                int32_t ptr_mode, void* stream, rlsq_problem* out) {
    return guarded([&]() -> int {
        if (!out || !rowptr || (!colidx && m > 0) || (!vals && m > 0))
            throw ApiError(RLSQ_ERR_ARG, "null argument");
        *out = nullptr;
        if (!(m > n && n > 0)) throw ApiError(RLSQ_ERR_SHAPE, "need m > n > 0");
        if (m >= (int64_t(1) << 31)) throw ApiError(RLSQ_ERR_SHAPE, "m must be < 2^31");
        std::unique_ptr<rlsq_problem_s> P(new rlsq_problem_s());
        P->m = m;
        P->n = n;
        HostCSR& A = P->A;
        A.rows = m;
        A.cols = n;
        A.ptr.resize(static_cast<size_t>(m) + 1);
        const bool dev = ptr_mode == RLSQ_DEVICE_PTRS;
        cudaStream_t user = static_cast<cudaStream_t>(stream);
        if (dev) {
            RLSQ_CUDA(cudaMemcpyAsync(A.ptr.data(), rowptr, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost, user));
            RLSQ_CUDA(cudaStreamSynchronize(user));
        } else {
            std::memcpy(A.ptr.data(), rowptr, sizeof(int64_t) * (m + 1));
        }
        if (A.ptr[0] != 0) throw ApiError(RLSQ_ERR_CSR, "rowptr[0] must be 0");
        for (int64_t i = 0; i < m; ++i)
            if (A.ptr[i + 1] < A.ptr[i]) throw ApiError(RLSQ_ERR_CSR, "rowptr must be nondecreasing");
        const int64_t nnz = A.ptr[m];
        if (nnz >= (int64_t(1) << 31)) throw ApiError(RLSQ_ERR_SHAPE, "nnz must be < 2^31");
        A.idx.resize(static_cast<size_t>(nnz));
        A.val.resize(static_cast<size_t>(nnz));
        if (dev) {
            RLSQ_CUDA(cudaMemcpyAsync(A.idx.data(), colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, user));
            RLSQ_CUDA(cudaMemcpyAsync(A.val.data(), vals, sizeof(double) * nnz, cudaMemcpyDeviceToHost, user));
            RLSQ_CUDA(cudaStreamSynchronize(user));
        } else {
            std::memcpy(A.idx.data(), colidx, sizeof(int32_t) * nnz);
            std::memcpy(A.val.data(), vals, sizeof(double) * nnz);
        }
        std::vector<char> seen(static_cast<size_t>(n), 0);
        for (int64_t i = 0; i < m; ++i)
            for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
                const int32_t c = A.idx[e];
                if (c < 0 || c >= n) throw ApiError(RLSQ_ERR_CSR, "column index out of range");
                if (e > A.ptr[i] && c <= A.idx[e - 1])
                    throw ApiError(RLSQ_ERR_CSR, "column indices must be strictly increasing within a row");
                if (!std::isfinite(A.val[e])) throw ApiError(RLSQ_ERR_CSR, "non-finite value");
                if (A.val[e] != 0.0) seen[c] = 1;
            }
        for (int64_t j = 0; j < n; ++j)
            if (!seen[j]) throw ApiError(RLSQ_ERR_RANK, "column " + std::to_string(j) + " is empty");
        P->nnz = nnz;
        RLSQ_CUDA(cudaGetDevice(&P->device));
        RLSQ_CUDA(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device));
        RLSQ_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
        RLSQ_CUDA(cudaEventCreateWithFlags(&P->ev[0], cudaEventDisableTiming));
        RLSQ_CUDA(cudaEventCreateWithFlags(&P->ev[1], cudaEventDisableTiming));
        RLSQ_CUDA(cudaMallocHost(reinterpret_cast<void**>(&P->pinned_state), sizeof(LsmrState)));
        RLSQ_CUDA(cudaMallocHost(reinterpret_cast<void**>(&P->pinned_done), 2 * sizeof(int)));
        cudaStream_t st = P->stream;
        layout_A(P.get(), auto_dense_threshold(A));
        P->qr.alloc(static_cast<size_t>(m));
        P->tx.alloc(static_cast<size_t>(n));
        P->b.alloc(static_cast<size_t>(m));
        for (auto* v : {&P->s, &P->h, &P->hb}) v->alloc(static_cast<size_t>(n));
        P->S.alloc(3);  // the solve's state, a scratch state, the adaptive-CG gate
        P->part.alloc(static_cast<size_t>(max_grid(P.get())) * 2);
        P->counter.alloc(1);
        RLSQ_CUDA(cudaMemsetAsync(P->counter.p, 0, sizeof(unsigned), st));
        P->tickets.alloc(kMaxSlots);
        P->barriers.alloc(kMaxSlots);
        {
            coop_attributes<double>();
            coop_attributes<float>();
            int occ = 0;
            RLSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trsv_coop<double, RHS_VEC, 8>, kCoopBlock,
                                                                    coop_smem_bytes<double>(8)));
            int occ32 = 0;
            RLSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, k_trsv_coop<float, RHS_VEC, 8>, kCoopBlock,
                                                                    coop_smem_bytes<float>(8)));
            P->coop_blocks = std::max(1, std::min(occ, occ32)) * P->num_sms;
        }
        default_mapping(P.get());
        P->anorm = power_norm(P.get(), 50);
        *out = P.release();
        return RLSQ_OK;
    });
}

int rlsq_factor(rlsq_problem h, const rlsq_factor_opts* o) {
    return guarded([&]() -> int {
        if (!h) throw ApiError(RLSQ_ERR_ARG, "null handle");
        if (h->served.load() > 0) throw ApiError(RLSQ_ERR_ARG, "the problem is registered with a server");
        rlsq_factor_opts opts;
        rlsq_factor_opts_default(&opts);
        if (o) opts = *o;
        if (!(opts.mu > 0.0 && opts.mu <= 1.0) || !(opts.tau >= 0.0) || !(opts.small > 0.0) ||
            opts.cg_steps < 1 || opts.correction < 0 || opts.correction > RLSQ_CORR_AUTO ||
            (opts.precision != RLSQ_PREC_FP64 && opts.precision != RLSQ_PREC_FP32))
            throw ApiError(RLSQ_ERR_ARG, "bad factor option");
        if (opts.cg_steps > 16) throw ApiError(RLSQ_ERR_ARG, "cg_steps must be <= 16");
        if (opts.trsv_rows != 0 && opts.trsv_rows != 1 && opts.trsv_rows != 2 && opts.trsv_rows != 4)
            throw ApiError(RLSQ_ERR_ARG, "trsv_rows must be 0, 1, 2 or 4");
        if (!(opts.cg_tol >= 0.0 && opts.cg_tol < 1.0)) throw ApiError(RLSQ_ERR_ARG, "cg_tol must be in [0, 1)");
        if (opts.sliced < -1 || opts.sliced > 1) throw ApiError(RLSQ_ERR_ARG, "sliced must be -1, 0 or 1");
        const auto t0 = std::chrono::steady_clock::now();
        h->factored = false;
        drop_graphs(h);
        IlupParams prm;
        prm.p = opts.p;
        prm.tau = opts.tau;
        prm.mu = opts.mu;
        prm.small = opts.small;
        prm.scale = opts.scale_columns != 0;
        prm.threads = ilup_threads(opts.host_threads, h->m, h->n);
        // The host factor depends only on (p, tau, mu, small, scaling): a call
        // that changes the correction, precision or schedule re-uses it.
        std::unique_ptr<IlupResult> F;
        const bool same = h->F && h->opts.p == opts.p && h->opts.tau == opts.tau &&
                          h->opts.mu == opts.mu && h->opts.small == opts.small &&
                          h->opts.scale_columns == opts.scale_columns;
        if (same) {
            F = std::move(h->F);
        } else {
            h->F.reset();
            h->sinv_valid = false;
            try {
                const auto t_ilup = std::chrono::steady_clock::now();
                F.reset(new IlupResult(ilup_factor(h->A, prm)));
                h->ilup_seconds =
                    std::chrono::duration<double>(std::chrono::steady_clock::now() - t_ilup).count();
                h->ilup_threads = prm.threads;
            } catch (const std::runtime_error& e) {
                throw ApiError(RLSQ_ERR_RANK, e.what());
            }
        }
        int corr = opts.correction;
        const int64_t m2 = h->m - h->n;
        // the dense S is formed through Z = L1^{-T} L2^T (n x (m-n) float64), so the
        // automatic choice also keeps that within 2 GiB
        if (corr == RLSQ_CORR_AUTO)
            corr = (m2 <= opts.dense_cap && static_cast<double>(h->n) * static_cast<double>(m2) * 8.0 <= 2147483648.0)
                       ? RLSQ_CORR_DENSE
                       : RLSQ_CORR_CG;
        std::vector<double> sinv;
        bool sinv_on_device = false;
        if (corr == RLSQ_CORR_DENSE) {
            if (h->sinv_valid) {
                sinv = h->sinv_host;  // formed for this factor, or updated with its rows
            } else if (!opts.dense_host) {
                sinv_on_device = true;  // formed below, once the factor is on the device
            } else {
                int th = opts.host_threads > 0 ? opts.host_threads
                                               : static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
                const bool keep = static_cast<double>(F->n) * static_cast<double>(F->m - F->n) * 8.0 <= 2147483648.0;
                h->sinv_z.clear();
                if (!dense_schur_inverse(*F, sinv, th, keep ? &h->sinv_z : nullptr))
                    throw ApiError(RLSQ_ERR_NUMERIC, "dense S is not positive definite");
                h->sinv_host = sinv;
                h->sinv_valid = true;
            }
        }
        cudaStream_t st = h->stream;
        // fused levels per system (0: the grouping of least modelled time
        // under the cost model of host_setup.h)
        h->merged.clear();
        {
            const HostCSR* parts[4] = {&F->L1, &F->L1t, &F->U, &F->Ut};
            const Levels* levs[4] = {&F->lev_L1, &F->lev_L1t, &F->lev_U, &F->lev_Ut};
            const double wv = opts.precision == RLSQ_PREC_FP32 ? 4.0 : 8.0;
            const double entry_s = (wv + 4.0) / 12.0 * kEntryCost;
            // candidates per system: 0 = as is, 1 = groups grown level by level
            // (a level joins while its fill costs less than the level it saves),
            // 2..4 = fixed k; every candidate is a pure function of the factor,
            // so they are built on separate host threads
            const int ncand = opts.level_merge >= 1 ? 1 : 5;
            std::vector<std::vector<MergedTri>> cand(4, std::vector<MergedTri>(static_cast<size_t>(ncand)));
            std::exception_ptr failed;
            std::mutex fail_mu;
            std::vector<std::thread> pool;
            for (int w = 0; w < 4; ++w)
                for (int c = 0; c < ncand; ++c)
                    pool.emplace_back([&, w, c]() {
                        try {
                            const double* dg = w >= 2 ? F->Udiag.data() : nullptr;
                            MergedTri& out = cand[static_cast<size_t>(w)][static_cast<size_t>(c)];
                            if (opts.level_merge >= 1) out = merge_levels(*parts[w], dg, *levs[w], opts.level_merge);
                            else if (c == 0) out = merge_levels(*parts[w], dg, *levs[w], 1);
                            else if (c == 1)
                                out = merge_levels_adaptive(*parts[w], dg, *levs[w], kLevelCost / entry_s, kMaxFusedGroup);
                            else
                                out = merge_levels(*parts[w], dg, *levs[w], c, 4 * std::max<int64_t>(parts[w]->nnz(), h->n));
                        } catch (...) {
                            std::lock_guard<std::mutex> lock(fail_mu);
                            if (!failed) failed = std::current_exception();
                        }
                    });
            for (auto& t : pool) t.join();
            if (failed) std::rethrow_exception(failed);
            auto cost = [&](const MergedTri& M) {
                return M.lev.nlevels * kLevelCost + entry_s * static_cast<double>(M.T.nnz() + M.R.nnz());
            };
            for (int w = 0; w < 4; ++w) {
                auto& cw = cand[static_cast<size_t>(w)];
                size_t best = 0;
                double cbest = cost(cw[0]);
                // earlier candidates win ties; fixed k stops at the first k the fill cap rejects
                for (size_t c = 1; c < cw.size(); ++c) {
                    if (c >= 2 && cw[c].k == 0) break;
                    const double cc = cost(cw[c]);
                    if (cc < cbest) {
                        cbest = cc;
                        best = c;
                    }
                }
                h->merged.push_back(std::move(cw[best]));
            }
        }
        h->f64.clear();
        h->f32.clear();
        // the sliced copies of the products' matrices only where they may run
        const bool want_sliced = opts.sliced == 1 || (opts.sliced < 0 && opts.autotune != 0);
        if (opts.precision == RLSQ_PREC_FP32) h->f32.upload(*F, h->merged.data(), sinv, st, want_sliced);
        else h->f64.upload(*F, h->merged.data(), sinv, st, want_sliced);
        if (sinv_on_device) {
            DevArray<double> sd;
            device_schur_inverse(*F, sd, st, h->num_sms);
            const size_t cnt = static_cast<size_t>(m2) * static_cast<size_t>(m2);
            if (opts.precision == RLSQ_PREC_FP32) {
                h->f32.sinv.alloc(cnt);
                const int grid = static_cast<int>(std::max<size_t>(1, std::min<size_t>((cnt + kBlock - 1) / kBlock, 4096)));
                k_convert<float, double><<<grid, kBlock, 0, st>>>(static_cast<int>(cnt), sd.p, h->f32.sinv.p);
                RLSQ_CUDA(cudaGetLastError());
            } else {
                h->f64.sinv.alloc(cnt);
                RLSQ_CUDA(cudaMemcpyAsync(h->f64.sinv.p, sd.p, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
            }
            RLSQ_CUDA(cudaStreamSynchronize(st));
        }
        if (opts.dense_row_min != 0) {
            // an explicit dense-row threshold (< 0: none) replaces the automatic one
            layout_A(h, opts.dense_row_min, want_sliced);
            h->anorm = power_norm(h, 50);
        } else if (want_sliced && (h->dA.snpos == 0 || h->dAt.snpos == 0)) {
            layout_A(h, h->layout_threshold, true);
        }
        h->F = std::move(F);
        h->opts = opts;
        h->correction = corr;
        h->precision = opts.precision;
        default_mapping(h);
        h->map.sl_A = h->map.sl_At = h->map.sl_L2 = h->map.sl_L2t = (opts.sliced == 1) ? 1 : 0;
        if (opts.trsv_schedule == RLSQ_TRSV_LEVEL || opts.trsv_schedule == RLSQ_TRSV_SYNCFREE ||
            opts.trsv_schedule == RLSQ_TRSV_COOP || opts.trsv_schedule == RLSQ_TRSV_WAVE ||
            opts.trsv_schedule == RLSQ_TRSV_BINNED)
            for (int w = 0; w < 4; ++w) h->map.sched[w] = opts.trsv_schedule;
        for (int w = 0; w < 4; ++w) {
            h->map.sf_rows[w] = opts.trsv_rows;
            // the warp-ticketed solve takes at most 8 lanes per row
            if (opts.trsv_rows > 0) h->map.G_tri[w] = std::min(h->map.G_tri[w], 8);
        }
        h->factored = true;
        if (opts.autotune) autotune(h, opts.autotune == 2 ? 2 : 1);
        h->factor_seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return RLSQ_OK;
    });
}

// Sec. 3.4 on a GPU handle: the host factor is updated (rows join A2 / A2
// rows leave, L1 and U kept), then A's device layout, the m-sized vectors and
// the device factor are rebuilt with the handle's own options (rlsq_factor
// finds the ILUP parameters unchanged and keeps the updated host factor).
static void refresh_after_rows(rlsq_problem_s* h) {
    cudaStream_t st = h->stream;
    h->m = h->A.rows;
    h->nnz = h->A.nnz();
    const int64_t thr = h->opts.dense_row_min != 0 ? h->opts.dense_row_min : auto_dense_threshold(h->A);
    layout_A(h, thr);
    h->qr.alloc(static_cast<size_t>(h->m));
    h->b.alloc(static_cast<size_t>(h->m));
    RLSQ_CUDA(cudaStreamSynchronize(st));
    h->anorm = power_norm(h, 50);
    const rlsq_factor_opts o = h->opts;
    const int code = rlsq_factor(h, &o);
    if (code != RLSQ_OK) throw ApiError(code, "refactor after the row update failed");
}

int rlsq_add_rows(rlsq_problem h, int64_t k, const int64_t* rowptr, const int32_t* colidx, const double* vals) {
    return guarded([&]() -> int {
        if (!h || !rowptr || (k > 0 && (!colidx || !vals)) || k < 0) throw ApiError(RLSQ_ERR_ARG, "bad argument");
        if (h->served.load() > 0) throw ApiError(RLSQ_ERR_ARG, "the problem is registered with a server");
        if (!h->factored || !h->F) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        if (rowptr[0] != 0) throw ApiError(RLSQ_ERR_CSR, "rowptr[0] must be 0");
        const int64_t n = h->n;
        for (int64_t i = 0; i < k; ++i) {
            if (rowptr[i + 1] < rowptr[i]) throw ApiError(RLSQ_ERR_CSR, "rowptr must be nondecreasing");
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                if (colidx[e] < 0 || colidx[e] >= n) throw ApiError(RLSQ_ERR_CSR, "column index out of range");
                if (e > rowptr[i] && colidx[e] <= colidx[e - 1])
                    throw ApiError(RLSQ_ERR_CSR, "column indices must be strictly increasing within a row");
                if (!std::isfinite(vals[e])) throw ApiError(RLSQ_ERR_CSR, "non-finite value");
            }
        }
        if (h->m + k >= (int64_t(1) << 31) || h->A.nnz() + rowptr[k] >= (int64_t(1) << 31))
            throw ApiError(RLSQ_ERR_SHAPE, "sizes must stay < 2^31");
        HostCSR rows;
        rows.rows = k;
        rows.cols = n;
        rows.ptr.assign(rowptr, rowptr + k + 1);
        rows.idx.assign(colidx, colidx + rowptr[k]);
        rows.val.assign(vals, vals + rowptr[k]);
        IlupParams prm;
        prm.p = h->opts.p;
        prm.tau = h->opts.tau;
        prm.mu = h->opts.mu;
        prm.small = h->opts.small;
        prm.scale = h->opts.scale_columns != 0;
        add_rows(*h->F, rows, prm);
        if (h->sinv_valid) {
            try {
                if (h->sinv_z.empty()) throw std::runtime_error("Z is not kept");
                schur_inverse_add(*h->F, k, h->sinv_host, h->sinv_z);
            } catch (const std::exception&) {
                h->sinv_valid = false;  // formed again by the refresh if needed
            }
        }
        HostCSR& A = h->A;
        const int64_t base = A.nnz();
        for (int64_t i = 0; i < k; ++i) A.ptr.push_back(base + rowptr[i + 1]);
        A.idx.insert(A.idx.end(), rows.idx.begin(), rows.idx.end());
        A.val.insert(A.val.end(), rows.val.begin(), rows.val.end());
        A.rows += k;
        refresh_after_rows(h);
        return RLSQ_OK;
    });
}

int rlsq_remove_rows(rlsq_problem h, int64_t k, const int32_t* ids) {
    return guarded([&]() -> int {
        if (!h || (k > 0 && !ids) || k < 0) throw ApiError(RLSQ_ERR_ARG, "bad argument");
        if (h->served.load() > 0) throw ApiError(RLSQ_ERR_ARG, "the problem is registered with a server");
        if (!h->factored || !h->F) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        std::vector<int32_t> v(ids, ids + k);
        // positions of the rows in A2 before the removal (for S^{-1})
        const int64_t m2_before = h->F->m - h->F->n;
        std::vector<int64_t> pos;
        for (const int32_t r : v)
            pos.push_back(std::lower_bound(h->F->a2rows.begin(), h->F->a2rows.end(), r) - h->F->a2rows.begin());
        try {
            remove_rows(*h->F, v);
        } catch (const std::invalid_argument& e) {
            throw ApiError(RLSQ_ERR_ARG, e.what());
        } catch (const std::length_error& e) {
            throw ApiError(RLSQ_ERR_SHAPE, e.what());
        }
        if (h->sinv_valid) {
            try {
                if (h->sinv_z.empty()) throw std::runtime_error("Z is not kept");
                schur_inverse_remove(pos, m2_before, h->sinv_host, h->sinv_z);
            } catch (const std::exception&) {
                h->sinv_valid = false;
            }
        }
        HostCSR& A = h->A;
        HostCSR B;
        B.cols = A.cols;
        B.ptr.push_back(0);
        size_t t = 0;
        for (int64_t i = 0; i < A.rows; ++i) {
            if (t < v.size() && v[t] == i) { ++t; continue; }
            for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
                B.idx.push_back(A.idx[e]);
                B.val.push_back(A.val[e]);
            }
            B.ptr.push_back(static_cast<int64_t>(B.idx.size()));
        }
        B.rows = A.rows - static_cast<int64_t>(v.size());
        h->A = std::move(B);
        refresh_after_rows(h);
        return RLSQ_OK;
    });
}

int rlsq_solve(rlsq_problem h, const double* b, double* x, const rlsq_solve_opts* opts, rlsq_info* info) {
    return guarded([&]() -> int {
        if (!h) throw ApiError(RLSQ_ERR_ARG, "null handle");
        return run_solve(h, b, x, opts, info, false);
    });
}

int rlsq_solve_plain(rlsq_problem h, const double* b, double* x, const rlsq_solve_opts* opts,
                     rlsq_info* info) {
    return guarded([&]() -> int {
        if (!h) throw ApiError(RLSQ_ERR_ARG, "null handle");
        return run_solve(h, b, x, opts, info, true);
    });
}

int rlsq_apply(rlsq_problem h, const double* s, double* t, int32_t ptr_mode, void* stream) {
    return guarded([&]() -> int {
        if (!h || !s || !t) throw ApiError(RLSQ_ERR_ARG, "null argument");
        if (!h->factored) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        cudaStream_t st = h->stream;
        const bool dev = ptr_mode == RLSQ_DEVICE_PTRS;
        cudaStream_t user = static_cast<cudaStream_t>(stream);
        if (dev) {
            RLSQ_CUDA(cudaEventRecord(h->ev[0], user));
            RLSQ_CUDA(cudaStreamWaitEvent(st, h->ev[0], 0));
        }
        LsmrState* S = state_ptr(h, 1);
        put_state(h, S, initial_state(h, 0.0, 0), st);
        RLSQ_CUDA(cudaMemcpyAsync(h->s.p, s, sizeof(double) * h->n,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        enqueue_apply_any<true>(h, h->s.p, S, st, false);
        LsmrState hs;
        RLSQ_CUDA(cudaMemcpyAsync(h->pinned_state, S, sizeof(LsmrState), cudaMemcpyDeviceToHost, st));
        copy_half(t, h->tx.p, h->n, 0, dev, h->s.p, st);  // t_j lives at tx[j].x
        RLSQ_CUDA(cudaStreamSynchronize(st));
        hs = *h->pinned_state;
        if (dev) {
            RLSQ_CUDA(cudaEventRecord(h->ev[0], st));
            RLSQ_CUDA(cudaStreamWaitEvent(user, h->ev[0], 0));
        }
        if (hs.error) throw ApiError(RLSQ_ERR_DEVICE_TIMEOUT, "a sync-free triangular solve timed out");
        return RLSQ_OK;
    });
}

int rlsq_apply_residual(rlsq_problem h, const double* r, double* t, int32_t ptr_mode, void* stream) {
    return guarded([&]() -> int {
        if (!h || !r || !t) throw ApiError(RLSQ_ERR_ARG, "null argument");
        if (!h->factored) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        if (h->md > 0) throw ApiError(RLSQ_ERR_ARG, "the split apply does not take dense-row problems");
        cudaStream_t st = h->stream;
        const bool dev = ptr_mode == RLSQ_DEVICE_PTRS;
        cudaStream_t user = static_cast<cudaStream_t>(stream);
        if (dev) {
            RLSQ_CUDA(cudaEventRecord(h->ev[0], user));
            RLSQ_CUDA(cudaStreamWaitEvent(st, h->ev[0], 0));
        }
        LsmrState* S = state_ptr(h, 1);
        put_state(h, S, initial_state(h, 0.0, 0), st);
        // r into b (length m); s = 0 only feeds the unused scalar step
        RLSQ_CUDA(cudaMemcpyAsync(h->b.p, r, sizeof(double) * h->m,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        RLSQ_CUDA(cudaMemsetAsync(h->s.p, 0, sizeof(double) * h->n, st));
        enqueue_apply_any<true, true>(h, h->s.p, S, st, false, h->b.p, 1);
        RLSQ_CUDA(cudaMemcpyAsync(h->pinned_state, S, sizeof(LsmrState), cudaMemcpyDeviceToHost, st));
        copy_half(t, h->tx.p, h->n, 0, dev, h->s.p, st);  // t_j lives at tx[j].x
        RLSQ_CUDA(cudaStreamSynchronize(st));
        const LsmrState hs = *h->pinned_state;
        if (dev) {
            RLSQ_CUDA(cudaEventRecord(h->ev[0], st));
            RLSQ_CUDA(cudaStreamWaitEvent(user, h->ev[0], 0));
        }
        if (hs.error) throw ApiError(RLSQ_ERR_DEVICE_TIMEOUT, "a sync-free triangular solve timed out");
        return RLSQ_OK;
    });
}

int rlsq_matvec(rlsq_problem h, int32_t trans, const double* x, double* y, int32_t ptr_mode, void* stream) {
    return guarded([&]() -> int {
        if (!h || !x || !y) throw ApiError(RLSQ_ERR_ARG, "null argument");
        cudaStream_t st = h->stream;
        const bool dev = ptr_mode == RLSQ_DEVICE_PTRS;
        cudaStream_t user = static_cast<cudaStream_t>(stream);
        const int64_t nin = trans ? h->m : h->n, nout = trans ? h->n : h->m;
        if (dev) {
            RLSQ_CUDA(cudaEventRecord(h->ev[0], user));
            RLSQ_CUDA(cudaStreamWaitEvent(st, h->ev[0], 0));
        }
        double* in = trans ? h->b.p : h->s.p;
        double* outv = trans ? h->s.p : h->b.p;
        double* tmp = reinterpret_cast<double*>(h->qr.p);  // 2m doubles
        const bool dense = h->md > 0;
        const auto kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (trans && dense) {
            // user row order -> internal order
            RLSQ_CUDA(cudaMemcpyAsync(tmp, x, sizeof(double) * nin, kind, st));
            k_gather<<<grid_rows(h, h->m, 1), kBlock, 0, st>>>(static_cast<int>(h->m), h->row_perm_d.p, tmp, in);
        } else {
            RLSQ_CUDA(cudaMemcpyAsync(in, x, sizeof(double) * nin, kind, st));
        }
        const Csr<double> M = trans ? h->dAt.view() : h->dA.view();
        const int G = trans ? h->map.G_At : h->map.G_A;
        with_G(G, [&](auto g) {
            k_csr_mv<double, decltype(g)::value><<<grid_rows(h, nout, decltype(g)::value), kBlock, 0, st>>>(
                M, in, outv, nullptr);
        });
        if (dense && !trans) {
            enqueue_dense_av<false>(h, in, nullptr, st);
            k_put_dense<<<static_cast<int>((h->md + kBlock - 1) / kBlock), kBlock, 0, st>>>(
                static_cast<int>(h->md), static_cast<int>(h->ms), h->dense_av.p, outv, nullptr);
            // internal order -> user row order
            k_scatter<<<grid_rows(h, h->m, 1), kBlock, 0, st>>>(static_cast<int>(h->m), h->row_perm_d.p, outv, tmp);
            outv = tmp;
        } else if (dense && trans) {
            enqueue_dense_atv<false>(h, in + h->ms, nullptr, st);
            k_add_x<<<grid_rows(h, h->n, 1), kBlock, 0, st>>>(static_cast<int>(h->n), h->dense_atv.p, outv);
        }
        RLSQ_CUDA(cudaGetLastError());
        RLSQ_CUDA(cudaMemcpyAsync(y, outv, sizeof(double) * nout,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        RLSQ_CUDA(cudaStreamSynchronize(st));
        if (dev) {
            RLSQ_CUDA(cudaEventRecord(h->ev[0], st));
            RLSQ_CUDA(cudaStreamWaitEvent(user, h->ev[0], 0));
        }
        return RLSQ_OK;
    });
}

int rlsq_trsv(rlsq_problem h, int32_t which, const double* b, double* x, int32_t ptr_mode, void* stream) {
    return guarded([&]() -> int {
        if (!h || !b || !x) throw ApiError(RLSQ_ERR_ARG, "null argument");
        if (which < 0 || which > 3) throw ApiError(RLSQ_ERR_ARG, "bad system id");
        if (!h->factored) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        cudaStream_t st = h->stream;
        const bool dev = ptr_mode == RLSQ_DEVICE_PTRS;
        cudaStream_t user = static_cast<cudaStream_t>(stream);
        if (dev) {
            RLSQ_CUDA(cudaEventRecord(h->ev[0], user));
            RLSQ_CUDA(cudaStreamWaitEvent(st, h->ev[0], 0));
        }
        const int n = static_cast<int>(h->n);
        LsmrState* S = state_ptr(h, 1);
        put_state(h, S, initial_state(h, 0.0, 0), st);
        RLSQ_CUDA(cudaMemcpyAsync(h->s.p, b, sizeof(double) * n,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        RLSQ_CUDA(cudaMemsetAsync(h->tickets.p, 0, sizeof(unsigned) * kMaxSlots, st));
        RLSQ_CUDA(cudaMemsetAsync(h->barriers.p, 0, sizeof(unsigned) * kMaxSlots, st));
        const int grid = grid_rows(h, n, 1);
        if (h->precision == RLSQ_PREC_FP32) {
            DevFactor<float>& F = h->f32;
            k_convert<float, double><<<grid, kBlock, 0, st>>>(n, h->s.p, F.vn[3].p);
            launch_trsv<float>(h, F, which, RHS_VEC, Rhs<float>{F.vn[3].p, nullptr, nullptr}, F.vn[4].p, 0,
                               S, st);
            k_convert<double, float><<<grid, kBlock, 0, st>>>(n, F.vn[4].p, h->h.p);
        } else {
            DevFactor<double>& F = h->f64;
            launch_trsv<double>(h, F, which, RHS_VEC, Rhs<double>{h->s.p, nullptr, nullptr}, h->h.p, 0, S, st);
        }
        RLSQ_CUDA(cudaGetLastError());
        RLSQ_CUDA(cudaMemcpyAsync(h->pinned_state, S, sizeof(LsmrState), cudaMemcpyDeviceToHost, st));
        RLSQ_CUDA(cudaMemcpyAsync(x, h->h.p, sizeof(double) * n,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        RLSQ_CUDA(cudaStreamSynchronize(st));
        if (dev) {
            RLSQ_CUDA(cudaEventRecord(h->ev[0], st));
            RLSQ_CUDA(cudaStreamWaitEvent(user, h->ev[0], 0));
        }
        if (h->pinned_state->error)
            throw ApiError(RLSQ_ERR_DEVICE_TIMEOUT, "a sync-free triangular solve timed out");
        return RLSQ_OK;
    });
}

int rlsq_profile(rlsq_problem h, const double* b, int32_t warmup, int32_t iters, int32_t plain,
                 rlsq_profile_out* out) {
    return guarded([&]() -> int {
        if (!h || !b || !out || iters < 1 || warmup < 0) throw ApiError(RLSQ_ERR_ARG, "bad argument");
        if (!plain && !h->factored) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        std::memset(out, 0, sizeof(*out));
        cudaStream_t st = h->stream;
        LsmrState* S = state_ptr(h, 0);
        const int big = 1 << 30;
        upload_b(h, b, false, st);
        put_state(h, S, initial_state(h, 0.0, big), st);
        enqueue_start(h, S, st, plain != 0);
        cudaGraphExec_t g1 = iteration_graph(h, 1, plain != 0);
        for (int i = 0; i < warmup; ++i) RLSQ_CUDA(cudaGraphLaunch(g1, st));
        cudaEvent_t a, e;
        RLSQ_CUDA(cudaEventCreate(&a));
        RLSQ_CUDA(cudaEventCreate(&e));
        RLSQ_CUDA(cudaStreamSynchronize(st));
        RLSQ_CUDA(cudaEventRecord(a, st));
        for (int i = 0; i < iters; ++i) RLSQ_CUDA(cudaGraphLaunch(g1, st));
        RLSQ_CUDA(cudaEventRecord(e, st));
        RLSQ_CUDA(cudaEventSynchronize(e));
        float ms = 0.f;
        RLSQ_CUDA(cudaEventElapsedTime(&ms, a, e));
        cudaEventDestroy(a);
        cudaEventDestroy(e);
        out->total_ms = ms;
        out->iters = iters;
        // Per-kernel times: one iteration captured with an event-record node
        // before and after every launch, replayed `iters` times; the graph runs
        // exactly like the timed one, so no host gap enters the times.
        std::unique_ptr<Recorder> rec(new Recorder());
        h->rec = rec.get();
        cudaGraph_t pg = nullptr;
        RLSQ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_iteration(h, S, st, plain != 0);
        } catch (...) {
            h->rec = nullptr;
            cudaStreamEndCapture(st, &pg);
            if (pg) cudaGraphDestroy(pg);
            throw;
        }
        h->rec = nullptr;
        RLSQ_CUDA(cudaStreamEndCapture(st, &pg));
        cudaGraphExec_t pex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&pex, pg, 0);
        cudaGraphDestroy(pg);
        if (ie != cudaSuccess) throw_cuda(ie, "cudaGraphInstantiate", __LINE__);
        std::vector<double> acc(rec->entries.size(), 0.0);
        for (int i = 0; i < iters; ++i) {
            RLSQ_CUDA(cudaGraphLaunch(pex, st));
            RLSQ_CUDA(cudaStreamSynchronize(st));
            for (size_t q = 0; q < rec->entries.size(); ++q) {
                float t = 0.f;
                RLSQ_CUDA(cudaEventElapsedTime(&t, rec->entries[q].a, rec->entries[q].b));
                acc[q] += t;
            }
        }
        cudaGraphExecDestroy(pex);
        for (size_t q = 0; q < rec->entries.size(); ++q) {
            const auto& en = rec->entries[q];
            out->class_ms[en.cls] += acc[q] / iters;
            out->class_launches[en.cls] += en.launches;
            out->class_bytes[en.cls] += en.bytes;
        }
        LsmrState hs;
        RLSQ_CUDA(cudaMemcpy(&hs, S, sizeof(LsmrState), cudaMemcpyDeviceToHost));
        out->status = hs.done ? (hs.error ? RLSQ_ERR_DEVICE_TIMEOUT : hs.status) : RLSQ_OK;
        out->bytes_per_iter = algorithmic_bytes(h, plain != 0);
        return RLSQ_OK;
    });
}

int rlsq_get_info(rlsq_problem h, rlsq_info* info) {
    return guarded([&]() -> int {
        if (!h || !info) throw ApiError(RLSQ_ERR_ARG, "null argument");
        std::memset(info, 0, sizeof(*info));
        fill_factor_info(h, info);
        return RLSQ_OK;
    });
}

int rlsq_get_split(rlsq_problem h, int32_t* prow, int32_t* a2rows, double* d, double* udiag) {
    return guarded([&]() -> int {
        if (!h) throw ApiError(RLSQ_ERR_ARG, "null handle");
        if (!h->F) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        const IlupResult& F = *h->F;
        if (prow) std::copy(F.prow.begin(), F.prow.end(), prow);
        if (a2rows) std::copy(F.a2rows.begin(), F.a2rows.end(), a2rows);
        if (d) std::copy(F.d.begin(), F.d.end(), d);
        if (udiag) std::copy(F.Udiag.begin(), F.Udiag.end(), udiag);
        return RLSQ_OK;
    });
}

int rlsq_get_factor(rlsq_problem h, int32_t part, int64_t* ptr, int32_t* idx, double* val) {
    return guarded([&]() -> int {
        if (!h) throw ApiError(RLSQ_ERR_ARG, "null handle");
        if (!h->F) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        const IlupResult& F = *h->F;
        const HostCSR* c = nullptr;
        if (part == RLSQ_PART_L1) c = &F.L1;
        else if (part == RLSQ_PART_L2) c = &F.L2;
        else if (part == RLSQ_PART_U) c = &F.U;
        else throw ApiError(RLSQ_ERR_ARG, "bad part id");
        if (ptr) std::copy(c->ptr.begin(), c->ptr.end(), ptr);
        if (idx) std::copy(c->idx.begin(), c->idx.end(), idx);
        if (val) std::copy(c->val.begin(), c->val.end(), val);
        return RLSQ_OK;
    });
}

int rlsq_get_levels(rlsq_problem h, int32_t which, int32_t* level) {
    return guarded([&]() -> int {
        if (!h || !level) throw ApiError(RLSQ_ERR_ARG, "null argument");
        if (!h->F) throw ApiError(RLSQ_ERR_NOT_FACTORED, "rlsq_factor has not succeeded");
        const IlupResult& F = *h->F;
        const Levels* L = nullptr;
        switch (which) {
            case RLSQ_SYS_L1: L = &F.lev_L1; break;
            case RLSQ_SYS_L1T: L = &F.lev_L1t; break;
            case RLSQ_SYS_U: L = &F.lev_U; break;
            case RLSQ_SYS_UT: L = &F.lev_Ut; break;
            default: throw ApiError(RLSQ_ERR_ARG, "bad system id");
        }
        std::copy(L->level.begin(), L->level.end(), level);
        return RLSQ_OK;
    });
}

void rlsq_destroy(rlsq_problem h) {
    // a live server still reads the problem's device data: keep it (and say so)
    if (h && h->served.load() > 0) {
        (void)guarded([&]() -> int { throw ApiError(RLSQ_ERR_ARG, "the problem is registered with a server"); });
        return;
    }
    delete h;
}

}  // extern "C"
