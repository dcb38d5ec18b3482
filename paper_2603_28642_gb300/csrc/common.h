// Shared host-side plumbing of the rlsq library: error reporting across the
// C ABI, owning device arrays and the problem handle.
#pragma once

#include <atomic>

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "host_setup.h"
#include "kernels.cuh"
#include "rlsq.h"

namespace rlsq {

// An error carrying an RLSQ_ERR_* code; caught at the C boundary.
struct ApiError : std::runtime_error {
    int code;
    ApiError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] void throw_cuda(cudaError_t e, const char* what, int line);

#define RLSQ_CUDA(call)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) ::rlsq::throw_cuda(e_, #call, __LINE__); \
    } while (0)

void set_last_error(const std::string& msg);

// Runs f, mapping exceptions to status codes and the thread's last error.
template <class F>
int guarded(F&& f) {
    try {
        set_last_error("");
        return f();
    } catch (const ApiError& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return RLSQ_ERR_OOM;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return RLSQ_ERR_ARG;
    }
}

template <typename T>
struct DevArray {
    T* p = nullptr;
    size_t n = 0;
    DevArray() = default;
    DevArray(const DevArray&) = delete;
    DevArray& operator=(const DevArray&) = delete;
    ~DevArray() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        RLSQ_CUDA(cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T)));
        n = count;
    }
    void upload(const T* host, size_t count, cudaStream_t s) {
        alloc(count);
        if (count) RLSQ_CUDA(cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

// Rows per window within which the sliced layout sorts rows by length.
constexpr int kSliceWindow = 1024;

template <typename T>
struct DevCsr {
    int32_t rows = 0, cols = 0;
    int64_t nnz = 0;
    DevArray<int32_t> ptr, idx;
    DevArray<T> val;
    // the sliced layout (Csr::sperm ...), built on request
    DevArray<int32_t> sperm, sbase, sidx;
    DevArray<T> sval;
    int32_t snpos = 0;
    int64_t sentries = 0;  // stored entries of the sliced layout, padding included
    Csr<T> view() const {
        return Csr<T>{rows, cols, ptr.p, idx.p, val.p, sperm.p, sbase.p, sidx.p, sval.p, snpos};
    }
    // sliced: also build the sliced layout (kept off when its padded size
    // would not fit 32-bit offsets)
    void upload(const HostCSR& h, cudaStream_t s, bool sliced = false);
};

// Kernel mapping choices for one problem (set by heuristics or the autotuner).
struct Mapping {
    int G_A = 8, G_At = 16;             // lanes per row of the A and A^T products
    int G_tri[4] = {4, 4, 4, 4};        // lanes per row: L1, L1^T, U, U^T
    int sched[4] = {RLSQ_TRSV_SYNCFREE, RLSQ_TRSV_SYNCFREE, RLSQ_TRSV_SYNCFREE, RLSQ_TRSV_SYNCFREE};
    int G_L2 = 4, G_L2t = 4;
    // the products in the sliced layout (one lane per row) instead of CSR
    // with G lanes: A, A^T, L2, L2^T
    int sl_A = 0, sl_At = 0, sl_L2 = 0, sl_L2t = 0;
    int sf_blocks[4] = {2, 2, 2, 2};    // sync-free solve: resident blocks per SM (bounds the polling rows)
    int sf_rows[4] = {0, 0, 0, 0};      // sync-free solve: 0 = block tickets (k_trsv_sentinel); R = 1, 2, 4:
                                        // warp tickets, R rows per lane group (k_trsv_warp)
    int wave_kp[4] = {4, 4, 4, 4};      // wavefront solve: entries per row loaded ahead (4 or 8)
};

template <typename T>
struct DevFactor {
    DevCsr<T> tri[4];          // strictly triangular parts: L1, L1^T, U, U^T (after level fusing)
    DevCsr<T> rtri[4];         // right-hand-side terms of fused rows (empty when not fused)
    DevArray<T> diag[4];       // inverse U diagonal for U and U^T, by position (unit for L1, L1^T)
    DevArray<int32_t> order[4];
    std::vector<int32_t> level_ptr[4];
    DevArray<int32_t> level_ptr_d[4];  // device copies for the persistent solve
    // first ell_kp[w] entries of every row, position-major ([q * n + t];
    // idx -1 and value 0 past the row's end): the persistent solve loads a
    // level's structure with independent, coalesced reads
    DevArray<int32_t> ell_idx[4];
    DevArray<T> ell_val[4];
    int ell_kp[4] = {4, 4, 4, 4};
    // the binned form of each system (k_trsv_binned): rows of a level group
    // sorted by the lanes they need, right-hand-side terms in the entry list
    DevArray<int32_t> bidx[4], border[4], bgseg[4], bgitems[4], bgpos[4], bgentry[4];
    DevArray<T> bval[4], bdiag[4];
    DevArray<BinSeg> bseg[4];
    int bngroups[4] = {0, 0, 0, 0};
    int64_t bentries[4] = {0, 0, 0, 0};
    DevCsr<T> L2, L2t;
    DevArray<T> d;
    DevArray<T> sinv;          // dense S^{-1} (DENSE mode)
    DevArray<int32_t> prow, a2rows;  // rows of A1 (by position) and of A2: Algorithm 3's input split
    DevArray<T> vn[6], vm[4];  // work vectors
    // sliced: also the sliced layout of L2 and L2^T
    void upload(const IlupResult& F, const MergedTri* merged, const std::vector<double>& sinv_h, cudaStream_t s,
                bool sliced = false);
    void clear() {
        for (int w = 0; w < 4; ++w) {
            tri[w].ptr.release(); tri[w].idx.release(); tri[w].val.release();
            rtri[w].ptr.release(); rtri[w].idx.release(); rtri[w].val.release(); rtri[w].nnz = 0;
            diag[w].release(); order[w].release(); level_ptr[w].clear(); level_ptr_d[w].release();
            ell_idx[w].release(); ell_val[w].release();
            for (auto* a : {&bidx[w], &border[w], &bgseg[w], &bgitems[w], &bgpos[w], &bgentry[w]}) a->release();
            bval[w].release(); bdiag[w].release(); bseg[w].release();
            bngroups[w] = 0;
            bentries[w] = 0;
        }
        for (auto* c : {&L2, &L2t}) { c->ptr.release(); c->idx.release(); c->val.release(); }
        d.release(); sinv.release(); prow.release(); a2rows.release();
        for (auto& v : vn) v.release();
        for (auto& v : vm) v.release();
    }
    BinTri<T> bview(int which) const {
        return BinTri<T>{tri[which].rows, bngroups[which], bidx[which].p, bval[which].p,
                         border[which].p, (which >= 2) ? bdiag[which].p : nullptr, bseg[which].p,
                         bgseg[which].p, bgitems[which].p, bgpos[which].p, bgentry[which].p};
    }
    // tri[w], diag[w] are stored by solve position (rows in level order)
    Tri<T> tview(int which) const {
        const bool fused = rtri[which].nnz > 0;
        return Tri<T>{tri[which].rows, tri[which].ptr.p, tri[which].idx.p, tri[which].val.p,
                      (which >= 2) ? diag[which].p : nullptr, order[which].p,
                      fused ? rtri[which].ptr.p : nullptr, fused ? rtri[which].idx.p : nullptr,
                      fused ? rtri[which].val.p : nullptr, ell_idx[which].p, ell_val[which].p};
    }
};

// Event pairs around launches, attributed to RLSQ_KCLASS_* (profiling only).
struct Recorder {
    struct Entry {
        int cls;
        double bytes;
        cudaEvent_t a, b;
        int launches;
    };
    std::vector<Entry> entries;
    ~Recorder() {
        for (auto& e : entries) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
    }
};

// dst[i] = pairs[i].x (half 0) or .y (half 1), i < n, on stream st: a kernel
// writes either dst itself (device destination) or the device staging buffer,
// which one contiguous copy then brings to the host
void copy_half(double* dst, const double2* pairs, int64_t n, int half, bool dev, double* staging, cudaStream_t st);

}  // namespace rlsq

struct rlsq_problem_s {
    int64_t m = 0, n = 0, nnz = 0;
    // servers this problem is registered with: while > 0 its device data must
    // not change (refactor, row updates) or go (destroy)
    std::atomic<int32_t> served{0};
    rlsq::HostCSR A;                 // host copy (the set-up runs on the host)
    rlsq::DevCsr<double> dA, dAt;    // CSR and CSC (= CSR of A^T) of the sparse rows, internal row order
    // Dense rows (sparse-dense problems): rows with many nonzeros sit at the end
    // of the internal row order (empty in dA) and are kept row-major in Ad.
    int64_t ms = 0, md = 0;          // sparse and dense row counts (ms + md = m)
    int64_t layout_threshold = 0;    // the dense-row threshold A's device layout was built with
    std::vector<int32_t> row_perm;   // internal row i holds user row row_perm[i] (empty: identity)
    rlsq::DevArray<int32_t> row_perm_d;
    rlsq::DevArray<double> Ad;       // md x n
    rlsq::DevArray<double2> dense_part, dense_av, dense_atv;
    int dense_chunks = 0;
    double anorm = 0.0;
    cudaStream_t stream = nullptr;   // internal stream
    int device = 0;
    int num_sms = 0;

    bool factored = false;
    rlsq_factor_opts opts{};
    int correction = RLSQ_CORR_NONE;
    int precision = RLSQ_PREC_FP64;
    double factor_seconds = 0.0;
    double ilup_seconds = 0.0;       // the host set-up of the factor in use
    int32_t ilup_threads = 0;
    std::unique_ptr<rlsq::IlupResult> F;
    // S^{-1} of the dense correction for F, kept on the host once formed so
    // that row updates can update it (valid only while it belongs to F)
    std::vector<double> sinv_host;
    std::vector<double> sinv_z;  // Z = L1^{-T} L2^T beside it (empty: updates form S^{-1} again)
    bool sinv_valid = false;
    std::vector<rlsq::MergedTri> merged;  // the four systems as the GPU solves them
    rlsq::DevFactor<double> f64;
    rlsq::DevFactor<float> f32;
    rlsq::Mapping map;

    // LSMR work vectors (float64); qr[i] = (q_i, r_i), tx[j] = (t_j, x_j)
    rlsq::DevArray<double2> qr, tx;
    rlsq::DevArray<double> b, s, h, hb;
    rlsq::DevArray<rlsq::LsmrState> S;   // [0] solve, [1] standalone calls
    rlsq::DevArray<double> part;
    rlsq::DevArray<unsigned> counter, tickets, barriers;  // barriers: one per triangular-solve slot
    int coop_blocks = 0;                                    // co-resident blocks of the persistent solve
    rlsq::LsmrState* pinned_state = nullptr;   // host-pinned mirror
    int* pinned_done = nullptr;                // [2]
    cudaEvent_t ev[2] = {nullptr, nullptr};

    rlsq::Recorder* rec = nullptr;                  // set while profiling one eager iteration
    // iteration graphs: [plain + 2 cgls], and 4 for CGLS with the split (residual) apply
    cudaGraphExec_t graph[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int graph_iters[5] = {0, 0, 0, 0, 0};

    ~rlsq_problem_s();
};
