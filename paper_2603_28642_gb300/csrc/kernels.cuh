// Device kernels of the preconditioned LSMR iteration (sm_103a).
//
// The path is sparse and bandwidth-bound (about 0.1-0.25 flop per byte), so
// there is no tensor-core work here: the kernels stream CSR arrays with
// coalesced loads, gather vector entries through L2, reduce rows with warp
// shuffles inside groups of G lanes, and reduce norms with fixed-shape
// block trees plus a "last block finishes" step, so every result is
// deterministic for a given launch shape.
//
// Scalars of the iteration live in device memory (LsmrState) so that one
// iteration can be captured once in a CUDA graph and replayed; a kernel whose
// state says `done` returns at once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rlsq {

constexpr int kBlock = 256;          // threads per block for every kernel here
constexpr int kMinBlocks = 6;        // resident blocks per SM asked of the register allocator
constexpr int kMaxSlots = 64;        // triangular-solve launches per apply
// Blocks per SM of a row-parallel launch at most (grid-stride loops cover the
// rest).  Every block of a reduction kernel adds one partial and one atomic to
// the grid-wide total, so a smaller grid makes the reductions cheaper: at
// 2M x 1M the iteration takes 1.607 / 1.552 / 1.558 / 1.536 ms with 32 / 16 /
// 8 / 4 blocks per SM.
constexpr int kGridBlocksPerSm = 4;
constexpr long long kWaitNs = 1000000000LL;  // bounded wait of a sync-free solve: 1 s

// status codes mirrored from rlsq.h
constexpr int kOk = 0, kErrBreakdown = -7, kErrMaxit = -8, kErrTimeout = -9;

struct LsmrState {
    // Golub-Kahan quantities: u = q * inv_beta, v^ = t * inv_alpha, w = s * inv_alpha
    double alpha, inv_alpha, beta, inv_beta;
    double alphabar, zetabar, rho, rhobar, cbar, sbar;
    double c_hbar, c_x, c_h;  // coefficients of the h-bar, x and h updates
    double rnorm, arnorm, ratio, anorm, atol;
    double ts;                // <t, s>
    double sum_q, sum_r;      // partial sums carried between kernels
    double cg_rr, cg_a, cg_beta;
    double cg_rr0;            // ||r_0||^2 of the CG iteration on S in the current apply
    int32_t k;                // index of the current iterate x_k
    int32_t maxit;
    int32_t done;
    int32_t status;
    int32_t apply_count;      // number of finished preconditioner applications (flag epochs)
    int32_t error;            // device-side error word (wait timeout)
    int32_t check;            // 1: this iteration forms the explicit residual pair (A x_k, A^T r_k)
    int32_t pad1;
};

// When an iteration forms the explicit residual r_k = b - A x_k and A^T r_k
// (half the float64 work of the two products) for the stopping ratio of x_k:
// in the first kResidualFirst iterations, whenever the last explicit ratio is
// below kResidualNear * atol, at the iteration limit, and otherwise every
// kResidualEvery-th iteration.  A solve stops only on an explicit ratio, so
// the returned x_k carries its exact ratio; a stop is found later than the
// first k with ratio_k < atol only if the ratio fell by more than
// kResidualNear within kResidualEvery - 1 iterations.
constexpr int kResidualFirst = 4;
constexpr int kResidualEvery = 4;
constexpr double kResidualNear = 1000.0;

__device__ __forceinline__ int residual_check_next(const LsmrState* S) {
    const int kn = S->k + 1;
    return (kn < kResidualFirst) || (S->ratio < kResidualNear * S->atol) || (kn % kResidualEvery == 0) ||
           (kn >= S->maxit);
}

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
template <typename T>
__device__ __forceinline__ T ld_l2(const T* p) {
    return __ldcg(p);
}

template <int G>
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, G);
    return v;
}
template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, G);
    return v;
}
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 1) {
        return 1u << (threadIdx.x & 31u);
    } else if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

// Block-wide sum of NV values; result valid in thread 0.  Fixed tree.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double red[NV][kBlock / 32];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) red[i][warp] = v[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double x = (lane < kBlock / 32) ? red[i][lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            v[i] = x;
        }
    }
    __syncthreads();
}

// Every block contributes NV partial sums; the last block to finish adds the
// partials in block order (deterministic) and returns true with the totals
// in `tot` (thread 0 only; the whole last block returns true).
// (bid, nblocks) name this block among the blocks that reduce together: the
// whole grid for a single problem, one slot's blocks in a batch.
template <int NV>
__device__ bool last_block_total_ctx(double (&v)[NV], double* part, unsigned* counter,
                                     double (&tot)[NV], unsigned bid, unsigned nblocks) {
    block_sum<NV>(v);
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) part[(size_t)bid * NV + i] = v[i];
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += ld_l2(&part[(size_t)b * NV + i]);
    block_sum<NV>(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) tot[i] = acc[i];
        *counter = 0u;
    }
    return true;
}

template <int NV>
__device__ __forceinline__ bool last_block_total(double (&v)[NV], double* part, unsigned* counter,
                                                 double (&tot)[NV]) {
    return last_block_total_ctx<NV>(v, part, counter, tot, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// CSR views
// ---------------------------------------------------------------------------
template <typename T>
struct Csr {
    int32_t rows, cols;
    const int32_t* ptr;
    const int32_t* idx;
    const T* val;
    // The same matrix sliced for one lane per row (null when not built): the
    // rows in the order sperm (sorted by length within windows; -1 marks the
    // padding positions up to snpos, a multiple of 32) form slices of 32
    // positions; slice q stores its entries column-major from sbase[q]
    // (entry k of position t at sbase[t / 32] + 32 k + t % 32), its width
    // (sbase[q + 1] - sbase[q]) / 32 the longest of its rows, shorter rows
    // padded with index -1.  Every row keeps its CSR entry order.
    const int32_t* sperm;
    const int32_t* sbase;
    const int32_t* sidx;
    const T* sval;
    int32_t snpos;
};

// Dot product of position t's row in the sliced layout with x.  Entries are
// added in their CSR order, as by one lane of row_dot<1>, so the sums equal
// the one-lane CSR products bit for bit; a warp walks one slice, every load
// of the 32 lanes one 128-byte (index) or 256-byte (value) line.
template <typename TV, typename TX, typename TA>
__device__ __forceinline__ void sliced_dot(const Csr<TV>& a, int t, const TX* __restrict__ x, TA& s) {
    const int q = t >> 5;
    const int e0 = a.sbase[q];
    const int w = (a.sbase[q + 1] - e0) >> 5;
    int e = e0 + (t & 31);
    int k = 0;
    for (; k + 4 <= w; k += 4, e += 128) {
        const int j0 = a.sidx[e], j1 = a.sidx[e + 32], j2 = a.sidx[e + 64], j3 = a.sidx[e + 96];
        const TA a0 = (TA)a.sval[e], a1 = (TA)a.sval[e + 32], a2 = (TA)a.sval[e + 64], a3 = (TA)a.sval[e + 96];
        const TA x0 = j0 >= 0 ? (TA)x[j0] : (TA)0, x1 = j1 >= 0 ? (TA)x[j1] : (TA)0;
        const TA x2 = j2 >= 0 ? (TA)x[j2] : (TA)0, x3 = j3 >= 0 ? (TA)x[j3] : (TA)0;
        if (j0 >= 0) s = fma(a0, x0, s);
        if (j1 >= 0) s = fma(a1, x1, s);
        if (j2 >= 0) s = fma(a2, x2, s);
        if (j3 >= 0) s = fma(a3, x3, s);
    }
    if (k < w) {  // the last (< 4) columns of the slice, loads first
        const bool h1 = k + 1 < w, h2 = k + 2 < w;
        const int j0 = a.sidx[e], j1 = h1 ? a.sidx[e + 32] : -1, j2 = h2 ? a.sidx[e + 64] : -1;
        const TA a0 = (TA)a.sval[e], a1 = h1 ? (TA)a.sval[e + 32] : (TA)0, a2 = h2 ? (TA)a.sval[e + 64] : (TA)0;
        const TA x0 = j0 >= 0 ? (TA)x[j0] : (TA)0, x1 = j1 >= 0 ? (TA)x[j1] : (TA)0;
        const TA x2 = j2 >= 0 ? (TA)x[j2] : (TA)0;
        if (j0 >= 0) s = fma(a0, x0, s);
        if (j1 >= 0) s = fma(a1, x1, s);
        if (j2 >= 0) s = fma(a2, x2, s);
    }
}

// The same against both halves of an interleaved pair vector (p[j].x, p[j].y)
// (PAIR), or its first halves only.
template <bool PAIR, typename TV>
__device__ __forceinline__ void sliced_dot_pair(const Csr<TV>& a, int t, const double2* __restrict__ p,
                                                double& s1, double& s2) {
    const double* px = reinterpret_cast<const double*>(p);
    const int q = t >> 5;
    const int e0 = a.sbase[q];
    const int w = (a.sbase[q + 1] - e0) >> 5;
    int e = e0 + (t & 31);
    int k = 0;
    for (; k + 4 <= w; k += 4, e += 128) {
        int j[4];
        double v[4];
        double2 y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            j[u] = a.sidx[e + 32 * u];
            v[u] = a.sval[e + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (PAIR) y[u] = j[u] >= 0 ? p[j[u]] : make_double2(0.0, 0.0);
            else y[u].x = j[u] >= 0 ? px[2 * (size_t)j[u]] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (j[u] >= 0) {
                s1 = fma(v[u], y[u].x, s1);
                if (PAIR) s2 = fma(v[u], y[u].y, s2);
            }
        }
    }
    if (k < w) {  // the last (< 4) columns of the slice, loads first
        int j[3];
        double v[3];
        double2 y[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const bool h = k + u < w;
            j[u] = h ? a.sidx[e + 32 * u] : -1;
            v[u] = h ? (double)a.sval[e + 32 * u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            if (PAIR) y[u] = j[u] >= 0 ? p[j[u]] : make_double2(0.0, 0.0);
            else y[u].x = j[u] >= 0 ? px[2 * (size_t)j[u]] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            if (j[u] >= 0) {
                s1 = fma(v[u], y[u].x, s1);
                if (PAIR) s2 = fma(v[u], y[u].y, s2);
            }
        }
    }
}

// group-of-G row dot products against two vectors
template <int G, typename TV, typename TX, typename TA>
__device__ __forceinline__ void row_dot2(const Csr<TV>& a, int row, int lane, const TX* x1,
                                         const TX* x2, TA& s1, TA& s2) {
    const int e1 = a.ptr[row + 1];
    for (int e = a.ptr[row] + lane; e < e1; e += G) {
        const int j = a.idx[e];
        const TA v = (TA)a.val[e];
        s1 += v * (TA)x1[j];
        s2 += v * (TA)x2[j];
    }
}
// one row's dot product, four entries in flight per lane
template <int G, typename TV, typename TX, typename TA>
__device__ __forceinline__ void row_dot(const Csr<TV>& a, int row, int lane, const TX* x, TA& s) {
    const int e1 = a.ptr[row + 1];
    int e = a.ptr[row] + lane;
    for (; e + 3 * G < e1; e += 4 * G) {
        const int j0 = a.idx[e], j1 = a.idx[e + G], j2 = a.idx[e + 2 * G], j3 = a.idx[e + 3 * G];
        const TA a0 = (TA)a.val[e], a1 = (TA)a.val[e + G], a2 = (TA)a.val[e + 2 * G], a3 = (TA)a.val[e + 3 * G];
        const TA x0 = (TA)x[j0], x1 = (TA)x[j1], x2 = (TA)x[j2], x3 = (TA)x[j3];
        s = fma(a0, x0, s);
        s = fma(a1, x1, s);
        s = fma(a2, x2, s);
        s = fma(a3, x3, s);
    }
    // the lane's last (< 4) entries: every load issued before the first
    // multiply-add (an absent entry re-reads entry e), added in entry order
    if (e < e1) {
        const bool h1 = e + G < e1, h2 = e + 2 * G < e1;
        const int j0 = a.idx[e];
        const int j1 = h1 ? a.idx[e + G] : j0, j2 = h2 ? a.idx[e + 2 * G] : j0;
        const TA a0 = (TA)a.val[e];
        const TA a1 = h1 ? (TA)a.val[e + G] : a0, a2 = h2 ? (TA)a.val[e + 2 * G] : a0;
        const TA x0 = (TA)x[j0], x1 = (TA)x[j1], x2 = (TA)x[j2];
        s = fma(a0, x0, s);
        if (h1) s = fma(a1, x1, s);
        if (h2) s = fma(a2, x2, s);
    }
}

// ---------------------------------------------------------------------------
// LSMR products with A (float64)
// ---------------------------------------------------------------------------

// Dot products of one row with the two halves of an interleaved vector pair
// (p[j].x, p[j].y): one 16-byte gather per entry, four entries in flight per
// lane.
template <int G, typename TV>
__device__ __forceinline__ void row_dot_pair(const Csr<TV>& a, int row, int lane, const double2* __restrict__ p,
                                             double& s1, double& s2) {
    const int e1 = a.ptr[row + 1];
    int e = a.ptr[row] + lane;
    for (; e + 3 * G < e1; e += 4 * G) {
        const int j0 = a.idx[e], j1 = a.idx[e + G], j2 = a.idx[e + 2 * G], j3 = a.idx[e + 3 * G];
        const double a0 = a.val[e], a1 = a.val[e + G], a2 = a.val[e + 2 * G], a3 = a.val[e + 3 * G];
        const double2 p0 = p[j0], p1 = p[j1], p2 = p[j2], p3 = p[j3];
        // one fused multiply-add per entry and vector: float64 issue slots
        // are the scarce resource of these products on this GPU
        s1 = fma(a0, p0.x, s1);
        s2 = fma(a0, p0.y, s2);
        s1 = fma(a1, p1.x, s1);
        s2 = fma(a1, p1.y, s2);
        s1 = fma(a2, p2.x, s1);
        s2 = fma(a2, p2.y, s2);
        s1 = fma(a3, p3.x, s1);
        s2 = fma(a3, p3.y, s2);
    }
    if (e < e1) {  // the lane's last (< 4) entries, loads first (as in row_dot)
        const bool h1 = e + G < e1, h2 = e + 2 * G < e1;
        const int j0 = a.idx[e];
        const int j1 = h1 ? a.idx[e + G] : j0, j2 = h2 ? a.idx[e + 2 * G] : j0;
        const double a0 = a.val[e];
        const double a1 = h1 ? (double)a.val[e + G] : a0, a2 = h2 ? (double)a.val[e + 2 * G] : a0;
        const double2 p0 = p[j0], p1 = p[j1], p2 = p[j2];
        s1 = fma(a0, p0.x, s1);
        s2 = fma(a0, p0.y, s2);
        if (h1) {
            s1 = fma(a1, p1.x, s1);
            s2 = fma(a1, p1.y, s2);
        }
        if (h2) {
            s1 = fma(a2, p2.x, s1);
            s2 = fma(a2, p2.y, s2);
        }
    }
}

// The first halves only: p[j].x (an 8-byte gather per entry).
template <int G, typename TV>
__device__ __forceinline__ void row_dot_first(const Csr<TV>& a, int row, int lane, const double2* __restrict__ p,
                                              double& s1) {
    const double* px = reinterpret_cast<const double*>(p);
    const int e1 = a.ptr[row + 1];
    int e = a.ptr[row] + lane;
    for (; e + 3 * G < e1; e += 4 * G) {
        const int j0 = a.idx[e], j1 = a.idx[e + G], j2 = a.idx[e + 2 * G], j3 = a.idx[e + 3 * G];
        const double a0 = a.val[e], a1 = a.val[e + G], a2 = a.val[e + 2 * G], a3 = a.val[e + 3 * G];
        const double p0 = px[2 * (size_t)j0], p1 = px[2 * (size_t)j1], p2 = px[2 * (size_t)j2], p3 = px[2 * (size_t)j3];
        s1 = fma(a0, p0, s1);
        s1 = fma(a1, p1, s1);
        s1 = fma(a2, p2, s1);
        s1 = fma(a3, p3, s1);
    }
    if (e < e1) {  // the lane's last (< 4) entries, loads first (as in row_dot)
        const bool h1 = e + G < e1, h2 = e + 2 * G < e1;
        const int j0 = a.idx[e];
        const int j1 = h1 ? a.idx[e + G] : j0, j2 = h2 ? a.idx[e + 2 * G] : j0;
        const double a0 = a.val[e];
        const double a1 = h1 ? (double)a.val[e + G] : a0, a2 = h2 ? (double)a.val[e + 2 * G] : a0;
        const double p0 = px[2 * (size_t)j0], p1 = px[2 * (size_t)j1], p2 = px[2 * (size_t)j2];
        s1 = fma(a0, p0, s1);
        if (h1) s1 = fma(a1, p1, s1);
        if (h2) s1 = fma(a2, p2, s1);
    }
}

// Row epilogue of the A product (shared by the CSR and sliced kernels): s1 =
// (A t)_row, s2 = (A x_k)_row (when chk); dense rows add their GEMV values.
__device__ __forceinline__ void spmv_row_out(int row, double s1, double s2, bool chk, double inv_alpha,
                                             double alpha, double inv_beta, double2* __restrict__ qr,
                                             const double* __restrict__ b, int ms,
                                             const double2* __restrict__ dense_av, double (&acc)[2]) {
    if (dense_av && row >= ms) {
        const double2 dv = dense_av[row - ms];
        s1 += dv.x;
        s2 += dv.y;
    }
    const double2 old = qr[row];
    const double qn = s1 * inv_alpha - alpha * (old.x * inv_beta);
    const double rr = chk ? b[row] - s2 : old.y;
    qr[row] = make_double2(qn, rr);
    acc[0] += qn * qn;
    if (chk) acc[1] += rr * rr;
}

__device__ __forceinline__ void spmv_totals(LsmrState* S, const double (&tot)[2], bool chk) {
    const double beta = sqrt(tot[0]);
    S->beta = beta;
    S->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
    if (chk) S->rnorm = sqrt(tot[1]);
}

// tx[j] = (t_j, x_j): v^ = t * inv_alpha and the current iterate x_k.
// qr[i] = (q_i, r_i) with u = q * inv_beta.
// q <- A v^ - alpha u  (= beta_{k+2} u_{k+2}),  r <- b - A x_k
// totals: beta = ||q||, rnorm = ||r||
// Dense rows (ms <= row < m, empty in the CSR) take their two products from
// dense_av (the dense-row GEMV ran just before); dense_av = nullptr if none.
template <int G>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
k_spmv_lsmr(Csr<double> A, const double2* __restrict__ tx, double2* __restrict__ qr,
            const double* __restrict__ b, LsmrState* S, double* part, unsigned* counter,
            int ms = 0, const double2* __restrict__ dense_av = nullptr) {
    if (S->done) return;
    const double inv_alpha = S->inv_alpha, alpha = S->alpha, inv_beta = S->inv_beta;
    const bool chk = S->check != 0;  // uniform: form r = b - A x_k as well
    double acc[2] = {0.0, 0.0};
    if constexpr (G == 0) {  // sliced layout, one lane per row
        for (int t = blockIdx.x * kBlock + threadIdx.x; t < A.snpos; t += gridDim.x * kBlock) {
            const int row = A.sperm[t];
            double s1 = 0.0, s2 = 0.0;
            if (chk) sliced_dot_pair<true>(A, t, tx, s1, s2);
            else sliced_dot_pair<false>(A, t, tx, s1, s2);
            if (row >= 0) spmv_row_out(row, s1, s2, chk, inv_alpha, alpha, inv_beta, qr, b, ms, dense_av, acc);
        }
    } else {
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (gridDim.x * kBlock) / G;
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < A.rows; row += groups) {
            double s1 = 0.0, s2 = 0.0;
            if (chk) row_dot_pair<G>(A, row, lane, tx, s1, s2);
            else row_dot_first<G>(A, row, lane, tx, s1);
            if (G > 1) {
                s1 = group_sum<G>(s1, mask);
                if (chk) s2 = group_sum<G>(s2, mask);
            }
            if (lane == 0) spmv_row_out(row, s1, s2, chk, inv_alpha, alpha, inv_beta, qr, b, ms, dense_av, acc);
        }
    }
    double tot[2];
    if (last_block_total<2>(acc, part, counter, tot) && threadIdx.x == 0) spmv_totals(S, tot, chk);
}

// Column epilogue of the A^T product (CSR and sliced kernels): s1 = (A^T q)_col,
// s2 = (A^T r)_col (when chk).
template <bool FIRST>
__device__ __forceinline__ void spmvt_row_out(int col, double s1, double s2, bool chk, double inv_alpha,
                                              double beta, double inv_beta, double* __restrict__ s,
                                              const double2* __restrict__ dense_atv, double (&acc)[1]) {
    if (dense_atv) {
        const double2 dv = dense_atv[col];
        s1 += dv.x;
        s2 += dv.y;
    }
    s[col] = FIRST ? s1 * inv_beta : s1 * inv_beta - beta * (s[col] * inv_alpha);
    if (chk) acc[0] += s2 * s2;
}

__device__ __forceinline__ void spmvt_totals(LsmrState* S, const double (&tot)[1], bool chk) {
    if (chk) {
        const double arn = sqrt(tot[0]);
        S->arnorm = arn;
        const double ratio = S->rnorm > 0.0 ? arn / (S->anorm * S->rnorm) : 0.0;
        S->ratio = ratio;
        if (ratio < S->atol) {
            S->done = 1;
            S->status = kOk;
        } else if (S->k >= S->maxit) {
            S->done = 1;
            S->status = kErrMaxit;
        }
    }
    S->check = residual_check_next(S);
}

// s <- A^T q * inv_beta - beta * (s * inv_alpha)      [s of the next apply]
// z  = A^T r                                            [only its norm]
// totals: arnorm = ||z||; ratio check on x_k; FIRST: s = A^T q * inv_beta.
// dense_atv[col] (nullptr if no dense rows): the dense rows' contribution
// to A^T u and A^T r, computed just before.
template <int G, bool FIRST>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
k_spmvt_lsmr(Csr<double> At, const double2* __restrict__ qr, double* __restrict__ s, LsmrState* S,
             double* part, unsigned* counter, const double2* __restrict__ dense_atv = nullptr) {
    if (S->done) return;
    const double inv_alpha = S->inv_alpha, beta = S->beta, inv_beta = S->inv_beta;
    const bool chk = FIRST || S->check != 0;  // uniform: form A^T r as well
    double acc[1] = {0.0};
    if constexpr (G == 0) {  // sliced layout, one lane per column
        for (int t = blockIdx.x * kBlock + threadIdx.x; t < At.snpos; t += gridDim.x * kBlock) {
            const int col = At.sperm[t];
            double s1 = 0.0, s2 = 0.0;
            if (chk) sliced_dot_pair<true>(At, t, qr, s1, s2);
            else sliced_dot_pair<false>(At, t, qr, s1, s2);
            if (col >= 0) spmvt_row_out<FIRST>(col, s1, s2, chk, inv_alpha, beta, inv_beta, s, dense_atv, acc);
        }
    } else {
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (gridDim.x * kBlock) / G;
        for (int col = (blockIdx.x * kBlock + threadIdx.x) / G; col < At.rows; col += groups) {
            double s1 = 0.0, s2 = 0.0;
            if (chk) row_dot_pair<G>(At, col, lane, qr, s1, s2);
            else row_dot_first<G>(At, col, lane, qr, s1);
            if (G > 1) {
                s1 = group_sum<G>(s1, mask);
                if (chk) s2 = group_sum<G>(s2, mask);
            }
            if (lane == 0) spmvt_row_out<FIRST>(col, s1, s2, chk, inv_alpha, beta, inv_beta, s, dense_atv, acc);
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0 && !FIRST) spmvt_totals(S, tot, chk);
}

struct PowerState {
    double lambda, inv_lambda;
};

// ---------------------------------------------------------------------------
// dense-row block (sparse-dense problems, Sec. 3.3): Ad is m_d x n row-major
// ---------------------------------------------------------------------------
constexpr int kDenseChunk = 1024;  // columns per block of the A_d products
constexpr int kDenseRowsPerBlock = kBlock / 32;

// Partial dot products of every dense row with (v1, v2) over one chunk of
// columns: PAIR reads (v1, v2) = p[j], otherwise (v, 0).  One warp per dense
// row; the chunk of the vector is staged in shared memory once per block.
template <bool PAIR>
__global__ void __launch_bounds__(kBlock)
k_dense_av(const double* __restrict__ Ad, int md, int n, const void* __restrict__ vin,
           double2* __restrict__ part, const LsmrState* S) {
    if (S && S->done) return;
    __shared__ double2 vs[kDenseChunk];
    const int c0 = blockIdx.x * kDenseChunk;
    const int cn = min(kDenseChunk, n - c0);
    for (int i = threadIdx.x; i < cn; i += kBlock) {
        if (PAIR) vs[i] = reinterpret_cast<const double2*>(vin)[c0 + i];
        else vs[i] = make_double2(reinterpret_cast<const double*>(vin)[c0 + i], 0.0);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.y * kDenseRowsPerBlock + warp;
    if (r >= md) return;
    const double* a = Ad + (size_t)r * n + c0;
    double s1 = 0.0, s2 = 0.0;
    for (int i = lane; i < cn; i += 32) {
        const double av = a[i];
        s1 += av * vs[i].x;
        s2 += av * vs[i].y;
    }
    s1 = group_sum<32>(s1, 0xffffffffu);
    s2 = group_sum<32>(s2, 0xffffffffu);
    if (lane == 0) part[(size_t)r * gridDim.x + blockIdx.x] = make_double2(s1, s2);
}

// Sums the chunk partials of each dense row in chunk order.
static __global__ void __launch_bounds__(kBlock)
k_dense_av_finish(int md, int nchunks, const double2* __restrict__ part, double2* __restrict__ out,
                  const LsmrState* S) {
    if (S && S->done) return;
    const int r = blockIdx.x * kBlock + threadIdx.x;
    if (r >= md) return;
    double s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < nchunks; ++c) {
        const double2 p = part[(size_t)r * nchunks + c];
        s1 += p.x;
        s2 += p.y;
    }
    out[r] = make_double2(s1, s2);
}

// out[j] = (sum_r Ad[r, j] u1[r], sum_r Ad[r, j] u2[r]) with (u1, u2) = u[r]
// (PAIR) or (u[r], 0); one thread per column, dense rows in order, the u
// values staged in shared memory (dynamic, 16 * md bytes).
template <bool PAIR>
__global__ void __launch_bounds__(kBlock)
k_dense_atv(const double* __restrict__ Ad, int md, int n, const void* __restrict__ uin,
            double2* __restrict__ out, const LsmrState* S) {
    if (S && S->done) return;
    extern __shared__ double2 us[];
    for (int i = threadIdx.x; i < md; i += kBlock) {
        if (PAIR) us[i] = reinterpret_cast<const double2*>(uin)[i];
        else us[i] = make_double2(reinterpret_cast<const double*>(uin)[i], 0.0);
    }
    __syncthreads();
    for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock) {
        double s1 = 0.0, s2 = 0.0;
        for (int r = 0; r < md; ++r) {
            const double av = Ad[(size_t)r * n + j];
            s1 += av * us[r].x;
            s2 += av * us[r].y;
        }
        out[j] = make_double2(s1, s2);
    }
}

// y[j] += add[j].x (plain products with the dense block)
static __global__ void k_add_x(int n, const double2* __restrict__ add, double* __restrict__ y) {
    for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock) y[j] += add[j].x;
}
// y[ms + r] = d[r].x * scale (scale = P->inv_lambda when P is given)
static __global__ void k_put_dense(int md, int ms, const double2* __restrict__ d, double* __restrict__ y,
                            const PowerState* P) {
    const int r = blockIdx.x * kBlock + threadIdx.x;
    if (r < md) y[ms + r] = d[r].x * (P ? P->inv_lambda : 1.0);
}
// out[i] = in[i].x (H = 0) or in[i].y (H = 1): one half of an interleaved pair
template <int H>
static __global__ void k_half(int n, const double2* __restrict__ in, double* __restrict__ out) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) out[i] = H ? in[i].y : in[i].x;
}
// out[i] = in[perm[i]]
static __global__ void k_gather(int m, const int32_t* __restrict__ perm, const double* __restrict__ in,
                         double* __restrict__ out) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < m; i += gridDim.x * kBlock) out[i] = in[perm[i]];
}
// out[perm[i]] = in[i]
static __global__ void k_scatter(int m, const int32_t* __restrict__ perm, const double* __restrict__ in,
                          double* __restrict__ out) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < m; i += gridDim.x * kBlock) out[perm[i]] = in[i];
}

// ---------------------------------------------------------------------------
// triangular solves
// ---------------------------------------------------------------------------
// right-hand side variants
enum RhsKind { RHS_VEC = 0, RHS_SCALED = 1, RHS_SUB = 2 };

template <typename T>
struct Rhs {
    const T* a;        // VEC, SUB: a;  SCALED: scale d
    const T* b;        // SUB: subtracted vector
    const double* s;   // SCALED: float64 source vector
};

template <typename T, int K>
__device__ __forceinline__ T rhs_at(const Rhs<T>& h, int i) {
    if (K == RHS_VEC) return h.a[i];
    if (K == RHS_SUB) return h.a[i] - h.b[i];
    return h.a[i] * (T)h.s[i];
}

// A triangular system stored by solve position: position t solves unknown
// order[t] (rows sorted by level, then id), and the row's entries (the
// strictly triangular part; column ids are unknown ids) and its diagonal are
// stored at position t, so every level is one contiguous range.
template <typename T>
struct Tri {
    int32_t n;
    const int32_t* ptr;    // n + 1, by position
    const int32_t* idx;    // unknown ids of the entries
    const T* val;
    const T* idiag;        // inverse diagonal by position; nullptr: unit diagonal
    const int32_t* order;  // order[t]: unknown solved at position t
    // right-hand-side terms of rows whose same-group dependencies were
    // substituted (fused levels): x_i uses rhs_i + sum rval * rhs(ridx);
    // rptr == nullptr when no levels are fused
    const int32_t* rptr;
    const int32_t* ridx;
    const T* rval;
    // the first entries of every row again, position-major (see DevFactor)
    const int32_t* eidx;
    const T* eval;
};

template <typename T, int K>
__device__ __forceinline__ T rhs_full(const Tri<T>& tri, const Rhs<T>& rhs, int t, int row) {
    T rv = rhs_at<T, K>(rhs, row);
    if (tri.rptr) {
        const int q1 = tri.rptr[t + 1];
        int q = tri.rptr[t];
        for (; q + 3 < q1; q += 4) {
            const int i0 = tri.ridx[q], i1 = tri.ridx[q + 1], i2 = tri.ridx[q + 2], i3 = tri.ridx[q + 3];
            const T c0 = tri.rval[q], c1 = tri.rval[q + 1], c2 = tri.rval[q + 2], c3 = tri.rval[q + 3];
            const T r0 = rhs_at<T, K>(rhs, i0), r1 = rhs_at<T, K>(rhs, i1), r2 = rhs_at<T, K>(rhs, i2),
                    r3 = rhs_at<T, K>(rhs, i3);
            rv += c0 * r0;
            rv += c1 * r1;
            rv += c2 * r2;
            rv += c3 * r3;
        }
        for (; q < q1; ++q) rv += tri.rval[q] * rhs_at<T, K>(rhs, tri.ridx[q]);
    }
    return rv;
}

// Waits until flag == epoch.  Gives up after kWaitNs or when another thread
// has already given up; returns false then.
__device__ __forceinline__ bool wait_flag(const int* flag, int epoch, int* err) {
    if (ld_acquire(flag) == epoch) return true;
    const unsigned long long t0 = globaltimer();
    for (int spin = 1;; ++spin) {
        if (ld_acquire(flag) == epoch) return true;
        if ((spin & 31) == 0) {
            if (*(volatile int*)err != 0) return false;
            if ((long long)(globaltimer() - t0) > kWaitNs) {
                atomicCAS(err, 0, 1);
                return false;
            }
        }
    }
}

// Sync-free solve with per-row ready flags (used by the allocation-free entry
// point, whose scratch holds the flags).  Blocks take chunks of positions
// from a ticket counter; every group of G lanes solves one row at a time,
// waiting on the flags of the unknowns it reads.  A dependency always sits at
// an earlier position, hence in a chunk taken earlier by a running block (or
// earlier in the same chunk), so every wait ends; the 1 s bound only guards
// against faults.  epoch = 1 + 64 * apply_count + slot.
template <typename T, int G, int K, int ROUNDS>
__global__ void __launch_bounds__(kBlock)
k_trsv_syncfree(Tri<T> tri, Rhs<T> rhs, T* x, int* flags, int slot, unsigned* tickets,
                const LsmrState* S, int* err) {
    if (S->done) return;
    const int epoch = 1 + kMaxSlots * S->apply_count + slot;
    const int n = tri.n;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    constexpr int per_round = kBlock / G;
    constexpr int chunk_rows = per_round * ROUNDS;
    __shared__ int chunk;
    for (;;) {
        // Lanes of one warp leave the spin-waits of the previous chunk at
        // different times; __syncthreads() is an aligned barrier, so every
        // warp reconverges first.
        __syncwarp();
        if (threadIdx.x == 0) chunk = (int)atomicAdd(&tickets[slot], 1u);
        __syncthreads();
        const long long c0 = (long long)chunk * chunk_rows;
        __syncthreads();
        if (c0 >= n) break;
#pragma unroll 1
        for (int rd = 0; rd < ROUNDS; ++rd) {
            const long long tpos = c0 + rd * per_round + threadIdx.x / G;
            if (tpos >= n) break;
            const int row = tri.order[tpos];
            T sum = (T)0;
            bool ok = true;
            const int e1 = tri.ptr[tpos + 1];
            for (int e = tri.ptr[tpos] + lane; e < e1; e += G) {
                const int j = tri.idx[e];
                if (!wait_flag(&flags[j], epoch, err)) {
                    ok = false;
                    break;
                }
                sum += tri.val[e] * ld_l2(&x[j]);
            }
            sum = group_sum<G>(sum, mask);
            ok = __all_sync(mask, ok);
            if (lane == 0) {
                T v = rhs_full<T, K>(tri, rhs, (int)tpos, row) - sum;
                if (tri.idiag) v = v * tri.idiag[tpos];
                if (!ok) v = (T)NAN;
                x[row] = v;
                st_release(&flags[row], epoch);
            }
        }
    }
}

// ---- sentinel-based sync-free solve ---------------------------------------
// Before the solve the output vector is filled with all-one bytes (a NaN
// whose bit pattern arithmetic never produces: the GPU's computed NaNs have a
// clear sign bit).  An unknown is ready once its value is no longer that
// pattern, so one relaxed load both tests readiness and delivers the value.
// The polled word is the datum itself, so no ordering with other accesses is
// needed: no "memory" clobber, which lets the compiler issue the row's other
// loads (position -> unknown, right-hand side, diagonal) before the wait.
__device__ __forceinline__ double ld_relaxed(const double* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
    return __longlong_as_double((long long)v);
}
__device__ __forceinline__ float ld_relaxed(const float* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return __uint_as_float(v);
}
__device__ __forceinline__ void st_relaxed(double* p, double x) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"((unsigned long long)__double_as_longlong(x)));
}
__device__ __forceinline__ void st_relaxed(float* p, float x) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(__float_as_uint(x)));
}
__device__ __forceinline__ bool is_pending(double v) { return __double_as_longlong(v) == -1LL; }
__device__ __forceinline__ bool is_pending(float v) { return __float_as_uint(v) == 0xffffffffu; }

// Spins until x[j] is written; NaN and ok = false after kWaitNs or once
// another thread has given up.
// Polls back off exponentially (64 ns .. 1 us): hundreds of thousands of
// waiting rows polling flat out would otherwise take the issue slots and L2
// bandwidth that the rows being solved need.
template <typename T>
__device__ __noinline__ T wait_value(const T* p, int* err, bool& ok) {
    const unsigned long long t0 = globaltimer();
    unsigned ns = 64;
    for (;;) {
        __nanosleep(ns);
        const T v = ld_relaxed(p);
        if (!is_pending(v)) return v;
        if (ns < 1024) ns <<= 1;
        if (*(volatile int*)err != 0 || (long long)(globaltimer() - t0) > kWaitNs) {
            atomicCAS(err, 0, 1);
            ok = false;
            return (T)NAN;
        }
    }
}

// One row per group of G lanes (G = 1: one thread per row); entries are read
// four at a time per lane so that several gathers are in flight.  Chunks of
// positions are handed out by a ticket counter as in k_trsv_syncfree.
template <typename T, int G, int K, int ROUNDS>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
k_trsv_sentinel(Tri<T> tri, Rhs<T> rhs, T* x, int slot, unsigned* tickets, const LsmrState* S,
                int* err) {
    if (S->done) return;
    const int n = tri.n;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    constexpr int per_round = kBlock / G;
    constexpr int chunk_rows = per_round * ROUNDS;
    __shared__ int chunk;
    for (;;) {
        __syncwarp();
        if (threadIdx.x == 0) chunk = (int)atomicAdd(&tickets[slot], 1u);
        __syncthreads();
        const long long c0 = (long long)chunk * chunk_rows;
        __syncthreads();
        if (c0 >= n) break;
#pragma unroll 1
        for (int rd = 0; rd < ROUNDS; ++rd) {
            const long long tpos = c0 + rd * per_round + threadIdx.x / G;
            if (tpos >= n) break;
            const int e1 = tri.ptr[tpos + 1];
            int e = tri.ptr[tpos] + lane;
            // everything that does not depend on other rows, loaded up front
            const int row = tri.order[tpos];
            const T rv = rhs_full<T, K>(tri, rhs, (int)tpos, row);
            const T dg = tri.idiag ? tri.idiag[tpos] : (T)1;
            T sum = (T)0;
            bool ok = true;
            for (; e + 3 * G < e1; e += 4 * G) {
                const int j0 = tri.idx[e], j1 = tri.idx[e + G], j2 = tri.idx[e + 2 * G], j3 = tri.idx[e + 3 * G];
                const T a0 = tri.val[e], a1 = tri.val[e + G], a2 = tri.val[e + 2 * G], a3 = tri.val[e + 3 * G];
                T v0 = ld_relaxed(&x[j0]), v1 = ld_relaxed(&x[j1]), v2 = ld_relaxed(&x[j2]), v3 = ld_relaxed(&x[j3]);
                if (is_pending(v0)) v0 = wait_value(&x[j0], err, ok);
                if (is_pending(v1)) v1 = wait_value(&x[j1], err, ok);
                if (is_pending(v2)) v2 = wait_value(&x[j2], err, ok);
                if (is_pending(v3)) v3 = wait_value(&x[j3], err, ok);
                sum += a0 * v0 + a1 * v1 + a2 * v2 + a3 * v3;
            }
            for (; e < e1; e += G) {
                const int j = tri.idx[e];
                T v = ld_relaxed(&x[j]);
                if (is_pending(v)) v = wait_value(&x[j], err, ok);
                sum += tri.val[e] * v;
            }
            if (G > 1) {
                sum = group_sum<G>(sum, mask);
                ok = __all_sync(mask, ok);
            }
            if (lane == 0) {
                T v = rv - sum;
                if (tri.idiag) v = v * dg;
                if (!ok) v = (T)NAN;
                st_relaxed(&x[row], v);
            }
        }
    }
}

// Sync-free solve with warp-level tickets.  A warp takes R * (32 / G)
// consecutive positions from the ticket counter; each group of G lanes
// solves R of them (row r of the group at chunk + r * (32 / G) + lane / G),
// reading the structure and the full right-hand sides of all R rows before
// it waits on any unknown, so those loads are in flight together.  There is
// no block-wide barrier: a warp whose rows wait holds up no other warp.
// Readiness as in k_trsv_sentinel (all-one bytes = not yet solved).  A row
// depends only on earlier positions, which sit in chunks taken earlier by
// running warps or earlier in this warp's own chunk (an earlier r, or the
// same r on a lower lane group), so every wait ends; the bound only guards
// against faults.
template <typename T, int G, int K, int R>
__global__ void __launch_bounds__(kBlock)
k_trsv_warp(Tri<T> tri, Rhs<T> rhs, T* x, int slot, unsigned* tickets, const LsmrState* S, int* err) {
    if (S->done) return;
    const int n = tri.n;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & 31;
    const int sub = lane & (G - 1);
    constexpr int per_pass = 32 / G;
    constexpr int chunk_rows = per_pass * R;
    for (;;) {
        __syncwarp();
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(&tickets[slot], 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        const long long c0 = (long long)c * chunk_rows;
        if (c0 >= n) break;
        int row[R], e0[R], e1[R];
        T rv[R], dg[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long t = c0 + r * per_pass + lane / G;
            row[r] = -1;
            e0[r] = 0;
            e1[r] = 0;
            rv[r] = (T)0;
            dg[r] = (T)1;
            if (t < n) {
                row[r] = tri.order[t];
                e0[r] = tri.ptr[t] + sub;
                e1[r] = tri.ptr[t + 1];
                if (sub == 0) {
                    rv[r] = rhs_full<T, K>(tri, rhs, (int)t, row[r]);
                    if (tri.idiag) dg[r] = tri.idiag[t];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            T sum = (T)0;
            bool ok = true;
            int e = e0[r];
            const int e_end = e1[r];
            for (; e + 3 * G < e_end; e += 4 * G) {
                const int j0 = tri.idx[e], j1 = tri.idx[e + G], j2 = tri.idx[e + 2 * G], j3 = tri.idx[e + 3 * G];
                const T a0 = tri.val[e], a1 = tri.val[e + G], a2 = tri.val[e + 2 * G], a3 = tri.val[e + 3 * G];
                T v0 = ld_relaxed(&x[j0]), v1 = ld_relaxed(&x[j1]), v2 = ld_relaxed(&x[j2]), v3 = ld_relaxed(&x[j3]);
                if (is_pending(v0)) v0 = wait_value(&x[j0], err, ok);
                if (is_pending(v1)) v1 = wait_value(&x[j1], err, ok);
                if (is_pending(v2)) v2 = wait_value(&x[j2], err, ok);
                if (is_pending(v3)) v3 = wait_value(&x[j3], err, ok);
                sum += a0 * v0 + a1 * v1 + a2 * v2 + a3 * v3;
            }
            for (; e < e_end; e += G) {
                const int j = tri.idx[e];
                T v = ld_relaxed(&x[j]);
                if (is_pending(v)) v = wait_value(&x[j], err, ok);
                sum += tri.val[e] * v;
            }
            if (G > 1) {
                sum = group_sum<G>(sum, mask);
                ok = __all_sync(mask, ok);
            }
            if (sub == 0 && row[r] >= 0) {
                T v = rv[r] - sum;
                if (tri.idiag) v = v * dg[r];
                if (!ok) v = (T)NAN;
                st_relaxed(&x[row[r]], v);
            }
        }
    }
}

// Persistent level-synchronous solve: one co-resident block of kCoopBlock
// threads per SM walks the levels in order, with a grid-wide barrier between
// levels.  The barrier is split: a block arrives as soon as its rows of level
// l are stored, then starts loading the structure of its rows of level l + 1
// (which depends on no unknown) while the other blocks finish, and only then
// waits.  The first KP entries of a row come from the position-major copy
// (Tri::eidx / eval) through cp.async into shared memory, so they cost no
// registers and a warp's loads are coalesced; only rows longer than KP read
// the CSR arrays as well.  Chunks of 32 consecutive positions go to warps in
// grid-cyclic order, so a level is spread over every SM.
// The barrier counter only grows (arrivals = level * blocks) and needs no
// reset within a launch; waits are bounded like every other wait here.  x is
// read through L2 (__ldcg) because other SMs wrote it.
constexpr int kCoopBlock = 1024;

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// every thread of the block has stored its level; one release-add per block
__device__ __forceinline__ void grid_arrive(unsigned* bar) {
    __syncthreads();
    if (threadIdx.x == 0) red_release_add(bar, 1u);
}

// one acquire-spin per block, then the block barrier hands the ordering on
__device__ __forceinline__ void grid_wait(unsigned* bar, unsigned target, int* err) {
    if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer();
        while ((unsigned)ld_acquire(reinterpret_cast<const int*>(bar)) < target) {
            if (*(volatile int*)err != 0) break;
            if ((long long)(globaltimer() - t0) > kWaitNs) {
                atomicCAS(err, 0, 1);
                break;
            }
        }
    }
    __syncthreads();
}

// One row's structure and right-hand side, loaded ahead (wavefront solve).
template <typename T, int KP>
struct RowAhead {
    int row, e0, e1;
    T rv, dg;
    int j[KP];
    T a[KP];
};

// From the CSR arrays (entries past the row's end: column 0, value 0).
template <typename T, int K, int KP>
__device__ __forceinline__ void read_ahead(const Tri<T>& tri, const Rhs<T>& rhs, int t, RowAhead<T, KP>& r) {
    r.row = tri.order[t];
    r.e0 = tri.ptr[t];
    r.e1 = tri.ptr[t + 1];
    r.rv = rhs_full<T, K>(tri, rhs, t, r.row);
    r.dg = tri.idiag ? tri.idiag[t] : (T)1;
#pragma unroll
    for (int q = 0; q < KP; ++q) {
        const bool in = r.e0 + q < r.e1;
        r.j[q] = in ? tri.idx[r.e0 + q] : 0;
        r.a[q] = in ? tri.val[r.e0 + q] : (T)0;
    }
}

// Asynchronous global -> shared copies (no registers involved).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <typename T>
__device__ __forceinline__ void cp_async_t(T* smem, const T* gmem) {
    if constexpr (sizeof(T) == 8) cp_async8(smem, gmem);
    else cp_async4(smem, gmem);
}

// The part of a row kept in registers while its level waits.
template <typename T>
struct RowHead {
    int row, e0, e1;  // e0: where the CSR remainder (entries past KP) starts
    T rv, dg;
};

// Shared-memory slots of one thread: KP values, then KP column ids, strided
// by the block size so that a warp's accesses hit distinct banks.
template <typename T, int K, int KP>
__device__ __forceinline__ void stage_row(const Tri<T>& tri, const Rhs<T>& rhs, int t, int32_t* js, T* as,
                                          RowHead<T>& h) {
    const size_t n = (size_t)tri.n;
#pragma unroll
    for (int q = 0; q < KP; ++q) {
        cp_async4(&js[q * kCoopBlock], &tri.eidx[q * n + t]);
        cp_async_t<T>(&as[q * kCoopBlock], &tri.eval[q * n + t]);
    }
    cp_async_commit();
    h.row = __ldg(&tri.order[t]);
    h.e0 = __ldg(&tri.ptr[t]) + KP;
    h.e1 = __ldg(&tri.ptr[t + 1]);
    h.dg = tri.idiag ? __ldg(&tri.idiag[t]) : (T)1;
    h.rv = rhs_full<T, K>(tri, rhs, t, h.row);
}

template <typename T, int KP>
__device__ __forceinline__ void solve_staged(const Tri<T>& tri, const RowHead<T>& h, const int32_t* js,
                                             const T* as, T* x) {
    cp_async_wait_all();
    int j[KP];
    T v[KP];
#pragma unroll
    for (int q = 0; q < KP; ++q) j[q] = js[q * kCoopBlock];
#pragma unroll
    for (int q = 0; q < KP; ++q) v[q] = j[q] >= 0 ? __ldcg(&x[j[q]]) : (T)0;
    T sum = (T)0;
#pragma unroll
    for (int q = 0; q < KP; ++q) sum += as[q * kCoopBlock] * v[q];
    // the CSR remainder (rows longer than KP), four gathers in flight
    int e = h.e0;
    for (; e + 3 < h.e1; e += 4) {
        const int j0 = __ldg(&tri.idx[e]), j1 = __ldg(&tri.idx[e + 1]), j2 = __ldg(&tri.idx[e + 2]),
                  j3 = __ldg(&tri.idx[e + 3]);
        const T a0 = __ldg(&tri.val[e]), a1 = __ldg(&tri.val[e + 1]), a2 = __ldg(&tri.val[e + 2]),
                a3 = __ldg(&tri.val[e + 3]);
        const T v0 = __ldcg(&x[j0]), v1 = __ldcg(&x[j1]), v2 = __ldcg(&x[j2]), v3 = __ldcg(&x[j3]);
        sum += a0 * v0;
        sum += a1 * v1;
        sum += a2 * v2;
        sum += a3 * v3;
    }
    for (; e < h.e1; ++e) sum += __ldg(&tri.val[e]) * __ldcg(&x[__ldg(&tri.idx[e])]);
    T res = h.rv - sum;
    if (tri.idiag) res = res * h.dg;
    x[h.row] = res;
}

// A row straight from the CSR arrays (rows past the first of a wide level).
template <typename T, int K>
__device__ __forceinline__ void solve_row_csr(const Tri<T>& tri, const Rhs<T>& rhs, int t, T* x) {
    const int row = __ldg(&tri.order[t]);
    const int e1 = __ldg(&tri.ptr[t + 1]);
    int e = __ldg(&tri.ptr[t]);
    const T dg = tri.idiag ? __ldg(&tri.idiag[t]) : (T)1;
    T sum = (T)0;
    for (; e + 3 < e1; e += 4) {
        const int j0 = __ldg(&tri.idx[e]), j1 = __ldg(&tri.idx[e + 1]), j2 = __ldg(&tri.idx[e + 2]),
                  j3 = __ldg(&tri.idx[e + 3]);
        const T a0 = __ldg(&tri.val[e]), a1 = __ldg(&tri.val[e + 1]), a2 = __ldg(&tri.val[e + 2]),
                a3 = __ldg(&tri.val[e + 3]);
        const T v0 = __ldcg(&x[j0]), v1 = __ldcg(&x[j1]), v2 = __ldcg(&x[j2]), v3 = __ldcg(&x[j3]);
        sum += a0 * v0;
        sum += a1 * v1;
        sum += a2 * v2;
        sum += a3 * v3;
    }
    for (; e < e1; ++e) sum += __ldg(&tri.val[e]) * __ldcg(&x[__ldg(&tri.idx[e])]);
    T res = rhs_full<T, K>(tri, rhs, t, row) - sum;
    if (tri.idiag) res = res * dg;
    x[row] = res;
}

// ---- binned persistent solve ----------------------------------------------
// A system stored for k_trsv_binned.  Rows are stored by "binned position":
// the positions of a level group are the group's rows, sorted by the lanes
// their entry count needs.  Each row is one flat entry list:
//   x_i = -(sum_e val_e * v_e) * d_i,
// where an entry with idx >= 0 reads the unknown x[idx] (a substituted or
// triangular dependency, val = its coefficient), an entry with idx < -1
// reads the right-hand side at (idx & 0x7fffffff) (the row's own term with
// val = -1, a fused right-hand-side term c with val = -c), and idx = -1 is
// padding.  The whole row is one dot product whose gathers can all be in
// flight together.  A segment is a run of rows of one group that all take G
// lanes each and round up to the same slot size `cap` (a multiple of G);
// each of its rows owns the slot at base + (t - p0) * cap, so a
// row's entries need no row-pointer lookup and lane `sub` reads entries
// sub, sub + G, ... (coalesced across the warp).  The warps of the grid deal
// the segment's work items (32 / G rows each) among themselves.
struct BinSeg {
    int32_t p0, p1;       // binned positions [p0, p1)
    int32_t G;            // lanes per row (1, 2, 4, 8, 16, 32)
    int32_t item0;        // first work item of the segment within its group
    int32_t cap;          // entries per row slot
    int32_t base;         // entry offset of the segment's first slot
};

template <typename T>
struct BinTri {
    int32_t n, ngroups;
    const int32_t* idx;      // see above
    const T* val;
    const int32_t* order;    // unknown solved at each binned position
    const T* idiag;          // inverse diagonal by binned position; nullptr: unit diagonal
    const BinSeg* seg;
    const int32_t* gseg;     // segments of group g: [gseg[g], gseg[g + 1])
    const int32_t* gitems;   // work items of group g
    const int32_t* gpos;     // first binned position of group g (ngroups + 1 entries)
    const int32_t* gentry;   // first entry of group g (ngroups + 1 entries)
};

// Bulk prefetch of [p, p + bytes) into L2, in pieces of at most 1 MiB.  Only
// whole 16-byte units inside the range are asked for (the instruction wants
// 16-byte aligned addresses and sizes), so nothing outside it is touched.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    uintptr_t lo = (a + 15) & ~(uintptr_t)15;
    const uintptr_t hi = (a + bytes) & ~(uintptr_t)15;
    while (lo < hi) {
        const uintptr_t piece = (hi - lo < ((uintptr_t)1 << 20)) ? hi - lo : ((uintptr_t)1 << 20);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)piece) : "memory");
        lo += piece;
    }
}

// What a lane holds of its row in a work item before the unknowns it needs
// are ready: where the row goes, and the first four entries of its share.
template <typename T>
struct BinLane {
    int t;        // binned position (-1: no row for this lane)
    int row;      // unknown solved there
    int slot;     // entry offset of the row's slot
    T dg;         // inverse diagonal (1: unit)
    int j[4];     // entry ids (-1: padding or none)
    T a[4];
};

// Work item `item` of segment sg: 32 / G consecutive binned positions, G
// lanes per row.  Reads the lane's first four entries and the row's
// placement, none of which depends on an unknown.
template <typename T>
__device__ __forceinline__ void binned_prepare(const BinTri<T>& bt, const BinSeg& sg, int item, int lane,
                                               BinLane<T>& L) {
    const int G = sg.G;
    const int t = sg.p0 + item * (32 / G) + lane / G;
    const int sub = lane & (G - 1);
    L.t = t < sg.p1 ? t : -1;
    L.row = 0;
    L.dg = (T)1;
    L.slot = sg.base + (t - sg.p0) * sg.cap;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = sub + q * G;
        const bool in = L.t >= 0 && k < sg.cap;
        L.j[q] = in ? __ldg(&bt.idx[L.slot + k]) : -1;
        L.a[q] = in ? __ldg(&bt.val[L.slot + k]) : (T)0;
    }
    if (L.t >= 0 && sub == 0) {
        L.row = __ldg(&bt.order[t]);
        if (bt.idiag) L.dg = __ldg(&bt.idiag[t]);
    }
}

template <typename T, int K>
__device__ __forceinline__ T binned_value(const Rhs<T>& rhs, const T* x, int j) {
    if (j >= 0) return __ldcg(&x[j]);
    if (j == -1) return (T)0;
    return rhs_at<T, K>(rhs, j & 0x7fffffff);
}

// The rest of the item once every unknown of earlier groups is stored: the
// gathers of the prepared entries (unknowns and right-hand sides together),
// the lane's remaining entries (rows longer than 4 G), the reduction over the
// row's lanes and the store.
template <typename T, int K>
__device__ __forceinline__ void binned_finish(const BinTri<T>& bt, const Rhs<T>& rhs, const BinSeg& sg, int lane,
                                              const BinLane<T>& L, T* x) {
    const int G = sg.G;
    const int sub = lane & (G - 1);
    T v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = binned_value<T, K>(rhs, x, L.j[q]);
    T sum = (T)0;
#pragma unroll
    for (int q = 0; q < 4; ++q) sum += L.a[q] * v[q];
    if (L.t >= 0) {
        for (int k = sub + 4 * G; k < sg.cap; k += 4 * G) {
            int jj[4];
            T aa[4], vv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool in = k + q * G < sg.cap;
                jj[q] = in ? __ldg(&bt.idx[L.slot + k + q * G]) : -1;
                aa[q] = in ? __ldg(&bt.val[L.slot + k + q * G]) : (T)0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) vv[q] = binned_value<T, K>(rhs, x, jj[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) sum += aa[q] * vv[q];
        }
    }
    // sum over the row's G lanes (all of them have the same t, so all take part)
    const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    for (int off = G / 2; off > 0; off >>= 1) sum += __shfl_xor_sync(mask, sum, off, G);
    if (L.t >= 0 && sub == 0) x[L.row] = (-sum) * L.dg;
}

// Finds the segment of work item k of a group: the last segment in
// [s, s1) whose first item is <= k (segments in item order; seg[s].item0 <= k).
__device__ __forceinline__ int binned_seg(const BinSeg* seg, int s, int s1, int k) {
    int lo = s, hi = s1 - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&seg[mid].item0) <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr int kBinBlock = 1024;

// Persistent level-synchronous solve over binned groups.  Every block walks
// the groups in order; within a group the warps of the whole grid deal the
// work items of its segments (warp w takes items w, w + W, ...; warps are
// numbered across blocks first, so a small group still spreads over every
// SM).  Between groups a grid barrier, split: a block arrives once its rows
// are stored, then every warp reads the entries of its first item of the
// next group -- they depend on no unknown -- and only then does the block
// wait (bounded by kWaitNs).  After the wait one round of gathers finishes
// the item.  Block 0 of each slice also asks L2 for the next-but-one group's
// entries (bulk prefetch).  x is read through L2 (__ldcg): other SMs wrote
// it.  No pre-fill of x is needed.
template <typename T, int K>
__global__ void __launch_bounds__(kBinBlock, 1)
k_trsv_binned(BinTri<T> bt, Rhs<T> rhs, T* x, unsigned* bar, const LsmrState* S, int* err) {
    if (S->done) return;
    const int warps_per_block = blockDim.x >> 5;
    const int W = gridDim.x * warps_per_block;
    const int gw = blockIdx.x + gridDim.x * (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    auto prefetch_group = [&](int g) {
        if (g >= bt.ngroups || threadIdx.x != 0) return;
        const long long e0 = __ldg(&bt.gentry[g]), e1 = __ldg(&bt.gentry[g + 1]);
        const long long per = (e1 - e0 + gridDim.x - 1) / gridDim.x;
        const long long a = e0 + per * blockIdx.x, b = min(e1, a + per);
        if (a < b) {
            prefetch_l2(bt.idx + a, (size_t)(b - a) * sizeof(int32_t));
            prefetch_l2(bt.val + a, (size_t)(b - a) * sizeof(T));
        }
        const int p0 = __ldg(&bt.gpos[g]), p1 = __ldg(&bt.gpos[g + 1]);
        const long long pp = (p1 - p0 + gridDim.x - 1) / gridDim.x;
        const long long q0 = p0 + pp * blockIdx.x, q1 = min((long long)p1, q0 + pp);
        if (q0 < q1) {
            prefetch_l2(bt.order + q0, (size_t)(q1 - q0) * sizeof(int32_t));
            if (bt.idiag) prefetch_l2(bt.idiag + q0, (size_t)(q1 - q0) * sizeof(T));
        }
    };
    prefetch_group(0);
    prefetch_group(1);
    BinLane<T> L;
    int s = __ldg(&bt.gseg[0]);
    bool have = false;
    if (gw < __ldg(&bt.gitems[0])) {
        s = binned_seg(bt.seg, s, __ldg(&bt.gseg[1]), gw);
        const BinSeg sg = bt.seg[s];
        binned_prepare<T>(bt, sg, gw - sg.item0, lane, L);
        have = true;
    }
    for (int g = 0; g < bt.ngroups; ++g) {
        const int s0 = __ldg(&bt.gseg[g]), s1 = __ldg(&bt.gseg[g + 1]);
        const int items = __ldg(&bt.gitems[g]);
        if (g > 0) {
            // first item of this group read while the other blocks finish
            have = gw < items;
            if (have) {
                s = binned_seg(bt.seg, s0, s1, gw);
                const BinSeg sg = bt.seg[s];
                binned_prepare<T>(bt, sg, gw - sg.item0, lane, L);
            }
            prefetch_group(g + 1);
            grid_wait(bar, (unsigned)g * gridDim.x, err);
            if (*(volatile int*)err != 0) return;
        }
        if (have) {
            binned_finish<T, K>(bt, rhs, bt.seg[s], lane, L, x);
            for (int k = gw + W; k < items; k += W) {
                s = binned_seg(bt.seg, s, s1, k);
                const BinSeg sg = bt.seg[s];
                binned_prepare<T>(bt, sg, k - sg.item0, lane, L);
                binned_finish<T, K>(bt, rhs, sg, lane, L, x);
            }
        }
        if (g + 1 < bt.ngroups) grid_arrive(bar);
    }
}

// Dynamic shared memory of k_trsv_coop.
template <typename T>
constexpr size_t coop_smem_bytes(int kp) {
    return (size_t)kp * kCoopBlock * (sizeof(int32_t) + sizeof(T));
}

template <typename T, int K, int KP>
__global__ void __launch_bounds__(kCoopBlock, 1)
k_trsv_coop(Tri<T> tri, Rhs<T> rhs, T* x, const int32_t* __restrict__ level_ptr, int nlevels, unsigned* bar,
            const LsmrState* S, int* err) {
    if (S->done) return;
    extern __shared__ __align__(16) unsigned char coop_smem[];
    T* as = reinterpret_cast<T*>(coop_smem) + threadIdx.x;
    int32_t* js = reinterpret_cast<int32_t*>(coop_smem + (size_t)KP * kCoopBlock * sizeof(T)) + threadIdx.x;
    const int nthreads = gridDim.x * kCoopBlock;
    const int tid = (((threadIdx.x >> 5) * gridDim.x + blockIdx.x) << 5) + (threadIdx.x & 31);
    RowHead<T> h;
    int lo = __ldg(&level_ptr[0]), hi = __ldg(&level_ptr[1]);
    if (lo + tid < hi) stage_row<T, K, KP>(tri, rhs, lo + tid, js, as, h);
    for (int l = 0; l < nlevels; ++l) {
        const int t = lo + tid;
        if (t < hi) {
            solve_staged<T, KP>(tri, h, js, as, x);
            for (int t2 = t + nthreads; t2 < hi; t2 += nthreads) solve_row_csr<T, K>(tri, rhs, t2, x);
        }
        if (l + 1 < nlevels) {
            grid_arrive(bar);
            lo = hi;
            hi = __ldg(&level_ptr[l + 2]);
            if (lo + tid < hi) stage_row<T, K, KP>(tri, rhs, lo + tid, js, as, h);
            grid_wait(bar, (unsigned)(l + 1) * gridDim.x, err);
        }
    }
}

// Wavefront solve: a co-resident grid in which every thread owns a fixed,
// increasing sequence of level-ordered positions and solves them one after
// another, waiting on each unknown it reads (all-one bit pattern = not yet
// written, as in k_trsv_sentinel).  There are no tickets and no barriers:
// a row starts as soon as its own inputs exist, so rows of many levels are in
// flight at once and the solve pipelines across levels.  Chunks of 32
// consecutive positions go to warps in grid-cyclic order (warp ids run across
// blocks first), which keeps the structure reads coalesced and spreads each
// level over all SMs.  While a row waits, the structure of the thread's next
// row is already loading (it does not depend on any unknown).
// Progress: the smallest unsolved position has all its inputs solved and its
// thread has finished every earlier position it owns, so it is being worked
// on; this needs every thread resident, hence the cooperative launch.
constexpr int kWaveBlock = 256;

template <typename T, int K, int KP>
__global__ void __launch_bounds__(kWaveBlock)
k_trsv_wave(Tri<T> tri, Rhs<T> rhs, T* x, const LsmrState* S, int* err) {
    if (S->done) return;
    const int n = tri.n;
    const int lane = threadIdx.x & 31;
    const int warp = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int stride = 32 * gridDim.x * (kWaveBlock / 32);
    int t = 32 * warp + lane;
    if (t >= n) return;
    RowAhead<T, KP> cur;
    read_ahead<T, K, KP>(tri, rhs, t, cur);
    bool ok = true;
    for (;;) {
        const int tn = t + stride;
        RowAhead<T, KP> nxt;
        if (tn < n) read_ahead<T, K, KP>(tri, rhs, tn, nxt);
        T v[KP];
#pragma unroll
        for (int q = 0; q < KP; ++q) v[q] = (cur.e0 + q < cur.e1) ? ld_relaxed(&x[cur.j[q]]) : (T)0;
        T sum = (T)0;
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            if (is_pending(v[q])) v[q] = wait_value(&x[cur.j[q]], err, ok);
            sum += cur.a[q] * v[q];
        }
        for (int e = cur.e0 + KP; e < cur.e1; ++e) {
            const int j = tri.idx[e];
            T w = ld_relaxed(&x[j]);
            if (is_pending(w)) w = wait_value(&x[j], err, ok);
            sum += tri.val[e] * w;
        }
        T r = cur.rv - sum;
        if (tri.idiag) r = r * cur.dg;
        if (!ok) r = (T)NAN;
        st_relaxed(&x[cur.row], r);
        if (tn >= n) break;
        cur = nxt;
        t = tn;
    }
}

// Level-scheduled solve: one launch per level, positions [lo, hi).
template <typename T, int G, int K>
__global__ void __launch_bounds__(kBlock)
k_trsv_level(Tri<T> tri, Rhs<T> rhs, T* x, int lo, int hi, const LsmrState* S) {
    if (S->done) return;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    for (int tpos = lo + (blockIdx.x * kBlock + threadIdx.x) / G; tpos < hi; tpos += groups) {
        const int row = tri.order[tpos];
        const T rv = rhs_full<T, K>(tri, rhs, tpos, row);
        const T dg = tri.idiag ? tri.idiag[tpos] : (T)1;
        T sum = (T)0;
        const int e1 = tri.ptr[tpos + 1];
        int e = tri.ptr[tpos] + lane;
        for (; e + 3 * G < e1; e += 4 * G) {
            const int j0 = tri.idx[e], j1 = tri.idx[e + G], j2 = tri.idx[e + 2 * G], j3 = tri.idx[e + 3 * G];
            const T a0 = tri.val[e], a1 = tri.val[e + G], a2 = tri.val[e + 2 * G], a3 = tri.val[e + 3 * G];
            const T v0 = x[j0], v1 = x[j1], v2 = x[j2], v3 = x[j3];
            sum += a0 * v0;
            sum += a1 * v1;
            sum += a2 * v2;
            sum += a3 * v3;
        }
        for (; e < e1; e += G) sum += tri.val[e] * x[tri.idx[e]];
        if (G > 1) sum = group_sum<G>(sum, mask);
        if (lane == 0) {
            T v = rv - sum;
            if (tri.idiag) v = v * dg;
            x[row] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// correction pieces (precision T)
// ---------------------------------------------------------------------------

// y = M x, or y = M x - sub when sub is given (no state check when S == nullptr)
template <typename T, int G>
__global__ void __launch_bounds__(kBlock)
k_csr_mv(Csr<T> M, const T* __restrict__ x, T* __restrict__ y, const LsmrState* S,
         const T* __restrict__ sub = nullptr) {
    if (S && S->done) return;
    if constexpr (G == 0) {  // sliced layout
        for (int t = blockIdx.x * kBlock + threadIdx.x; t < M.snpos; t += gridDim.x * kBlock) {
            const int row = M.sperm[t];
            T s = (T)0;
            sliced_dot(M, t, x, s);
            if (row >= 0) y[row] = sub ? s - sub[row] : s;
        }
    } else {
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (gridDim.x * kBlock) / G;
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < M.rows; row += groups) {
            T s = (T)0;
            row_dot<G>(M, row, lane, x, s);
            s = group_sum<G>(s, mask);
            if (lane == 0) y[row] = sub ? s - sub[row] : s;
        }
    }
}

// e = L2 q1 (or L2 q1 - sub), CG start: r = e (and p = e implied), rr = <e, e>
template <typename T, int G>
__global__ void __launch_bounds__(kBlock)
k_l2_start(Csr<T> L2, const T* __restrict__ q1, T* __restrict__ r, LsmrState* S, double* part,
           unsigned* counter, LsmrState* gate, const T* __restrict__ sub = nullptr) {
    if (S->done) return;
    double acc[1] = {0.0};
    auto out = [&](int row, T s) {
        if (sub) s -= sub[row];
        r[row] = s;
        acc[0] += (double)(s * s);
    };
    if constexpr (G == 0) {  // sliced layout
        for (int t = blockIdx.x * kBlock + threadIdx.x; t < L2.snpos; t += gridDim.x * kBlock) {
            const int row = L2.sperm[t];
            T s = (T)0;
            sliced_dot(L2, t, q1, s);
            if (row >= 0) out(row, s);
        }
    } else {
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (gridDim.x * kBlock) / G;
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < L2.rows; row += groups) {
            T s = (T)0;
            row_dot<G>(L2, row, lane, q1, s);
            s = group_sum<G>(s, mask);
            if (lane == 0) out(row, s);
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        S->cg_rr = tot[0];
        S->cg_rr0 = tot[0];
        S->cg_beta = 0.0;
        if (gate) gate->done = 0;
    }
}

// c1 = L2^T p' with p' = r (first step) or r + beta p.  After the first step
// L2^T p' = L2^T r + beta (L2^T p), and c1 still holds L2^T p from the step
// before, so only L2^T r is formed (one multiply-add per entry).
template <typename T, int G, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_l2t_cg(Csr<T> L2t, const T* __restrict__ r, const T* __restrict__ p, T* __restrict__ c1,
         const LsmrState* S, const LsmrState* gate) {
    if (S->done || (gate && gate->done)) return;
    const T beta = (T)S->cg_beta;
    if constexpr (G == 0) {  // sliced layout
        for (int t = blockIdx.x * kBlock + threadIdx.x; t < L2t.snpos; t += gridDim.x * kBlock) {
            const int row = L2t.sperm[t];
            T s = (T)0;
            sliced_dot(L2t, t, r, s);
            if (row >= 0) c1[row] = FIRST ? s : s + beta * c1[row];
        }
    } else {
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (gridDim.x * kBlock) / G;
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < L2t.rows; row += groups) {
            T s = (T)0;
            row_dot<G>(L2t, row, lane, r, s);
            s = group_sum<G>(s, mask);
            if (lane == 0) c1[row] = FIRST ? s : s + beta * c1[row];
        }
    }
    (void)p;
}

// p <- r (+ beta p); Sp = p + L2 c3; totals: a = rr / <p, Sp>
template <typename T, int G, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_l2_sp(Csr<T> L2, const T* __restrict__ c3, const T* __restrict__ r, T* __restrict__ p,
        T* __restrict__ sp, LsmrState* S, double* part, unsigned* counter, const LsmrState* gate) {
    if (S->done || (gate && gate->done)) return;
    const T beta = (T)S->cg_beta;
    double acc[1] = {0.0};
    auto out = [&](int row, T s) {
        const T pv = FIRST ? r[row] : r[row] + beta * p[row];
        const T spv = pv + s;
        p[row] = pv;
        sp[row] = spv;
        acc[0] += (double)(pv * spv);
    };
    if constexpr (G == 0) {  // sliced layout
        for (int t = blockIdx.x * kBlock + threadIdx.x; t < L2.snpos; t += gridDim.x * kBlock) {
            const int row = L2.sperm[t];
            T s = (T)0;
            sliced_dot(L2, t, c3, s);
            if (row >= 0) out(row, s);
        }
    } else {
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (gridDim.x * kBlock) / G;
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < L2.rows; row += groups) {
            T s = (T)0;
            row_dot<G>(L2, row, lane, c3, s);
            s = group_sum<G>(s, mask);
            if (lane == 0) out(row, s);
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double rr = S->cg_rr;
        S->cg_a = (rr != 0.0 && tot[0] != 0.0) ? rr / tot[0] : 0.0;
    }
}

// w += a p (FIRST: w = a p); r -= a Sp; totals: beta = rr' / rr.  With a
// gate (adaptive steps): once rr' <= tol2 rr_0 the gate is closed and the
// kernels of the remaining CG steps return at once.
//
// With z (n entries): z += a c3 (FIRST: z = a c3) instead of the w update,
// c3 = L1^{-1} L1^{-T} L2^T p being this step's direction carried through
// both solves.  Since w = sum_j a_j p_j, z = L1^{-1} L1^{-T} L2^T w, the
// term Algorithm 3 forms from w with one more L2^T product and two more
// solves (steps 3-4); w itself is then not needed (w == nullptr).
template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_cg_update(int m2, const T* __restrict__ p, const T* __restrict__ sp, T* __restrict__ r,
            T* __restrict__ w, LsmrState* S, double* part, unsigned* counter, LsmrState* gate, double tol2,
            int n = 0, const T* __restrict__ c3 = nullptr, T* __restrict__ z = nullptr) {
    if (S->done || (gate && gate->done)) return;
    const T a = (T)S->cg_a;
    double acc[1] = {0.0};
    const int len = m2 > n ? m2 : n;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += gridDim.x * kBlock) {
        if (i < m2) {
            if (w) {
                const T pi = p[i];
                w[i] = FIRST ? a * pi : w[i] + a * pi;
            }
            const T ri = r[i] - a * sp[i];
            r[i] = ri;
            acc[0] += (double)(ri * ri);
        }
        if (i < n) z[i] = FIRST ? a * c3[i] : z[i] + a * c3[i];
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double rr = S->cg_rr;
        S->cg_beta = rr != 0.0 ? tot[0] / rr : 0.0;
        S->cg_rr = tot[0];
        if (gate && tot[0] <= tol2 * S->cg_rr0) gate->done = 1;
    }
}

// w = Sinv e (dense symmetric, row-major m2 x m2): one warp per row
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_dense_gemv(int m2, const T* __restrict__ Sinv, const T* __restrict__ e, T* __restrict__ w,
             const LsmrState* S) {
    if (S && S->done) return;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * kBlock) / 32;
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / 32; row < m2; row += warps) {
        const T* a = Sinv + (size_t)row * m2;
        T s = (T)0;
        for (int j = lane; j < m2; j += 32) s += a[j] * e[j];
        s = group_sum<32>(s, 0xffffffffu);
        if (lane == 0) w[row] = s;
    }
}

// ---------------------------------------------------------------------------
// end of the apply and the LSMR vector updates (float64)
// ---------------------------------------------------------------------------

// Advances the LSMR scalars after <t, s> is known (INIT: the first alpha, else
// one pair of rotations P_k, Pbar_k and the update coefficients); also counts
// the application and maps a device wait timeout to the solve's status.
template <bool INIT>
__device__ void lsmr_scalar_step(LsmrState* S, double ts) {
    S->apply_count += 1;
    if (S->error != 0) {
        S->done = 1;
        S->status = kErrTimeout;
        return;
    }
    S->ts = ts;
    if (!(ts >= 0.0) || !isfinite(ts)) {
        S->done = 1;
        S->status = kErrBreakdown;
        return;
    }
    const double alpha = sqrt(ts);
    if (INIT) {
        S->alphabar = alpha;
        S->zetabar = alpha * S->beta;
        S->rho = 1.0;
        S->rhobar = 1.0;
        S->cbar = 1.0;
        S->sbar = 0.0;
    } else {
        const double beta = S->beta;
        // rotation P_k
        const double rhoold = S->rho;
        const double ab = S->alphabar;
        const double rho = sqrt(ab * ab + beta * beta);
        const double c = ab / rho, sn = beta / rho;
        const double theta = sn * alpha;
        S->alphabar = c * alpha;
        // rotation Pbar_k
        const double rhobarold = S->rhobar;
        const double thetabar = S->sbar * rho;
        const double crho = S->cbar * rho;
        const double rhobar = sqrt(crho * crho + theta * theta);
        const double cbar = crho / rhobar, sbar = theta / rhobar;
        const double zeta = cbar * S->zetabar;
        S->zetabar = -sbar * S->zetabar;
        S->c_hbar = thetabar * rho / (rhoold * rhobarold);
        S->c_x = zeta / (rho * rhobar);
        S->c_h = theta / rho;
        S->rho = rho;
        S->rhobar = rhobar;
        S->cbar = cbar;
        S->sbar = sbar;
    }
    S->alpha = alpha;
    S->inv_alpha = alpha > 0.0 ? 1.0 / alpha : 0.0;
}

// t = d * g5 (IDENT: t = s, the unpreconditioned case), <t, s>; INIT: start the recurrences, else one LSMR
// rotation step; either way the apply counter advances.
// CGLS (Algorithm 1) scalars after h = M^{-1} z: rho' = <z, h> (step 13),
// beta = rho' / rho (step 14; INIT: the first rho, beta = 0).  The CGLS
// quantities reuse LsmrState fields: rho -> alphabar, beta -> zetabar,
// the step length alpha -> alpha.
template <bool INIT>
__device__ void cgls_scalar_step(LsmrState* S, double rho_new) {
    S->apply_count += 1;
    if (S->error != 0) {
        S->done = 1;
        S->status = kErrTimeout;
        return;
    }
    if (!(rho_new > 0.0) || !isfinite(rho_new)) {
        S->done = 1;
        S->status = kErrBreakdown;
        return;
    }
    S->zetabar = INIT ? 0.0 : rho_new / S->alphabar;
    S->alphabar = rho_new;
}

// t = D g5 (IDENT: t = s) into tx[i].x and <t, s>; the last block runs the
// solver's scalar step (LSMR, or CGLS when CGLS is set).
template <typename T, bool INIT, bool IDENT = false, bool CGLS = false>
__global__ void __launch_bounds__(kBlock)
k_finish_apply(int n, const T* __restrict__ d, const T* __restrict__ g5, const double* __restrict__ s,
               double2* __restrict__ tx, LsmrState* S, double* part, unsigned* counter) {
    if (S->done) return;
    double* t = reinterpret_cast<double*>(tx);  // t_i lives at tx[i].x
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const double ti = IDENT ? s[i] : (double)(d[i] * g5[i]);
        t[2 * i] = ti;
        acc[0] += ti * s[i];
    }
    double tot[1];
    if (!(last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0)) return;
    if (CGLS) cgls_scalar_step<INIT>(S, tot[0]);
    else lsmr_scalar_step<INIT>(S, tot[0]);
}

// Algorithm 3's input split of an m-vector r (user row order, stride
// `stride` doubles between entries): r1 = r[prow] (the rows of A1), r2 =
// r[a2rows] (the rows of A2), in the apply precision.
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_split_gather(int n, int m2, const int32_t* __restrict__ prow, const int32_t* __restrict__ a2rows,
               const double* __restrict__ r, int stride, T* __restrict__ r1, T* __restrict__ r2,
               const LsmrState* S) {
    if (S->done) return;
    const int len = n > m2 ? n : m2;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += gridDim.x * kBlock) {
        if (i < n) r1[i] = (T)r[(size_t)prow[i] * stride];
        if (i < m2) r2[i] = (T)r[(size_t)a2rows[i] * stride];
    }
}

// ---- preconditioned CGLS (Algorithm 1) ------------------------------------
// Vectors: (q, r) interleaved in qr, (h, x) in tx (h = the preconditioner's
// output t), z = A^T r in s, p in pv.

// step 1 from x0 = 0: r = b, x = 0; rnorm = ||r||
static __global__ void __launch_bounds__(kBlock)
k_cgls_begin(int m, int n, const double* __restrict__ b, double2* __restrict__ qr, double2* __restrict__ tx,
             LsmrState* S, double* part, unsigned* counter) {
    double acc[1] = {0.0};
    const int len = m > n ? m : n;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += gridDim.x * kBlock) {
        if (i < m) {
            const double v = b[i];
            qr[i] = make_double2(0.0, v);
            acc[0] += v * v;
        }
        if (i < n) tx[i] = make_double2(0.0, 0.0);
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) S->rnorm = sqrt(tot[0]);
}

// step 11: z = A^T r (columns of A = rows of At, r = qr[i].y); the stopping
// test on the current iterate: ratio = ||z|| / (||A|| ||r||)
template <int G>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
k_cgls_z(Csr<double> At, const double2* __restrict__ qr, double* __restrict__ z, LsmrState* S, double* part,
         unsigned* counter) {
    if (S->done) return;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    const double* r = reinterpret_cast<const double*>(qr) + 1;  // r_i at r[2 i]
    double acc[1] = {0.0};
    for (int col = (blockIdx.x * kBlock + threadIdx.x) / G; col < At.rows; col += groups) {
        double sum = 0.0;
        const int e1 = At.ptr[col + 1];
        int e = At.ptr[col] + lane;
        for (; e + 3 * G < e1; e += 4 * G) {
            const int j0 = At.idx[e], j1 = At.idx[e + G], j2 = At.idx[e + 2 * G], j3 = At.idx[e + 3 * G];
            const double a0 = At.val[e], a1 = At.val[e + G], a2 = At.val[e + 2 * G], a3 = At.val[e + 3 * G];
            const double v0 = r[2 * j0], v1 = r[2 * j1], v2 = r[2 * j2], v3 = r[2 * j3];
            sum = fma(a0, v0, sum);
            sum = fma(a1, v1, sum);
            sum = fma(a2, v2, sum);
            sum = fma(a3, v3, sum);
        }
        if (e < e1) {  // the lane's last (< 4) entries, loads first (as in row_dot)
            const bool h1 = e + G < e1, h2 = e + 2 * G < e1;
            const int j0 = At.idx[e];
            const int j1 = h1 ? At.idx[e + G] : j0, j2 = h2 ? At.idx[e + 2 * G] : j0;
            const double a0 = At.val[e];
            const double a1 = h1 ? At.val[e + G] : a0, a2 = h2 ? At.val[e + 2 * G] : a0;
            const double v0 = r[2 * j0], v1 = r[2 * j1], v2 = r[2 * j2];
            sum = fma(a0, v0, sum);
            if (h1) sum = fma(a1, v1, sum);
            if (h2) sum = fma(a2, v2, sum);
        }
        if (G > 1) sum = group_sum<G>(sum, mask);
        if (lane == 0) {
            z[col] = sum;
            acc[0] += sum * sum;
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double zn = sqrt(tot[0]);
        S->arnorm = zn;
        const double ratio = S->rnorm > 0.0 ? zn / (S->anorm * S->rnorm) : 0.0;
        S->ratio = ratio;
        if (ratio < S->atol) {
            S->done = 1;
            S->status = kOk;
        } else if (S->k >= S->maxit) {
            S->done = 1;
            S->status = kErrMaxit;
        }
    }
}

// step 15: p = h + beta p (INIT: step 5, p = h)
template <bool INIT>
__global__ void __launch_bounds__(kBlock)
k_cgls_p(int n, const double2* __restrict__ tx, double* __restrict__ pv, const LsmrState* S) {
    if (S->done) return;
    const double beta = S->zetabar;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock)
        pv[i] = INIT ? tx[i].x : tx[i].x + beta * pv[i];
}

// steps 7-8: q = A p, alpha = rho / <q, q>
template <int G>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
k_cgls_q(Csr<double> A, const double* __restrict__ pv, double2* __restrict__ qr, LsmrState* S, double* part,
         unsigned* counter) {
    if (S->done) return;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    double acc[1] = {0.0};
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < A.rows; row += groups) {
        double sum = 0.0;
        row_dot<G>(A, row, lane, pv, sum);
        if (G > 1) sum = group_sum<G>(sum, mask);
        if (lane == 0) {
            qr[row].x = sum;
            acc[0] += sum * sum;
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double qq = tot[0];
        if (!(qq > 0.0) || !isfinite(qq)) {
            S->done = 1;
            S->status = kErrBreakdown;
        } else {
            S->alpha = S->alphabar / qq;
        }
    }
}

// steps 9-10: x += alpha p, r -= alpha q; rnorm = ||r||, k += 1
static __global__ void __launch_bounds__(kBlock)
k_cgls_xr(int m, int n, const double* __restrict__ pv, double2* __restrict__ qr, double2* __restrict__ tx,
          LsmrState* S, double* part, unsigned* counter) {
    if (S->done) return;
    const double a = S->alpha;
    double acc[1] = {0.0};
    const int len = m > n ? m : n;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += gridDim.x * kBlock) {
        if (i < m) {
            double2 v = qr[i];
            v.y = v.y - a * v.x;
            qr[i] = v;
            acc[0] += v.y * v.y;
        }
        if (i < n) tx[i].y = tx[i].y + a * pv[i];
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        S->rnorm = sqrt(tot[0]);
        S->k += 1;
    }
}

// INIT: h = v^_1, h-bar = 0, x = 0.  Else: h-bar, x, h updates, k += 1.
template <bool INIT>
__global__ void __launch_bounds__(kBlock)
k_lsmr_update(int n, double2* __restrict__ tx, double* __restrict__ h, double* __restrict__ hb,
              LsmrState* S) {
    if (S->done) return;
    const double ia = S->inv_alpha;
    const double chb = S->c_hbar, cx = S->c_x, ch = S->c_h;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const double2 p = tx[i];
        const double vh = p.x * ia;
        if (INIT) {
            h[i] = vh;
            hb[i] = 0.0;
            tx[i] = make_double2(p.x, 0.0);
        } else {
            const double hbi = h[i] - chb * hb[i];
            hb[i] = hbi;
            tx[i] = make_double2(p.x, p.y + cx * hbi);
            h[i] = vh - ch * h[i];
        }
    }
    if (!INIT && blockIdx.x == 0 && threadIdx.x == 0) S->k += 1;
}

// (q, r) = (b, b), totals: beta = ||b||
template <int UNUSED = 0>
__global__ void __launch_bounds__(kBlock)
k_start_b(int m, const double* __restrict__ b, double2* __restrict__ qr, LsmrState* S, double* part,
          unsigned* counter) {
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < m; i += gridDim.x * kBlock) {
        const double v = b[i];
        qr[i] = make_double2(v, v);  // q = beta_1 u_1 = b, r_0 = b
        acc[0] += v * v;
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double beta = sqrt(tot[0]);
        S->beta = beta;
        S->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
        if (!isfinite(tot[0])) {
            S->done = 1;
            S->status = kErrBreakdown;
        }
    }
}

// float64 -> T conversion and back
template <typename TO, typename TI>
__global__ void k_convert(int n, const TI* __restrict__ a, TO* __restrict__ b) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) b[i] = (TO)a[i];
}

// ---------------------------------------------------------------------------
// plain products and the power method for ||A||_2
// ---------------------------------------------------------------------------

// y = A (v * scale) with scale = inv_lambda (1/sqrt(n) at start via v)
template <int G>
__global__ void __launch_bounds__(kBlock)
k_power_av(Csr<double> A, const double* __restrict__ v, double* __restrict__ y, const PowerState* P) {
    const double sc = P->inv_lambda;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < A.rows; row += groups) {
        double s = 0.0;
        row_dot<G>(A, row, lane, v, s);
        s = group_sum<G>(s, mask);
        if (lane == 0) y[row] = s * sc;
    }
}
// w = A^T y; lambda = ||w||
template <int G>
__global__ void __launch_bounds__(kBlock)
k_power_atv(Csr<double> At, const double* __restrict__ y, double* __restrict__ w, PowerState* P,
            double* part, unsigned* counter, const double2* __restrict__ dense_atv = nullptr) {
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    double acc[1] = {0.0};
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < At.rows; row += groups) {
        double s = 0.0;
        row_dot<G>(At, row, lane, y, s);
        s = group_sum<G>(s, mask);
        if (lane == 0) {
            if (dense_atv) s += dense_atv[row].x;
            w[row] = s;
            acc[0] += s * s;
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double lam = sqrt(tot[0]);
        P->lambda = lam;
        P->inv_lambda = lam > 0.0 ? 1.0 / lam : 0.0;
    }
}

}  // namespace rlsq
