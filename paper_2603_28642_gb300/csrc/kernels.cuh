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
constexpr int kMaxSlots = 64;        // triangular-solve launches per apply
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
    int32_t k;                // index of the current iterate x_k
    int32_t maxit;
    int32_t done;
    int32_t status;
    int32_t apply_count;      // number of finished preconditioner applications (flag epochs)
    int32_t error;            // device-side error word (wait timeout)
    int32_t pad[2];
};

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
    if constexpr (G == 32) {
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
template <int NV>
__device__ bool last_block_total(double (&v)[NV], double* part, unsigned* counter,
                                 double (&tot)[NV]) {
    block_sum<NV>(v);
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) part[(size_t)blockIdx.x * NV + i] = v[i];
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
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

// ---------------------------------------------------------------------------
// CSR views
// ---------------------------------------------------------------------------
template <typename T>
struct Csr {
    int32_t rows, cols;
    const int32_t* ptr;
    const int32_t* idx;
    const T* val;
};

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
template <int G, typename TV, typename TX, typename TA>
__device__ __forceinline__ void row_dot(const Csr<TV>& a, int row, int lane, const TX* x, TA& s) {
    const int e1 = a.ptr[row + 1];
    for (int e = a.ptr[row] + lane; e < e1; e += G) s += (TA)a.val[e] * (TA)x[a.idx[e]];
}

// ---------------------------------------------------------------------------
// LSMR products with A (float64)
// ---------------------------------------------------------------------------

// q <- A (t * inv_alpha) - alpha * (q * inv_beta)   [u_{k+1} beta_{k+2}]
// r <- b - A x                                        [r_k]
// totals: beta = ||q||, rnorm = ||r||
template <int G>
__global__ void __launch_bounds__(kBlock)
k_spmv_lsmr(Csr<double> A, const double* __restrict__ t, const double* __restrict__ x,
            double* __restrict__ q, const double* __restrict__ b, double* __restrict__ r,
            LsmrState* S, double* part, unsigned* counter) {
    if (S->done) return;
    const double inv_alpha = S->inv_alpha, alpha = S->alpha, inv_beta = S->inv_beta;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    double acc[2] = {0.0, 0.0};
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < A.rows; row += groups) {
        double s1 = 0.0, s2 = 0.0;
        row_dot2<G>(A, row, lane, t, x, s1, s2);
        s1 = group_sum<G>(s1, mask);
        s2 = group_sum<G>(s2, mask);
        if (lane == 0) {
            const double qn = s1 * inv_alpha - alpha * (q[row] * inv_beta);
            const double rr = b[row] - s2;
            q[row] = qn;
            r[row] = rr;
            acc[0] += qn * qn;
            acc[1] += rr * rr;
        }
    }
    double tot[2];
    if (last_block_total<2>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double beta = sqrt(tot[0]);
        S->beta = beta;
        S->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
        S->rnorm = sqrt(tot[1]);
    }
}

// s <- A^T q * inv_beta - beta * (s * inv_alpha)      [s of the next apply]
// z  = A^T r                                            [only its norm]
// totals: arnorm = ||z||; ratio check on x_k; FIRST: s = A^T q * inv_beta.
template <int G, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_spmvt_lsmr(Csr<double> At, const double* __restrict__ q, const double* __restrict__ r,
             double* __restrict__ s, LsmrState* S, double* part, unsigned* counter) {
    if (S->done) return;
    const double inv_alpha = S->inv_alpha, beta = S->beta, inv_beta = S->inv_beta;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    double acc[1] = {0.0};
    for (int col = (blockIdx.x * kBlock + threadIdx.x) / G; col < At.rows; col += groups) {
        double s1 = 0.0, s2 = 0.0;
        if (FIRST) {
            row_dot<G>(At, col, lane, q, s1);
        } else {
            row_dot2<G>(At, col, lane, q, r, s1, s2);
        }
        s1 = group_sum<G>(s1, mask);
        if (!FIRST) s2 = group_sum<G>(s2, mask);
        if (lane == 0) {
            s[col] = FIRST ? s1 * inv_beta : s1 * inv_beta - beta * (s[col] * inv_alpha);
            acc[0] += s2 * s2;
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0 && !FIRST) {
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

template <typename T>
struct Tri {
    Csr<T> a;             // strictly triangular part (rows = unknowns)
    const T* diag;        // nullptr: unit diagonal
    const int32_t* order; // rows sorted by (level, id)
};

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

// Sync-free solve.  Blocks take chunks of the level order from a ticket
// counter; every group of G lanes solves one row at a time, waiting on the
// ready flags of the unknowns it reads.  A dependency always sits earlier
// in the level order, hence in a chunk taken earlier by a running block (or
// earlier in the same chunk), so every wait ends; the 1 s bound only guards
// against faults.  epoch = 1 + 64 * apply_count + slot.
template <typename T, int G, int K, int ROUNDS>
__global__ void __launch_bounds__(kBlock)
k_trsv_syncfree(Tri<T> tri, Rhs<T> rhs, T* x, int* flags, int slot, unsigned* tickets,
                const LsmrState* S, int* err) {
    if (S->done) return;
    const int epoch = 1 + kMaxSlots * S->apply_count + slot;
    const int n = tri.a.rows;
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
            const int e1 = tri.a.ptr[row + 1];
            for (int e = tri.a.ptr[row] + lane; e < e1; e += G) {
                const int j = tri.a.idx[e];
                if (!wait_flag(&flags[j], epoch, err)) {
                    ok = false;
                    break;
                }
                sum += tri.a.val[e] * ld_l2(&x[j]);
            }
            sum = group_sum<G>(sum, mask);
            ok = __all_sync(mask, ok);
            if (lane == 0) {
                T v = rhs_at<T, K>(rhs, row) - sum;
                if (tri.diag) v = v / tri.diag[row];
                if (!ok) v = (T)NAN;
                x[row] = v;
                st_release(&flags[row], epoch);
            }
        }
    }
}

// Level-scheduled solve: one launch per level, rows order[lo..hi).
template <typename T, int G, int K>
__global__ void __launch_bounds__(kBlock)
k_trsv_level(Tri<T> tri, Rhs<T> rhs, T* x, int lo, int hi, const LsmrState* S) {
    if (S->done) return;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    for (int tpos = lo + (blockIdx.x * kBlock + threadIdx.x) / G; tpos < hi; tpos += groups) {
        const int row = tri.order[tpos];
        T sum = (T)0;
        row_dot<G>(tri.a, row, lane, x, sum);
        sum = group_sum<G>(sum, mask);
        if (lane == 0) {
            T v = rhs_at<T, K>(rhs, row) - sum;
            if (tri.diag) v = v / tri.diag[row];
            x[row] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// correction pieces (precision T)
// ---------------------------------------------------------------------------

// y = M x for a CSR matrix (no state check when S == nullptr)
template <typename T, int G>
__global__ void __launch_bounds__(kBlock)
k_csr_mv(Csr<T> M, const T* __restrict__ x, T* __restrict__ y, const LsmrState* S) {
    if (S && S->done) return;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < M.rows; row += groups) {
        T s = (T)0;
        row_dot<G>(M, row, lane, x, s);
        s = group_sum<G>(s, mask);
        if (lane == 0) y[row] = s;
    }
}

// e = L2 q1, CG start: r = e (and p = e implied), rr = <e, e>
template <typename T, int G>
__global__ void __launch_bounds__(kBlock)
k_l2_start(Csr<T> L2, const T* __restrict__ q1, T* __restrict__ r, LsmrState* S, double* part,
           unsigned* counter) {
    if (S->done) return;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    double acc[1] = {0.0};
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < L2.rows; row += groups) {
        T s = (T)0;
        row_dot<G>(L2, row, lane, q1, s);
        s = group_sum<G>(s, mask);
        if (lane == 0) {
            r[row] = s;
            acc[0] += (double)(s * s);
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        S->cg_rr = tot[0];
        S->cg_beta = 0.0;
    }
}

// c1 = L2^T p' with p' = r (first step) or r + beta p
template <typename T, int G, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_l2t_cg(Csr<T> L2t, const T* __restrict__ r, const T* __restrict__ p, T* __restrict__ c1,
         const LsmrState* S) {
    if (S->done) return;
    const T beta = (T)S->cg_beta;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < L2t.rows; row += groups) {
        T s = (T)0;
        const int e1 = L2t.ptr[row + 1];
        for (int e = L2t.ptr[row] + lane; e < e1; e += G) {
            const int j = L2t.idx[e];
            const T pj = FIRST ? r[j] : r[j] + beta * p[j];
            s += L2t.val[e] * pj;
        }
        s = group_sum<G>(s, mask);
        if (lane == 0) c1[row] = s;
    }
}

// p <- r (+ beta p); Sp = p + L2 c3; totals: a = rr / <p, Sp>
template <typename T, int G, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_l2_sp(Csr<T> L2, const T* __restrict__ c3, const T* __restrict__ r, T* __restrict__ p,
        T* __restrict__ sp, LsmrState* S, double* part, unsigned* counter) {
    if (S->done) return;
    const T beta = (T)S->cg_beta;
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    double acc[1] = {0.0};
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < L2.rows; row += groups) {
        T s = (T)0;
        row_dot<G>(L2, row, lane, c3, s);
        s = group_sum<G>(s, mask);
        if (lane == 0) {
            const T pv = FIRST ? r[row] : r[row] + beta * p[row];
            const T spv = pv + s;
            p[row] = pv;
            sp[row] = spv;
            acc[0] += (double)(pv * spv);
        }
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double rr = S->cg_rr;
        S->cg_a = (rr != 0.0 && tot[0] != 0.0) ? rr / tot[0] : 0.0;
    }
}

// w += a p (FIRST: w = a p); r -= a Sp; totals: beta = rr' / rr
template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_cg_update(int m2, const T* __restrict__ p, const T* __restrict__ sp, T* __restrict__ r,
            T* __restrict__ w, LsmrState* S, double* part, unsigned* counter) {
    if (S->done) return;
    const T a = (T)S->cg_a;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < m2; i += gridDim.x * kBlock) {
        const T pi = p[i];
        w[i] = FIRST ? a * pi : w[i] + a * pi;
        const T ri = r[i] - a * sp[i];
        r[i] = ri;
        acc[0] += (double)(ri * ri);
    }
    double tot[1];
    if (last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0) {
        const double rr = S->cg_rr;
        S->cg_beta = rr != 0.0 ? tot[0] / rr : 0.0;
        S->cg_rr = tot[0];
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

// t = d * g5 (IDENT: t = s, the unpreconditioned case), <t, s>; INIT: start the recurrences, else one LSMR
// rotation step; either way the apply counter advances.
template <typename T, bool INIT, bool IDENT = false>
__global__ void __launch_bounds__(kBlock)
k_finish_apply(int n, const T* __restrict__ d, const T* __restrict__ g5, const double* __restrict__ s,
               double* __restrict__ t, LsmrState* S, double* part, unsigned* counter) {
    if (S->done) return;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const double ti = IDENT ? s[i] : (double)(d[i] * g5[i]);
        t[i] = ti;
        acc[0] += ti * s[i];
    }
    double tot[1];
    if (!(last_block_total<1>(acc, part, counter, tot) && threadIdx.x == 0)) return;
    S->apply_count += 1;
    if (S->error != 0) {
        S->done = 1;
        S->status = kErrTimeout;
        return;
    }
    const double ts = tot[0];
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

// INIT: h = v^_1, h-bar = 0, x = 0.  Else: h-bar, x, h updates, k += 1.
template <bool INIT>
__global__ void __launch_bounds__(kBlock)
k_lsmr_update(int n, const double* __restrict__ t, double* __restrict__ h, double* __restrict__ hb,
              double* __restrict__ x, LsmrState* S) {
    if (S->done) return;
    const double ia = S->inv_alpha;
    const double chb = S->c_hbar, cx = S->c_x, ch = S->c_h;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const double vh = t[i] * ia;
        if (INIT) {
            h[i] = vh;
            hb[i] = 0.0;
            x[i] = 0.0;
        } else {
            const double hbi = h[i] - chb * hb[i];
            hb[i] = hbi;
            x[i] = x[i] + cx * hbi;
            h[i] = vh - ch * h[i];
        }
    }
    if (!INIT && blockIdx.x == 0 && threadIdx.x == 0) S->k += 1;
}

// q = b, totals: beta = ||b||
template <int UNUSED = 0>
__global__ void __launch_bounds__(kBlock)
k_start_b(int m, const double* __restrict__ b, double* __restrict__ q, LsmrState* S, double* part,
          unsigned* counter) {
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < m; i += gridDim.x * kBlock) {
        const double v = b[i];
        q[i] = v;
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
struct PowerState {
    double lambda, inv_lambda;
};

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
            double* part, unsigned* counter) {
    const unsigned mask = group_mask<G>();
    const int lane = threadIdx.x & (G - 1);
    const int groups = (gridDim.x * kBlock) / G;
    double acc[1] = {0.0};
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < At.rows; row += groups) {
        double s = 0.0;
        row_dot<G>(At, row, lane, y, s);
        s = group_sum<G>(s, mask);
        if (lane == 0) {
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
