// Batched and served forms of the preconditioned LSMR iteration.
//
// A batch is a table of slots; slot s is described by a BSlot (its matrix A,
// its factors, its vectors, its LSMR state) and a phase word (0 empty, 1
// starting, 2 iterating).  Every kernel here takes the table and works on
// slot blockIdx.y, so one launch advances every slot; a slot whose phase
// differs, or whose solve is done, returns at once.  Inside a slot each kernel
// runs exactly the block grid it would run alone (own_blocks) with the
// slot's own reduction scratch, so a problem's iterates do not depend on the
// other slots: a problem gives the same bits alone and in any mix.
//
// The triangular solves run as one persistent launch per solve for all slots
// (grid barrier per level), or, for more slots than a block has threads, one
// launch per level.  One LSMR iteration for the whole table is captured in one
// CUDA graph and replayed; a server tick that admits requests runs one graph
// in which the new slots start while the others iterate.
//
// rlsq_batch_solve points the slots at the problems' own buffers;
// the server (rlsq_server_*) points them at slot-owned buffers over shared,
// resident matrices and admits requests between iterations (continuous
// batching): new requests join the running ones in the very next launches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <type_traits>
#include <unordered_map>

#include "common.h"

namespace rlsq {
namespace {

// Lanes per row of a slot's products (A, A^T, L2, L2^T) come from its own
// problem's mapping (the heuristic of rlsq_factor, or its autotuner when the
// problem was factored with autotune != 0), so a slot's arithmetic depends on
// its problem only, never on the batch it runs in.  Launch grids are sized
// for the widest mapping (kBG_Max lanes); blocks a slot does not own return.
constexpr int kBG_Max = 32;

// dispatch on a slot's lanes per row (1 .. 32), uniform per block
template <class F>
__device__ __forceinline__ void with_slot_lanes(int g, F&& f) {
    switch (g) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 16: f(std::integral_constant<int, 16>{}); break;
        default: f(std::integral_constant<int, 32>{}); break;
    }
}

enum Cond { C_ALL = 0, C_CORR = 1, C_NOCORR = 2, C_CG = 3, C_E = 4, C_DENSE = 5 };
constexpr int SEL_W = 100;  // "w of the correction": vm[0] for S^ = I, vm[3] otherwise

template <typename T>
struct BSlot {
    int32_t m, n, m2, corr, cg_steps;
    int32_t gA, gAt, gL2, gL2t;  // lanes per row of the A, A^T, L2, L2^T products
    int32_t nlev[4];
    Csr<double> A, At;
    Tri<T> tri[4];
    BinTri<T> bt[4];  // the binned form of each system (kb_trsv_bin)
    const int32_t* lp[4];
    Csr<T> L2, L2t;
    const T* d;
    const T* sinv;
    double2* qr;
    double2* tx;
    double* b;
    double* s;
    double* h;
    double* hb;
    T* vn[6];
    T* vm[4];
    LsmrState* S;
    double* part;
    unsigned* counter;
};

// Blocks a slot may use in one launch.  A constant, so a problem's launch
// shape (and its bits) never depends on the mix; small enough that a launch
// over many slots stays a few waves of blocks (every slot's share of the grid
// is launched even when that slot has less work).
constexpr int kSlotBlocks = 64;

// phase selector of the preconditioner application shared by starting
// (phase 1) and iterating (phase 2) slots in one server tick
constexpr int kPhaseActive = 3;

__device__ __forceinline__ int own_blocks(long long rows, int G, int cap) {
    const long long g = (rows * G + kBlock - 1) / kBlock;
    return (int)max(1LL, min(g, (long long)cap));
}

template <typename T>
__device__ __forceinline__ bool cond_ok(const BSlot<T>& D, int cond) {
    switch (cond) {
        case C_CORR: return D.corr != RLSQ_CORR_NONE;
        case C_NOCORR: return D.corr == RLSQ_CORR_NONE;
        case C_CG: return D.corr == RLSQ_CORR_CG;
        case C_E: return D.corr == RLSQ_CORR_SI || D.corr == RLSQ_CORR_DENSE;
        case C_DENSE: return D.corr == RLSQ_CORR_DENSE;
        default: return true;
    }
}

// The slot of this block if it must work, else nullptr (uniform per block).
template <typename T>
__device__ __forceinline__ const BSlot<T>* gate(const BSlot<T>* slots, const int32_t* phase, int want,
                                                int cond) {
    const int ph = phase[blockIdx.y];
    if (want == kPhaseActive ? (ph != 1 && ph != 2) : ph != want) return nullptr;
    const BSlot<T>* D = &slots[blockIdx.y];
    if (D->S->done || !cond_ok(*D, cond)) return nullptr;
    return D;
}

template <typename T>
__device__ __forceinline__ T* vsel(const BSlot<T>& D, int sel) {
    if (sel == SEL_W) return D.corr == RLSQ_CORR_SI ? D.vm[0] : D.vm[3];
    return sel >= 0 ? D.vn[sel] : D.vm[-sel - 1];
}

// ---- kernels (bodies follow the single-problem kernels in kernels.cuh) ------

template <typename T>
__global__ void __launch_bounds__(kBlock) kb_start(const BSlot<T>* slots, const int32_t* phase, int cap) {
    const BSlot<T>* D = gate(slots, phase, 1, C_ALL);
    if (!D) return;
    const int own = own_blocks(D->m, 1, cap);
    if ((int)blockIdx.x >= own) return;
    LsmrState* S = D->S;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < D->m; i += own * kBlock) {
        const double v = D->b[i];
        D->qr[i] = make_double2(v, v);
        acc[0] += v * v;
    }
    double tot[1];
    if (last_block_total_ctx<1>(acc, D->part, D->counter, tot, blockIdx.x, own) && threadIdx.x == 0) {
        const double beta = sqrt(tot[0]);
        S->beta = beta;
        S->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
        if (!isfinite(tot[0])) {
            S->done = 1;
            S->status = kErrBreakdown;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
kb_spmv(const BSlot<T>* slots, const int32_t* phase, int cap) {
    const BSlot<T>* D = gate(slots, phase, 2, C_ALL);
    if (!D) return;
    with_slot_lanes(D->gA, [&](auto gc) {
        constexpr int G = decltype(gc)::value;
        const int own = own_blocks(D->m, G, cap);
        if ((int)blockIdx.x >= own) return;
        LsmrState* S = D->S;
        const double inv_alpha = S->inv_alpha, alpha = S->alpha, inv_beta = S->inv_beta;
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (own * kBlock) / G;
        double acc[2] = {0.0, 0.0};
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < D->m; row += groups) {
            double s1 = 0.0, s2 = 0.0;
            row_dot_pair<G>(D->A, row, lane, D->tx, s1, s2);
            s1 = group_sum<G>(s1, mask);
            s2 = group_sum<G>(s2, mask);
            if (lane == 0) {
                const double2 old = D->qr[row];
                const double qn = s1 * inv_alpha - alpha * (old.x * inv_beta);
                const double rr = D->b[row] - s2;
                D->qr[row] = make_double2(qn, rr);
                acc[0] += qn * qn;
                acc[1] += rr * rr;
            }
        }
        double tot[2];
        if (last_block_total_ctx<2>(acc, D->part, D->counter, tot, blockIdx.x, own) && threadIdx.x == 0) {
            const double beta = sqrt(tot[0]);
            S->beta = beta;
            S->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
            S->rnorm = sqrt(tot[1]);
        }
    });
}

template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
kb_spmvt(const BSlot<T>* slots, const int32_t* phase, int cap) {
    const BSlot<T>* D = gate(slots, phase, FIRST ? 1 : 2, C_ALL);
    if (!D) return;
    with_slot_lanes(D->gAt, [&](auto gc) {
        constexpr int G = decltype(gc)::value;
        const int own = own_blocks(D->n, G, cap);
        if ((int)blockIdx.x >= own) return;
        LsmrState* S = D->S;
        const double inv_alpha = S->inv_alpha, beta = S->beta, inv_beta = S->inv_beta;
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (own * kBlock) / G;
        double acc[1] = {0.0};
        for (int col = (blockIdx.x * kBlock + threadIdx.x) / G; col < D->n; col += groups) {
            double s1 = 0.0, s2 = 0.0;
            row_dot_pair<G>(D->At, col, lane, D->qr, s1, s2);
            s1 = group_sum<G>(s1, mask);
            s2 = group_sum<G>(s2, mask);
            if (lane == 0) {
                D->s[col] = FIRST ? s1 * inv_beta : s1 * inv_beta - beta * (D->s[col] * inv_alpha);
                acc[0] += s2 * s2;
            }
        }
        double tot[1];
        if (last_block_total_ctx<1>(acc, D->part, D->counter, tot, blockIdx.x, own) && threadIdx.x == 0 && !FIRST) {
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
    });
}

// slot s if it takes part (phase, not done, condition), else nullptr
template <typename T>
__device__ __forceinline__ const BSlot<T>* gate_s(const BSlot<T>* slots, const int32_t* phase, int s, int want,
                                                  int cond) {
    const int ph = phase[s];
    if (want == kPhaseActive ? (ph != 1 && ph != 2) : ph != want) return nullptr;
    const BSlot<T>* D = &slots[s];
    if (D->S->done || !cond_ok(*D, cond)) return nullptr;
    return D;
}

// The right-hand side of a slot's solve, selected as in the single-problem apply.
template <typename T, int K>
__device__ __forceinline__ Rhs<T> slot_rhs(const BSlot<T>& D, int ia, int ib) {
    Rhs<T> rhs;
    if (K == RHS_SCALED) {
        rhs.a = D.d;
        rhs.b = nullptr;
        rhs.s = D.s;
    } else {
        rhs.a = D.vn[ia];
        rhs.b = (K == RHS_SUB) ? D.vn[ib] : nullptr;
        rhs.s = nullptr;
    }
    return rhs;
}

// One fused level group of a triangular solve for every slot, one launch per
// group (the path for more than kCoopBlock slots): the slot's blocks (blockIdx.y
// = slot) deal its items of group g; rows are solved exactly as in kb_trsv_bin,
// so the bits do not depend on the schedule or the mix.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock)
kb_trsv_level(const BSlot<T>* slots, const int32_t* phase, int want, int cond, int which, int group, int ia,
              int ib, int io) {
    const BSlot<T>* D = gate(slots, phase, want, cond);
    if (!D) return;
    const BinTri<T> bt = D->bt[which];
    if (group >= bt.ngroups) return;
    const int lane = threadIdx.x & 31;
    const int W = gridDim.x * (kBlock / 32);
    const int gw = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
    const int s0 = __ldg(&bt.gseg[group]), s1 = __ldg(&bt.gseg[group + 1]);
    const int items = __ldg(&bt.gitems[group]);
    const Rhs<T> rhs = slot_rhs<T, K>(*D, ia, ib);
    T* const x = D->vn[io];
    for (int k = gw; k < items; k += W) {
        const BinSeg sg = bt.seg[binned_seg(bt.seg, s0, s1, k)];
        BinLane<T> L;
        binned_prepare<T>(bt, sg, k - sg.item0, lane, L);
        binned_finish<T, K>(bt, rhs, sg, lane, L, x);
    }
}

// The binned solve (see k_trsv_binned) for every slot at once: one persistent
// launch walks the fused level groups 0..ngroups-1; for group g every block
// builds, in shared memory, the prefix over the slots (one per thread) of the
// work items the taking-part slots have in g, and the warps of the grid deal
// the union of those items.  A row's arithmetic is exactly the single-problem
// binned solve's (its own segment, lanes and slot), so the bits do not depend
// on the mix.  A grid barrier separates the groups (bounded waits).  At most
// kCoopBlock slots.
template <typename T, int K>
__global__ void __launch_bounds__(kCoopBlock, 1)
kb_trsv_bin(const BSlot<T>* slots, const int32_t* phase, int nslots, int want, int cond, int which, int ngroups,
            int ia, int ib, int io, unsigned* bar, int* err) {
    __shared__ int pre[kCoopBlock + 1];
    __shared__ int wsum[kCoopBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = gridDim.x * (kCoopBlock / 32);
    const int gw = blockIdx.x + gridDim.x * warp;
    for (int g = 0; g < ngroups; ++g) {
        int w = 0;
        if ((int)threadIdx.x < nslots) {
            const BSlot<T>* D = gate_s(slots, phase, threadIdx.x, want, cond);
            if (D && g < D->bt[which].ngroups) w = D->bt[which].gitems[g];
        }
        // inclusive scan of the item counts over the block (slot = thread)
        int v = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int z = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, z, off);
                if (lane >= off) z += y;
            }
            wsum[lane] = z;
        }
        __syncthreads();
        pre[threadIdx.x + 1] = v + (warp > 0 ? wsum[warp - 1] : 0);
        if (threadIdx.x == 0) pre[0] = 0;
        __syncthreads();
        const int total = pre[nslots];
        for (int k = gw; k < total; k += W) {
            // the last slot s with pre[s] <= k (slots without items have pre[s] == pre[s + 1])
            int lo = 0, hi = nslots;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pre[mid] <= k) lo = mid;
                else hi = mid;
            }
            const BSlot<T>& D = slots[lo];
            const BinTri<T> bt = D.bt[which];
            const int item = k - pre[lo];
            const int sidx = binned_seg(bt.seg, __ldg(&bt.gseg[g]), __ldg(&bt.gseg[g + 1]), item);
            const BinSeg sg = bt.seg[sidx];
            const Rhs<T> rhs = slot_rhs<T, K>(D, ia, ib);
            BinLane<T> L;
            binned_prepare<T>(bt, sg, item - sg.item0, lane, L);
            binned_finish<T, K>(bt, rhs, sg, lane, L, D.vn[io]);
        }
        if (g + 1 < ngroups) {
            grid_arrive(bar);
            grid_wait(bar, (unsigned)(g + 1) * gridDim.x, err);
            if (*(volatile int*)err != 0) return;
        }
    }
}

// y = M x with M = L2 (mat 0, rows m2) or L2^T (mat 1, rows n)
template <typename T>
__global__ void __launch_bounds__(kBlock)
kb_csr_mv(const BSlot<T>* slots, const int32_t* phase, int want, int cond, int mat, int in_sel, int out_sel,
          int cap) {
    const BSlot<T>* D = gate(slots, phase, want, cond);
    if (!D) return;
    const Csr<T>& M = mat == 0 ? D->L2 : D->L2t;
    const int G = mat == 0 ? D->gL2 : D->gL2t;
    const int own = own_blocks(M.rows, G, cap);
    if ((int)blockIdx.x >= own) return;
    const T* x = vsel(*D, in_sel);
    T* y = vsel(*D, out_sel);
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = (G == 32) ? 0xffffffffu : ((1u << G) - 1u) << ((threadIdx.x & 31u) & ~(unsigned)(G - 1));
    const int groups = (own * kBlock) / G;
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < M.rows; row += groups) {
        T s = (T)0;
        for (int e = M.ptr[row] + lane; e < M.ptr[row + 1]; e += G) s += M.val[e] * x[M.idx[e]];
        for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(mask, s, off, G);
        if (lane == 0) y[row] = s;
    }
}

// e = L2 q1 -> r (vm0), rr = <e, e>
template <typename T>
__global__ void __launch_bounds__(kBlock) kb_l2_start(const BSlot<T>* slots, const int32_t* phase, int want, int cap) {
    const BSlot<T>* D = gate(slots, phase, want, C_CG);
    if (!D) return;
    with_slot_lanes(D->gL2, [&](auto gc) {
        constexpr int G = decltype(gc)::value;
        const int own = own_blocks(D->m2, G, cap);
        if ((int)blockIdx.x >= own) return;
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (own * kBlock) / G;
        const T* q1 = D->vn[2];
        T* r = D->vm[0];
        double acc[1] = {0.0};
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < D->m2; row += groups) {
            T s = (T)0;
            row_dot<G>(D->L2, row, lane, q1, s);
            s = group_sum<G>(s, mask);
            if (lane == 0) {
                r[row] = s;
                acc[0] += (double)(s * s);
            }
        }
        double tot[1];
        if (last_block_total_ctx<1>(acc, D->part, D->counter, tot, blockIdx.x, own) && threadIdx.x == 0) {
            D->S->cg_rr = tot[0];
            D->S->cg_beta = 0.0;
        }
    });
}

template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock)
kb_l2t_cg(const BSlot<T>* slots, const int32_t* phase, int want, int it, int cap) {
    const BSlot<T>* D = gate(slots, phase, want, C_CG);
    if (!D || it >= D->cg_steps) return;
    with_slot_lanes(D->gL2t, [&](auto gc) {
        constexpr int G = decltype(gc)::value;
        const int own = own_blocks(D->n, G, cap);
        if ((int)blockIdx.x >= own) return;
        const T beta = (T)D->S->cg_beta;
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (own * kBlock) / G;
        const T* r = D->vm[0];
        const T* p = D->vm[1];
        T* c1 = D->vn[3];
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < D->n; row += groups) {
            T s = (T)0;
            const int e1 = D->L2t.ptr[row + 1];
            for (int e = D->L2t.ptr[row] + lane; e < e1; e += G) {
                const int j = D->L2t.idx[e];
                const T pj = FIRST ? r[j] : r[j] + beta * p[j];
                s += D->L2t.val[e] * pj;
            }
            s = group_sum<G>(s, mask);
            if (lane == 0) c1[row] = s;
        }
    });
}

template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock)
kb_l2_sp(const BSlot<T>* slots, const int32_t* phase, int want, int it, int cap) {
    const BSlot<T>* D = gate(slots, phase, want, C_CG);
    if (!D || it >= D->cg_steps) return;
    with_slot_lanes(D->gL2, [&](auto gc) {
        constexpr int G = decltype(gc)::value;
        const int own = own_blocks(D->m2, G, cap);
        if ((int)blockIdx.x >= own) return;
        LsmrState* S = D->S;
        const T beta = (T)S->cg_beta;
        const unsigned mask = group_mask<G>();
        const int lane = threadIdx.x & (G - 1);
        const int groups = (own * kBlock) / G;
        const T* c3 = D->vn[5];
        const T* r = D->vm[0];
        T* p = D->vm[1];
        T* sp = D->vm[2];
        double acc[1] = {0.0};
        for (int row = (blockIdx.x * kBlock + threadIdx.x) / G; row < D->m2; row += groups) {
            T s = (T)0;
            row_dot<G>(D->L2, row, lane, c3, s);
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
        if (last_block_total_ctx<1>(acc, D->part, D->counter, tot, blockIdx.x, own) && threadIdx.x == 0) {
            const double rr = S->cg_rr;
            S->cg_a = (rr != 0.0 && tot[0] != 0.0) ? rr / tot[0] : 0.0;
        }
    });
}

template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock)
kb_cg_update(const BSlot<T>* slots, const int32_t* phase, int want, int it, int cap) {
    const BSlot<T>* D = gate(slots, phase, want, C_CG);
    if (!D || it >= D->cg_steps) return;
    const int len = D->m2 > D->n ? D->m2 : D->n;
    const int own = own_blocks(len, 1, cap);
    if ((int)blockIdx.x >= own) return;
    LsmrState* S = D->S;
    const T a = (T)S->cg_a;
    const T* p = D->vm[1];
    const T* sp = D->vm[2];
    T* r = D->vm[0];
    // z = sum_j a_j c3_j in vn[0] (as k_cg_update); after the last step vn[0]
    // holds q1 - z, the input of the U solve
    const T* c3 = D->vn[5];
    const T* q1 = D->vn[2];
    T* z = D->vn[0];
    const bool last = it + 1 == D->cg_steps;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += own * kBlock) {
        if (i < D->m2) {
            const T ri = r[i] - a * sp[i];
            r[i] = ri;
            acc[0] += (double)(ri * ri);
        }
        if (i < D->n) {
            const T zi = FIRST ? a * c3[i] : z[i] + a * c3[i];
            z[i] = last ? q1[i] - zi : zi;
        }
    }
    double tot[1];
    if (last_block_total_ctx<1>(acc, D->part, D->counter, tot, blockIdx.x, own) && threadIdx.x == 0) {
        const double rr = S->cg_rr;
        S->cg_beta = rr != 0.0 ? tot[0] / rr : 0.0;
        S->cg_rr = tot[0];
    }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) kb_dense_gemv(const BSlot<T>* slots, const int32_t* phase, int want) {
    const BSlot<T>* D = gate(slots, phase, want, C_DENSE);
    if (!D) return;
    const int m2 = D->m2;
    const T* e = D->vm[0];
    T* w = D->vm[3];
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * kBlock) / 32;
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / 32; row < m2; row += warps) {
        const T* a = D->sinv + (size_t)row * m2;
        T s = (T)0;
        for (int j = lane; j < m2; j += 32) s += a[j] * e[j];
        s = group_sum<32>(s, 0xffffffffu);
        if (lane == 0) w[row] = s;
    }
}

template <typename T, bool INIT>
__global__ void __launch_bounds__(kBlock) kb_finish(const BSlot<T>* slots, const int32_t* phase, int cap) {
    const BSlot<T>* D = gate(slots, phase, INIT ? 1 : 2, C_ALL);
    if (!D) return;
    const int own = own_blocks(D->n, 1, cap);
    if ((int)blockIdx.x >= own) return;
    const T* g5 = D->vn[2];
    double* t = reinterpret_cast<double*>(D->tx);
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < D->n; i += own * kBlock) {
        const double ti = (double)(D->d[i] * g5[i]);
        t[2 * i] = ti;
        acc[0] += ti * D->s[i];
    }
    double tot[1];
    if (last_block_total_ctx<1>(acc, D->part, D->counter, tot, blockIdx.x, own) && threadIdx.x == 0)
        lsmr_scalar_step<INIT>(D->S, tot[0]);
}

template <typename T, bool INIT>
__global__ void __launch_bounds__(kBlock) kb_update(const BSlot<T>* slots, const int32_t* phase, int cap) {
    const BSlot<T>* D = gate(slots, phase, INIT ? 1 : 2, C_ALL);
    if (!D) return;
    const int own = own_blocks(D->n, 1, cap);
    if ((int)blockIdx.x >= own) return;
    LsmrState* S = D->S;
    const double ia = S->inv_alpha;
    const double chb = S->c_hbar, cx = S->c_x, ch = S->c_h;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < D->n; i += own * kBlock) {
        const double2 p = D->tx[i];
        const double vh = p.x * ia;
        if (INIT) {
            D->h[i] = vh;
            D->hb[i] = 0.0;
            D->tx[i] = make_double2(p.x, 0.0);
        } else {
            const double hbi = D->h[i] - chb * D->hb[i];
            D->hb[i] = hbi;
            D->tx[i] = make_double2(p.x, p.y + cx * hbi);
            D->h[i] = vh - ch * D->h[i];
        }
    }
    if (!INIT && blockIdx.x == 0 && threadIdx.x == 0) S->k += 1;
}

// phase 1 -> 2 for the slots that have just been started
__global__ void kb_begin(int nslots, int32_t* phase) {
    const int s = blockIdx.x * kBlock + threadIdx.x;
    if (s < nslots && phase[s] == 1) phase[s] = 2;
}

// needs[s] = 1 while slot s still iterates
template <typename T>
__global__ void kb_collect(const BSlot<T>* slots, const int32_t* phase, int nslots, int32_t* needs) {
    const int s = blockIdx.x * kBlock + threadIdx.x;
    if (s >= nslots) return;
    needs[s] = (phase[s] == 2 && !slots[s].S->done) ? 1 : 0;
}

// ---- host engine -----------------------------------------------------------

template <typename T>
DevFactor<T>& factor_of(rlsq_problem_s* P);
template <>
DevFactor<double>& factor_of<double>(rlsq_problem_s* P) { return P->f64; }
template <>
DevFactor<float>& factor_of<float>(rlsq_problem_s* P) { return P->f32; }

// Buffers of one slot when the slot does not borrow a problem's buffers.
template <typename T>
struct SlotBuffers {
    DevArray<double2> qr, tx;
    DevArray<double> b, s, h, hb, part;
    DevArray<T> vn[6], vm[4];
    DevArray<LsmrState> S;
    DevArray<unsigned> counter;
    int64_t cap_m = 0, cap_n = 0, cap_m2 = 0;
    void ensure(int64_t m, int64_t n, int64_t m2, int max_blocks) {
        if (m <= cap_m && n <= cap_n && m2 <= cap_m2 && S.p) return;
        cap_m = std::max(cap_m, m);
        cap_n = std::max(cap_n, n);
        cap_m2 = std::max<int64_t>(cap_m2, std::max<int64_t>(m2, 1));
        qr.alloc(cap_m);
        tx.alloc(cap_n);
        b.alloc(cap_m);
        for (auto* v : {&s, &h, &hb}) v->alloc(cap_n);
        for (auto& v : vn) v.alloc(cap_n);
        for (auto& v : vm) v.alloc(cap_m2);
        part.alloc(static_cast<size_t>(max_blocks) * 2);
        S.alloc(1);
        counter.alloc(1);
        RLSQ_CUDA(cudaMemset(counter.p, 0, sizeof(unsigned)));
    }
};

// per-slot footprint of the LSMR state (vectors and scratch) in bytes
int64_t state_bytes(int64_t m, int64_t n, int64_t m2, int prec) {
    const int64_t w = prec == RLSQ_PREC_FP32 ? 4 : 8;
    return 16 * m + 16 * n + 8 * m + 24 * n + 6 * w * n + 4 * w * std::max<int64_t>(m2, 1) + 4096;
}

template <typename T>
struct Engine {
    int nslots = 0;
    int cap = 1;
    cudaStream_t st = nullptr;
    std::vector<BSlot<T>> h_slots;
    DevArray<BSlot<T>> d_slots;
    std::vector<int32_t> h_phase;
    DevArray<int32_t> d_phase, d_needs;
    int32_t* pinned_needs = nullptr;  // nslots flags, then the device error word
    DevArray<unsigned> d_bars;        // grid-barrier counters of the persistent solves of one apply
    DevArray<int> d_err;              // set when a bounded device wait gave up
    int bar_next = 0;
    int coop_grid = 0;                // co-resident blocks of kb_trsv_bin (0: level launches only)
    // maxima over everything the graphs must cover
    int maxlev[4] = {0, 0, 0, 0};
    int maxcg = 0;
    int64_t max_m = 0, max_n = 0, max_m2 = 0, max_levw = 0;
    bool any_corr = false, any_none = false, any_cg = false, any_e = false, any_dense = false;
    cudaGraphExec_t g_start = nullptr, g_iter = nullptr, g_tick = nullptr;
    int iter_reps = 0;

    ~Engine() {
        if (g_start) cudaGraphExecDestroy(g_start);
        if (g_iter) cudaGraphExecDestroy(g_iter);
        if (g_tick) cudaGraphExecDestroy(g_tick);
        if (pinned_needs) cudaFreeHost(pinned_needs);
    }

    void init(int slots, int max_blocks, cudaStream_t stream, int num_sms) {
        nslots = slots;
        cap = max_blocks;
        st = stream;
        d_bars.alloc(kMaxSlots);
        d_err.alloc(1);
        RLSQ_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int), st));
        coop_grid = 0;
        if (slots <= kCoopBlock) {
            int occ = 1 << 30;
            auto prep = [&](auto kern) {
                int o = 0;
                RLSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kCoopBlock, 0));
                occ = std::min(occ, o);
            };
            prep(kb_trsv_bin<T, RHS_VEC>);
            prep(kb_trsv_bin<T, RHS_SCALED>);
            prep(kb_trsv_bin<T, RHS_SUB>);
            coop_grid = occ * num_sms;
        }
        h_slots.assign(static_cast<size_t>(slots), BSlot<T>{});
        h_phase.assign(static_cast<size_t>(slots), 0);
        d_slots.alloc(slots);
        d_phase.alloc(slots);
        d_needs.alloc(slots);
        RLSQ_CUDA(cudaMallocHost(reinterpret_cast<void**>(&pinned_needs), sizeof(int32_t) * (slots + 1)));
    }

    // cover a matrix (its levels, sizes, correction) in the captured graphs
    void cover(const rlsq_problem_s* P) {
        // the solves walk the fused levels (the ones uploaded with the factor)
        const IlupResult& F = *P->F;
        const Levels* L[4] = {&F.lev_L1, &F.lev_L1t, &F.lev_U, &F.lev_Ut};
        if (P->merged.size() == 4)
            for (int w = 0; w < 4; ++w) L[w] = &P->merged[w].lev;
        bool grow = false;
        for (int w = 0; w < 4; ++w) {
            if (L[w]->nlevels > maxlev[w]) { maxlev[w] = L[w]->nlevels; grow = true; }
            if (L[w]->max_width > max_levw) { max_levw = L[w]->max_width; grow = true; }
        }
        auto upd = [&](int64_t& a, int64_t b) { if (b > a) { a = b; grow = true; } };
        upd(max_m, P->m);
        upd(max_n, P->n);
        upd(max_m2, P->m - P->n);
        auto flag = [&](bool& f, bool v) { if (v && !f) { f = true; grow = true; } };
        flag(any_corr, P->correction != RLSQ_CORR_NONE);
        flag(any_none, P->correction == RLSQ_CORR_NONE);
        flag(any_cg, P->correction == RLSQ_CORR_CG);
        flag(any_e, P->correction == RLSQ_CORR_SI || P->correction == RLSQ_CORR_DENSE);
        flag(any_dense, P->correction == RLSQ_CORR_DENSE);
        if (P->correction == RLSQ_CORR_CG && P->opts.cg_steps > maxcg) { maxcg = P->opts.cg_steps; grow = true; }
        if (grow) drop_graphs();
    }

    void drop_graphs() {
        if (g_start) cudaGraphExecDestroy(g_start);
        if (g_iter) cudaGraphExecDestroy(g_iter);
        if (g_tick) cudaGraphExecDestroy(g_tick);
        g_start = g_iter = g_tick = nullptr;
    }

    // descriptor of slot s: matrix from P, vectors from P (own == nullptr) or own
    void set_slot(int s, rlsq_problem_s* P, SlotBuffers<T>* own) {
        BSlot<T> D{};
        DevFactor<T>& F = factor_of<T>(P);
        D.m = static_cast<int32_t>(P->m);
        D.n = static_cast<int32_t>(P->n);
        D.m2 = static_cast<int32_t>(P->m - P->n);
        D.corr = P->correction;
        D.cg_steps = P->opts.cg_steps;
        D.gA = P->map.G_A;
        D.gAt = P->map.G_At;
        D.gL2 = P->map.G_L2;
        D.gL2t = P->map.G_L2t;
        for (int w = 0; w < 4; ++w) {
            D.nlev[w] = static_cast<int32_t>(F.level_ptr[w].size()) - 1;
            D.tri[w] = F.tview(w);
            D.bt[w] = F.bview(w);
            D.lp[w] = F.level_ptr_d[w].p;
        }
        D.A = P->dA.view();
        D.At = P->dAt.view();
        D.L2 = F.L2.view();
        D.L2t = F.L2t.view();
        D.d = F.d.p;
        D.sinv = F.sinv.p;
        if (own) {
            D.qr = own->qr.p; D.tx = own->tx.p; D.b = own->b.p; D.s = own->s.p; D.h = own->h.p; D.hb = own->hb.p;
            for (int i = 0; i < 6; ++i) D.vn[i] = own->vn[i].p;
            for (int i = 0; i < 4; ++i) D.vm[i] = own->vm[i].p;
            D.S = own->S.p; D.part = own->part.p; D.counter = own->counter.p;
        } else {
            D.qr = P->qr.p; D.tx = P->tx.p; D.b = P->b.p; D.s = P->s.p; D.h = P->h.p; D.hb = P->hb.p;
            for (int i = 0; i < 6; ++i) D.vn[i] = F.vn[i].p;
            for (int i = 0; i < 4; ++i) D.vm[i] = F.vm[i].p;
            D.S = P->S.p; D.part = P->part.p; D.counter = P->counter.p;
        }
        h_slots[s] = D;
    }

    void push_table() {
        RLSQ_CUDA(cudaMemcpyAsync(d_slots.p, h_slots.data(), sizeof(BSlot<T>) * nslots, cudaMemcpyHostToDevice, st));
        RLSQ_CUDA(cudaMemcpyAsync(d_phase.p, h_phase.data(), sizeof(int32_t) * nslots, cudaMemcpyHostToDevice, st));
    }

    int gx(int64_t rows, int G) const {
        const int64_t g = (rows * G + kBlock - 1) / kBlock;
        return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, cap)));
    }

    void trsv(int want, int cond, int which, int kind, int ia, int ib, int io) {
        if (coop_grid > 0 && maxlev[which] > 0) {
            // one persistent launch for every level of every slot
            if (bar_next >= kMaxSlots) throw ApiError(RLSQ_ERR_ARG, "too many triangular solves in one apply");
            unsigned* bar = d_bars.p + bar_next++;
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(static_cast<unsigned>(coop_grid));
            cfg.blockDim = dim3(kCoopBlock);
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const BSlot<T>* sl = d_slots.p;
            const int32_t* ph = d_phase.p;
            const int nl = maxlev[which];
            if (kind == RHS_SCALED)
                RLSQ_CUDA(cudaLaunchKernelEx(&cfg, kb_trsv_bin<T, RHS_SCALED>, sl, ph, nslots, want, cond, which, nl,
                                             ia, ib, io, bar, d_err.p));
            else if (kind == RHS_SUB)
                RLSQ_CUDA(cudaLaunchKernelEx(&cfg, kb_trsv_bin<T, RHS_SUB>, sl, ph, nslots, want, cond, which, nl, ia,
                                             ib, io, bar, d_err.p));
            else
                RLSQ_CUDA(cudaLaunchKernelEx(&cfg, kb_trsv_bin<T, RHS_VEC>, sl, ph, nslots, want, cond, which, nl, ia,
                                             ib, io, bar, d_err.p));
            return;
        }
        const dim3 grid(static_cast<unsigned>(std::min(gx(max_levw, 1), 64)), static_cast<unsigned>(nslots));
        for (int l = 0; l < maxlev[which]; ++l) {
            if (kind == RHS_SCALED)
                kb_trsv_level<T, RHS_SCALED><<<grid, kBlock, 0, st>>>(d_slots.p, d_phase.p, want, cond, which, l, ia, ib, io);
            else if (kind == RHS_SUB)
                kb_trsv_level<T, RHS_SUB><<<grid, kBlock, 0, st>>>(d_slots.p, d_phase.p, want, cond, which, l, ia, ib, io);
            else
                kb_trsv_level<T, RHS_VEC><<<grid, kBlock, 0, st>>>(d_slots.p, d_phase.p, want, cond, which, l, ia, ib, io);
        }
    }

    // t = M^{-1} s for every slot in phase `want` (same sequence as the single path)
    void apply(int want) {
        const unsigned ns = static_cast<unsigned>(nslots);
        RLSQ_CUDA(cudaMemsetAsync(d_bars.p, 0, sizeof(unsigned) * kMaxSlots, st));
        bar_next = 0;
        trsv(want, C_ALL, 3, RHS_SCALED, 0, 0, 0);  // U^{-T} D s -> vn0
        trsv(want, C_ALL, 1, RHS_VEC, 0, 0, 1);     // L1^{-T} -> vn1
        if (any_corr) {
            trsv(want, C_CORR, 0, RHS_VEC, 1, 0, 2);  // L1^{-1} -> vn2
            if (any_cg) {
                kb_l2_start<T><<<dim3(gx(max_m2, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, cap);
                for (int it = 0; it < maxcg; ++it) {
                    if (it == 0)
                        kb_l2t_cg<T, true><<<dim3(gx(max_n, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, it, cap);
                    else
                        kb_l2t_cg<T, false><<<dim3(gx(max_n, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, it, cap);
                    trsv(want, C_CG, 1, RHS_VEC, 3, 0, 4);
                    trsv(want, C_CG, 0, RHS_VEC, 4, 0, 5);
                    if (it == 0) {
                        kb_l2_sp<T, true><<<dim3(gx(max_m2, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, it, cap);
                        kb_cg_update<T, true><<<dim3(gx(std::max(max_m2, max_n), 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, it, cap);
                    } else {
                        kb_l2_sp<T, false><<<dim3(gx(max_m2, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, it, cap);
                        kb_cg_update<T, false><<<dim3(gx(std::max(max_m2, max_n), 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, it, cap);
                    }
                }
            }
            if (any_e) {
                kb_csr_mv<T><<<dim3(gx(max_m2, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, C_E, 0, 2, -1, cap);
                if (any_dense)
                    kb_dense_gemv<T><<<dim3(gx(max_m2, 32), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want);
            }
            // S^ = I or dense: Algorithm 3's steps 3-4; the CG slots already hold
            // L1^{-1}(g2 - L1^{-T} L2^T w) = q1 - z in vn0 (kb_cg_update)
            if (any_e) {
                kb_csr_mv<T><<<dim3(gx(max_n, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, want, C_E, 1, SEL_W, 3, cap);
                trsv(want, C_E, 1, RHS_VEC, 3, 0, 4);  // L1^{-T} Y^T w -> vn4
                trsv(want, C_E, 0, RHS_SUB, 1, 4, 0);  // L1^{-1}(g2 - .) -> vn0
            }
        }
        if (any_none) trsv(want, C_NOCORR, 0, RHS_VEC, 1, 0, 0);
        trsv(want, C_ALL, 2, RHS_VEC, 0, 0, 2);  // U^{-1} -> vn2
    }

    void enqueue_start() {
        const unsigned ns = static_cast<unsigned>(nslots);
        kb_start<T><<<dim3(gx(max_m, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_spmvt<T, true><<<dim3(gx(max_n, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        apply(1);
        kb_finish<T, true><<<dim3(gx(max_n, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_update<T, true><<<dim3(gx(max_n, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_begin<<<(nslots + kBlock - 1) / kBlock, kBlock, 0, st>>>(nslots, d_phase.p);
    }

    void enqueue_iteration() {
        const unsigned ns = static_cast<unsigned>(nslots);
        kb_spmv<T><<<dim3(gx(max_m, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_spmvt<T, false><<<dim3(gx(max_n, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        apply(2);
        kb_finish<T, false><<<dim3(gx(max_n, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_update<T, false><<<dim3(gx(max_n, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
    }

    // one server tick: newly admitted slots (phase 1) start while the others
    // (phase 2) iterate, sharing one preconditioner application
    void enqueue_tick() {
        const unsigned ns = static_cast<unsigned>(nslots);
        kb_start<T><<<dim3(gx(max_m, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_spmv<T><<<dim3(gx(max_m, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_spmvt<T, true><<<dim3(gx(max_n, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_spmvt<T, false><<<dim3(gx(max_n, kBG_Max), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        apply(kPhaseActive);
        kb_finish<T, true><<<dim3(gx(max_n, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_finish<T, false><<<dim3(gx(max_n, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_update<T, true><<<dim3(gx(max_n, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_update<T, false><<<dim3(gx(max_n, 1), ns), kBlock, 0, st>>>(d_slots.p, d_phase.p, cap);
        kb_begin<<<(nslots + kBlock - 1) / kBlock, kBlock, 0, st>>>(nslots, d_phase.p);
    }

    // start (0), reps iterations (1) or one tick (2)
    cudaGraphExec_t capture(int kind, int reps) {
        RLSQ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            if (kind == 0) enqueue_start();
            else if (kind == 2) enqueue_tick();
            else
                for (int i = 0; i < reps; ++i) enqueue_iteration();
            kb_collect<T><<<(nslots + kBlock - 1) / kBlock, kBlock, 0, st>>>(d_slots.p, d_phase.p, nslots, d_needs.p);
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
        return ex;
    }

    void launch_start() {
        if (!g_start) g_start = capture(0, 0);
        RLSQ_CUDA(cudaGraphLaunch(g_start, st));
    }
    void launch_tick() {
        if (!g_tick) g_tick = capture(2, 1);
        RLSQ_CUDA(cudaGraphLaunch(g_tick, st));
    }
    void launch_iterations(int reps) {
        if (!g_iter || iter_reps != reps) {
            if (g_iter) cudaGraphExecDestroy(g_iter);
            g_iter = capture(1, reps);
            iter_reps = reps;
        }
        RLSQ_CUDA(cudaGraphLaunch(g_iter, st));
    }
    // copies the per-slot "still iterating" flags to the host (after sync)
    void read_needs() {
        RLSQ_CUDA(cudaMemcpyAsync(pinned_needs, d_needs.p, sizeof(int32_t) * nslots, cudaMemcpyDeviceToHost, st));
        RLSQ_CUDA(cudaMemcpyAsync(pinned_needs + nslots, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RLSQ_CUDA(cudaStreamSynchronize(st));
    }
};

LsmrState fresh_state(double anorm, double atol, int maxit) {
    LsmrState s;
    std::memset(&s, 0, sizeof(s));
    s.anorm = anorm;
    s.atol = atol;
    s.maxit = maxit;
    s.rho = s.rhobar = s.cbar = 1.0;
    return s;
}

void fill_info(const rlsq_problem_s* P, const LsmrState& hs, double seconds, rlsq_info* info) {
    std::memset(info, 0, sizeof(*info));
    rlsq_get_info(const_cast<rlsq_problem_s*>(P), info);
    info->status = hs.error ? RLSQ_ERR_DEVICE_TIMEOUT : hs.status;
    info->iterations = hs.k;
    info->ratio = hs.ratio;
    info->rnorm = hs.rnorm;
    info->arnorm = hs.arnorm;
    info->solve_seconds = seconds;
}

template <typename T>
int batch_solve_impl(rlsq_problem const* hs, const double* const* bs, double* const* xs, int count,
                     const rlsq_solve_opts& opts, rlsq_info* infos) {
    const auto t0 = std::chrono::steady_clock::now();
    rlsq_problem_s* P0 = hs[0];
    // one stream for the whole batch: the first problem's
    cudaStream_t st = P0->stream;
    const bool dev = opts.ptr_mode == RLSQ_DEVICE_PTRS;
    cudaStream_t user = static_cast<cudaStream_t>(opts.stream);
    if (dev) {
        RLSQ_CUDA(cudaEventRecord(P0->ev[0], user));
        RLSQ_CUDA(cudaStreamWaitEvent(st, P0->ev[0], 0));
    }
    // finish whatever the problems' own streams still hold
    for (int i = 0; i < count; ++i) RLSQ_CUDA(cudaStreamSynchronize(hs[i]->stream));
    Engine<T> E;
    E.init(count, kSlotBlocks, st, P0->num_sms);
    for (int i = 0; i < count; ++i) {
        rlsq_problem_s* P = hs[i];
        E.cover(P);
        E.set_slot(i, P, nullptr);
        E.h_phase[i] = 1;
        RLSQ_CUDA(cudaMemcpyAsync(P->b.p, bs[i], sizeof(double) * P->m,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        const LsmrState s0 = fresh_state(P->anorm, opts.atol, opts.maxit);
        RLSQ_CUDA(cudaMemcpyAsync(P->S.p, &s0, sizeof(LsmrState), cudaMemcpyHostToDevice, st));
        RLSQ_CUDA(cudaStreamSynchronize(st));  // s0 and b live on this frame / caller memory
    }
    E.push_table();
    E.launch_start();
    const int reps = std::max(1, opts.check_every);
    const int64_t max_launches = static_cast<int64_t>(opts.maxit) / reps + 4;
    for (int64_t l = 0;; ++l) {
        E.launch_iterations(reps);
        E.read_needs();
        if (E.pinned_needs[count] != 0)
            throw ApiError(RLSQ_ERR_DEVICE_TIMEOUT, "a bounded wait of the batched triangular solve gave up");
        bool any = false;
        for (int i = 0; i < count; ++i) any |= E.pinned_needs[i] != 0;
        if (!any) break;
        if (l > max_launches) throw ApiError(RLSQ_ERR_CUDA, "batched solve did not reach a stopping point");
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int first_bad = RLSQ_OK;
    for (int i = 0; i < count; ++i) {
        rlsq_problem_s* P = hs[i];
        copy_half(xs[i], P->tx.p, P->n, 1, dev, P->s.p, st);
        LsmrState h;
        RLSQ_CUDA(cudaMemcpyAsync(&h, P->S.p, sizeof(LsmrState), cudaMemcpyDeviceToHost, st));
        RLSQ_CUDA(cudaStreamSynchronize(st));
        const int status = h.error ? RLSQ_ERR_DEVICE_TIMEOUT : h.status;
        if (infos) fill_info(P, h, secs, &infos[i]);
        if (status != RLSQ_OK && first_bad == RLSQ_OK) first_bad = status;
    }
    if (dev) {
        RLSQ_CUDA(cudaEventRecord(P0->ev[0], st));
        RLSQ_CUDA(cudaStreamWaitEvent(user, P0->ev[0], 0));
    }
    return first_bad;
}

}  // namespace
}  // namespace rlsq

using namespace rlsq;

// ---------------------------------------------------------------------------
// server
// ---------------------------------------------------------------------------
struct rlsq_server_s {
    rlsq_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    std::string error;

    struct Request {
        int64_t ticket;
        int32_t matrix;
        std::vector<double> b;
        std::chrono::steady_clock::time_point submitted;
    };
    struct Result {
        std::vector<double> x;
        rlsq_info info;
        int status;
    };
    std::vector<rlsq_problem_s*> matrices;
    std::deque<Request> queue;
    std::unordered_map<int64_t, Result> results;
    int64_t next_ticket = 1;
    int64_t submitted = 0, completed = 0, ticks = 0, peak_bytes = 0, active = 0;
    double tick_s = 0.0, tick_device_s = 0.0;  // summed over ticks
    std::vector<double> latencies_ms;
    std::chrono::steady_clock::time_point first_submit, last_done;
    bool any_submit = false;
    int precision = -1;

    // device side (worker thread only)
    cudaStream_t st = nullptr;
    int num_sms = 0;
    std::unique_ptr<Engine<double>> e64;
    std::unique_ptr<Engine<float>> e32;
    std::vector<std::unique_ptr<SlotBuffers<double>>> b64;
    std::vector<std::unique_ptr<SlotBuffers<float>>> b32;
    struct SlotInfo {
        bool busy = false;
        Request req;
        int64_t bytes = 0;
    };
    std::vector<SlotInfo> slots;
    int64_t used_bytes = 0;
    bool dirty = true;  // matrices changed: slot buffers / graphs must cover them

    ~rlsq_server_s() {
        {
            std::lock_guard<std::mutex> lock(mu);
            stop = true;
        }
        cv.notify_all();
        if (worker.joinable()) worker.join();
        for (rlsq_problem_s* p : matrices) p->served.fetch_sub(1);
        e64.reset();
        e32.reset();
        b64.clear();
        b32.clear();
        if (st) cudaStreamDestroy(st);
    }

    template <typename T>
    void run_loop(std::unique_ptr<Engine<T>>& E, std::vector<std::unique_ptr<SlotBuffers<T>>>& bufs);
    void loop();
};

template <typename T>
void rlsq_server_s::run_loop(std::unique_ptr<Engine<T>>& E, std::vector<std::unique_ptr<SlotBuffers<T>>>& bufs) {
    const int nslots = opts.max_slots;
    for (;;) {
        std::vector<int> admitted;
        {
            std::unique_lock<std::mutex> lock(mu);
            if (!stop && queue.empty() && active == 0)
                cv.wait_for(lock, std::chrono::milliseconds(50));
            if (stop) return;
            if (dirty) {
                if (active > 0) {
                    // new matrices are covered once the running requests have finished
                } else {
                    if (!E) {
                        E.reset(new Engine<T>());
                        E->init(nslots, kSlotBlocks, st, num_sms);
                        bufs.resize(nslots);
                        slots.assign(nslots, SlotInfo{});
                    }
                    int64_t mm = 0, mn = 0, mm2 = 0;
                    for (rlsq_problem_s* P : matrices) {
                        E->cover(P);
                        mm = std::max(mm, P->m);
                        mn = std::max(mn, P->n);
                        mm2 = std::max(mm2, P->m - P->n);
                    }
                    for (auto& b : bufs) {
                        if (!b) b.reset(new SlotBuffers<T>());
                        b->ensure(mm, mn, mm2, kSlotBlocks);
                    }
                    dirty = false;
                }
            }
            if (!dirty || E) {
                // admission: FIFO, a free slot and room in the HBM budget
                while (!queue.empty() && E && !dirty) {
                    int free_slot = -1;
                    for (int s = 0; s < nslots; ++s)
                        if (!slots[s].busy) { free_slot = s; break; }
                    if (free_slot < 0) break;
                    const Request& rq = queue.front();
                    rlsq_problem_s* P = matrices[rq.matrix];
                    const int64_t need = state_bytes(P->m, P->n, P->m - P->n, precision);
                    if (used_bytes + need > opts.hbm_budget_bytes) break;
                    slots[free_slot].busy = true;
                    slots[free_slot].req = std::move(queue.front());
                    slots[free_slot].bytes = need;
                    queue.pop_front();
                    used_bytes += need;
                    peak_bytes = std::max(peak_bytes, used_bytes);
                    ++active;
                    admitted.push_back(free_slot);
                }
            }
        }
        if (!E) continue;
        const auto tick0 = std::chrono::steady_clock::now();
        if (!admitted.empty()) {
            for (int s : admitted) {
                rlsq_problem_s* P = matrices[slots[s].req.matrix];
                E->set_slot(s, P, bufs[s].get());
                E->h_phase[s] = 1;
                RLSQ_CUDA(cudaMemcpyAsync(bufs[s]->b.p, slots[s].req.b.data(), sizeof(double) * P->m,
                                          cudaMemcpyHostToDevice, st));
                const LsmrState s0 = fresh_state(P->anorm, opts.atol, opts.maxit);
                RLSQ_CUDA(cudaMemcpyAsync(bufs[s]->S.p, &s0, sizeof(LsmrState), cudaMemcpyHostToDevice, st));
                RLSQ_CUDA(cudaStreamSynchronize(st));
            }
            E->push_table();
        }
        bool running = false;
        for (int s = 0; s < nslots; ++s) running |= slots[s].busy;
        if (!running) continue;
        const auto dev0 = std::chrono::steady_clock::now();
        if (!admitted.empty()) {
            E->launch_tick();  // the new slots start, the others iterate
            for (int s : admitted) E->h_phase[s] = 2;
        } else {
            E->launch_iterations(1);
        }
        E->read_needs();
        const auto dev1 = std::chrono::steady_clock::now();
        ++ticks;
        // a bounded device wait gave up: every running request ends with that error
        const bool dev_err = E->pinned_needs[nslots] != 0;
        if (dev_err) RLSQ_CUDA(cudaMemsetAsync(E->d_err.p, 0, sizeof(int), st));
        // finished slots: results out, slot freed
        for (int s = 0; s < nslots; ++s) {
            if (!slots[s].busy || (E->pinned_needs[s] && !dev_err)) continue;
            rlsq_problem_s* P = matrices[slots[s].req.matrix];
            Result res;
            res.x.resize(static_cast<size_t>(P->n));
            copy_half(res.x.data(), bufs[s]->tx.p, P->n, 1, false, bufs[s]->s.p, st);
            LsmrState h;
            RLSQ_CUDA(cudaMemcpyAsync(&h, bufs[s]->S.p, sizeof(LsmrState), cudaMemcpyDeviceToHost, st));
            RLSQ_CUDA(cudaStreamSynchronize(st));
            const auto now = std::chrono::steady_clock::now();
            const double lat = std::chrono::duration<double, std::milli>(now - slots[s].req.submitted).count();
            fill_info(P, h, lat / 1000.0, &res.info);
            res.status = dev_err ? RLSQ_ERR_DEVICE_TIMEOUT : res.info.status;
            E->h_phase[s] = 0;
            {
                std::lock_guard<std::mutex> lock(mu);
                results[slots[s].req.ticket] = std::move(res);
                latencies_ms.push_back(lat);
                ++completed;
                --active;
                used_bytes -= slots[s].bytes;
                last_done = now;
                slots[s].busy = false;
                slots[s].req.b.clear();
            }
        }
        // the phase table changed for freed slots
        RLSQ_CUDA(cudaMemcpyAsync(E->d_phase.p, E->h_phase.data(), sizeof(int32_t) * nslots, cudaMemcpyHostToDevice, st));
        {
            const auto tick1 = std::chrono::steady_clock::now();
            std::lock_guard<std::mutex> lock(mu);
            tick_s += std::chrono::duration<double>(tick1 - tick0).count();
            tick_device_s += std::chrono::duration<double>(dev1 - dev0).count();
        }
    }
}

void rlsq_server_s::loop() {
    try {
        // wait for the first registration: it fixes the device and the precision
        for (;;) {
            std::unique_lock<std::mutex> lock(mu);
            if (stop) return;
            if (precision >= 0) break;
            cv.wait_for(lock, std::chrono::milliseconds(20));
        }
        {
            std::lock_guard<std::mutex> lock(mu);
            RLSQ_CUDA(cudaSetDevice(matrices[0]->device));
        }
        RLSQ_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        int dev = 0;
        RLSQ_CUDA(cudaGetDevice(&dev));
        RLSQ_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        if (precision == RLSQ_PREC_FP32) run_loop<float>(e32, b32);
        else run_loop<double>(e64, b64);
    } catch (const std::exception& e) {
        std::lock_guard<std::mutex> lock(mu);
        error = e.what();
        stop = true;
    }
}

extern "C" {

int rlsq_batch_solve(rlsq_problem const* hs, const double* const* bs, double* const* xs, int32_t count,
                     const rlsq_solve_opts* o, rlsq_info* infos) {
    return guarded([&]() -> int {
        if (!hs || !bs || !xs || count <= 0) throw ApiError(RLSQ_ERR_ARG, "null argument or empty batch");
        if (count > 65535) throw ApiError(RLSQ_ERR_ARG, "at most 65535 problems per batch");
        rlsq_solve_opts opts;
        rlsq_solve_opts_default(&opts);
        if (o) opts = *o;
        const int prec = hs[0] ? hs[0]->precision : 0;
        for (int i = 0; i < count; ++i) {
            if (!hs[i] || !bs[i] || !xs[i]) throw ApiError(RLSQ_ERR_ARG, "null problem, b or x");
            if (!hs[i]->factored) throw ApiError(RLSQ_ERR_NOT_FACTORED, "problem " + std::to_string(i) + " is not factored");
            if (hs[i]->correction == RLSQ_CORR_CG && hs[i]->opts.cg_tol > 0.0)
                throw ApiError(RLSQ_ERR_ARG, "problem " + std::to_string(i) +
                                                 ": adaptive CG steps (cg_tol > 0) are for single-problem solves");
            if (hs[i]->precision != prec) throw ApiError(RLSQ_ERR_ARG, "all problems of a batch need the same precision");
            if (hs[i]->md > 0) throw ApiError(RLSQ_ERR_ARG, "batched solves take problems without dense rows");
            for (int j = 0; j < i; ++j)
                if (hs[j] == hs[i]) throw ApiError(RLSQ_ERR_ARG, "a problem appears twice in the batch");
        }
        if (prec == RLSQ_PREC_FP32) return batch_solve_impl<float>(hs, bs, xs, count, opts, infos);
        return batch_solve_impl<double>(hs, bs, xs, count, opts, infos);
    });
}

int rlsq_server_create(const rlsq_server_opts* o, rlsq_server* out) {
    return guarded([&]() -> int {
        if (!o || !out) throw ApiError(RLSQ_ERR_ARG, "null argument");
        if (o->max_slots < 1 || o->max_slots > 65535 || o->hbm_budget_bytes <= 0 || o->maxit < 0 || !(o->atol >= 0.0))
            throw ApiError(RLSQ_ERR_ARG, "bad server option");
        std::unique_ptr<rlsq_server_s> S(new rlsq_server_s());
        S->opts = *o;
        rlsq_server_s* raw = S.get();
        S->worker = std::thread([raw]() { raw->loop(); });
        *out = S.release();
        return RLSQ_OK;
    });
}

int rlsq_server_register(rlsq_server s, rlsq_problem h, int32_t* matrix_id) {
    return guarded([&]() -> int {
        if (!s || !h || !matrix_id) throw ApiError(RLSQ_ERR_ARG, "null argument");
        if (!h->factored) throw ApiError(RLSQ_ERR_NOT_FACTORED, "register a factored problem");
        if (h->correction == RLSQ_CORR_CG && h->opts.cg_tol > 0.0)
            throw ApiError(RLSQ_ERR_ARG, "adaptive CG steps (cg_tol > 0) are for single-problem solves");
        if (h->md > 0) throw ApiError(RLSQ_ERR_ARG, "served matrices must have no dense rows");
        const int64_t need = state_bytes(h->m, h->n, h->m - h->n, h->precision);
        if (need > s->opts.hbm_budget_bytes) throw ApiError(RLSQ_ERR_ADMISSION, "one request does not fit the budget");
        std::lock_guard<std::mutex> lock(s->mu);
        if (!s->error.empty()) throw ApiError(RLSQ_ERR_CUDA, s->error);
        if (s->precision >= 0 && s->precision != h->precision)
            throw ApiError(RLSQ_ERR_ARG, "all served matrices need the same precision");
        s->precision = h->precision;
        s->matrices.push_back(h);
        h->served.fetch_add(1);
        s->dirty = true;
        *matrix_id = static_cast<int32_t>(s->matrices.size() - 1);
        s->cv.notify_all();
        return RLSQ_OK;
    });
}

int rlsq_server_submit(rlsq_server s, int32_t matrix_id, const double* b, int64_t* ticket) {
    return guarded([&]() -> int {
        if (!s || !b || !ticket) throw ApiError(RLSQ_ERR_ARG, "null argument");
        std::lock_guard<std::mutex> lock(s->mu);
        if (!s->error.empty()) throw ApiError(RLSQ_ERR_CUDA, s->error);
        if (matrix_id < 0 || matrix_id >= static_cast<int32_t>(s->matrices.size()))
            throw ApiError(RLSQ_ERR_NOT_FOUND, "unknown matrix id");
        rlsq_problem_s* P = s->matrices[matrix_id];
        rlsq_server_s::Request r;
        r.ticket = s->next_ticket++;
        r.matrix = matrix_id;
        r.b.assign(b, b + P->m);
        r.submitted = std::chrono::steady_clock::now();
        if (!s->any_submit) {
            s->first_submit = r.submitted;
            s->any_submit = true;
        }
        *ticket = r.ticket;
        s->queue.push_back(std::move(r));
        ++s->submitted;
        s->cv.notify_all();
        return RLSQ_OK;
    });
}

int rlsq_server_poll(rlsq_server s, int64_t ticket, double* x, rlsq_info* info) {
    return guarded([&]() -> int {
        if (!s || !x) throw ApiError(RLSQ_ERR_ARG, "null argument");
        std::lock_guard<std::mutex> lock(s->mu);
        if (!s->error.empty()) throw ApiError(RLSQ_ERR_CUDA, s->error);
        auto it = s->results.find(ticket);
        if (it == s->results.end()) {
            if (ticket >= 1 && ticket < s->next_ticket) return RLSQ_PENDING;
            throw ApiError(RLSQ_ERR_NOT_FOUND, "unknown or already collected ticket");
        }
        std::copy(it->second.x.begin(), it->second.x.end(), x);
        if (info) *info = it->second.info;
        const int status = it->second.status;
        s->results.erase(it);
        return status;
    });
}

int rlsq_server_get_stats(rlsq_server s, rlsq_server_stats* st) {
    return guarded([&]() -> int {
        if (!s || !st) throw ApiError(RLSQ_ERR_ARG, "null argument");
        std::lock_guard<std::mutex> lock(s->mu);
        std::memset(st, 0, sizeof(*st));
        st->submitted = s->submitted;
        st->completed = s->completed;
        st->queued = static_cast<int64_t>(s->queue.size());
        st->active = s->active;
        st->ticks = s->ticks;
        st->peak_bytes = s->peak_bytes;
        st->tick_ms = s->ticks ? 1000.0 * s->tick_s / s->ticks : 0.0;
        st->tick_device_ms = s->ticks ? 1000.0 * s->tick_device_s / s->ticks : 0.0;
        if (!s->latencies_ms.empty()) {
            std::vector<double> l = s->latencies_ms;
            std::sort(l.begin(), l.end());
            auto pct = [&](double q) {
                const size_t i = static_cast<size_t>(std::min<double>(l.size() - 1, std::floor(q * (l.size() - 1) + 0.5)));
                return l[i];
            };
            st->p50_ms = pct(0.50);
            st->p99_ms = pct(0.99);
            double sum = 0;
            for (double v : l) sum += v;
            st->mean_ms = sum / l.size();
            const double span = std::chrono::duration<double>(s->last_done - s->first_submit).count();
            st->solves_per_s = span > 0 ? s->completed / span : 0.0;
        }
        return RLSQ_OK;
    });
}

void rlsq_server_destroy(rlsq_server s) { delete s; }

}  // extern "C"
