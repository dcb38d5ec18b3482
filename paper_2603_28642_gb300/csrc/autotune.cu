// Autotuner for the kernel mappings of one problem: lanes per row (G) of the
// A / A^T products and of the L2 / L2^T products, and (mode 1), for each of
// the four triangular systems, the schedule and its parameters.  Each
// candidate is timed with CUDA events on the problem's stream (median of a
// few runs after a warm-up) on the problem's own matrices; the fastest wins.
// Results are cached on the handle until the next factor.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.h"

namespace rlsq {

namespace {

template <class F>
void with_lanes(int G, F&& f) {
    switch (G) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 16: f(std::integral_constant<int, 16>{}); break;
        default: f(std::integral_constant<int, 32>{}); break;
    }
}

template <class Body>
float time_median(cudaStream_t st, Body&& body, int reps = 5) {
    cudaEvent_t a, b;
    RLSQ_CUDA(cudaEventCreate(&a));
    RLSQ_CUDA(cudaEventCreate(&b));
    body();  // warm-up
    std::vector<float> ts;
    for (int i = 0; i < reps; ++i) {
        RLSQ_CUDA(cudaEventRecord(a, st));
        body();
        RLSQ_CUDA(cudaEventRecord(b, st));
        RLSQ_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        RLSQ_CUDA(cudaEventElapsedTime(&ms, a, b));
        ts.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

int grid_for(const rlsq_problem_s* P, int64_t rows, int G) {
    const int64_t g = (rows * G + kBlock - 1) / kBlock;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, std::max(1, P->num_sms * kGridBlocksPerSm))));
}

// the grid of kernels without a grid-wide reduction (as the apply launches them)
int grid_for_wide(const rlsq_problem_s* P, int64_t rows, int G) {
    const int64_t g = (rows * G + kBlock - 1) / kBlock;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, std::max(1, P->num_sms * 32))));
}

// Best CSR lanes of the L2 (L2T = false) or L2^T product, timed with the
// CG kernels the apply runs (k_l2_start, with its epilogue and reduction,
// for L2; k_l2t_cg for L2^T) on a scratch state; with try_sliced, also the
// sliced layout (when built): *sliced = 1 when it beats the best CSR lanes.
template <typename T, bool L2T>
int best_l2_lanes(rlsq_problem_s* P, const Csr<T>& M, const T* x, T* y, LsmrState* S, bool try_sliced,
                  int* sliced) {
    static const int cands[] = {1, 2, 4, 8, 16, 32};
    auto launch = [&](auto g, int grid) {
        constexpr int GG = decltype(g)::value;
        if (L2T) k_l2t_cg<T, GG, false><<<grid, kBlock, 0, P->stream>>>(M, x, nullptr, y, S, nullptr);
        else k_l2_start<T, GG><<<grid, kBlock, 0, P->stream>>>(M, x, y, S, P->part.p, P->counter.p, nullptr);
    };
    int best = 8;
    float tbest = 1e30f;
    for (int G : cands) {
        const float t = time_median(P->stream, [&]() {
            with_lanes(G, [&](auto g) {
                constexpr int GG = decltype(g)::value;
                launch(g, L2T ? grid_for_wide(P, M.rows, GG) : grid_for(P, M.rows, GG));
            });
            RLSQ_CUDA(cudaGetLastError());
        });
        if (t < tbest) {
            tbest = t;
            best = G;
        }
    }
    if (try_sliced && M.snpos > 0) {
        const float t = time_median(P->stream, [&]() {
            launch(std::integral_constant<int, 0>{}, L2T ? grid_for_wide(P, M.snpos, 1) : grid_for(P, M.snpos, 1));
            RLSQ_CUDA(cudaGetLastError());
        });
        *sliced = t < tbest ? 1 : 0;
    }
    return best;
}

// A scratch LSMR state that no kernel stops on (for timing).
static LsmrState* scratch_state(rlsq_problem_s* P) {
    LsmrState* S = P->S.p + 1;
    LsmrState h;
    std::memset(&h, 0, sizeof(h));
    h.alpha = h.inv_alpha = h.beta = h.inv_beta = 1.0;
    h.anorm = 1.0;
    h.atol = -1.0;  // the stopping test never fires while timing
    h.maxit = 0x7fffffff;
    RLSQ_CUDA(cudaMemcpy(S, &h, sizeof(h), cudaMemcpyHostToDevice));
    return S;
}

}  // namespace

int rlsq_trsv_time(rlsq_problem_s* P, int which, float* ms);

template <typename T>
static void tune_factor(rlsq_problem_s* P, DevFactor<T>& F, bool schedules) {
    const int n = static_cast<int>(P->n);
    // inputs: any finite vectors will do for timing
    std::vector<T> ones(static_cast<size_t>(std::max<int64_t>(P->m, 1)), (T)1);
    RLSQ_CUDA(cudaMemcpyAsync(F.vn[3].p, ones.data(), sizeof(T) * n, cudaMemcpyHostToDevice, P->stream));
    RLSQ_CUDA(cudaMemcpyAsync(F.vm[0].p, ones.data(), sizeof(T) * F.vm[0].n, cudaMemcpyHostToDevice, P->stream));
    RLSQ_CUDA(cudaStreamSynchronize(P->stream));
    if (P->correction != RLSQ_CORR_NONE) {
        const bool try_sl = P->opts.sliced < 0;
        LsmrState* S = scratch_state(P);
        P->map.G_L2 = best_l2_lanes<T, false>(P, F.L2.view(), F.vn[3].p, F.vm[1].p, S, try_sl, &P->map.sl_L2);
        P->map.G_L2t = best_l2_lanes<T, true>(P, F.L2t.view(), F.vm[0].p, F.vn[4].p, S, try_sl, &P->map.sl_L2t);
    }
    if (!schedules) return;
    static const int cands[] = {1, 2, 4, 8, 16, 32};
    const bool log = std::getenv("RLSQ_TUNE_LOG") != nullptr;
    for (int w = 0; w < 4; ++w) {
        int bestG = P->map.G_tri[w], bestS = P->map.sched[w];
        float tbest = 1e30f;
        int bestB = P->map.sf_blocks[w], bestK = P->map.wave_kp[w], bestR = P->map.sf_rows[w];
        for (int sched : {RLSQ_TRSV_WAVE, RLSQ_TRSV_SYNCFREE, RLSQ_TRSV_LEVEL, RLSQ_TRSV_COOP, RLSQ_TRSV_BINNED}) {
            for (int G : cands) {
                // the persistent and wavefront solves run one thread per row; the
                // binned solve picks lanes per row itself
                if ((sched == RLSQ_TRSV_COOP || sched == RLSQ_TRSV_WAVE || sched == RLSQ_TRSV_BINNED) && G != 1)
                    continue;
                for (int R : {0, 1, 2, 4}) {
                    // R: rows per lane group of the warp-ticketed sync-free solve (0: block tickets)
                    if (R > 0 && (sched != RLSQ_TRSV_SYNCFREE || G > 8)) continue;
                    for (int nb : {1, 2, 3, 4, 6, 8}) {
                        // nb: resident blocks per SM (sync-free) or entries loaded ahead (wavefront: 4, 8)
                        if (sched == RLSQ_TRSV_WAVE ? (nb != 1 && nb != 2) : (sched != RLSQ_TRSV_SYNCFREE && nb != 1))
                            continue;
                        if (sched == RLSQ_TRSV_SYNCFREE && R == 0 && (nb == 4 || nb == 8)) continue;
                        P->map.sched[w] = sched;
                        P->map.G_tri[w] = G;
                        P->map.sf_rows[w] = R;
                        if (sched == RLSQ_TRSV_WAVE) P->map.wave_kp[w] = 4 * nb;
                        else P->map.sf_blocks[w] = nb;
                        float ms = 0.f;
                        if (rlsq_trsv_time(P, w, &ms) != RLSQ_OK) continue;
                        if (log)
                            std::fprintf(stderr, "tune system %d sched %d G %d R %d nb %d: %.4f ms\n", w, sched, G, R,
                                         nb, ms);
                        if (ms < tbest) {
                            tbest = ms;
                            bestG = G;
                            bestS = sched;
                            bestR = R;
                            if (sched == RLSQ_TRSV_WAVE) bestK = 4 * nb;
                            else bestB = nb;
                        }
                    }
                }
            }
        }
        P->map.G_tri[w] = bestG;
        P->map.sched[w] = bestS;
        P->map.sf_blocks[w] = bestB;
        P->map.wave_kp[w] = bestK;
        P->map.sf_rows[w] = bestR;
    }
}

// Lanes per row of the fused LSMR products, timed on a scratch state (the
// kernels write only the work vectors, which a solve re-initialises).
static void tune_products(rlsq_problem_s* P) {
    static const int cands[] = {1, 2, 4, 8, 16, 32};
    LsmrState* S = scratch_state(P);
    RLSQ_CUDA(cudaMemsetAsync(P->tx.p, 0, sizeof(double2) * P->n, P->stream));
    RLSQ_CUDA(cudaMemsetAsync(P->qr.p, 0, sizeof(double2) * P->m, P->stream));
    RLSQ_CUDA(cudaMemsetAsync(P->b.p, 0, sizeof(double) * P->m, P->stream));
    float best_a = 1e30f, best_t = 1e30f;
    for (int G : cands) {
        const float ta = time_median(P->stream, [&]() {
            with_lanes(G, [&](auto g) {
                constexpr int GG = decltype(g)::value;
                k_spmv_lsmr<GG><<<grid_for(P, P->m, GG), kBlock, 0, P->stream>>>(
                    P->dA.view(), P->tx.p, P->qr.p, P->b.p, S, P->part.p, P->counter.p);
            });
            RLSQ_CUDA(cudaGetLastError());
        });
        if (ta < best_a) {
            best_a = ta;
            P->map.G_A = G;
        }
        const float tt = time_median(P->stream, [&]() {
            with_lanes(G, [&](auto g) {
                constexpr int GG = decltype(g)::value;
                k_spmvt_lsmr<GG, false><<<grid_for(P, P->n, GG), kBlock, 0, P->stream>>>(
                    P->dAt.view(), P->qr.p, P->s.p, S, P->part.p, P->counter.p);
            });
            RLSQ_CUDA(cudaGetLastError());
        });
        if (tt < best_t) {
            best_t = tt;
            P->map.G_At = G;
        }
    }
    if (P->opts.sliced >= 0) return;  // the layout was chosen by the caller
    if (P->dA.snpos > 0) {
        const float ta = time_median(P->stream, [&]() {
            k_spmv_lsmr<0><<<grid_for(P, P->dA.snpos, 1), kBlock, 0, P->stream>>>(
                P->dA.view(), P->tx.p, P->qr.p, P->b.p, S, P->part.p, P->counter.p);
            RLSQ_CUDA(cudaGetLastError());
        });
        P->map.sl_A = ta < best_a ? 1 : 0;
    }
    if (P->dAt.snpos > 0) {
        const float tt = time_median(P->stream, [&]() {
            k_spmvt_lsmr<0, false><<<grid_for(P, P->dAt.snpos, 1), kBlock, 0, P->stream>>>(
                P->dAt.view(), P->qr.p, P->s.p, S, P->part.p, P->counter.p);
            RLSQ_CUDA(cudaGetLastError());
        });
        P->map.sl_At = tt < best_t ? 1 : 0;
    }
}

// mode 1: every mapping; mode 2: the lanes of the sparse products only (A,
// A^T, L2, L2^T), which is all the batched and served forms use.
void autotune(rlsq_problem_s* P, int mode) {
    tune_products(P);
    if (!P->factored) return;
    if (P->precision == RLSQ_PREC_FP32) tune_factor<float>(P, P->f32, mode == 1);
    else tune_factor<double>(P, P->f64, mode == 1);
}

}  // namespace rlsq
