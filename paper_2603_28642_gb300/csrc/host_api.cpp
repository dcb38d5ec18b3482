// Host-only entry points of the set-up (rlsq_setup_*): the same code path
// that rlsq_factor runs before uploading, usable without a GPU.
#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "host_setup.h"

#include <algorithm>
#include "rlsq.h"

namespace rlsq {
void set_last_error(const std::string& msg);
}

struct rlsq_setup_s {
    rlsq::IlupResult F;
    rlsq::IlupParams prm;   // the drop rule, reused when rows are added
    rlsq::MergedTri fused;  // the last rlsq_setup_fuse result
    std::vector<double> sinv;  // S^{-1} of the dense correction, once asked for (kept current by row updates)
    std::vector<double> Z;     // Z = L1^{-T} L2^T beside it (empty: row updates form S^{-1} again)
    bool has_sinv = false;
};

namespace {

struct SetupError : std::runtime_error {
    int code;
    SetupError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

template <class F>
int run(F&& f) {
    try {
        rlsq::set_last_error("");
        return f();
    } catch (const SetupError& e) {
        rlsq::set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        rlsq::set_last_error("host allocation failed");
        return RLSQ_ERR_OOM;
    } catch (const std::exception& e) {
        rlsq::set_last_error(e.what());
        return RLSQ_ERR_ARG;
    }
}

}  // namespace

// Validates a host CSR matrix; shared with rlsq_create's checks in spirit but
// kept here so the host API has no CUDA dependency.
static void validate_csr(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v) {
    if (!(m > n && n > 0)) throw SetupError(RLSQ_ERR_SHAPE, "need m > n > 0");
    if (m >= (int64_t(1) << 31)) throw SetupError(RLSQ_ERR_SHAPE, "m must be < 2^31");
    if (rp[0] != 0) throw SetupError(RLSQ_ERR_CSR, "rowptr[0] must be 0");
    for (int64_t i = 0; i < m; ++i)
        if (rp[i + 1] < rp[i]) throw SetupError(RLSQ_ERR_CSR, "rowptr must be nondecreasing");
    if (rp[m] >= (int64_t(1) << 31)) throw SetupError(RLSQ_ERR_SHAPE, "nnz must be < 2^31");
    std::unique_ptr<char[]> seen(new char[static_cast<size_t>(n)]());
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] < 0 || ci[e] >= n) throw SetupError(RLSQ_ERR_CSR, "column index out of range");
            if (e > rp[i] && ci[e] <= ci[e - 1])
                throw SetupError(RLSQ_ERR_CSR, "column indices must be strictly increasing within a row");
            if (!std::isfinite(v[e])) throw SetupError(RLSQ_ERR_CSR, "non-finite value");
            if (v[e] != 0.0) seen[ci[e]] = 1;
        }
    for (int64_t j = 0; j < n; ++j)
        if (!seen[j]) throw SetupError(RLSQ_ERR_RANK, "column " + std::to_string(j) + " is empty");
}

extern "C" {

int rlsq_setup_create(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* vals,
                      const rlsq_factor_opts* opts, rlsq_setup* out) {
    return run([&]() -> int {
        if (!out || !rowptr || !colidx || !vals) throw SetupError(RLSQ_ERR_ARG, "null argument");
        *out = nullptr;
        rlsq_factor_opts o;
        rlsq_factor_opts_default(&o);
        if (opts) o = *opts;
        if (!(o.mu > 0.0 && o.mu <= 1.0) || !(o.tau >= 0.0) || !(o.small > 0.0))
            throw SetupError(RLSQ_ERR_ARG, "bad factor option");
        validate_csr(m, n, rowptr, colidx, vals);
        rlsq::HostCSR A;
        A.rows = m;
        A.cols = n;
        A.ptr.assign(rowptr, rowptr + m + 1);
        A.idx.assign(colidx, colidx + rowptr[m]);
        A.val.assign(vals, vals + rowptr[m]);
        rlsq::IlupParams prm;
        prm.p = o.p;
        prm.tau = o.tau;
        prm.mu = o.mu;
        prm.small = o.small;
        prm.scale = o.scale_columns != 0;
        prm.threads = rlsq::ilup_threads(o.host_threads, m, n);
        std::unique_ptr<rlsq_setup_s> s(new rlsq_setup_s());
        s->prm = prm;
        try {
            s->F = rlsq::ilup_factor(A, prm);
        } catch (const std::runtime_error& e) {
            throw SetupError(RLSQ_ERR_RANK, e.what());
        }
        *out = s.release();
        return RLSQ_OK;
    });
}

int32_t rlsq_setup_threads(int32_t requested, int64_t m, int64_t n) {
    return rlsq::ilup_threads(requested, m, n);
}

int rlsq_setup_sizes(rlsq_setup s, int64_t* sizes) {
    return run([&]() -> int {
        if (!s || !sizes) throw SetupError(RLSQ_ERR_ARG, "null argument");
        const rlsq::IlupResult& F = s->F;
        sizes[0] = F.L1.nnz();
        sizes[1] = F.L2.nnz();
        sizes[2] = F.U.nnz();
        sizes[3] = F.nmod;
        sizes[4] = F.lev_L1.nlevels;
        sizes[5] = F.lev_L1t.nlevels;
        sizes[6] = F.lev_U.nlevels;
        sizes[7] = F.lev_Ut.nlevels;
        return RLSQ_OK;
    });
}

int rlsq_setup_split(rlsq_setup s, int32_t* prow, int32_t* a2rows, double* d, double* udiag) {
    return run([&]() -> int {
        if (!s) throw SetupError(RLSQ_ERR_ARG, "null argument");
        const rlsq::IlupResult& F = s->F;
        if (prow) std::memcpy(prow, F.prow.data(), F.prow.size() * sizeof(int32_t));
        if (a2rows && !F.a2rows.empty()) std::memcpy(a2rows, F.a2rows.data(), F.a2rows.size() * sizeof(int32_t));
        if (d) std::memcpy(d, F.d.data(), F.d.size() * sizeof(double));
        if (udiag) std::memcpy(udiag, F.Udiag.data(), F.Udiag.size() * sizeof(double));
        return RLSQ_OK;
    });
}

int rlsq_setup_factor(rlsq_setup s, int32_t part, int64_t* ptr, int32_t* idx, double* val) {
    return run([&]() -> int {
        if (!s) throw SetupError(RLSQ_ERR_ARG, "null argument");
        const rlsq::HostCSR* c = nullptr;
        if (part == RLSQ_PART_L1) c = &s->F.L1;
        else if (part == RLSQ_PART_L2) c = &s->F.L2;
        else if (part == RLSQ_PART_U) c = &s->F.U;
        else throw SetupError(RLSQ_ERR_ARG, "bad part id");
        if (ptr) std::memcpy(ptr, c->ptr.data(), c->ptr.size() * sizeof(int64_t));
        if (idx && !c->idx.empty()) std::memcpy(idx, c->idx.data(), c->idx.size() * sizeof(int32_t));
        if (val && !c->val.empty()) std::memcpy(val, c->val.data(), c->val.size() * sizeof(double));
        return RLSQ_OK;
    });
}

int rlsq_setup_levels(rlsq_setup s, int32_t which, int32_t* level) {
    return run([&]() -> int {
        if (!s || !level) throw SetupError(RLSQ_ERR_ARG, "null argument");
        const rlsq::IlupResult& F = s->F;
        const rlsq::Levels* L = nullptr;
        switch (which) {
            case RLSQ_SYS_L1: L = &F.lev_L1; break;
            case RLSQ_SYS_L1T: L = &F.lev_L1t; break;
            case RLSQ_SYS_U: L = &F.lev_U; break;
            case RLSQ_SYS_UT: L = &F.lev_Ut; break;
            default: throw SetupError(RLSQ_ERR_ARG, "bad system id");
        }
        std::memcpy(level, L->level.data(), L->level.size() * sizeof(int32_t));
        return RLSQ_OK;
    });
}

int rlsq_setup_fuse(rlsq_setup s, int32_t which, int32_t k, int64_t* out) {
    return run([&]() -> int {
        if (!s || !out) throw SetupError(RLSQ_ERR_ARG, "null argument");
        if (k < 0) throw SetupError(RLSQ_ERR_ARG, "k must be >= 0");
        const rlsq::IlupResult& F = s->F;
        const rlsq::HostCSR* parts[4] = {&F.L1, &F.L1t, &F.U, &F.Ut};
        const rlsq::Levels* levs[4] = {&F.lev_L1, &F.lev_L1t, &F.lev_U, &F.lev_Ut};
        if (which < 0 || which > 3) throw SetupError(RLSQ_ERR_ARG, "bad system id");
        const double* dg = which >= 2 ? F.Udiag.data() : nullptr;
        s->fused = k >= 1 ? rlsq::merge_levels(*parts[which], dg, *levs[which], k)
                          : rlsq::merge_levels_adaptive(*parts[which], dg, *levs[which],
                                                        rlsq::kLevelCost / rlsq::kEntryCost, rlsq::kMaxFusedGroup);
        out[0] = s->fused.T.nnz();
        out[1] = s->fused.R.nnz();
        out[2] = s->fused.lev.nlevels;
        out[3] = s->fused.k;
        return RLSQ_OK;
    });
}

int rlsq_setup_fused(rlsq_setup s, int32_t part, int64_t* ptr, int32_t* idx, double* val) {
    return run([&]() -> int {
        if (!s || !ptr || !idx || !val) throw SetupError(RLSQ_ERR_ARG, "null argument");
        if (part != 0 && part != 1) throw SetupError(RLSQ_ERR_ARG, "part must be 0 (T) or 1 (R)");
        const rlsq::HostCSR& M = part == 0 ? s->fused.T : s->fused.R;
        if (M.ptr.empty()) throw SetupError(RLSQ_ERR_ARG, "no fused system: call rlsq_setup_fuse first");
        std::memcpy(ptr, M.ptr.data(), M.ptr.size() * sizeof(int64_t));
        std::memcpy(idx, M.idx.data(), M.idx.size() * sizeof(int32_t));
        std::memcpy(val, M.val.data(), M.val.size() * sizeof(double));
        return RLSQ_OK;
    });
}

int rlsq_setup_add_rows(rlsq_setup s, int64_t k, const int64_t* rowptr, const int32_t* colidx,
                        const double* vals) {
    return run([&]() -> int {
        if (!s || !rowptr || (k > 0 && (!colidx || !vals))) throw SetupError(RLSQ_ERR_ARG, "null argument");
        if (k < 0) throw SetupError(RLSQ_ERR_ARG, "k must be >= 0");
        if (rowptr[0] != 0) throw SetupError(RLSQ_ERR_CSR, "rowptr[0] must be 0");
        const int64_t n = s->F.n;
        for (int64_t i = 0; i < k; ++i) {
            if (rowptr[i + 1] < rowptr[i]) throw SetupError(RLSQ_ERR_CSR, "rowptr must be nondecreasing");
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                if (colidx[e] < 0 || colidx[e] >= n) throw SetupError(RLSQ_ERR_CSR, "column index out of range");
                if (e > rowptr[i] && colidx[e] <= colidx[e - 1])
                    throw SetupError(RLSQ_ERR_CSR, "column indices must be strictly increasing within a row");
                if (!std::isfinite(vals[e])) throw SetupError(RLSQ_ERR_CSR, "non-finite value");
            }
        }
        if (s->F.m + k >= (int64_t(1) << 31)) throw SetupError(RLSQ_ERR_SHAPE, "m must stay < 2^31");
        rlsq::HostCSR rows;
        rows.rows = k;
        rows.cols = n;
        rows.ptr.assign(rowptr, rowptr + k + 1);
        rows.idx.assign(colidx, colidx + rowptr[k]);
        rows.val.assign(vals, vals + rowptr[k]);
        rlsq::add_rows(s->F, rows, s->prm);
        if (s->has_sinv) {
            try {
                if (s->Z.empty()) throw std::runtime_error("Z is not kept");
                rlsq::schur_inverse_add(s->F, k, s->sinv, s->Z);
            } catch (const std::exception&) {
                s->has_sinv = false;  // formed again when next asked for
            }
        }
        return RLSQ_OK;
    });
}

int rlsq_setup_remove_rows(rlsq_setup s, int64_t k, const int32_t* ids) {
    return run([&]() -> int {
        if (!s || (k > 0 && !ids) || k < 0) throw SetupError(RLSQ_ERR_ARG, "bad argument");
        std::vector<int32_t> v(ids, ids + k);
        const int64_t m2 = s->F.m - s->F.n;
        std::vector<int64_t> pos;
        for (const int32_t r : v) {
            const auto it = std::lower_bound(s->F.a2rows.begin(), s->F.a2rows.end(), r);
            pos.push_back(it - s->F.a2rows.begin());
        }
        try {
            rlsq::remove_rows(s->F, v);
        } catch (const std::invalid_argument& e) {
            throw SetupError(RLSQ_ERR_ARG, e.what());
        } catch (const std::length_error& e) {
            throw SetupError(RLSQ_ERR_SHAPE, e.what());
        }
        if (s->has_sinv) {
            try {
                if (s->Z.empty()) throw std::runtime_error("Z is not kept");
                rlsq::schur_inverse_remove(pos, m2, s->sinv, s->Z);
            } catch (const std::exception&) {
                s->has_sinv = false;
            }
        }
        return RLSQ_OK;
    });
}

int rlsq_setup_schur_inverse(rlsq_setup s, int32_t recompute, double* out) {
    return run([&]() -> int {
        if (!s || !out) throw SetupError(RLSQ_ERR_ARG, "null argument");
        if (recompute || !s->has_sinv) {
            s->has_sinv = false;
            // Z is kept for later row updates while it fits in 2 GiB
            const bool keep = static_cast<double>(s->F.n) * static_cast<double>(s->F.m - s->F.n) * 8.0 <= 2147483648.0;
            s->Z.clear();
            if (!rlsq::dense_schur_inverse(s->F, s->sinv, std::max(1, s->prm.threads), keep ? &s->Z : nullptr))
                throw SetupError(RLSQ_ERR_NUMERIC, "dense S is not positive definite");
            s->has_sinv = true;
        }
        std::copy(s->sinv.begin(), s->sinv.end(), out);
        return RLSQ_OK;
    });
}

void rlsq_setup_destroy(rlsq_setup s) { delete s; }

}  // extern "C"
