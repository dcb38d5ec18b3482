// The dense correction's S^{-1} formed on the device (Sec. 3.2, eq. 3.9,
// Table 2's dense S): S = I + Z^T Z with Z = L1^{-T} L2^T (n x (m - n)),
// its Cholesky factor S = L L^T, and S^{-1} = L^{-T} L^{-1}, kept explicitly
// so that the apply is one dense symmetric GEMV.
//
//   Z      a level-scheduled solve with L1^T for all m - n right-hand sides
//          at once: Z is row-major (row i holds z_i for every column), so a
//          warp updates 32 consecutive columns of a row with coalesced reads
//          of its dependencies' rows; one launch per level of L1^T.
//   S      cuBLAS DSYRK (a plain library GEMM), then the upper triangle
//          mirrored and the identity added.
//   L      left-looking Cholesky, two launches per column: the pivot (one
//          warp), then a warp per row below it.  A pivot that is not
//          positive sets an error word (S must be positive definite; its
//          eigenvalues are >= 1 in exact arithmetic).
//   L^{-1} one thread per column, forward substitution down that column.
//   S^{-1} cuBLAS DGEMM: L^{-T} L^{-1}.
#include <algorithm>
#include <map>
#include <mutex>

#include <cublas_v2.h>

#include "common.h"

namespace rlsq {

namespace {

void check_cublas(cublasStatus_t s, const char* what) {
    if (s != CUBLAS_STATUS_SUCCESS)
        throw ApiError(s == CUBLAS_STATUS_ALLOC_FAILED ? RLSQ_ERR_OOM : RLSQ_ERR_CUDA,
                       std::string("cuBLAS error ") + std::to_string(static_cast<int>(s)) + " in " + what);
}

// one cuBLAS handle per device, made on first use and kept until exit
std::mutex g_blas_mu;
std::map<int, cublasHandle_t> g_blas;

cublasHandle_t blas_handle() {
    int dev = 0;
    RLSQ_CUDA(cudaGetDevice(&dev));
    auto it = g_blas.find(dev);
    if (it != g_blas.end()) return it->second;
    cublasHandle_t h = nullptr;
    check_cublas(cublasCreate(&h), "cublasCreate");
    g_blas[dev] = h;
    return h;
}

// Z[j, c] = L2(c, j): the right-hand sides of the solves (Z zeroed before)
__global__ void k_z_scatter(Csr<double> L2, double* __restrict__ Z, int m2) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < L2.rows; c += gridDim.x * blockDim.x)
        for (int e = L2.ptr[c]; e < L2.ptr[c + 1]; ++e) Z[(size_t)L2.idx[e] * m2 + c] = L2.val[e];
}

// one level of the unit upper solve with L1^T, in place on every column:
// z_i -= sum_k L1t(i, k) z_k for the rows i of positions [lo, hi)
__global__ void __launch_bounds__(256)
k_z_level(Csr<double> L1t, const int32_t* __restrict__ order, int lo, int hi, double* __restrict__ Z, int m2) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int chunks = (m2 + 31) >> 5;
    const long long items = (long long)(hi - lo) * chunks;
    for (long long it = gw; it < items; it += warps) {
        const int t = lo + (int)(it / chunks);
        const int c = (int)(it % chunks) * 32 + lane;
        const int i = order[t];
        if (c >= m2) continue;
        double s = Z[(size_t)i * m2 + c];
        for (int e = L1t.ptr[i]; e < L1t.ptr[i + 1]; ++e) s -= L1t.val[e] * Z[(size_t)L1t.idx[e] * m2 + c];
        Z[(size_t)i * m2 + c] = s;
    }
}

// S (column-major lower triangle from DSYRK) -> full symmetric, plus I
__global__ void k_sym_plus_identity(double* __restrict__ S, int m2) {
    const long long total = (long long)m2 * m2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q / m2), r = (int)(q % m2);  // element (r, c) at S[c * m2 + r]
        if (r < c) S[(size_t)c * m2 + r] = S[(size_t)r * m2 + c];
        else if (r == c) S[(size_t)c * m2 + r] += 1.0;
    }
}

// Pivot of column j of the Cholesky factor, in place (row-major, lower
// triangle): L(j, j) = sqrt(S(j, j) - sum_{k<j} L(j, k)^2); one warp.
__global__ void k_chol_pivot(double* __restrict__ L, int m2, int j, int* err) {
    const int lane = threadIdx.x & 31;
    const double* Lj = L + (size_t)j * m2;
    double d = 0.0;
    for (int k = lane; k < j; k += 32) d += Lj[k] * Lj[k];
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (lane == 0) {
        const double piv = Lj[j] - d;
        if (!(piv > 0.0)) {
            atomicExch(err, 1);
            L[(size_t)j * m2 + j] = 1.0;  // keeps the rest finite; the error is reported
        } else {
            L[(size_t)j * m2 + j] = sqrt(piv);
        }
    }
}

// The rest of column j (after its pivot): L(i, j) = (S(i, j) -
// sum_{k<j} L(i, k) L(j, k)) / L(j, j), i > j; one warp per row.
__global__ void __launch_bounds__(256) k_chol_column(double* __restrict__ L, int m2, int j) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const double* Lj = L + (size_t)j * m2;
    const double ljj = Lj[j];
    for (int i = j + 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m2; i += warps) {
        const double* Li = L + (size_t)i * m2;
        double s = 0.0;
        for (int k = lane; k < j; k += 32) s += Li[k] * Lj[k];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) L[(size_t)i * m2 + j] = (Li[j] - s) / ljj;
    }
}

// Y = L^{-1} (row-major, lower), one thread per column c:
// Y(i, c) = (delta_ic - sum_{k=c}^{i-1} L(i, k) Y(k, c)) / L(i, i)
__global__ void k_lower_inverse(const double* __restrict__ L, double* __restrict__ Y, int m2) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m2) return;
    for (int i = 0; i < c; ++i) Y[(size_t)i * m2 + c] = 0.0;
    for (int i = c; i < m2; ++i) {
        const double* Li = L + (size_t)i * m2;
        double s = (i == c) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) s -= Li[k] * Y[(size_t)k * m2 + c];
        Y[(size_t)i * m2 + c] = s / Li[i];
    }
}

}  // namespace

// S^{-1} of factor F into out (row-major (m - n)^2 float64), on stream st.
// Throws RLSQ_ERR_NUMERIC when S is not positive definite, RLSQ_ERR_OOM when
// Z (n x (m - n) float64) does not fit in 80% of the free device memory.
void device_schur_inverse(const IlupResult& F, DevArray<double>& out, cudaStream_t st, int num_sms) {
    const int64_t n = F.n, m2 = F.m - F.n;
    if (m2 <= 0) {
        out.release();
        return;
    }
    size_t free_b = 0, total_b = 0;
    RLSQ_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double zbytes = 8.0 * static_cast<double>(n) * static_cast<double>(m2);
    if (zbytes + 3.0 * 8.0 * static_cast<double>(m2) * static_cast<double>(m2) > 0.8 * static_cast<double>(free_b))
        throw ApiError(RLSQ_ERR_OOM, "the dense correction's Z (n x (m - n) float64) does not fit on the device");
    const int m2i = static_cast<int>(m2);
    // L1^T and L2 (unfused) and the level order of L1^T
    DevCsr<double> L1t, L2;
    L1t.upload(F.L1t, st);
    L2.upload(F.L2, st);
    DevArray<int32_t> order;
    order.upload(F.lev_L1t.order.data(), F.lev_L1t.order.size(), st);
    DevArray<double> Z, S, Y;
    Z.alloc(static_cast<size_t>(n) * static_cast<size_t>(m2));
    S.alloc(static_cast<size_t>(m2) * static_cast<size_t>(m2));
    Y.alloc(static_cast<size_t>(m2) * static_cast<size_t>(m2));
    out.alloc(static_cast<size_t>(m2) * static_cast<size_t>(m2));
    DevArray<int> err;
    err.alloc(1);
    RLSQ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    RLSQ_CUDA(cudaMemsetAsync(Z.p, 0, sizeof(double) * Z.n, st));
    k_z_scatter<<<std::max(1, std::min(4096, (m2i + 255) / 256)), 256, 0, st>>>(L2.view(), Z.p, m2i);
    const std::vector<int32_t>& lp = F.lev_L1t.level_ptr;
    for (size_t l = 0; l + 1 < lp.size(); ++l) {
        const long long items = static_cast<long long>(lp[l + 1] - lp[l]) * ((m2 + 31) / 32);
        const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>((items + 7) / 8, 32LL * num_sms)));
        k_z_level<<<grid, 256, 0, st>>>(L1t.view(), order.p, lp[l], lp[l + 1], Z.p, m2i);
    }
    RLSQ_CUDA(cudaGetLastError());
    std::lock_guard<std::mutex> lock(g_blas_mu);
    cublasHandle_t h = blas_handle();
    check_cublas(cublasSetStream(h, st), "cublasSetStream");
    const double one = 1.0, zero = 0.0;
    // Z row-major n x m2 is the column-major m2 x n matrix Zc; Z^T Z = Zc Zc^T
    check_cublas(cublasDsyrk(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, m2i, static_cast<int>(n), &one, Z.p, m2i, &zero,
                             S.p, m2i),
                 "cublasDsyrk");
    const long long total = static_cast<long long>(m2) * m2;
    k_sym_plus_identity<<<static_cast<int>(std::min<long long>((total + 255) / 256, 65535)), 256, 0, st>>>(S.p, m2i);
    for (int j = 0; j < m2i; ++j) {
        k_chol_pivot<<<1, 32, 0, st>>>(S.p, m2i, j, err.p);
        const int rows = m2i - j - 1;
        if (rows > 0) {
            const int grid = std::max(1, std::min(8 * num_sms, (rows + 7) / 8));
            k_chol_column<<<grid, 256, 0, st>>>(S.p, m2i, j);
        }
    }
    k_lower_inverse<<<(m2i + 127) / 128, 128, 0, st>>>(S.p, Y.p, m2i);
    // Y row-major is the column-major Yc = Y^T; S^{-1} = Y^T Y = Yc Yc^T
    check_cublas(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, m2i, m2i, m2i, &one, Y.p, m2i, Y.p, m2i, &zero, out.p, m2i),
                 "cublasDgemm");
    RLSQ_CUDA(cudaGetLastError());
    int herr = 0;
    RLSQ_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RLSQ_CUDA(cudaStreamSynchronize(st));
    if (herr) throw ApiError(RLSQ_ERR_NUMERIC, "dense S is not positive definite");
}

}  // namespace rlsq
