// C ABI of the strip solve (include/boxcode.h, bc_strip_*): argument checks,
// the one-warp-per-system kernel for blocks up to 32 x 32, and the
// whole-GPU sequence for larger blocks: block LU of the tridiagonal part by
// blocked LU per element (kernels_strip.cu) with the rank updates as plain
// cuBLAS DGEMMs, back substitution, and the Woodbury correction.
#include <cublas_v2.h>

#include <algorithm>
#include <cstdint>

#include "bc_internal.h"

namespace bc {
namespace {

bool strip_on_device(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

constexpr int kSmallM = 32;     // blocks up to this size: one warp per system
constexpr int kLargeM = 448;    // the panel kernel stages (2m x 32) FP64 in shared memory (227 KB)

bool strip_shape_ok(int64_t nsys, int64_t N, int m, int r)
{
    return nsys >= 0 && nsys <= INT32_MAX && N >= 1 && m >= 1 && m <= kLargeM && r >= 1 && r <= 32 &&
           (m <= kSmallM || N * int64_t(m) <= INT32_MAX / 4);
}

// doubles of scratch: small blocks, per system; large blocks, one system's
// H, G, the augmented block, the capacitance system, pivots and a status word
size_t strip_scratch_doubles(int64_t nsys, int64_t N, int m, int r)
{
    if (m <= kSmallM) return size_t(nsys) * strip_work_doubles(N, m, r);
    const size_t R = size_t(r) + 2 * m, Wc = 2 * size_t(m) + R;
    return strip_work_doubles(N, m, r) + size_t(m) * Wc + size_t(2 * m) * (2 * m + r) + size_t(2 * m) + 2;
}

// Row-major DGEMM: C (rows x cols, ldc) = alpha A (rows x k, lda) B (k x cols, ldb) + beta C
cublasStatus_t gemm_rm(cublasHandle_t h, int rows, int cols, int k, double alpha, const double *A, int lda,
                       const double *B, int ldb, double beta, double *C, int ldc)
{
    return cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, cols, rows, k, &alpha, B, ldb, A, lda, &beta, C, ldc);
}

struct Blas {
    cublasHandle_t h = nullptr;
    int device = -1;
};
thread_local Blas t_blas;

cublasHandle_t blas_for(int device)
{
    if (t_blas.h && t_blas.device == device) return t_blas.h;
    if (t_blas.h) cublasDestroy(t_blas.h);
    t_blas.h = nullptr;
    if (cublasCreate(&t_blas.h) != CUBLAS_STATUS_SUCCESS) return nullptr;
    t_blas.device = device;
    return t_blas.h;
}

// LU with partial pivoting of M[:, 0:n] (row-major, ld), carried to the
// columns [n, c_end), then back substitution on the columns [c_rhs, c_end):
// those columns end as M[:, 0:n]^-1 times their input.
bool lu_solve(cublasHandle_t h, double *M, int n, int ld, int c_rhs, int c_end, int32_t *piv, int32_t *status,
              cudaStream_t st)
{
    const int nb = strip_panel_width();
    for (int j0 = 0; j0 < n; j0 += nb) {
        const int jb = std::min(nb, n - j0), c0 = j0 + jb;
        if (launch_strip_panel(M, n, ld, j0, jb, piv, status, st) != cudaSuccess) return false;
        if (c0 < c_end) {
            if (launch_strip_cols(0, M, ld, j0, jb, piv, c0, c_end, st) != cudaSuccess) return false;
            if (launch_strip_cols(1, M, ld, j0, jb, piv, c0, c_end, st) != cudaSuccess) return false;
            if (c0 < n &&
                gemm_rm(h, n - c0, c_end - c0, jb, -1.0, M + size_t(c0) * ld + j0, ld, M + size_t(j0) * ld + c0, ld,
                        1.0, M + size_t(c0) * ld + c0, ld) != CUBLAS_STATUS_SUCCESS)
                return false;
        }
    }
    const int last = ((n - 1) / nb) * nb;
    for (int j0 = last; j0 >= 0; j0 -= nb) {
        const int jb = std::min(nb, n - j0);
        if (launch_strip_cols(2, M, ld, j0, jb, piv, c_rhs, c_end, st) != cudaSuccess) return false;
        if (j0 > 0 && gemm_rm(h, j0, c_end - c_rhs, jb, -1.0, M + j0, ld, M + size_t(j0) * ld + c_rhs, ld, 1.0,
                              M + c_rhs, ld) != CUBLAS_STATUS_SUCCESS)
            return false;
    }
    return true;
}

// One system with m > 32, on `st`; returns a CUDA/cuBLAS failure as false.
bool solve_large(cublasHandle_t h, int64_t N, int m, int r, const double *A, const double *B, const double *C,
                 const double *b, double *x, double *work, int32_t *status, cudaStream_t st)
{
    const int R = r + 2 * m, Wc = 2 * m + R, n2 = 2 * m, ldk = n2 + r;
    const size_t mm = size_t(m) * m;
    double *H = work, *G = H + size_t(N) * mm, *aug = G + size_t(N) * m * R, *K = aug + size_t(m) * Wc;
    int32_t *piv = reinterpret_cast<int32_t *>(K + size_t(n2) * ldk);
    for (int64_t k = 0; k < N; k++) {
        if (launch_strip_aug(N, m, r, k, A, B, C, b, aug, Wc, st) != cudaSuccess) return false;
        if (k > 0) {
            // D_k = A_k - C_k H_{k-1};  rhs_k -= C_k g_{k-1}
            if (gemm_rm(h, m, m, m, -1.0, C + k * mm, m, H + (k - 1) * mm, m, 1.0, aug, Wc) != CUBLAS_STATUS_SUCCESS ||
                gemm_rm(h, m, R, m, -1.0, C + k * mm, m, G + (k - 1) * size_t(m) * R, R, 1.0, aug + 2 * m, Wc) !=
                    CUBLAS_STATUS_SUCCESS)
                return false;
        }
        if (!lu_solve(h, aug, m, Wc, m, Wc, piv, status, st)) return false;
        if (k < N - 1 && cudaMemcpy2DAsync(H + k * mm, sizeof(double) * m, aug + m, sizeof(double) * Wc,
                                           sizeof(double) * m, m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return false;
        if (cudaMemcpy2DAsync(G + k * size_t(m) * R, sizeof(double) * R, aug + 2 * m, sizeof(double) * Wc,
                              sizeof(double) * R, m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return false;
    }
    // X_k = g_k - H_k X_{k+1}
    for (int64_t k = N - 2; k >= 0; k--)
        if (gemm_rm(h, m, R, m, -1.0, H + k * mm, m, G + (k + 1) * size_t(m) * R, R, 1.0, G + k * size_t(m) * R, R) !=
            CUBLAS_STATUS_SUCCESS)
            return false;
    // Woodbury: w = (I + [Z_{N-1}; Z_0])^-1 [y_{N-1}; y_0];  x = y - Z w
    if (launch_strip_cap(G, N, m, r, R, K, st) != cudaSuccess) return false;
    if (!lu_solve(h, K, n2, ldk, n2, ldk, piv, status, st)) return false;
    if (cudaMemcpy2DAsync(x, sizeof(double) * r, G, sizeof(double) * R, sizeof(double) * r, size_t(N) * m,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return false;
    return gemm_rm(h, int(N * m), r, n2, -1.0, G + r, R, K + n2, ldk, 1.0, x, r) == CUBLAS_STATUS_SUCCESS;
}

}  // namespace
}  // namespace bc

using namespace bc;

bc_status bc_strip_workspace(int64_t nsys, int64_t N, int m, int r, int64_t *bytes)
{
    if (!bytes || !strip_shape_ok(nsys, N, m, r)) {
        set_error("bc_strip_workspace: need nsys >= 0, N >= 1, 1 <= m <= 448, 1 <= r <= 32");
        return BC_ERR_ARG;
    }
    *bytes = int64_t(sizeof(double) * strip_scratch_doubles(nsys, N, m, r));
    return BC_OK;
}

bc_status bc_strip_solve(int64_t nsys, int64_t N, int m, int r, const double *A, const double *B, const double *C,
                         const double *b, double *x, void *work, int32_t *status, void *stream)
{
    if (!strip_shape_ok(nsys, N, m, r)) {
        set_error("bc_strip_solve: need nsys >= 0, N >= 1, 1 <= m <= 448, 1 <= r <= 32");
        return BC_ERR_ARG;
    }
    if (nsys == 0) return BC_OK;
    if (!A || !B || !C || !b || !x || !work) { set_error("bc_strip_solve: NULL argument"); return BC_ERR_ARG; }
    for (const void *p : {(const void *)A, (const void *)B, (const void *)C, (const void *)b, (const void *)x,
                          (const void *)work})
        if (!strip_on_device(p)) { set_error("bc_strip_solve: every array must be device memory"); return BC_ERR_ARG; }
    if (status && !strip_on_device(status)) { set_error("bc_strip_solve: status must be device memory"); return BC_ERR_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m <= kSmallM) {
        const cudaError_t e = launch_strip(nsys, N, m, r, A, B, C, b, x, static_cast<double *>(work), status, st);
        if (e != cudaSuccess) {
            set_error("bc_strip_solve: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
            return BC_ERR_CUDA;
        }
        return BC_OK;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cublasHandle_t h = blas_for(dev);
    if (!h || cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) {
        set_error("bc_strip_solve: cuBLAS handle unavailable");
        return BC_ERR_CUDA;
    }
    double *wk = static_cast<double *>(work);
    const size_t per = strip_work_doubles(N, m, r) + size_t(m) * (2 * size_t(m) + r + 2 * m) +
                       size_t(2 * m) * (2 * m + r);
    int32_t *scratch_status = reinterpret_cast<int32_t *>(wk + per + size_t(2 * m) / 2 + 1);
    const size_t mm = size_t(m) * m;
    for (int64_t s = 0; s < nsys; s++) {
        int32_t *st_s = status ? status + s : scratch_status;
        if (cudaMemsetAsync(st_s, 0, sizeof(int32_t), st) != cudaSuccess ||
            !solve_large(h, N, m, r, A + s * N * mm, B + s * N * mm, C + s * N * mm, b + s * N * m * r,
                         x + s * N * m * r, wk, st_s, st)) {
            const cudaError_t e = cudaGetLastError();
            set_error("bc_strip_solve: %s", e != cudaSuccess ? cudaGetErrorString(e) : "cuBLAS call failed");
            return BC_ERR_CUDA;
        }
    }
    return BC_OK;
}
