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

// large blocks, one system: H and G for the N - 1 blocks of T' (R = r + m),
// the augmented block (2m + R columns) and the border system (m + r columns)
size_t large_work_doubles(int64_t N, int m, int r)
{
    const size_t nt = size_t(std::max<int64_t>(N - 1, 1)), R = size_t(r) + m;
    return nt * (size_t(m) * m + size_t(m) * R) + size_t(m) * (2 * m + R) + size_t(m) * (m + r);
}

// doubles of scratch: small blocks, per system; large blocks, one system's
// arrays, the pivots and a status word
size_t strip_scratch_doubles(int64_t nsys, int64_t N, int m, int r)
{
    if (m <= kSmallM) return size_t(nsys) * strip_work_doubles(N, m, r);
    return large_work_doubles(N, m, r) + size_t(m) + 2;
}

// Row-major DGEMM: C (rows x cols, ldc) = alpha A (rows x k, lda) B (k x cols, ldb) + beta C
cublasStatus_t gemm_rm(cublasHandle_t h, int rows, int cols, int k, double alpha, const double *A, int lda,
                       const double *B, int ldb, double beta, double *C, int ldc)
{
    return cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, cols, rows, k, &alpha, B, ldb, A, lda, &beta, C, ldc);
}

// Per thread and device: a cuBLAS handle with its own workspace (so that its
// calls can be captured into a graph), a private capture stream, and the
// graph of the last large-block solve with its arguments.
struct StripKey {
    const void *p[7] = {};
    int64_t nsys = 0, N = 0;
    int m = 0, r = 0;
    bool operator==(const StripKey &o) const
    {
        for (int i = 0; i < 7; i++)
            if (p[i] != o.p[i]) return false;
        return nsys == o.nsys && N == o.N && m == o.m && r == o.r;
    }
};
constexpr int kMaxPanels = 64;   // panels of one LU: up to 448 rows / 16, with room
struct Blas {
    cublasHandle_t h = nullptr, h2 = nullptr;   // one per capture stream (own workspaces)
    int device = -1;
    void *ws = nullptr, *ws2 = nullptr;
    cudaStream_t cap = nullptr, cap2 = nullptr;
    cudaEvent_t evA[kMaxPanels] = {}, evB[kMaxPanels] = {};
    cudaGraphExec_t exec = nullptr;
    StripKey key;
};
thread_local Blas t_blas;
constexpr size_t kBlasWorkspace = size_t(32) << 20;

Blas *blas_for(int device)
{
    if (t_blas.h && t_blas.device == device) return &t_blas;
    if (t_blas.exec) cudaGraphExecDestroy(t_blas.exec);
    if (t_blas.h) cublasDestroy(t_blas.h);
    if (t_blas.h2) cublasDestroy(t_blas.h2);
    if (t_blas.ws) cudaFree(t_blas.ws);
    if (t_blas.ws2) cudaFree(t_blas.ws2);
    if (t_blas.cap) cudaStreamDestroy(t_blas.cap);
    if (t_blas.cap2) cudaStreamDestroy(t_blas.cap2);
    for (int i = 0; i < kMaxPanels; i++) {
        if (t_blas.evA[i]) cudaEventDestroy(t_blas.evA[i]);
        if (t_blas.evB[i]) cudaEventDestroy(t_blas.evB[i]);
    }
    t_blas = Blas();
    if (cublasCreate(&t_blas.h) != CUBLAS_STATUS_SUCCESS) { t_blas.h = nullptr; return nullptr; }
    if (cublasCreate(&t_blas.h2) != CUBLAS_STATUS_SUCCESS) { t_blas.h2 = nullptr; return nullptr; }
    bool ok = cudaMalloc(&t_blas.ws, kBlasWorkspace) == cudaSuccess &&
              cudaMalloc(&t_blas.ws2, kBlasWorkspace) == cudaSuccess &&
              cublasSetWorkspace(t_blas.h, t_blas.ws, kBlasWorkspace) == CUBLAS_STATUS_SUCCESS &&
              cublasSetWorkspace(t_blas.h2, t_blas.ws2, kBlasWorkspace) == CUBLAS_STATUS_SUCCESS &&
              cudaStreamCreateWithFlags(&t_blas.cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&t_blas.cap2, cudaStreamNonBlocking) == cudaSuccess &&
              strip_prepare(2 * 448) == cudaSuccess;
    for (int i = 0; ok && i < kMaxPanels; i++)
        ok = cudaEventCreateWithFlags(&t_blas.evA[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&t_blas.evB[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return nullptr;
    }
    t_blas.device = device;
    return &t_blas;
}

// LU with partial pivoting of M[:, 0:n] (row-major, ld), carried to the
// columns [n, c_end), then back substitution on the columns [c_rhs, c_end):
// those columns end as M[:, 0:n]^-1 times their input.
// The panels' updates of the columns right of the next panel run on a second
// captured stream (look-ahead): while they run, the first stream updates the
// next panel's columns alone and factors that panel, which is the critical
// path.  A column block gets its row exchanges and updates in panel order:
// the next panel's columns wait for the second stream's previous update.
bool lu_solve(const Blas &bl, double *M, int n, int ld, int c_rhs, int c_end, int32_t *piv, int32_t *status,
              cudaStream_t A)
{
    const int nb = strip_panel_width(), np = (n + nb - 1) / nb;
    cudaStream_t B = bl.cap2;
    if (np > kMaxPanels || cublasSetStream(bl.h2, B) != CUBLAS_STATUS_SUCCESS) return false;
    if (cudaEventRecord(bl.evA[0], A) != cudaSuccess || cudaStreamWaitEvent(B, bl.evA[0], 0) != cudaSuccess)
        return false;
    if (launch_strip_panel(M, n, ld, 0, std::min(nb, n), piv, status, A) != cudaSuccess) return false;
    for (int p = 0; p < np; p++) {
        const int j0 = p * nb, jb = std::min(nb, n - j0), c0 = j0 + jb;
        const int nx1 = c0 < n ? std::min(c0 + nb, n) : c0;   // end of the next panel's columns
        if (cudaEventRecord(bl.evA[p], A) != cudaSuccess) return false;   // panel p factored
        if (c0 < n) {
            if (p > 0 && cudaStreamWaitEvent(A, bl.evB[p - 1], 0) != cudaSuccess) return false;
            if (launch_strip_swap(M, ld, j0, jb, piv, c0, nx1, A) != cudaSuccess ||
                launch_strip_trsm(M, ld, j0, jb, false, c0, nx1, A) != cudaSuccess ||
                gemm_rm(bl.h, n - c0, nx1 - c0, jb, -1.0, M + size_t(c0) * ld + j0, ld, M + size_t(j0) * ld + c0,
                        ld, 1.0, M + size_t(c0) * ld + c0, ld) != CUBLAS_STATUS_SUCCESS ||
                launch_strip_panel(M, n, ld, c0, nx1 - c0, piv, status, A) != cudaSuccess)
                return false;
        }
        if (nx1 < c_end) {
            if (cudaStreamWaitEvent(B, bl.evA[p], 0) != cudaSuccess ||
                launch_strip_swap(M, ld, j0, jb, piv, nx1, c_end, B) != cudaSuccess ||
                launch_strip_trsm(M, ld, j0, jb, false, nx1, c_end, B) != cudaSuccess)
                return false;
            if (c0 < n && gemm_rm(bl.h2, n - c0, c_end - nx1, jb, -1.0, M + size_t(c0) * ld + j0, ld,
                                  M + size_t(j0) * ld + nx1, ld, 1.0, M + size_t(c0) * ld + nx1, ld) !=
                              CUBLAS_STATUS_SUCCESS)
                return false;
        }
        if (cudaEventRecord(bl.evB[p], B) != cudaSuccess) return false;
    }
    if (cudaStreamWaitEvent(A, bl.evB[np - 1], 0) != cudaSuccess) return false;
    const int last = ((n - 1) / nb) * nb;
    for (int j0 = last; j0 >= 0; j0 -= nb) {
        const int jb = std::min(nb, n - j0);
        if (launch_strip_trsm(M, ld, j0, jb, true, c_rhs, c_end, A) != cudaSuccess) return false;
        if (j0 > 0 && gemm_rm(bl.h, j0, c_end - c_rhs, jb, -1.0, M + j0, ld, M + size_t(j0) * ld + c_rhs, ld, 1.0,
                              M + c_rhs, ld) != CUBLAS_STATUS_SUCCESS)
            return false;
    }
    return true;
}

// One system with m > 32, on `st` (the bordered form of the corner
// correction, kernels_strip.cu); returns a CUDA/cuBLAS failure as false.
bool solve_large(const Blas &bl, int64_t N, int m, int r, const double *A, const double *B, const double *C,
                 const double *b, double *x, double *work, int32_t *status, cudaStream_t st)
{
    cublasHandle_t h = bl.h;
    const int R = r + m, Wc = 2 * m + R, ldS = m + r;
    const size_t mm = size_t(m) * m;
    const int64_t Nt = N - 1;   // blocks of T'
    double *H = work, *G = H + size_t(std::max<int64_t>(Nt, 1)) * mm;
    double *aug = G + size_t(std::max<int64_t>(Nt, 1)) * m * R, *S = aug + size_t(m) * Wc;
    int32_t *piv = reinterpret_cast<int32_t *>(S + size_t(m) * ldS);
    for (int64_t k = 0; k < Nt; k++) {
        if (launch_strip_aug(N, m, r, k, A, B, C, b, aug, Wc, st) != cudaSuccess) return false;
        if (k > 0) {
            // D_k = A_k - C_k H_{k-1};  [b_k | E_k] -= C_k [Y_{k-1} | Z_{k-1}]
            if (gemm_rm(h, m, m, m, -1.0, C + k * mm, m, H + (k - 1) * mm, m, 1.0, aug, Wc) != CUBLAS_STATUS_SUCCESS ||
                gemm_rm(h, m, R, m, -1.0, C + k * mm, m, G + (k - 1) * size_t(m) * R, R, 1.0, aug + 2 * m, Wc) !=
                    CUBLAS_STATUS_SUCCESS)
                return false;
        }
        if (!lu_solve(bl, aug, m, Wc, m, Wc, piv, status, st)) return false;
        if (k < Nt - 1 && cudaMemcpy2DAsync(H + k * mm, sizeof(double) * m, aug + m, sizeof(double) * Wc,
                                            sizeof(double) * m, m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return false;
        if (cudaMemcpy2DAsync(G + k * size_t(m) * R, sizeof(double) * R, aug + 2 * m, sizeof(double) * Wc,
                              sizeof(double) * R, m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return false;
    }
    // T'^-1 [b | E]: X_k = g_k - H_k X_{k+1}
    for (int64_t k = Nt - 2; k >= 0; k--)
        if (gemm_rm(h, m, R, m, -1.0, H + k * mm, m, G + (k + 1) * size_t(m) * R, R, 1.0, G + k * size_t(m) * R, R) !=
            CUBLAS_STATUS_SUCCESS)
            return false;
    // border: [S | s] = [A_{N-1} | b_{N-1}] - B_{N-1} [Z_0 | Y_0] - C_{N-1} [Z_{N-2} | Y_{N-2}]
    if (launch_strip_border(N, m, r, A, B, C, b, S, st) != cudaSuccess) return false;
    if (Nt > 0) {
        const double *Bl = B + (N - 1) * mm, *Cl = C + (N - 1) * mm;
        const double *G0 = G, *Gl = G + (Nt - 1) * size_t(m) * R;
        if (gemm_rm(h, m, m, m, -1.0, Bl, m, G0 + r, R, 1.0, S, ldS) != CUBLAS_STATUS_SUCCESS ||
            gemm_rm(h, m, r, m, -1.0, Bl, m, G0, R, 1.0, S + m, ldS) != CUBLAS_STATUS_SUCCESS ||
            gemm_rm(h, m, m, m, -1.0, Cl, m, Gl + r, R, 1.0, S, ldS) != CUBLAS_STATUS_SUCCESS ||
            gemm_rm(h, m, r, m, -1.0, Cl, m, Gl, R, 1.0, S + m, ldS) != CUBLAS_STATUS_SUCCESS)
            return false;
    }
    if (!lu_solve(bl, S, m, ldS, m, ldS, piv, status, st)) return false;
    // x_{N-1} from the border, x_k = Y_k - Z_k x_{N-1}
    if (cudaMemcpy2DAsync(x + size_t(Nt) * m * r, sizeof(double) * r, S + m, sizeof(double) * ldS,
                          sizeof(double) * r, m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return false;
    if (Nt == 0) return true;
    if (cudaMemcpy2DAsync(x, sizeof(double) * r, G, sizeof(double) * R, sizeof(double) * r, size_t(Nt) * m,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return false;
    return gemm_rm(h, int(Nt * m), r, m, -1.0, G + r, R, S + m, ldS, 1.0, x, r) == CUBLAS_STATUS_SUCCESS;
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
    Blas *bl = blas_for(dev);
    if (!bl) {
        set_error("bc_strip_solve: cuBLAS handle unavailable");
        return BC_ERR_CUDA;
    }
    cublasHandle_t h = bl->h;
    // The sequence (some 10^4 launches for the paper's strip) is captured
    // once into a CUDA graph on a private stream and replayed on `stream`
    // while the arguments stay the same.
    StripKey key;
    const void *ptrs[7] = {A, B, C, b, x, work, status};
    for (int i = 0; i < 7; i++) key.p[i] = ptrs[i];
    key.nsys = nsys; key.N = N; key.m = m; key.r = r;
    if (bl->exec && bl->key == key) {
        const cudaError_t e = cudaGraphLaunch(bl->exec, st);
        if (e == cudaSuccess) return BC_OK;
        set_error("bc_strip_solve: %s", cudaGetErrorString(e));
        return BC_ERR_CUDA;
    }
    if (bl->exec) {
        cudaGraphExecDestroy(bl->exec);
        bl->exec = nullptr;
    }
    cudaStream_t cs = bl->cap;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess ||
        cublasSetStream(h, cs) != CUBLAS_STATUS_SUCCESS) {
        set_error("bc_strip_solve: cannot capture");
        return BC_ERR_CUDA;
    }
    double *wk = static_cast<double *>(work);
    int32_t *scratch_status = reinterpret_cast<int32_t *>(wk + large_work_doubles(N, m, r) + size_t(m) / 2 + 1);
    const size_t mm = size_t(m) * m;
    bool ok = true;
    for (int64_t s = 0; s < nsys && ok; s++) {
        int32_t *st_s = status ? status + s : scratch_status;
        ok = cudaMemsetAsync(st_s, 0, sizeof(int32_t), cs) == cudaSuccess &&
             solve_large(*bl, N, m, r, A + s * N * mm, B + s * N * mm, C + s * N * mm, b + s * N * m * r,
                         x + s * N * m * r, wk, st_s, cs);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    cudaError_t e = ok ? ec : cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bl->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess) {
        bl->key = key;
        e = cudaGraphLaunch(bl->exec, st);
    } else {
        bl->exec = nullptr;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("bc_strip_solve: %s", ok ? cudaGetErrorString(e) : "a CUDA or cuBLAS call failed");
        return BC_ERR_CUDA;
    }
    return BC_OK;
}
