// Strip solve (Sec. 3.3): the multidomain collocation system of the strip
// couples each element only to its neighbours around the closed strip, so it
// is block tridiagonal with two corner blocks:
//
//   C[k] x[k-1] + A[k] x[k] + B[k] x[k+1] = b[k],   k = 0..N-1, indices mod N.
//
// Solved as the paper does, by block LU of the tridiagonal part T and the
// Woodbury identity for the corners: M = T + U V^T with U = [E_0 C[0] |
// E_{N-1} B[N-1]] (block rows 0 and N-1) and V^T x = [x[N-1]; x[0]], so
//
//   x = y - Z (I + V^T Z)^-1 V^T y,   y = T^-1 b,  Z = T^-1 U,
//
// where T^-1 is applied to the r columns of b and the 2m columns of U in one
// sweep (R = r + 2m right-hand sides).  The sweep: D_0 = A_0; D_k = A_k -
// C_k H_{k-1}; [H_k | g_k] = D_k^-1 [B_k | rhs_k - C_k g_{k-1}]; then
// X_{N-1} = g_{N-1}, X_k = g_k - H_k X_{k+1}.  Every D_k and the capacitance
// matrix I + V^T Z (2m x 2m) are factored by LU with partial pivoting.
//
// One warp per system (the batched small-dense-LU workload: many strips or
// many right-hand-side sets at once); the blocks of the current step live in
// shared memory, H_k and g_k / X_k in a global workspace.  FP64.
#include <cuda_runtime.h>

#include "bc_internal.h"

namespace bc {
namespace {

// In-place LU solve of M [n x n] (row-major, shared) with the right-hand
// sides S [n x ns] (row-major, leading dimension lds): partial pivoting, the
// warp's lanes over rows and columns.  Returns false (on every lane) if a
// pivot is zero or not finite.
__device__ bool warp_lu_solve(double *M, int n, double *S, int ns, int lds)
{
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int j = 0; j < n; j++) {
        double best = -1.0;
        int bi = j;
        for (int i = j + lane; i < n; i += 32) {
            const double v = fabs(M[i * n + j]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > 0.0) || !isfinite(best)) ok = false;
        if (bi != j) {
            for (int c = lane; c < n; c += 32) {
                const double t = M[j * n + c];
                M[j * n + c] = M[bi * n + c];
                M[bi * n + c] = t;
            }
            for (int c = lane; c < ns; c += 32) {
                const double t = S[j * lds + c];
                S[j * lds + c] = S[bi * lds + c];
                S[bi * lds + c] = t;
            }
        }
        __syncwarp();
        const double inv = ok ? 1.0 / M[j * n + j] : 0.0;
        for (int i = j + 1 + lane; i < n; i += 32) M[i * n + j] *= inv;   // multipliers
        __syncwarp();
        const int w = n - j - 1;
        for (int idx = lane; idx < w * w; idx += 32) {
            const int i = j + 1 + idx / w, c = j + 1 + idx % w;
            M[i * n + c] = fma(-M[i * n + j], M[j * n + c], M[i * n + c]);
        }
        for (int idx = lane; idx < w * ns; idx += 32) {
            const int i = j + 1 + idx / ns, c = idx % ns;
            S[i * lds + c] = fma(-M[i * n + j], S[j * lds + c], S[i * lds + c]);
        }
        __syncwarp();
    }
    // back substitution, the lanes over the right-hand sides
    for (int i = n - 1; i >= 0; i--) {
        const double inv = ok ? 1.0 / M[i * n + i] : 0.0;
        for (int c = lane; c < ns; c += 32) {
            double s = S[i * lds + c];
            for (int t = i + 1; t < n; t++) s = fma(-M[i * n + t], S[t * lds + c], s);
            S[i * lds + c] = s * inv;
        }
        __syncwarp();
    }
    return ok;
}

// out[i][c] (ld lo) -= P [m x m] (ld m) . Q[.][c] (ld lq), c < nc; lanes over (i, c)
__device__ __forceinline__ void warp_sub_mm(double *out, int lo, const double *P, const double *Q, int lq, int m,
                                            int nc)
{
    const int lane = threadIdx.x & 31;
    for (int idx = lane; idx < m * nc; idx += 32) {
        const int i = idx / nc, c = idx % nc;
        double s = out[i * lo + c];
        for (int t = 0; t < m; t++) s = fma(-P[i * m + t], Q[t * lq + c], s);
        out[i * lo + c] = s;
    }
}

__global__ void k_strip_solve(int64_t nsys, int64_t N, int m, int r, const double *__restrict__ A,
                              const double *__restrict__ B, const double *__restrict__ C,
                              const double *__restrict__ b, double *__restrict__ x, double *__restrict__ work,
                              int32_t *__restrict__ status)
{
    extern __shared__ double sh[];
    const int lane = threadIdx.x & 31;
    const int R = r + 2 * m, W = m + R;   // augmented columns: [H | g]
    const int64_t s = blockIdx.x;
    if (s >= nsys) return;
    const size_t mm = size_t(m) * m;
    const double *As = A + s * N * mm, *Bs = B + s * N * mm, *Cs = C + s * N * mm;
    const double *bs = b + s * N * m * r;
    double *xs = x + s * N * m * r;
    double *Hs = work + s * N * (mm + size_t(m) * R);   // [N][m][m] then [N][m][R]
    double *Gs = Hs + N * mm;
    double *sD = sh, *sC = sD + mm, *aug0 = sC + mm, *aug1 = aug0 + size_t(m) * W;
    double *prev = aug0, *next = aug1;
    bool ok = true;
    // ---- forward sweep
    for (int64_t k = 0; k < N; k++) {
        for (int i = lane; i < m * m; i += 32) {
            sD[i] = As[k * mm + i];
            if (k > 0) sC[i] = Cs[k * mm + i];
        }
        for (int idx = lane; idx < m * W; idx += 32) {
            const int i = idx / W, c = idx % W;
            double v = 0.0;
            if (c < m) v = k < N - 1 ? Bs[k * mm + i * m + c] : 0.0;
            else if (c < m + r) v = bs[(k * m + i) * r + (c - m)];
            else if (c < m + r + m) v = k == 0 ? Cs[i * m + (c - m - r)] : 0.0;   // corner C[0]
            else v = k == N - 1 ? Bs[(N - 1) * mm + i * m + (c - m - r - m)] : 0.0;   // corner B[N-1]
            next[idx] = v;
        }
        __syncwarp();
        if (k > 0) {
            warp_sub_mm(sD, m, sC, prev, W, m, m);                       // D = A_k - C_k H_{k-1}
            warp_sub_mm(next + m, W, sC, prev + m, W, m, R);             // rhs - C_k g_{k-1}
            __syncwarp();
        }
        ok = warp_lu_solve(sD, m, next, W, W) && ok;
        for (int idx = lane; idx < m * W; idx += 32) {
            const int i = idx / W, c = idx % W;
            if (c < m) Hs[k * mm + i * m + c] = next[idx];
            else Gs[(k * m + i) * R + (c - m)] = next[idx];
        }
        __syncwarp();
        double *t = prev;
        prev = next;
        next = t;
    }
    // ---- backward sweep: X_k = g_k - H_k X_{k+1}, X overwrites g in place;
    // X_{k+1} is kept in `prev` (columns m..W-1), H_k staged in sD
    for (int64_t k = N - 2; k >= 0; k--) {
        for (int i = lane; i < m * m; i += 32) sD[i] = Hs[k * mm + i];
        for (int idx = lane; idx < m * R; idx += 32) next[(idx / R) * W + m + idx % R] = Gs[k * m * R + idx];
        __syncwarp();
        warp_sub_mm(next + m, W, sD, prev + m, W, m, R);
        __syncwarp();
        for (int idx = lane; idx < m * R; idx += 32) Gs[k * m * R + idx] = next[(idx / R) * W + m + idx % R];
        __syncwarp();
        double *t = prev;
        prev = next;
        next = t;
    }
    // ---- Woodbury: K = I + [Z_{N-1}; Z_0], w = K^-1 [y_{N-1}; y_0]
    const int n2 = 2 * m;
    double *sK = sh, *sW = sK + size_t(n2) * n2;   // reuses the sweep's space
    __syncwarp();
    for (int idx = lane; idx < n2 * R; idx += 32) {
        const int i = idx / R, c = idx % R;
        const int64_t blk = i < m ? N - 1 : 0;
        const double v = Gs[(blk * m + (i % m)) * R + c];
        if (c < r) sW[i * r + c] = v;
        else sK[i * n2 + (c - r)] = v + ((c - r) == i ? 1.0 : 0.0);
    }
    __syncwarp();
    ok = warp_lu_solve(sK, n2, sW, r, r) && ok;
    // x_k = y_k - Z_k w
    for (int64_t k = 0; k < N; k++) {
        for (int idx = lane; idx < m * r; idx += 32) {
            const int i = idx / r, c = idx % r;
            const double *row = Gs + (k * m + i) * R;
            double v = row[c];
            for (int t = 0; t < n2; t++) v = fma(-row[r + t], sW[t * r + c], v);
            xs[(k * m + i) * r + c] = v;
        }
    }
    if (status && lane == 0) status[s] = ok ? 0 : 1;
}

}  // namespace

size_t strip_smem_bytes(int m, int r)
{
    const size_t R = size_t(r) + 2 * m, W = m + R;
    const size_t sweep = 2 * size_t(m) * m + 2 * size_t(m) * W;
    const size_t wood = size_t(2 * m) * (2 * m) + size_t(2 * m) * r;
    return sizeof(double) * (sweep > wood ? sweep : wood);
}

size_t strip_work_doubles(int64_t N, int m, int r) { return size_t(N) * (size_t(m) * m + size_t(m) * (r + 2 * m)); }

cudaError_t launch_strip(int64_t nsys, int64_t N, int m, int r, const double *A, const double *B, const double *C,
                         const double *b, double *x, double *work, int32_t *status, cudaStream_t st)
{
    const size_t sm = strip_smem_bytes(m, r);
    cudaError_t e = cudaFuncSetAttribute(k_strip_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    k_strip_solve<<<dim3(unsigned(nsys)), 32, sm, st>>>(nsys, N, m, r, A, B, C, b, x, work, status);
    return cudaGetLastError();
}

}  // namespace bc
