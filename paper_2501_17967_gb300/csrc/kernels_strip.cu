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
// Blocks up to 32 x 32 (interface-sized blocks): one warp per system, the
// batched small-dense-LU workload (many strips or right-hand-side sets at
// once); the blocks of the current step live in shared memory, H_k and g_k /
// X_k in a global workspace.  Larger blocks (the paper's elements of 16 x 24
// nodes): one system at a time on the whole GPU, below.  FP64.
#include <cuda_runtime.h>

#include <algorithm>

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

// ---------------------------------------------------------------------------
// Large blocks (m > 32, the element blocks of the paper's strip: 16 x 24 =
// 384 nodes): one system at a time on the whole GPU.  The host loops over
// the elements; each step factors the augmented block [D_k | B_k | rhs_k]
// (row-major, Wc = m + m + R columns) by right-looking blocked LU with
// partial pivoting (panels of kPanel columns: k_strip_panel factors a panel
// in shared memory in one CTA, k_strip_swap carries its row exchanges to the
// columns on its right, k_strip_trsm applies L11^-1 to them (one thread per
// column, so the many columns spread over the SMs), and a DGEMM updates the
// trailing block), then back-substitutes the right-hand columns (k_strip_trsm
// with U11 per diagonal block, DGEMM for the rows above).  Narrow panels keep
// the single-CTA FP64 work of each panel small: one SM's FP64 pipe does 4
// flop per clock.
// ---------------------------------------------------------------------------
constexpr int kPanel = 16;
constexpr int kPanelThreads = 256;

// Large blocks take the corners as a border: x_{N-1} is eliminated last.  The
// first N - 1 block rows form a tridiagonal T' whose right-hand side also
// carries the border column E (C_0 in row 0, B_{N-2} in row N-2: they couple
// to x_{N-1}), so only m extra columns ride through the sweep; then the
// Schur complement S = A_{N-1} - F T'^-1 E (F: B_{N-1} at column 0, C_{N-1}
// at column N-2) gives x_{N-1}, and x_k = Y_k - Z_k x_{N-1}.  This is the
// rank-m form of the corner correction.
// Step k's augmented block (k < N - 1): [A_k | B_k (k < N-2) | b_k | E_k].
__global__ void k_strip_aug(int64_t N, int m, int r, int64_t k, const double *__restrict__ A,
                            const double *__restrict__ B, const double *__restrict__ C,
                            const double *__restrict__ b, double *__restrict__ aug, int Wc)
{
    const size_t mm = size_t(m) * m;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < int64_t(m) * Wc;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(idx / Wc), c = int(idx % Wc);
        double v = 0.0;
        if (c < m) v = A[k * mm + size_t(i) * m + c];
        else if (c < 2 * m) v = k < N - 2 ? B[k * mm + size_t(i) * m + (c - m)] : 0.0;
        else if (c < 2 * m + r) v = b[(k * m + i) * r + (c - 2 * m)];
        else {
            const int q = c - 2 * m - r;
            if (k == 0) v += C[size_t(i) * m + q];
            if (k == N - 2) v += B[k * mm + size_t(i) * m + q];
        }
        aug[idx] = v;
    }
}

// the border system [A_{N-1} | b_{N-1}] (N = 1: [A_0 + B_0 + C_0 | b_0]),
// before the products with T'^-1 [b | E] are taken off
__global__ void k_strip_border(int64_t N, int m, int r, const double *__restrict__ A, const double *__restrict__ B,
                               const double *__restrict__ C, const double *__restrict__ b, double *__restrict__ S)
{
    const size_t mm = size_t(m) * m;
    const int ld = m + r;
    const int64_t k = N - 1;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < int64_t(m) * ld;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(idx / ld), c = int(idx % ld);
        double v;
        if (c < m) {
            v = A[k * mm + size_t(i) * m + c];
            if (N == 1) v += B[size_t(i) * m + c] + C[size_t(i) * m + c];
        } else {
            v = b[(k * m + i) * r + (c - m)];
        }
        S[idx] = v;
    }
}

// LU with partial pivoting of the panel: rows [j0, n), columns [j0, j0 + jb)
// of M (row-major, leading dimension ld), staged in shared memory; the pivot
// rows go to piv[j] (absolute); a zero or non-finite pivot sets *status.
// Thread t owns the rows t, t + nt, ...: it searches them for the pivot and
// applies the rank-1 update to them, so a column step needs three barriers
// (pivot found, pivot row in place, and the next step's search).
__global__ void __launch_bounds__(kPanelThreads)
k_strip_panel(double *__restrict__ M, int n, int ld, int j0, int jb, int32_t *__restrict__ piv,
              int32_t *__restrict__ status)
{
    extern __shared__ double sp[];   // [n - j0][jb]
    __shared__ unsigned long long s_key[kPanelThreads / 32];
    __shared__ int s_row[kPanelThreads / 32];
    __shared__ int s_piv;
    __shared__ double s_inv;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nt = blockDim.x, nw = nt >> 5;
    const int rows = n - j0;
    for (int idx = t; idx < rows * jb; idx += nt) sp[idx] = M[size_t(j0 + idx / jb) * ld + j0 + idx % jb];
    __syncthreads();
    // |x| compared through its bit pattern (sign cleared): an integer order
    // that matches the order of the magnitudes, so the search leaves the FP64
    // pipe to the updates (a NaN sorts above every number and is flagged)
    constexpr unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
    for (int jj = 0; jj < jb; jj++) {
        unsigned long long key = 0;
        int bi = rows;
        for (int i = jj + ((t - jj) % nt + nt) % nt; i < rows; i += nt) {   // owned rows >= jj
            const unsigned long long v = static_cast<unsigned long long>(__double_as_longlong(sp[i * jb + jj])) & kMag;
            if (bi == rows || v > key) { key = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi < rows && (bi == rows || ok > key || (ok == key && oi < bi))) { key = ok; bi = oi; }
        }
        if (lane == 0) { s_key[w] = key; s_row[w] = bi; }
        __syncthreads();
        if (w == 0) {
            key = lane < nw ? s_key[lane] : 0ull;
            bi = lane < nw ? s_row[lane] : rows;
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (oi < rows && (bi == rows || ok > key || (ok == key && oi < bi))) { key = ok; bi = oi; }
            }
            if (lane == 0) {
                const int p = bi < rows ? bi : jj;
                const double d = sp[p * jb + jj];
                const bool good = d != 0.0 && isfinite(d);
                s_piv = p;
                s_inv = good ? 1.0 / d : 0.0;
                piv[j0 + jj] = j0 + p;
                if (!good) *status = 1;
            }
        }
        __syncthreads();
        const int p = s_piv;
        if (p != jj)
            for (int c = t; c < jb; c += nt) {
                const double x = sp[jj * jb + c];
                sp[jj * jb + c] = sp[p * jb + c];
                sp[p * jb + c] = x;
            }
        __syncthreads();
        const double inv = s_inv;
        for (int i = jj + 1 + ((t - jj - 1) % nt + nt) % nt; i < rows; i += nt) {   // owned rows > jj
            const double l = sp[i * jb + jj] * inv;
            sp[i * jb + jj] = l;
            for (int c = jj + 1; c < jb; c++) sp[i * jb + c] = fma(-l, sp[jj * jb + c], sp[i * jb + c]);
        }
    }
    __syncthreads();
    for (int idx = t; idx < rows * jb; idx += nt) M[size_t(j0 + idx / jb) * ld + j0 + idx % jb] = sp[idx];
}

// the panel's row exchanges on columns [c0, c1)
__global__ void k_strip_swap(double *__restrict__ M, int ld, int j0, int jb, const int32_t *__restrict__ piv,
                             int c0, int c1)
{
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    for (int j = j0; j < j0 + jb; j++) {
        const int p = piv[j];
        if (p != j) {
            const double x = M[size_t(j) * ld + c];
            M[size_t(j) * ld + c] = M[size_t(p) * ld + c];
            M[size_t(p) * ld + c] = x;
        }
    }
}

// Triangular solve with the jb x jb diagonal block at j0, in place on rows
// [j0, j0 + jb) of the columns [c0, c1), one thread per column (jb <= kPanel):
// upper = false: the unit lower block (L11^-1 A12); upper = true: the upper
// block (U11^-1 Y).  A zero diagonal gives zero (the panel flagged it).
__global__ void k_strip_trsm(double *__restrict__ M, int ld, int j0, int jb, bool upper, int c0, int c1)
{
    __shared__ double sa[kPanel * kPanel];
    __shared__ double sr[kPanel];   // reciprocals of the diagonal (upper)
    for (int idx = threadIdx.x; idx < jb * jb; idx += blockDim.x)
        sa[idx] = M[size_t(j0 + idx / jb) * ld + j0 + idx % jb];
    __syncthreads();
    if (upper && threadIdx.x < jb) {
        const double d = sa[threadIdx.x * jb + threadIdx.x];
        sr[threadIdx.x] = d != 0.0 ? 1.0 / d : 0.0;
    }
    __syncthreads();
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    double x[kPanel];
#pragma unroll
    for (int i = 0; i < kPanel; i++) x[i] = i < jb ? M[size_t(j0 + i) * ld + c] : 0.0;
    if (!upper) {
#pragma unroll
        for (int i = 1; i < kPanel; i++)
#pragma unroll
            for (int q = 0; q < i; q++) x[i] = fma(-sa[i * jb + q], x[q], x[i]);   // x[q] = 0 past jb
    } else {
#pragma unroll
        for (int i = kPanel - 1; i >= 0; i--) {
            if (i >= jb) continue;
#pragma unroll
            for (int q = i + 1; q < kPanel; q++)
                if (q < jb) x[i] = fma(-sa[i * jb + q], x[q], x[i]);
            x[i] *= sr[i];
        }
    }
#pragma unroll
    for (int i = 0; i < kPanel; i++)
        if (i < jb) M[size_t(j0 + i) * ld + c] = x[i];
}

}  // namespace

int strip_panel_width() { return kPanel; }

cudaError_t launch_strip_aug(int64_t N, int m, int r, int64_t k, const double *A, const double *B, const double *C,
                             const double *b, double *aug, int Wc, cudaStream_t st)
{
    const int64_t n = int64_t(m) * Wc;
    k_strip_aug<<<int(std::min<int64_t>((n + 255) / 256, 152 * 8)), 256, 0, st>>>(N, m, r, k, A, B, C, b, aug, Wc);
    return cudaGetLastError();
}

cudaError_t strip_prepare(int nmax)
{
    return cudaFuncSetAttribute(k_strip_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(sizeof(double) * size_t(nmax) * kPanel));
}

cudaError_t launch_strip_panel(double *M, int n, int ld, int j0, int jb, int32_t *piv, int32_t *status,
                               cudaStream_t st)
{
    const size_t sm = sizeof(double) * size_t(n - j0) * jb;
    k_strip_panel<<<1, kPanelThreads, sm, st>>>(M, n, ld, j0, jb, piv, status);
    return cudaGetLastError();
}

cudaError_t launch_strip_swap(double *M, int ld, int j0, int jb, const int32_t *piv, int c0, int c1, cudaStream_t st)
{
    if (c1 <= c0) return cudaSuccess;
    k_strip_swap<<<(c1 - c0 + 127) / 128, 128, 0, st>>>(M, ld, j0, jb, piv, c0, c1);
    return cudaGetLastError();
}

cudaError_t launch_strip_trsm(double *M, int ld, int j0, int jb, bool upper, int c0, int c1, cudaStream_t st)
{
    if (c1 <= c0) return cudaSuccess;
    k_strip_trsm<<<(c1 - c0 + 31) / 32, 32, 0, st>>>(M, ld, j0, jb, upper, c0, c1);
    return cudaGetLastError();
}

cudaError_t launch_strip_border(int64_t N, int m, int r, const double *A, const double *B, const double *C,
                                const double *b, double *S, cudaStream_t st)
{
    const int64_t n = int64_t(m) * (m + r);
    k_strip_border<<<int(std::min<int64_t>((n + 255) / 256, 152 * 8)), 256, 0, st>>>(N, m, r, A, B, C, b, S);
    return cudaGetLastError();
}

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
