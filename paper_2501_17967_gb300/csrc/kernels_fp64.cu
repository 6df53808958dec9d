// FP64 passes of the box code (forward and adjoint).
//
// The forward apply u = A f runs four kernel shapes:
//   leafA : per leaf,  box expansion  = s * Op * (leaf vector)     P2M
//   up    : per box,   parent expansion = sum_q Op_q * child_q     M2M (bottom-up)
//   down  : per box,   local = Op_q * parent + sum_V Op_d * src
//                      + sum_X Op_e * (leaf vector) + log terms    L2L + M2L + P2L (top-down)
//   leafB : per leaf,  nodes = Re(Op * own expansion) + sum_W Re(Op * src)
//                      + sum_near T * (leaf vector) + log terms    L2P + M2P + near field
// The adjoint h = A^T g runs the same four shapes in the same order with the
// conjugate-transposed operator of each forward step (L2P^H, L2L^H, M2M^H +
// M2L^H + M2P^H, P2M^H + P2L^H + T^T); only the scale factors differ, which
// the template flag ADJ selects.  Operators are stored so that every kernel
// computes out[l] = sum_k Op[k*P1 + l] * in[k].
#include <cuda_runtime.h>

#include <algorithm>

#include "bc_internal.h"

namespace bc {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ double r_at(double half_L, int lv) { return ldexp(half_L, -lv); }

// -------------------------------------------------------------------------
// leaf_up: per leaf, the box expansion from the leaf vector, then the upward
// pass without per-level launches: a parent's expansion is computed by the
// block whose child arrives last (arrival counter per box, no waiting).
//   leaf:   ex[box(leaf)][l] = s * sum_j OpA[j][l] v[leaf][j]
//           forward (P2M): OpA = Q^T, s = r^2;  adjoint (L2P^H): OpA = E^H, s = 1
//   parent: ex[p][l] = sum_q sum_k OpUp[q][k][l] ex[child_q(p)][k]    (levels >= 2)
//           forward: M2M; adjoint: L2L^H
// cnt[] must be zero on entry (the apply clears it).
// -------------------------------------------------------------------------
template <bool ADJ>
__global__ void __launch_bounds__(64)
k_leaf_up(int64_t nleaf, const int32_t *__restrict__ order, const int32_t *__restrict__ leaf_box,
          const int32_t *__restrict__ leaf_level, const int32_t *__restrict__ box_parent,
          const int32_t *__restrict__ box_level, const int32_t *__restrict__ box_child0,
          const double *__restrict__ vin, const double2 *__restrict__ OpA, const double2 *__restrict__ OpUp,
          double2 *ex, int32_t *cnt, int NP, int P1, double half_L)
{
    extern __shared__ double2 shu[];
    double2 *sc = shu;                                     // 4 * P1
    double *sv = reinterpret_cast<double *>(shu + 4 * P1); // NP
    __shared__ int s_go;
    for (int64_t li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int leaf = order[li];
        int b = leaf_box[leaf];
        __syncthreads();
        for (int j = threadIdx.x; j < NP; j += blockDim.x) sv[j] = vin[int64_t(leaf) * NP + j];
        __syncthreads();
        const double r = r_at(half_L, leaf_level[leaf]);
        const double s = ADJ ? 1.0 : r * r;
        for (int l = threadIdx.x; l < P1; l += blockDim.x) {
            double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
            for (int j = 0; j < NP; j += 2) {
                double2 o0 = OpA[j * P1 + l], o1 = OpA[(j + 1) * P1 + l];
                re0 = fma(o0.x, sv[j], re0);
                im0 = fma(o0.y, sv[j], im0);
                re1 = fma(o1.x, sv[j + 1], re1);
                im1 = fma(o1.y, sv[j + 1], im1);
            }
            ex[int64_t(b) * P1 + l] = make_double2(s * (re0 + re1), s * (im0 + im1));
        }
        for (; cnt;) {
            const int p = box_parent[b];
            if (p < 0 || box_level[p] < 2) break;
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_go = atomicAdd(&cnt[p], 1) == 3;
            __syncthreads();
            if (!s_go) break;
            __threadfence();
            const int c0 = box_child0[p];
            for (int i = threadIdx.x; i < 4 * P1; i += blockDim.x) sc[i] = __ldcg(&ex[int64_t(c0) * P1 + i]);
            __syncthreads();
            for (int l = threadIdx.x; l < P1; l += blockDim.x) {
                double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
                for (int k = 0; k < P1; k++) {
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        double2 o = OpUp[(q * P1 + k) * P1 + l], a = sc[q * P1 + k];
                        re[q] = fma(o.x, a.x, fma(-o.y, a.y, re[q]));
                        im[q] = fma(o.x, a.y, fma(o.y, a.x, im[q]));
                    }
                }
                ex[int64_t(p) * P1 + l] = make_double2((re[0] + re[1]) + (re[2] + re[3]), (im[0] + im[1]) + (im[2] + im[3]));
            }
            b = p;
        }
    }
}

// -------------------------------------------------------------------------
// m2l: for every box b at level >= 2 (one launch over all levels)
//   out[b] = sum_{s in V(b)} M2L(d_s) in[s] + log(r) sum_s in[s][0] e_0
//          + sum_{c in X(b)} (s1 * OpX[code] x[c] + s2 (lvec . x[c]) e_0)
// M2L in factored form (d = (c_s - c_t)/r, complex):
//   forward  a_k = (-1)^k d^-k A_k (k >= 1),
//            B_l += d^-l sum_{k>=1} C(k+l-1, l) a_k + (l = 0 ? log|d| A_0 : -d^-l A_0 / l)
//   adjoint  (exact conjugate transpose of the forward map of the reversed pair)
//            a_l = (-1)^l conj(d)^-l in_l (l >= 0),
//            out_k += conj(d)^-k sum_{l>=0} C(k+l-1, l) a_l   (k >= 1)
//            out_0 += log|d| in_0 - sum_{l>=1} a_l / l
// tri = 1 keeps only the terms with k + l <= P (and exactly their transpose).
// The binomial table is shared by every offset and lives in shared memory;
// each of the two warps of a block takes every other V source.
// -------------------------------------------------------------------------
template <bool ADJ>
__global__ void __launch_bounds__(64)
k_m2l(int64_t b0, int64_t b1, const int32_t *__restrict__ box_level, const int32_t *__restrict__ v_ptr,
      const int32_t *__restrict__ v_src, const int32_t *__restrict__ v_code, const int32_t *__restrict__ x_ptr,
      const int32_t *__restrict__ x_src, const int32_t *__restrict__ x_code, const double2 *__restrict__ dpow,
      const double *__restrict__ logd, const double *__restrict__ binom, const double2 *__restrict__ OpX,
      const double *__restrict__ xvec, const int32_t *__restrict__ leaf_box, const double2 *__restrict__ in,
      double2 *out, int NP, int P1, double half_L, int tri)
{
    extern __shared__ double smem[];
    const int ldc = P1 + 1;
    double *Cb = smem;                                           // [P1][P1+1]
    double *inv = Cb + P1 * ldc;                                 // [P1] 1/l
    double2 *sa = reinterpret_cast<double2 *>(inv + P1);         // [2][64] scaled sources
    double2 *part = sa + 128;                                    // [2][64] warp partial sums
    double2 *mono = part + 128;                                  // [2] sum of in[s][0] per warp
    double *sx = reinterpret_cast<double *>(mono + 2);           // [NP]
    const int tid = threadIdx.x, h = tid >> 5, lane = tid & 31, P = P1 - 1;
    for (int i = tid; i < P1 * ldc; i += blockDim.x) {
        int r = i / ldc, c = i % ldc;
        // forward reads [k][l] = C(k+l-1, l); adjoint reads [l][k] = C(k+l-1, l),
        // with column k = 0 holding the coefficients -1/l of out_0 (l >= 1)
        if (ADJ)
            Cb[i] = (c >= 1 && c < P1 && r < P1) ? binom[c * ldc + r] : ((c == 0 && r >= 1 && r < P1) ? -1.0 / r : 0.0);
        else
            Cb[i] = binom[i];
    }
    for (int i = tid; i < P1; i += blockDim.x) inv[i] = i ? 1.0 / i : 0.0;
    __syncthreads();
    for (int64_t b = b0 + blockIdx.x; b < b1; b += gridDim.x) {
        const int lv = box_level[b];
        double ar[2] = {0.0, 0.0}, ai[2] = {0.0, 0.0};
        double mr = 0.0, mi = 0.0;
        double2 *a = sa + h * 64;
        for (int e = v_ptr[b] + h; e < v_ptr[b + 1]; e += 2) {
            const int s = v_src[e], c = v_code[e];
            const double2 *dp = dpow + size_t(c) * P1;
            for (int k = lane; k < P1; k += 32) {
                double2 A = in[int64_t(s) * P1 + k], D = dp[k];
                double zr = A.x * D.x - A.y * D.y, zi = A.x * D.y + A.y * D.x;
                if (k & 1) { zr = -zr; zi = -zi; }
                a[k] = make_double2(zr, zi);
            }
            __syncwarp();
            const double2 A0 = a[0];
            const double ld = logd[c];
            mr += A0.x;
            mi += A0.y;
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int o = lane + 32 * u;
                if (o >= P1) continue;
                double sr = 0.0, si = 0.0;
                if (!ADJ) {
                    // B_o += d^-o (sum_{k>=1} C(k+o-1, o) a_k + c_o A_0), c_0 = log|d| (d^0 = 1), c_o = -1/o
                    const int kmax = tri ? P - o : P;
                    for (int k = 1; k <= kmax; k++) {
                        double cf = Cb[k * ldc + o];
                        sr = fma(cf, a[k].x, sr);
                        si = fma(cf, a[k].y, si);
                    }
                    const double c0 = o == 0 ? ld : -inv[o];
                    sr = fma(c0, A0.x, sr);
                    si = fma(c0, A0.y, si);
                } else {
                    // out_o += conj(d)^-o sum_{l} Cb[l][o] a_l  (+ log|d| in_0 for o = 0)
                    const int lmax = (tri && o > 0) ? P - o : P;
                    for (int l = 0; l <= lmax; l++) {
                        double cf = Cb[l * ldc + o];
                        sr = fma(cf, a[l].x, sr);
                        si = fma(cf, a[l].y, si);
                    }
                    const double c0 = o == 0 ? ld : 0.0;
                    sr = fma(c0, A0.x, sr);
                    si = fma(c0, A0.y, si);
                }
                const double2 D = dp[o];
                ar[u] += sr * D.x - si * D.y;
                ai[u] += sr * D.y + si * D.x;
            }
            __syncwarp();
        }
        // combine the two warps: thread tid owns coefficient tid
#pragma unroll
        for (int u = 0; u < 2; u++) part[h * 64 + lane + 32 * u] = make_double2(ar[u], ai[u]);
        if (lane == 0) mono[h] = make_double2(mr, mi);
        __syncthreads();
        double orr = 0.0, oi = 0.0;
        if (tid < P1) {
            orr = part[tid].x + part[64 + tid].x;
            oi = part[tid].y + part[64 + tid].y;
        }
        if (tid == 0) {
            const double logr = log(r_at(half_L, lv));
            orr += logr * (mono[0].x + mono[1].x);
            oi += logr * (mono[0].y + mono[1].y);
        }
        // X list: leaf densities (forward) / leaf adjoint data (adjoint) of the
        // coarser neighbour leaves.  The log term uses coefficient 0 of the
        // leaf's own expansion from the upward pass: forward A_0 = r_c^2 (w.f)/2pi,
        // adjoint B_0 = sum_j g_j, so the term is log(r_c) * that coefficient.
        const double rc = r_at(half_L, lv - 1);
        const double s1 = ADJ ? 1.0 : rc * rc;
        const double logrc = log(rc);
        for (int e = x_ptr[b]; e < x_ptr[b + 1]; e++) {
            const int c = x_src[e];
            const double2 *op = OpX + size_t(x_code[e]) * NP * P1;
            __syncthreads();
            for (int j = tid; j < NP; j += blockDim.x) sx[j] = xvec[int64_t(c) * NP + j];
            __syncthreads();
            if (tid < P1) {
                double xr0 = 0.0, xi0 = 0.0, xr1 = 0.0, xi1 = 0.0;
                for (int j = 0; j < NP; j += 2) {
                    double2 o0 = op[j * P1 + tid], o1 = op[(j + 1) * P1 + tid];
                    xr0 = fma(o0.x, sx[j], xr0);
                    xi0 = fma(o0.y, sx[j], xi0);
                    xr1 = fma(o1.x, sx[j + 1], xr1);
                    xi1 = fma(o1.y, sx[j + 1], xi1);
                }
                orr = fma(s1, xr0 + xr1, orr);
                oi = fma(s1, xi0 + xi1, oi);
                if (tid == 0) orr = fma(logrc, in[int64_t(leaf_box[c]) * P1].x, orr);
            }
        }
        if (tid < P1) out[b * P1 + tid] = make_double2(orr, oi);
        __syncthreads();
    }
}

// -------------------------------------------------------------------------
// shift_down: out[b] += Par_q * out[parent(b)] for the boxes of one level >= 3
//   forward: L2L; adjoint: M2M^H.  Two independent FMA chains per thread.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(64)
k_shift_down(int64_t b0, int64_t b1, const int32_t *__restrict__ parent, const int32_t *__restrict__ box_ix,
             const int32_t *__restrict__ box_iy, const double2 *__restrict__ OpPar, double2 *__restrict__ out, int P1)
{
    extern __shared__ double2 se[];
    for (int64_t b = b0 + blockIdx.x; b < b1; b += gridDim.x) {
        const int pb = parent[b];
        const int q = (box_ix[b] & 1) + 2 * (box_iy[b] & 1);
        __syncthreads();
        for (int i = threadIdx.x; i < P1; i += blockDim.x) se[i] = out[int64_t(pb) * P1 + i];
        __syncthreads();
        for (int l = threadIdx.x; l < P1; l += blockDim.x) {
            const double2 *op = OpPar + size_t(q) * P1 * P1;
            const double2 acc = out[b * P1 + l];
            double re0 = acc.x, im0 = acc.y, re1 = 0.0, im1 = 0.0;
            int k = 0;
            for (; k + 1 < P1; k += 2) {
                double2 o0 = op[k * P1 + l], a0 = se[k], o1 = op[(k + 1) * P1 + l], a1 = se[k + 1];
                re0 = fma(o0.x, a0.x, fma(-o0.y, a0.y, re0));
                im0 = fma(o0.x, a0.y, fma(o0.y, a0.x, im0));
                re1 = fma(o1.x, a1.x, fma(-o1.y, a1.y, re1));
                im1 = fma(o1.x, a1.y, fma(o1.y, a1.x, im1));
            }
            if (k < P1) {
                double2 o0 = op[k * P1 + l], a0 = se[k];
                re0 = fma(o0.x, a0.x, fma(-o0.y, a0.y, re0));
                im0 = fma(o0.x, a0.y, fma(o0.y, a0.x, im0));
            }
            out[b * P1 + l] = make_double2(re0 + re1, im0 + im1);
        }
    }
}

// -------------------------------------------------------------------------
// leafB: for every leaf o, node j
//   out[o][j] = sE * Re(sum_l OpE[l][j] own[box(o)][l])                  (level >= 2)
//             + sum_{w in W(o)} [ sW * Re(sum_k OpW[code][k][j] src[w][k]) + cW_j * Re(src[w][0]) ]
//             + sum_{s in near(o)} [ sN * sum_k T[tab][k][j] v[s][k] + cN_j * Re(aux[box(s)][0]) ]
//   forward: sE = 1, sW = 1, cW = log r_o, sN = r_s^2, cN = log r_s (aux = multipoles: A_0 = r^2 w.f / 2pi)
//   adjoint: sE = r_o^2, sW = r_o^2, cW = r_o^2 log r_o w_j / 2pi, sN = r_o^2,
//            cN = r_o^2 log r_o w_j / 2pi (aux = adjoint locals: B_0 = sum_i g_i)
// -------------------------------------------------------------------------
template <bool ADJ>
__global__ void k_leaf_out(int64_t nleaf, const int32_t *__restrict__ order,
                           const int32_t *__restrict__ leaf_box, const int32_t *__restrict__ leaf_level,
                           const int32_t *__restrict__ w_ptr, const int32_t *__restrict__ w_src,
                           const int32_t *__restrict__ w_code, const int32_t *__restrict__ n_ptr,
                           const int32_t *__restrict__ n_src, const int32_t *__restrict__ n_tab,
                           const double2 *__restrict__ OpE, const double2 *__restrict__ OpW,
                           const double *__restrict__ T, const double *__restrict__ wvec,
                           const double2 *__restrict__ own, const double2 *__restrict__ src,
                           const double2 *__restrict__ aux, const double *__restrict__ vnear,
                           double *__restrict__ vout, int NP, int P1, double half_L, bool far,
                           const double *__restrict__ Pnear)
{
    extern __shared__ double2 sh[];
    double2 *se = sh;                                  // P1
    double *sv = reinterpret_cast<double *>(sh + P1);  // NP
    for (int64_t li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int o = order[li];
        const int lvo = leaf_level[o];
        const double ro = r_at(half_L, lvo);
        const int j = threadIdx.x;   // blockDim.x == NP
        const double wj = wvec[j];
        double acc = 0.0;
        if (far && lvo >= 2) {
            __syncthreads();
            for (int i = threadIdx.x; i < P1; i += blockDim.x) se[i] = own[int64_t(leaf_box[o]) * P1 + i];
            __syncthreads();
            double s = 0.0;
            for (int l = 0; l < P1; l++) {
                double2 op = OpE[l * NP + j], b = se[l];
                s = fma(op.x, b.x, fma(-op.y, b.y, s));
            }
            acc = ADJ ? ro * ro * s : s;
        }
        const double sW = ADJ ? ro * ro : 1.0;
        const double cW = ADJ ? ro * ro * log(ro) * wj / kTwoPi : log(ro);
        for (int e = w_ptr[o]; e < w_ptr[o + 1]; e++) {
            const double2 *op = OpW + size_t(w_code[e]) * P1 * NP;
            __syncthreads();
            for (int i = threadIdx.x; i < P1; i += blockDim.x) se[i] = src[int64_t(w_src[e]) * P1 + i];
            __syncthreads();
            double s = 0.0;
            for (int k = 0; k < P1; k++) {
                double2 opk = op[k * NP + j], b = se[k];
                s = fma(opk.x, b.x, fma(-opk.y, b.y, s));
            }
            acc = fma(sW, s, fma(cW, se[0].x, acc));
        }
        for (int e = n_ptr[o]; e < n_ptr[o + 1]; e++) {
            const int s = n_src[e];
            double t = 0.0;
            if (Pnear) {
                // split-precision result of this entry, alpha already applied
                t = Pnear[size_t(e) * NP + j];
            } else {
                const double *tb = T + size_t(n_tab[e]) * NP * NP;
                __syncthreads();
                for (int i = threadIdx.x; i < NP; i += blockDim.x) sv[i] = vnear[int64_t(s) * NP + i];
                __syncthreads();
                for (int k = 0; k < NP; k++) t = fma(tb[k * NP + j], sv[k], t);
            }
            double a0 = aux[int64_t(leaf_box[s]) * P1].x;
            double sN, cN;
            if (ADJ) {
                sN = ro * ro;
                cN = ro * ro * log(ro) * wj / kTwoPi;
            } else {
                double rs = r_at(half_L, leaf_level[s]);
                sN = rs * rs;
                cN = log(rs);
            }
            if (Pnear) sN = 1.0;
            acc = fma(sN, t, fma(cN, a0, acc));
        }
        vout[int64_t(o) * NP + j] = acc;
    }
}

// -------------------------------------------------------------------------
// Point evaluation by barycentric Chebyshev interpolation on the containing leaf.
// -------------------------------------------------------------------------
__global__ void k_eval_points(int64_t n, const double *__restrict__ xy, const double *__restrict__ u,
                              const int32_t *__restrict__ child0, const int32_t *__restrict__ box_leaf,
                              const int32_t *__restrict__ box_level, const int32_t *__restrict__ box_ix,
                              const int32_t *__restrict__ box_iy, double x0, double y0, double L, int p,
                              double *__restrict__ out)
{
    const double pi = 3.14159265358979323846;
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        double x = xy[2 * k], y = xy[2 * k + 1];
        if (!(x >= x0 && x <= x0 + L && y >= y0 && y <= y0 + L)) { out[k] = nan(""); continue; }
        int b = 0;
        while (box_leaf[b] < 0) {
            int lv = box_level[b];
            double h = ldexp(L, -lv);
            double mx = x0 + (box_ix[b] + 0.5) * h, my = y0 + (box_iy[b] + 0.5) * h;
            b = child0[b] + (x >= mx ? 1 : 0) + (y >= my ? 2 : 0);
        }
        int lv = box_level[b];
        double h = ldexp(L, -lv), r = 0.5 * h;
        double xi = (x - (x0 + (box_ix[b] + 0.5) * h)) / r, eta = (y - (y0 + (box_iy[b] + 0.5) * h)) / r;
        double lx[kMaxP], ly[kMaxP], sx = 0.0, sy = 0.0;
        int hx = -1, hy = -1;
        for (int m = 0; m < p; m++) {
            double th = (2.0 * m + 1.0) * pi / (2.0 * p);
            double xm = -cos(th), lam = ((m & 1) ? -1.0 : 1.0) * sin(th);
            double dx = xi - xm, dy = eta - xm;
            if (dx == 0.0) hx = m;
            if (dy == 0.0) hy = m;
            lx[m] = dx == 0.0 ? 0.0 : lam / dx;
            ly[m] = dy == 0.0 ? 0.0 : lam / dy;
            sx += lx[m];
            sy += ly[m];
        }
        for (int m = 0; m < p; m++) {
            lx[m] = hx >= 0 ? (m == hx ? 1.0 : 0.0) : lx[m] / sx;
            ly[m] = hy >= 0 ? (m == hy ? 1.0 : 0.0) : ly[m] / sy;
        }
        const double *ub = u + int64_t(box_leaf[b]) * p * p;
        double acc = 0.0;
        for (int jy = 0; jy < p; jy++) {
            double row = 0.0;
            for (int jx = 0; jx < p; jx++) row = fma(lx[jx], ub[jy * p + jx], row);
            acc = fma(ly[jy], row, acc);
        }
        out[k] = acc;
    }
}

inline int grid_for(int64_t n, int cap = 152 * 16)
{
    return int(n < cap ? (n > 0 ? n : 1) : cap);
}

// Per-tree arrays <-> the union's vectors for batched applies.
__global__ void k_batch_copy(BatchPtrs bp, bool gather, double *__restrict__ ubuf, int NP)
{
    const int64_t base = bp.off[0], total = (bp.off[bp.n] - base) * NP;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t leaf = base + i / NP;
        int lo = 0, hi = bp.n - 1;   // tree of this leaf: last k with off[k] <= leaf
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bp.off[mid] <= leaf) lo = mid; else hi = mid - 1;
        }
        const int64_t local = (leaf - bp.off[lo]) * NP + i % NP;
        if (gather) ubuf[base * NP + i] = bp.in[lo][local];
        else bp.out[lo][local] = ubuf[base * NP + i];
    }
}

}  // namespace

cudaError_t launch_apply(const PassArgs &a, const HostTree &h, const DevTree &d, const DevTables &tb,
                         bool adj, const double *vin, double *vout, cudaStream_t st, int pass_mask,
                         cudaEvent_t *ev, int m2l_tri, const SplitLaunch *split)
{
    const bool far = (pass_mask & 2) != 0, near = (pass_mask & 1) != 0;
    const double *Pnear = split ? split->tree->P : nullptr;
    if (ev) cudaEventRecord(ev[0], st);
    if (split && near) {
        cudaError_t e = launch_split_near(a, *split->tables, *split->tree, adj, vin, st);
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[1], st);
    const OpSet &op = adj ? tb.adj : tb.fwd;
    const int NP = a.NP, P1 = a.P1;
    double2 *first = adj ? d.expB : d.expA;    // leafA / up target
    double2 *second = adj ? d.expA : d.expB;   // down target
    // arrival counters of the upward pass start at zero
    cudaError_t ce = cudaMemsetAsync(d.cnt, 0, sizeof(int32_t) * size_t(a.nbox), st);
    if (ce != cudaSuccess) return ce;
    if (ev) cudaEventRecord(ev[2], st);
    // leafA + upward pass in one launch (leafA always runs: the near-field log
    // term reads coefficient 0 of its output; without the far field no climb)
    int32_t *cnt_up = d.cnt;
    const size_t shU = sizeof(double) * NP + sizeof(double2) * 4 * P1;
    if (adj)
        k_leaf_up<true><<<grid_for(a.nleaf, 152 * (a.leaf_bps ? a.leaf_bps : 16)), 64, shU, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                                                           d.box_parent, d.box_level, d.box_child0, vin, op.leafA,
                                                           op.up, first, far ? cnt_up : nullptr, NP, P1, a.half_L);
    else
        k_leaf_up<false><<<grid_for(a.nleaf, 152 * (a.leaf_bps ? a.leaf_bps : 16)), 64, shU, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                                                            d.box_parent, d.box_level, d.box_child0, vin, op.leafA,
                                                            op.up, first, far ? cnt_up : nullptr, NP, P1, a.half_L);
    if (ev) cudaEventRecord(ev[3], st);
    size_t shD = sizeof(double2) * P1 + sizeof(double) * NP;
    if (far && h.nlevels > 2) {
        const int64_t b0 = h.level_start[2], b1 = h.level_start[h.nlevels];
        size_t shM = sizeof(double) * (size_t(P1) * (P1 + 1) + P1) + sizeof(double2) * (128 + 128 + 2) +
                     sizeof(double) * NP;
        int grid = grid_for(b1 - b0, 152 * (a.m2l_bps ? a.m2l_bps : 12));
        if (adj)
            k_m2l<true><<<grid, 64, shM, st>>>(b0, b1, d.box_level, d.v_ptr, d.v_src, d.v_code, d.x_ptr, d.x_src,
                                               d.x_code, tb.dpow_a, tb.logd, tb.binom, op.x, vin, d.leaf_box, first,
                                               second, NP, P1, a.half_L, m2l_tri);
        else
            k_m2l<false><<<grid, 64, shM, st>>>(b0, b1, d.box_level, d.v_ptr, d.v_src, d.v_code, d.x_ptr, d.x_src,
                                                d.x_code, tb.dpow_f, tb.logd, tb.binom, op.x, vin, d.leaf_box, first,
                                                second, NP, P1, a.half_L, m2l_tri);
        for (int lv = 3; lv < h.nlevels; lv++) {
            int64_t c0 = h.level_start[lv], c1 = h.level_start[lv + 1];
            k_shift_down<<<grid_for(c1 - c0), 64, sizeof(double2) * P1, st>>>(c0, c1, d.box_parent, d.box_ix,
                                                                              d.box_iy, op.par, second, P1);
        }
    }
    // leafB: own expansion = second (local / adjoint multipole), W sources and
    // near log aux = first (multipole / adjoint local)
    if (ev) cudaEventRecord(ev[4], st);
    const int32_t *wp = far ? d.w_ptr : d.zero_ptr, *np_ = near ? d.near_ptr : d.zero_ptr;
    if (adj)
        k_leaf_out<true><<<grid_for(a.nleaf, 152 * (a.leaf_bps ? a.leaf_bps : 16)), NP, shD, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level, wp,
                                                            d.w_src, d.w_code, np_, d.near_src, d.near_tab, op.e,
                                                            op.w, op.t, tb.wvec, second, first, first, vin, vout, NP,
                                                            P1, a.half_L, far, Pnear);
    else
        k_leaf_out<false><<<grid_for(a.nleaf, 152 * (a.leaf_bps ? a.leaf_bps : 16)), NP, shD, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                                                             wp, d.w_src, d.w_code, np_, d.near_src,
                                                             d.near_tab, op.e, op.w, op.t, tb.wvec, second, first,
                                                             first, vin, vout, NP, P1, a.half_L, far, Pnear);
    if (ev) cudaEventRecord(ev[5], st);
    return cudaGetLastError();
}

cudaError_t launch_batch_copy(const BatchPtrs &bp, bool gather, double *union_buf, int NP, cudaStream_t st)
{
    const int64_t total = (bp.off[bp.n] - bp.off[0]) * NP;
    if (total <= 0) return cudaSuccess;
    const int grid = int(std::min<int64_t>((total + 255) / 256, 152 * 8));
    k_batch_copy<<<grid, 256, 0, st>>>(bp, gather, union_buf, NP);
    return cudaGetLastError();
}

cudaError_t launch_eval_points(const PassArgs &a, const DevTree &d, const double *u, const double *xy, int64_t n,
                               double *out, double x0, double y0, double L, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int grid = int(std::min<int64_t>((n + 255) / 256, 152 * 8));
    k_eval_points<<<grid, 256, 0, st>>>(n, xy, u, d.box_child0, d.box_leaf, d.box_level, d.box_ix, d.box_iy, x0,
                                        y0, L, a.p, out);
    return cudaGetLastError();
}

}  // namespace bc
