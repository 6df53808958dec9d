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
// leafA: out[box(leaf)][l] = s * sum_j Op[j][l] v[leaf][j]
//   forward (P2M): Op = Q^T, s = r^2;  adjoint (L2P^H): Op = E^H, s = 1
// -------------------------------------------------------------------------
template <bool ADJ>
__global__ void k_leaf_to_exp(int64_t nleaf, const int32_t *__restrict__ order,
                              const int32_t *__restrict__ leaf_box, const int32_t *__restrict__ leaf_level,
                              const double *__restrict__ vin, const double2 *__restrict__ Op,
                              double2 *__restrict__ out, int NP, int P1, double half_L)
{
    extern __shared__ double sv[];
    for (int64_t li = blockIdx.x; li < nleaf; li += gridDim.x) {
        int leaf = order[li];
        __syncthreads();
        for (int j = threadIdx.x; j < NP; j += blockDim.x) sv[j] = vin[int64_t(leaf) * NP + j];
        __syncthreads();
        double r = r_at(half_L, leaf_level[leaf]);
        double s = ADJ ? 1.0 : r * r;
        for (int l = threadIdx.x; l < P1; l += blockDim.x) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < NP; j++) {
                double2 o = Op[j * P1 + l];
                re = fma(o.x, sv[j], re);
                im = fma(o.y, sv[j], im);
            }
            out[int64_t(leaf_box[leaf]) * P1 + l] = make_double2(s * re, s * im);
        }
    }
}

// -------------------------------------------------------------------------
// up: exp[b][l] = sum_q sum_k Op[q][k][l] exp[child_q(b)][k]   (non-leaf b)
// -------------------------------------------------------------------------
__global__ void k_up(int64_t b0, int64_t b1, const int32_t *__restrict__ child0,
                     const double2 *__restrict__ Op, double2 *__restrict__ ex, int P1)
{
    extern __shared__ double2 se[];
    for (int64_t b = b0 + blockIdx.x; b < b1; b += gridDim.x) {
        int c0 = child0[b];
        if (c0 < 0) continue;   // leaf: uniform across the block
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * P1; i += blockDim.x) se[i] = ex[int64_t(c0) * P1 + i];
        __syncthreads();
        for (int l = threadIdx.x; l < P1; l += blockDim.x) {
            double re = 0.0, im = 0.0;
            for (int q = 0; q < 4; q++)
                for (int k = 0; k < P1; k++) {
                    double2 o = Op[(q * P1 + k) * P1 + l], a = se[q * P1 + k];
                    re = fma(o.x, a.x, fma(-o.y, a.y, re));
                    im = fma(o.x, a.y, fma(o.y, a.x, im));
                }
            ex[b * P1 + l] = make_double2(re, im);
        }
    }
}

// -------------------------------------------------------------------------
// down: for every box b at one level lv >= 2
//   out[b] = Par_q * out[parent]                  (lv >= 3)
//          + sum_{s in V(b)} OpV[code] * in[s]  ;  out[b][0] += log(r_lv) sum_V in[s][0]
//          + sum_{c in X(b)} s1 * OpX[code] * x[c] ;  out[b][0] += s2 * (lv . x[c])
//   forward: out = local, in = multipole, x = f,  s1 = r_c^2, s2 = r_c^2 log r_c / 2pi, lvec = w
//   adjoint: out = adj. multipole, in = adj. local, x = g, s1 = 1, s2 = log r_c, lvec = 1
//   (r_c = half-side at level lv-1, the level of the X-list leaves)
// -------------------------------------------------------------------------
template <bool ADJ>
__global__ void k_down(int64_t b0, int64_t b1, int lv, const int32_t *__restrict__ parent,
                       const int32_t *__restrict__ box_ix, const int32_t *__restrict__ box_iy,
                       const int32_t *__restrict__ v_ptr, const int32_t *__restrict__ v_src,
                       const int32_t *__restrict__ v_code, const int32_t *__restrict__ x_ptr,
                       const int32_t *__restrict__ x_src, const int32_t *__restrict__ x_code,
                       const double2 *__restrict__ OpPar, const double2 *__restrict__ OpV,
                       const double2 *__restrict__ OpX, const double *__restrict__ xvec,
                       const double *__restrict__ wvec, const double2 *__restrict__ in,
                       double2 *__restrict__ out, int NP, int P1, double half_L)
{
    extern __shared__ double2 sh[];
    double2 *se = sh;                                   // P1
    double *sx = reinterpret_cast<double *>(sh + P1);   // NP
    const double r = r_at(half_L, lv), logr = log(r);
    const double rc = r_at(half_L, lv - 1);
    const double s1 = ADJ ? 1.0 : rc * rc;
    const double s2 = ADJ ? log(rc) : rc * rc * log(rc) / kTwoPi;
    for (int64_t b = b0 + blockIdx.x; b < b1; b += gridDim.x) {
        double re[2] = {0.0, 0.0}, im[2] = {0.0, 0.0};   // two coefficients per thread max (P1 <= 64, 32+ threads)
        const int l0 = threadIdx.x, l1 = threadIdx.x + blockDim.x;
        if (lv >= 3) {
            int pb = parent[b];
            int q = (box_ix[b] & 1) + 2 * (box_iy[b] & 1);
            __syncthreads();
            for (int i = threadIdx.x; i < P1; i += blockDim.x) se[i] = out[int64_t(pb) * P1 + i];
            __syncthreads();
            const double2 *op = OpPar + size_t(q) * P1 * P1;
            for (int k = 0; k < P1; k++) {
                double2 a = se[k];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    int l = u ? l1 : l0;
                    if (l < P1) {
                        double2 o = op[k * P1 + l];
                        re[u] = fma(o.x, a.x, fma(-o.y, a.y, re[u]));
                        im[u] = fma(o.x, a.y, fma(o.y, a.x, im[u]));
                    }
                }
            }
        }
        double mono = 0.0;   // sum of in[s][0] (real part) for the log term
        double mono_i = 0.0;
        for (int e = v_ptr[b]; e < v_ptr[b + 1]; e++) {
            int s = v_src[e];
            const double2 *op = OpV + size_t(v_code[e]) * P1 * P1;
            __syncthreads();
            for (int i = threadIdx.x; i < P1; i += blockDim.x) se[i] = in[int64_t(s) * P1 + i];
            __syncthreads();
            mono += se[0].x;
            mono_i += se[0].y;
            for (int k = 0; k < P1; k++) {
                double2 a = se[k];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    int l = u ? l1 : l0;
                    if (l < P1) {
                        double2 o = op[k * P1 + l];
                        re[u] = fma(o.x, a.x, fma(-o.y, a.y, re[u]));
                        im[u] = fma(o.x, a.y, fma(o.y, a.x, im[u]));
                    }
                }
            }
        }
        double xdot = 0.0;
        for (int e = x_ptr[b]; e < x_ptr[b + 1]; e++) {
            int c = x_src[e];
            const double2 *op = OpX + size_t(x_code[e]) * NP * P1;
            __syncthreads();
            for (int j = threadIdx.x; j < NP; j += blockDim.x) sx[j] = xvec[int64_t(c) * NP + j];
            __syncthreads();
            if (threadIdx.x == 0) {
                double d = 0.0;
                for (int j = 0; j < NP; j++) d = fma(ADJ ? 1.0 : wvec[j], sx[j], d);
                xdot += d;
            }
            double xr[2] = {0.0, 0.0}, xi[2] = {0.0, 0.0};
            for (int j = 0; j < NP; j++) {
                double v = sx[j];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    int l = u ? l1 : l0;
                    if (l < P1) {
                        double2 o = op[j * P1 + l];
                        xr[u] = fma(o.x, v, xr[u]);
                        xi[u] = fma(o.y, v, xi[u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 2; u++) { re[u] = fma(s1, xr[u], re[u]); im[u] = fma(s1, xi[u], im[u]); }
        }
        if (threadIdx.x == 0) {
            re[0] += logr * mono + s2 * xdot;
            im[0] += logr * mono_i;
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
            int l = u ? l1 : l0;
            if (l < P1) out[b * P1 + l] = make_double2(re[u], im[u]);
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
                           double *__restrict__ vout, int NP, int P1, double half_L, bool far)
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
            const double *tb = T + size_t(n_tab[e]) * NP * NP;
            __syncthreads();
            for (int i = threadIdx.x; i < NP; i += blockDim.x) sv[i] = vnear[int64_t(s) * NP + i];
            __syncthreads();
            double t = 0.0;
            for (int k = 0; k < NP; k++) t = fma(tb[k * NP + j], sv[k], t);
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

}  // namespace

cudaError_t launch_apply(const PassArgs &a, const HostTree &h, const DevTree &d, const DevTables &tb,
                         bool adj, const double *vin, double *vout, cudaStream_t st, int pass_mask,
                         cudaEvent_t *ev)
{
    const bool far = (pass_mask & 2) != 0, near = (pass_mask & 1) != 0;
    if (ev) cudaEventRecord(ev[0], st);
    const OpSet &op = adj ? tb.adj : tb.fwd;
    const int NP = a.NP, P1 = a.P1;
    double2 *first = adj ? d.expB : d.expA;    // leafA / up target
    double2 *second = adj ? d.expA : d.expB;   // down target
    const int tA = 64;
    size_t shA = sizeof(double) * NP;
    // leafA always runs: the near-field log term reads coefficient 0 of its output
    if (adj)
        k_leaf_to_exp<true><<<grid_for(a.nleaf), tA, shA, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                                                               vin, op.leafA, first, NP, P1, a.half_L);
    else
        k_leaf_to_exp<false><<<grid_for(a.nleaf), tA, shA, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                                                                vin, op.leafA, first, NP, P1, a.half_L);
    if (ev) cudaEventRecord(ev[1], st);
    for (int lv = h.nlevels - 2; far && lv >= 2; lv--) {
        int64_t b0 = h.level_start[lv], b1 = h.level_start[lv + 1];
        k_up<<<grid_for(b1 - b0), 64, sizeof(double2) * 4 * P1, st>>>(b0, b1, d.box_child0, op.up, first, P1);
    }
    if (ev) cudaEventRecord(ev[2], st);
    size_t shD = sizeof(double2) * P1 + sizeof(double) * NP;
    for (int lv = 2; far && lv < h.nlevels; lv++) {
        int64_t b0 = h.level_start[lv], b1 = h.level_start[lv + 1];
        if (adj)
            k_down<true><<<grid_for(b1 - b0), 32, shD, st>>>(b0, b1, lv, d.box_parent, d.box_ix, d.box_iy, d.v_ptr,
                                                            d.v_src, d.v_code, d.x_ptr, d.x_src, d.x_code, op.par, op.v,
                                                            op.x, vin, tb.wvec, first, second, NP, P1, a.half_L);
        else
            k_down<false><<<grid_for(b1 - b0), 32, shD, st>>>(b0, b1, lv, d.box_parent, d.box_ix, d.box_iy, d.v_ptr,
                                                             d.v_src, d.v_code, d.x_ptr, d.x_src, d.x_code, op.par, op.v,
                                                             op.x, vin, tb.wvec, first, second, NP, P1, a.half_L);
    }
    // leafB: own expansion = second (local / adjoint multipole), W sources and
    // near log aux = first (multipole / adjoint local)
    if (ev) cudaEventRecord(ev[3], st);
    const int32_t *wp = far ? d.w_ptr : d.zero_ptr, *np_ = near ? d.near_ptr : d.zero_ptr;
    if (adj)
        k_leaf_out<true><<<grid_for(a.nleaf), NP, shD, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level, wp,
                                                            d.w_src, d.w_code, np_, d.near_src, d.near_tab, op.e,
                                                            op.w, op.t, tb.wvec, second, first, first, vin, vout, NP,
                                                            P1, a.half_L, far);
    else
        k_leaf_out<false><<<grid_for(a.nleaf), NP, shD, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                                                             wp, d.w_src, d.w_code, np_, d.near_src,
                                                             d.near_tab, op.e, op.w, op.t, tb.wvec, second, first,
                                                             first, vin, vout, NP, P1, a.half_L, far);
    if (ev) cudaEventRecord(ev[4], st);
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
