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

constexpr double kInvTwoPi = 0.15915494309189533576888376337251;   // 1 / (2 pi)

// Per-level constants of the tree (no FP64 log or divide in the kernels):
// lvtab[lv] = r_lv^2, lvtab[kLvTab + lv] = log r_lv, r_lv = (L/2) 2^-lv.

// -------------------------------------------------------------------------
// Grid-wide barrier of the persistent level-synchronous passes.  Their grids
// are sized so that every block is resident (occupancy calculator), so the
// wait ends once all blocks arrive; it is bounded all the same: a block whose
// wait runs out records the failure in *err (reported by bc_sync) and goes on.
// bar[0] counts arrivals, bar[1] is the generation.  Data written before the
// barrier is read after it with L2 loads (__ldcg).
// -------------------------------------------------------------------------
__device__ void grid_sync(uint32_t *bar, long long limit, int32_t *err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *vb = bar;
        const uint32_t gen = vb[1];
        __threadfence();
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            for (long long it = 0; vb[1] == gen; it++) {
                if (it >= limit) {
                    atomicExch(err, 2);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// -------------------------------------------------------------------------
// upward pass, one persistent launch:
//   leaves: ex[box(leaf)][l] = s * sum_j OpA[j][l] v[leaf][j]
//           forward (P2M): OpA = Q^T, s = r^2;  adjoint (L2P^H): OpA = E^H, s = 1
//           (OpA == nullptr: the leaf expansions are already in ex, split path)
//   then level by level, deepest first, separated by grid barriers:
//   parent: ex[p][l] = sum_q sum_k OpUp[q][k][l] ex[child_q(p)][k]    (levels >= 2)
//           forward: M2M; adjoint: L2L^H
// Four warps per block: in the leaf step warp w sums over the w-th quarter of
// the nodes, in a parent step warp q applies the operator of child q; the four
// partial sums meet in shared memory.
// -------------------------------------------------------------------------
template <bool ADJ>
__global__ void __launch_bounds__(128)
k_up_levels(int64_t nleaf, const int32_t *__restrict__ order, const int32_t *__restrict__ leaf_box,
            const int32_t *__restrict__ leaf_level, const int64_t *__restrict__ level_start, int nlevels,
            const int32_t *__restrict__ box_child0, const double *__restrict__ vin,
            const double2 *__restrict__ OpA, const double2 *__restrict__ OpUp, double2 *ex, int NP, int P1,
            const double *__restrict__ lvtab, bool climb, uint32_t *gbar, long long limit, int32_t *err)
{
    extern __shared__ double2 shu[];
    double2 *sc = shu;                                       // 4 * P1 children
    double2 *part = sc + 4 * P1;                             // [4][P1] partial sums
    double *sv = reinterpret_cast<double *>(part + 4 * P1);  // NP
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = NP / 4;
    for (int64_t li = blockIdx.x; OpA && li < nleaf; li += gridDim.x) {
        const int leaf = order[li];
        const int b = leaf_box[leaf];
        const double s = ADJ ? 1.0 : lvtab[leaf_level[leaf]];   // r^2
        __syncthreads();
        for (int j = threadIdx.x; j < NP; j += blockDim.x) sv[j] = vin[int64_t(leaf) * NP + j];
        __syncthreads();
        for (int l = lane; l < P1; l += 32) {
            double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
            for (int j = w * nq; j < (w + 1) * nq; j += 2) {
                double2 o0 = OpA[j * P1 + l], o1 = OpA[(j + 1) * P1 + l];
                re0 = fma(o0.x, sv[j], re0);
                im0 = fma(o0.y, sv[j], im0);
                re1 = fma(o1.x, sv[j + 1], re1);
                im1 = fma(o1.y, sv[j + 1], im1);
            }
            part[w * P1 + l] = make_double2(re0 + re1, im0 + im1);
        }
        __syncthreads();
        for (int l = threadIdx.x; l < P1; l += blockDim.x) {
            const double2 a0 = part[l], a1 = part[P1 + l], a2 = part[2 * P1 + l], a3 = part[3 * P1 + l];
            ex[int64_t(b) * P1 + l] =
                make_double2(s * ((a0.x + a1.x) + (a2.x + a3.x)), s * ((a0.y + a1.y) + (a2.y + a3.y)));
        }
    }
    if (!climb) return;
    for (int lv = nlevels - 2; lv >= 2; lv--) {
        grid_sync(gbar, limit, err);   // every box of the levels below is complete
        for (int64_t p = level_start[lv] + blockIdx.x; p < level_start[lv + 1]; p += gridDim.x) {
            const int c0 = box_child0[p];
            if (c0 < 0) continue;   // a leaf (uniform over the block)
            __syncthreads();
            for (int i = threadIdx.x; i < 4 * P1; i += blockDim.x) sc[i] = __ldcg(&ex[int64_t(c0) * P1 + i]);
            __syncthreads();
            const double2 *op = OpUp + size_t(w) * P1 * P1;
            const double2 *a = sc + w * P1;
            for (int l = lane; l < P1; l += 32) {
                double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
                for (int k0 = 0; k0 < P1; k0 += 8) {   // 8 operator loads in flight
                    double2 o[8];
#pragma unroll
                    for (int u = 0; u < 8; u++)
                        o[u] = k0 + u < P1 ? __ldg(&op[(k0 + u) * P1 + l]) : make_double2(0.0, 0.0);
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        if (k0 + u >= P1) break;
                        const double2 a0 = a[k0 + u], a1 = k0 + u + 1 < P1 ? a[k0 + u + 1] : make_double2(0.0, 0.0);
                        re0 = fma(o[u].x, a0.x, fma(-o[u].y, a0.y, re0));
                        im0 = fma(o[u].x, a0.y, fma(o[u].y, a0.x, im0));
                        re1 = fma(o[u + 1].x, a1.x, fma(-o[u + 1].y, a1.y, re1));
                        im1 = fma(o[u + 1].x, a1.y, fma(o[u + 1].y, a1.x, im1));
                    }
                }
                part[w * P1 + l] = make_double2(re0 + re1, im0 + im1);
            }
            __syncthreads();
            for (int l = threadIdx.x; l < P1; l += blockDim.x) {
                const double2 a0 = part[l], a1 = part[P1 + l], a2 = part[2 * P1 + l], a3 = part[3 * P1 + l];
                ex[int64_t(p) * P1 + l] = make_double2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
            }
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
      double2 *out, int NP, int P1, const double *__restrict__ lvtab, int tri, const double *__restrict__ PX)
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
            const double logr = lvtab[kLvTab + lv];
            orr += logr * (mono[0].x + mono[1].x);
            oi += logr * (mono[0].y + mono[1].y);
        }
        // X list: leaf densities (forward) / leaf adjoint data (adjoint) of the
        // coarser neighbour leaves.  The log term uses coefficient 0 of the
        // leaf's own expansion from the upward pass: forward A_0 = r_c^2 (w.f)/2pi,
        // adjoint B_0 = sum_j g_j, so the term is log(r_c) * that coefficient.
        const double s1 = ADJ ? 1.0 : lvtab[lv - 1];   // r_c^2
        const double logrc = lvtab[kLvTab + lv - 1];
        for (int e = x_ptr[b]; e < x_ptr[b + 1] && PX; e++) {
            // split path: the scaled product s1 * OpX x[c] comes from the tensor cores
            if (tid < P1) {
                orr += PX[size_t(e) * kSplitKE + 2 * tid];
                oi += PX[size_t(e) * kSplitKE + 2 * tid + 1];
                if (tid == 0) orr = fma(logrc, in[int64_t(leaf_box[x_src[e]]) * P1].x, orr);
            }
        }
        for (int e = x_ptr[b]; e < x_ptr[b + 1] && !PX; e++) {
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
// shift_levels: out[b] += Par_q * out[parent(b)] for every box of level >= 3,
// level by level (one persistent launch, grid barriers between levels)
//   forward: L2L; adjoint: M2M^H.  Two independent FMA chains per thread.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(64)
k_shift_levels(const int64_t *__restrict__ level_start, int nlevels, const int32_t *__restrict__ parent,
               const int32_t *__restrict__ box_ix, const int32_t *__restrict__ box_iy,
               const double2 *__restrict__ OpPar, double2 *out, int P1, uint32_t *gbar, long long limit,
               int32_t *err)
{
    extern __shared__ double2 se[];
    for (int lv = 3; lv < nlevels; lv++) {
        if (lv > 3) grid_sync(gbar, limit, err);   // the parents' level is complete
        for (int64_t b = level_start[lv] + blockIdx.x; b < level_start[lv + 1]; b += gridDim.x) {
            const int pb = parent[b];
            const int q = (box_ix[b] & 1) + 2 * (box_iy[b] & 1);
            __syncthreads();
            for (int i = threadIdx.x; i < P1; i += blockDim.x) se[i] = __ldcg(&out[int64_t(pb) * P1 + i]);
            __syncthreads();
            for (int l = threadIdx.x; l < P1; l += blockDim.x) {
                const double2 *op = OpPar + size_t(q) * P1 * P1;
                const double2 acc = __ldcg(&out[b * P1 + l]);
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
                           double *__restrict__ vout, int NP, int P1, const double *__restrict__ lvtab, bool far,
                           const double *__restrict__ Pnear, const double *__restrict__ PE,
                           const double *__restrict__ PW)
{
    extern __shared__ double2 sh[];
    double2 *se = sh;                                  // P1
    double *sv = reinterpret_cast<double *>(sh + P1);  // NP
    for (int64_t li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int o = order[li];
        const int lvo = leaf_level[o];
        const double r2o = lvtab[lvo], lgo = lvtab[kLvTab + lvo];
        const int j = threadIdx.x;   // blockDim.x == NP
        const double wj = wvec[j];
        // adjoint log term of a target leaf o: r_o^2 log(r_o) w_j / (2 pi)
        const double cO = ADJ ? r2o * lgo * wj * kInvTwoPi : lgo;
        double acc = 0.0;
        if (far && lvo >= 2 && PE) {
            acc = PE[int64_t(o) * NP + j];   // split path: scaled L2P from the tensor cores
        } else if (far && lvo >= 2) {
            __syncthreads();
            for (int i = threadIdx.x; i < P1; i += blockDim.x) se[i] = own[int64_t(leaf_box[o]) * P1 + i];
            __syncthreads();
            double s = 0.0;
            for (int l = 0; l < P1; l++) {
                double2 op = OpE[l * NP + j], b = se[l];
                s = fma(op.x, b.x, fma(-op.y, b.y, s));
            }
            acc = ADJ ? r2o * s : s;
        }
        const double sW = ADJ ? r2o : 1.0;
        const double cW = cO;
        for (int e = w_ptr[o]; e < w_ptr[o + 1] && PW; e++)
            acc = PW[size_t(e) * NP + j] + fma(cW, src[int64_t(w_src[e]) * P1].x, acc);
        for (int e = w_ptr[o]; e < w_ptr[o + 1] && !PW; e++) {
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
                sN = r2o;
                cN = cO;
            } else {
                const int ls = leaf_level[s];
                sN = lvtab[ls];
                cN = lvtab[kLvTab + ls];
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
    const OpSet &op = adj ? tb.adj : tb.fwd;
    const int NP = a.NP, P1 = a.P1, dir = adj ? 1 : 0;
    double2 *first = adj ? d.expB : d.expA;    // leafA / up target
    double2 *second = adj ? d.expA : d.expB;   // down target
    const double alpha0 = a.half_L * a.half_L;  // r^2 at level 0
    const SplitTables *sT = split ? split->tables : nullptr;
    const SplitTree *sp = split ? split->tree : nullptr;
    const int parts = split ? split->parts : 0;
    cudaError_t ce;
    if (ev) cudaEventRecord(ev[0], st);
    if (split) {
        // tensor group V: digits of alpha0 * vin; near field, leafA (P2M / L2P^H)
        // into `first`, X list into PX
        ce = launch_split_digits_vec(a.nleaf, vin, alpha0, sp->vdig, sp->vexp, st);
        if (ce != cudaSuccess) return ce;
        SplitGemm g;
        g.tiles = sp->tV[dir]; g.cols = sp->cV[dir]; g.ntiles = sp->ntV[dir];
        g.ops = sT->ops[0][dir]; g.op_exp = sT->op_exp[0][dir];
        g.dig = sp->vdig; g.dexp = sp->vexp;
        ce = launch_split_gemm(g, 256, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, st);
        if (ce != cudaSuccess) return ce;
    }
    if (ev) cudaEventRecord(ev[1], st);
    // the grid barrier of the persistent passes starts from zero (a barrier
    // wait that ran out in an earlier apply cannot leave it out of step)
    ce = cudaMemsetAsync(d.gbar, 0, 2 * sizeof(uint32_t), st);
    if (ce != cudaSuccess) return ce;
    if (ev) cudaEventRecord(ev[2], st);
    // grid-barrier polls go to L2 (about a microsecond each): a sixteenth of
    // the mbarrier poll limit
    const long long glimit = std::max(1ll, a.wait_limit / 16);
    // leafA + upward pass in one persistent launch (leafA always runs: the
    // near-field log term reads coefficient 0 of its output; without the far
    // field no climb).  Split path: leafA came from the tensor cores.
    const size_t shU = sizeof(double) * NP + sizeof(double2) * 8 * P1;
    const int grid_leaf = grid_for(a.nleaf, 152 * (a.leaf_bps ? a.leaf_bps : 16));
    const double2 *opA = (parts & 2) ? nullptr : op.leafA;
    const bool climb = far && h.nlevels > 3;
    if (opA || climb) {
        if (adj)
            k_up_levels<true><<<a.up_blocks, 128, shU, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                                                             d.level_start, h.nlevels, d.box_child0, vin, opA,
                                                             op.up, first, NP, P1, d.lvtab, climb, d.gbar,
                                                             glimit, a.err);
        else
            k_up_levels<false><<<a.up_blocks, 128, shU, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                                                              d.level_start, h.nlevels, d.box_child0, vin, opA,
                                                              op.up, first, NP, P1, d.lvtab, climb, d.gbar,
                                                              glimit, a.err);
    }
    if (ev) cudaEventRecord(ev[3], st);
    if (far && h.nlevels > 2) {
        const int64_t b0 = h.level_start[2], b1 = h.level_start[h.nlevels];
        size_t shM = sizeof(double) * (size_t(P1) * (P1 + 1) + P1) + sizeof(double2) * (128 + 128 + 2) +
                     sizeof(double) * NP;
        int grid = grid_for(b1 - b0, 152 * (a.m2l_bps ? a.m2l_bps : 12));
        const double *PX = (parts & 4) ? sp->PX : nullptr;
        if (adj)
            k_m2l<true><<<grid, 64, shM, st>>>(b0, b1, d.box_level, d.v_ptr, d.v_src, d.v_code, d.x_ptr, d.x_src,
                                               d.x_code, tb.dpow_a, tb.logd, tb.binom, op.x, vin, d.leaf_box, first,
                                               second, NP, P1, d.lvtab, m2l_tri, PX);
        else
            k_m2l<false><<<grid, 64, shM, st>>>(b0, b1, d.box_level, d.v_ptr, d.v_src, d.v_code, d.x_ptr, d.x_src,
                                                d.x_code, tb.dpow_f, tb.logd, tb.binom, op.x, vin, d.leaf_box, first,
                                                second, NP, P1, d.lvtab, m2l_tri, PX);
        if (h.nlevels > 3)
            k_shift_levels<<<a.shift_blocks, 64, sizeof(double2) * P1, st>>>(d.level_start, h.nlevels, d.box_parent,
                                                                            d.box_ix, d.box_iy, op.par, second, P1,
                                                                            d.gbar, glimit, a.err);
    }
    if (ev) cudaEventRecord(ev[4], st);
    if (split && far) {
        // tensor group E: digits of both expansion arrays (times alpha0 in the
        // adjoint), then L2P (P2M^H) of `second` into PE and the W list of
        // `first` into PW
        ce = launch_split_digits_exp(a.nbox, d.expA, d.expB, P1, adj ? alpha0 : 1.0, sT->escale[dir], sp->edig,
                                     sp->eexp, st);
        if (ce != cudaSuccess) return ce;
        SplitGemm g;
        g.tiles = sp->tE[dir]; g.cols = sp->cE[dir]; g.ntiles = sp->ntE[dir];
        g.ops = sT->ops[1][dir]; g.op_exp = sT->op_exp[1][dir];
        g.dig = sp->edig; g.dexp = sp->eexp;
        ce = launch_split_gemm(g, kSplitKE, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, st);
        if (ce != cudaSuccess) return ce;
    }
    if (ev) cudaEventRecord(ev[5], st);
    // leafB: own expansion = second (local / adjoint multipole), W sources and
    // near log aux = first (multipole / adjoint local)
    size_t shD = sizeof(double2) * P1 + sizeof(double) * NP;
    const int32_t *wp = far ? d.w_ptr : d.zero_ptr, *np_ = near ? d.near_ptr : d.zero_ptr;
    const double *Pnear = (parts & 1) ? sp->Pnear : nullptr, *PE = (parts & 8) ? sp->PE : nullptr,
                 *PW = (parts & 16) ? sp->PW : nullptr;
    if (adj)
        k_leaf_out<true><<<grid_leaf, NP, shD, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level, wp, d.w_src,
                                                     d.w_code, np_, d.near_src, d.near_tab, op.e, op.w, op.t,
                                                     tb.wvec, second, first, first, vin, vout, NP, P1, d.lvtab, far,
                                                     Pnear, PE, PW);
    else
        k_leaf_out<false><<<grid_leaf, NP, shD, st>>>(a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level, wp,
                                                      d.w_src, d.w_code, np_, d.near_src, d.near_tab, op.e, op.w,
                                                      op.t, tb.wvec, second, first, first, vin, vout, NP, P1,
                                                      d.lvtab, far, Pnear, PE, PW);
    if (ev) cudaEventRecord(ev[6], st);
    return cudaGetLastError();
}

cudaError_t fp64_prepare(int NP, int P1, int per_sm, int *up_blocks, int *shift_blocks)
{
    int dev = 0, sms = 0, bu0 = 0, bu1 = 0, bs = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t shU = sizeof(double) * NP + sizeof(double2) * 8 * P1;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu0, k_up_levels<false>, 128, shU);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu1, k_up_levels<true>, 128, shU);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_shift_levels, 64, sizeof(double2) * P1);
    if (e != cudaSuccess) return e;
    if (std::min(bu0, bu1) < 1 || bs < 1) return cudaErrorInvalidConfiguration;
    *up_blocks = sms * std::min(per_sm, std::min(bu0, bu1));
    *shift_blocks = sms * std::min(per_sm, bs);
    return cudaSuccess;
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
