// FMM evaluation of the glue layer potential at every leaf node of a tree.
//
// The glue step of the solver (Sec. 3.4) patches the bulk and strip
// solutions together with v_glue = S[sigma] - D[tau] on the fictitious curve,
// a single-layer and a double-layer Laplace potential with Phi = (1/2pi)
// log(1/|x - y|); discretised on the curve's quadrature nodes y_j (weights
// w_j, unit normals n_j) with q_j = w_j sigma_j and m_j = w_j tau_j n_j:
//
//   u(x) = -(1/2pi) sum_j [ q_j log|x - y_j| + Re(m_j / (x - y_j)) ]
//
// (points as complex numbers; Re(m / (x - y)) = m.(x - y)/|x - y|^2).  The
// sources are point charges and dipoles; the far field runs through the same
// expansions, lists and level passes as the volume potential (multipoles in
// the scaled form of the leaf-to-expansion step, M2M, M2L, L2L), with these
// point-source steps around them:
//   P2M  (leaf box of centre c, half-side r, eta = (y - c)/r):
//        M_0 = sum c_q,  M_k = sum [ -c_q eta^k / k + (c_m / r) eta^(k-1) ]
//   P2L  (X list: source leaf c, target box b one level finer, e = (c_b - c_c)/r_c,
//        w = e - eta, the target's own coordinate rho = (x - c_b)/r_b):
//        L_0 = sum [ c_q log|w| + (c_m / r_c) / w ]     (c_q log r_c: downward pass)
//        L_l = sum (-1)^l (2w)^-l [ -c_q / l + (c_m / r_c) / w ]
//   M2P  (W list) and L2P as for the volume potential, near field direct;
// with c_q = -q / (2 pi), c_m = -m / (2 pi).  A source that coincides with a
// target node contributes nothing.  FP64 throughout, except the split option's
// L2P (the volume apply's group-E tensor tiles over the same locals).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "bc_internal.h"

namespace bc {
namespace {

constexpr double kInvTwoPi = 0.159154943091895335768883763372514362;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cinv(double2 a)
{
    const double d = 1.0 / fma(a.x, a.x, a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
}
// ---------------------------------------------------------------------------
// log x and 1/x for the direct near sums, written for this GPU's FP64 rate
// (1/64 of FP32): a table-driven logarithm after Tang (ACM TOMS 16, 1990).
// With x = 2^e m, m in [1, 2), and j the top kLogBits bits of m's fraction,
// c_j is a short (9-bit) approximation of 1 / (1 + (j + 1/2) / 2^kLogBits)
// (c_0 = 1), so that r = m c_j - 1 is one FMA with a single rounding and
// |r| < 0.008; then
//     log x = e ln 2 - log c_j + log1p(r),  log1p(r) = r - r^2/2 + ... + r^7/7,
//     1/x   = 2^-e c_j / (1 + r),           1/(1 + r) = 1 - r + ... - r^7,
// both series truncated below 2e-17 relative.  ln 2 is split so that e ln2_hi
// is exact (42 bits); -log c_j is stored as a double-double.  About 13 FP64
// operations for the logarithm and 8 for the reciprocal.  Valid for normal x
// with 1/x normal (|e| <= 1021), which the near sums' squared distances meet.
// Table: g_logtab[4 j + 0..2] = c_j, hi, lo of -log c_j; [4 kLogN + 0..1] =
// ln2_hi, ln2_lo (set by layer_log_init).
// ---------------------------------------------------------------------------
constexpr int kLogBits = 7, kLogN = 1 << kLogBits, kLogTabLen = 4 * kLogN + 2;
__device__ double g_logtab[kLogTabLen];

__device__ __forceinline__ void log_inv(double x, const double *__restrict__ tab, double &lg, double &inv)
{
    const long long bits = __double_as_longlong(x);
    const int e = int(bits >> 52) - 1023;   // x > 0
    const int j = int((bits >> (52 - kLogBits)) & (kLogN - 1));
    const double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    const double c = tab[4 * j], Lh = tab[4 * j + 1], Ll = tab[4 * j + 2];
    const double r = fma(m, c, -1.0);
    double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);   // log1p(r) = r + r^2 q(r)
    q = fma(q, r, 0.2);
    q = fma(q, r, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double ed = double(e);
    lg = fma(ed, tab[4 * kLogN], Lh) + (fma(r * r, q, fma(ed, tab[4 * kLogN + 1], Ll)) + r);
    double s = 1.0 - r;   // 1 / (1 + r)
#pragma unroll
    for (int k = 0; k < 6; k++) s = fma(s, -r, 1.0);
    inv = __longlong_as_double(__double_as_longlong(c * s) - (static_cast<long long>(e) << 52));
}

__global__ void k_log_inv_check(const double *__restrict__ x, int64_t n, double *__restrict__ lg,
                                double *__restrict__ inv)
{
    __shared__ double tab[kLogTabLen];
    for (int i = threadIdx.x; i < kLogTabLen; i += blockDim.x) tab[i] = g_logtab[i];
    __syncthreads();
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        double a, b;
        log_inv(x[i], tab, a, b);
        lg[i] = a;
        inv[i] = b;
    }
}

struct BoxGeom {
    double cx, cy, r;
};
__device__ __forceinline__ BoxGeom box_geom(int b, const int32_t *box_level, const int32_t *box_ix,
                                            const int32_t *box_iy, double x0, double y0, double L)
{
    const double h = ldexp(L, -box_level[b]);
    return {x0 + (box_ix[b] + 0.5) * h, y0 + (box_iy[b] + 0.5) * h, 0.5 * h};
}

// the strengths in sorted order, scaled by -1/(2 pi)
__global__ void k_layer_gather(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ q,
                               const double *__restrict__ m, double *__restrict__ cq, double2 *__restrict__ cm)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = perm[i];
        cq[i] = -kInvTwoPi * q[j];
        cm[i] = make_double2(-kInvTwoPi * m[2 * j], -kInvTwoPi * m[2 * j + 1]);
    }
}

// Sum over the warp of each coefficient k < P1 (butterfly, the same order on
// every lane); lane k writes coefficient k to out[k].
template <int PMAX>
__device__ __forceinline__ void warp_sum_store(double2 (&acc)[PMAX], int P1, int lane, double2 *__restrict__ out)
{
#pragma unroll
    for (int k = 0; k < PMAX; k++) {
        if (k < P1) {   // uniform over the warp
            double re = acc[k].x, im = acc[k].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, o);
                im += __shfl_xor_sync(0xffffffffu, im, o);
            }
            if (lane == k) out[k] = make_double2(re, im);
        }
    }
}

// P2M: one warp per leaf, lane s the sources s, s + 32, ... of the leaf; each
// lane carries eta^k up the coefficients (one complex multiplication per
// term), then the warp sums each coefficient.  Every leaf box is written
// (zero without sources: the climb reads all children).  P1 <= PMAX.
template <int PMAX>
__global__ void __launch_bounds__(128)
k_layer_p2m(int64_t nleaf, const int32_t *__restrict__ src_ptr, const double2 *__restrict__ sxy,
            const double *__restrict__ cq, const double2 *__restrict__ cm, const int32_t *__restrict__ leaf_box,
            const int32_t *__restrict__ box_level, const int32_t *__restrict__ box_ix,
            const int32_t *__restrict__ box_iy, double x0, double y0, double L, int P1, double2 *__restrict__ ex)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t leaf = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5); leaf < nleaf; leaf += nw) {
        const int b = leaf_box[leaf];
        const int j0 = src_ptr[leaf], j1 = src_ptr[leaf + 1];
        if (j0 == j1) {   // most leaves: no source, no sums to form (uniform over the warp)
            for (int k = lane; k < P1; k += 32) ex[int64_t(b) * P1 + k] = make_double2(0.0, 0.0);
            continue;
        }
        const BoxGeom g = box_geom(b, box_level, box_ix, box_iy, x0, y0, L);
        const double ir = 1.0 / g.r;
        double2 acc[PMAX];
#pragma unroll
        for (int k = 0; k < PMAX; k++) acc[k] = make_double2(0.0, 0.0);
        for (int j = j0 + lane; j < j1; j += 32) {
            const double2 y = sxy[j];
            const double2 eta = make_double2((y.x - g.cx) * ir, (y.y - g.cy) * ir);
            const double c = cq[j];
            const double2 cmr = make_double2(cm[j].x * ir, cm[j].y * ir);   // c_m / r
            acc[0].x += c;
            double2 pw = make_double2(1.0, 0.0);   // eta^(k-1)
#pragma unroll
            for (int k = 1; k < PMAX; k++) {
                if (k < P1) {
                    const double2 d = cmul(cmr, pw);
                    pw = cmul(pw, eta);
                    const double ck = -c * (1.0 / double(k));
                    acc[k].x += fma(ck, pw.x, d.x);
                    acc[k].y += fma(ck, pw.y, d.y);
                }
            }
        }
        warp_sum_store(acc, P1, lane, ex + int64_t(b) * P1);
    }
}

// P2L of the X list: one warp per entry, lane s the sources s, s + 32, ... of
// the source leaf; each lane carries t^l = (-1/(2w))^l up the coefficients,
// then the warp sums each coefficient.  P1 <= PMAX.
template <int PMAX>
__global__ void __launch_bounds__(128)
k_layer_p2l(int64_t nx, const int32_t *__restrict__ x_box, const int32_t *__restrict__ x_src,
            const int32_t *__restrict__ src_ptr, const double2 *__restrict__ sxy, const double *__restrict__ cq,
            const double2 *__restrict__ cm, const int32_t *__restrict__ leaf_box,
            const int32_t *__restrict__ box_level, const int32_t *__restrict__ box_ix,
            const int32_t *__restrict__ box_iy, double x0, double y0, double L, int P1, double2 *__restrict__ PX)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t x = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5); x < nx; x += nw) {
        const int leaf = x_src[x];
        const BoxGeom gc = box_geom(leaf_box[leaf], box_level, box_ix, box_iy, x0, y0, L);
        const BoxGeom gb = box_geom(x_box[x], box_level, box_ix, box_iy, x0, y0, L);
        const double ir = 1.0 / gc.r;
        const double2 e = make_double2((gb.cx - gc.cx) * ir, (gb.cy - gc.cy) * ir);
        double2 acc[PMAX];
#pragma unroll
        for (int l = 0; l < PMAX; l++) acc[l] = make_double2(0.0, 0.0);
        for (int j = src_ptr[leaf] + lane; j < src_ptr[leaf + 1]; j += 32) {
            const double2 y = sxy[j];
            const double2 w = make_double2(e.x - (y.x - gc.cx) * ir, e.y - (y.y - gc.cy) * ir);
            const double2 iw = cinv(w);
            const double2 dm = cmul(make_double2(cm[j].x * ir, cm[j].y * ir), iw);   // (c_m / r_c) / w
            const double c = cq[j];
            acc[0].x += fma(c, 0.5 * log(fma(w.x, w.x, w.y * w.y)), dm.x);
            acc[0].y += dm.y;
            const double2 t = make_double2(-0.5 * iw.x, -0.5 * iw.y);   // -1 / (2w)
            double2 pw = make_double2(1.0, 0.0);
#pragma unroll
            for (int l = 1; l < PMAX; l++) {
                if (l < P1) {
                    pw = cmul(pw, t);
                    const double2 v = cmul(pw, make_double2(dm.x - c * (1.0 / double(l)), dm.y));
                    acc[l].x += v.x;
                    acc[l].y += v.y;
                }
            }
        }
        warp_sum_store(acc, P1, lane, PX + x * P1);
    }
}

// Leaf output: one block of NP threads per target leaf, thread j its node.
// u = L2P of the leaf's local expansion (levels >= 2; PE: its row from the
// tensor-core tiles, else in FP64 here) + the W list's
// multipoles at the nodes (M2P, with the log r term of the target level) +
// the direct sum over the sources of the leaf's near leaves.
constexpr int kSrcChunk = 128;
__global__ void __launch_bounds__(256)
k_layer_out(int64_t nleaf, const int32_t *__restrict__ order, const int32_t *__restrict__ leaf_box,
            const int32_t *__restrict__ box_level, const int32_t *__restrict__ box_ix,
            const int32_t *__restrict__ box_iy, double x0, double y0, double L, const int32_t *__restrict__ w_ptr,
            const int32_t *__restrict__ w_src, const int32_t *__restrict__ w_code,
            const int32_t *__restrict__ n_ptr, const int32_t *__restrict__ n_src,
            const int32_t *__restrict__ src_ptr, const double2 *__restrict__ sxy, const double *__restrict__ cq,
            const double2 *__restrict__ cm, const double2 *__restrict__ OpE, const double2 *__restrict__ OpW,
            const double2 *__restrict__ loc, const double2 *__restrict__ mul, const double *__restrict__ lvtab,
            int p, int P1, double *__restrict__ u, const double *__restrict__ PE)
{
    const int NP = p * p, j = threadIdx.x;
    __shared__ double2 se[32];
    __shared__ double2 s_xy[kSrcChunk], s_m[kSrcChunk];
    __shared__ double s_q[kSrcChunk];
    __shared__ double s_log[kLogTabLen];
    for (int i = j; i < kLogTabLen; i += blockDim.x) s_log[i] = g_logtab[i];   // read after the first barrier below
    const double pi = 3.14159265358979323846;
    const double xj = -cos((2.0 * (j % p) + 1.0) * pi / (2.0 * p)), yj = -cos((2.0 * (j / p) + 1.0) * pi / (2.0 * p));
    for (int64_t li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int o = order[li];
        const int b = leaf_box[o];
        const int lvo = box_level[b];
        const BoxGeom g = box_geom(b, box_level, box_ix, box_iy, x0, y0, L);
        const double zx = g.cx + g.r * xj, zy = g.cy + g.r * yj;
        double acc = 0.0;
        if (lvo >= 2 && PE) {
            acc = PE[int64_t(o) * NP + j];   // the L2P from the tensor cores
        } else if (lvo >= 2) {
            __syncthreads();
            for (int i = j; i < P1; i += blockDim.x) se[i] = loc[int64_t(b) * P1 + i];
            __syncthreads();
            double a1 = 0.0;
            int l = 0;
            for (; l + 1 < P1; l += 2) {
                const double2 op0 = OpE[l * NP + j], c0 = se[l], op1 = OpE[(l + 1) * NP + j], c1 = se[l + 1];
                acc = fma(op0.x, c0.x, fma(-op0.y, c0.y, acc));
                a1 = fma(op1.x, c1.x, fma(-op1.y, c1.y, a1));
            }
            if (l < P1) {
                const double2 op = OpE[l * NP + j], c = se[l];
                acc = fma(op.x, c.x, fma(-op.y, c.y, acc));
            }
            acc += a1;
        }
        double lw = 0.0;
        for (int e = w_ptr[o]; e < w_ptr[o + 1]; e++) {
            const double2 *op = OpW + size_t(w_code[e]) * P1 * NP;
            __syncthreads();
            for (int i = j; i < P1; i += blockDim.x) se[i] = mul[int64_t(w_src[e]) * P1 + i];
            __syncthreads();
            for (int k = 0; k < P1; k++) {
                const double2 opk = op[k * NP + j], c = se[k];
                acc = fma(opk.x, c.x, fma(-opk.y, c.y, acc));
            }
            lw += se[0].x;
        }
        acc = fma(lvtab[kLvTab + lvo], lw, acc);
        // near field, sources staged in chunks
        double near = 0.0;
        for (int e = n_ptr[o]; e < n_ptr[o + 1]; e++) {
            const int s = n_src[e];
            for (int c0 = src_ptr[s]; c0 < src_ptr[s + 1]; c0 += kSrcChunk) {
                const int cnt = min(kSrcChunk, src_ptr[s + 1] - c0);
                __syncthreads();
                for (int i = j; i < cnt; i += blockDim.x) {
                    s_xy[i] = sxy[c0 + i];
                    s_q[i] = 0.5 * cq[c0 + i];   // c_q log|x - y| = (c_q / 2) log r^2
                    s_m[i] = cm[c0 + i];
                }
                __syncthreads();
                for (int i = 0; i < cnt; i++) {
                    const double dx = zx - s_xy[i].x, dy = zy - s_xy[i].y;
                    const double r2 = fma(dx, dx, dy * dy);
                    if (r2 > 0.0) {
                        double lg, ir2;
                        log_inv(r2, s_log, lg, ir2);
                        near = fma(s_q[i], lg, near);
                        near = fma(fma(s_m[i].x, dx, s_m[i].y * dy), ir2, near);
                    }
                }
            }
        }
        u[int64_t(o) * NP + j] = acc + near;
    }
}

inline int grid_cap(int64_t n, int cap) { return int(n < cap ? (n > 0 ? n : 1) : cap); }

}  // namespace

cudaError_t layer_log_init()
{
    // c_j (9 bits), -log c_j as hi + lo from the host's extended-precision
    // logarithm, and ln 2 split so that its high part has 42 bits
    double t[kLogTabLen] = {};
    for (int j = 0; j < kLogN; j++) {
        const double F = 1.0 + (j + 0.5) / kLogN;
        const double c = j == 0 ? 1.0 : std::nearbyint(512.0 / F) / 512.0;
        const long double L = -logl(static_cast<long double>(c));
        t[4 * j] = c;
        t[4 * j + 1] = static_cast<double>(L);
        t[4 * j + 2] = static_cast<double>(L - static_cast<long double>(t[4 * j + 1]));
    }
    const long double ln2 = logl(2.0L);
    long long b;
    const double l2 = static_cast<double>(ln2);
    std::memcpy(&b, &l2, sizeof b);
    b &= ~((1ll << 11) - 1);
    double l2h;
    std::memcpy(&l2h, &b, sizeof b);
    t[4 * kLogN] = l2h;
    t[4 * kLogN + 1] = static_cast<double>(ln2 - static_cast<long double>(l2h));
    return cudaMemcpyToSymbol(g_logtab, t, sizeof t);
}

cudaError_t launch_log_inv_check(const double *x, int64_t n, double *lg, double *inv, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int grid = int(std::min<int64_t>((n + 255) / 256, 152 * 8));
    k_log_inv_check<<<grid, 256, 0, st>>>(x, n, lg, inv);
    return cudaGetLastError();
}

cudaError_t launch_layer(const PassArgs &a, const HostTree &h, const DevTree &d, const DevTables &tb,
                         const LayerDev &ly, const double *q, const double *m, double *u, cudaStream_t st,
                         const SplitLaunch *split)
{
    cudaError_t e;
    const int P1 = a.P1;
    if (ly.n > 0) {
        k_layer_gather<<<grid_cap((ly.n + 255) / 256, 152 * 8), 256, 0, st>>>(ly.n, ly.perm, q, m, ly.cq, ly.cm);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_layer_p2m<32><<<grid_cap((a.nleaf + 3) / 4, 152 * 8), 128, 0, st>>>(
        a.nleaf, ly.src_ptr, ly.sxy, ly.cq, ly.cm, d.leaf_box, d.box_level, d.box_ix, d.box_iy, h.x0, h.y0, h.L, P1,
        d.expA);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ly.nx > 0) {
        k_layer_p2l<32><<<grid_cap((ly.nx + 3) / 4, 152 * 8), 128, 0, st>>>(
            ly.nx, ly.x_box, ly.x_src, ly.src_ptr, ly.sxy, ly.cq, ly.cm, d.leaf_box, d.box_level, d.box_ix, d.box_iy,
            h.x0, h.y0, h.L, P1, ly.PX);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    FarLists fl;
    fl.v_ptr = ly.v_ptr; fl.v_src = ly.v_src; fl.v_code = ly.v_code;
    fl.x_ptr = ly.x_ptr; fl.x_src = ly.x_src; fl.PX = ly.PX;
    fl.live = ly.live;
    if ((e = launch_far_points(a, h, d, tb, fl, st)) != cudaSuccess) return e;
    const double *PE = nullptr;
    if (split) {
        // L2P of every leaf at level >= 2 on the tensor cores: digits of the
        // locals (expB, the forward apply's second array), then the forward
        // group-E tiles that evaluate them at the leaf nodes, into PE
        const SplitTables *sT = split->tables;
        const SplitTree *sp = split->tree;
        const int64_t nbox = a.nbox;
        e = launch_split_digits_exp(nbox, 2 * nbox, nbox, d.expA, d.expB, P1, 1.0, sT->escale[0], sp->edig,
                                    sp->eexp, st);
        if (e != cudaSuccess) return e;
        SplitGemm g;
        g.tiles = sp->tE[0]; g.cols = sp->cE[0]; g.ntiles = sp->ntL[0];
        g.ops = sT->ops[1][0]; g.op_exp = sT->op_exp[1][0];
        g.dig = sp->edig; g.dexp = sp->eexp;
        e = launch_split_gemm(g, kSplitKE, 1.0 / (a.half_L * a.half_L), sp->err, sT->wait_limit, sT->withhold_copy,
                              st);
        if (e != cudaSuccess) return e;
        PE = sp->PE;
    }
    k_layer_out<<<grid_cap(a.nleaf, 152 * 8), a.NP, 0, st>>>(
        a.nleaf, ly.order, d.leaf_box, d.box_level, d.box_ix, d.box_iy, h.x0, h.y0, h.L, ly.w_ptr, ly.w_src,
        ly.w_code, ly.n_ptr, ly.n_src, ly.src_ptr, ly.sxy, ly.cq, ly.cm, tb.fwd.e, tb.fwd.w, d.expB, d.expA, d.lvtab,
        a.p, P1, u, PE);
    return cudaGetLastError();
}

}  // namespace bc
