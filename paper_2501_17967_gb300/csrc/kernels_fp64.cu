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
#include "pdl.h"

namespace bc {

namespace {

constexpr double kInvTwoPi = 0.15915494309189533576888376337251;   // 1 / (2 pi)

// Per-level constants of the tree (no FP64 log or divide in the kernels):
// lvtab[lv] = r_lv^2, lvtab[kLvTab + lv] = log r_lv, r_lv = (L/2) 2^-lv.

// -------------------------------------------------------------------------
// Per-box completion flags of the persistent level passes.  A box's expansion
// is published by flag[box] (1: upward result, 2: downward result) once every
// thread of the producing block has written it; a consumer waits for the
// flags of exactly the boxes it reads (a parent for its children, a box for
// its parent) instead of for a whole level.  Each block takes its boxes in
// dependency order and every block is resident (the grids come from the
// occupancy calculator), so every wait ends; it is bounded all the same: a
// wait that runs out records the failure in *err (reported by bc_sync) and
// goes on.  Data published this way is read with L2 loads (__ldcg).
// -------------------------------------------------------------------------
__device__ __forceinline__ int flag_load(const int32_t *f)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    return v;
}

// called by every thread of the block after the box's expansion is written:
// the barrier orders the block's writes before thread 0's release store,
// which makes them visible at GPU scope to a reader that acquires the flag
__device__ __forceinline__ void flag_publish(int32_t *f, int v)
{
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}

// the calling thread waits until *f >= want
__device__ __forceinline__ void flag_wait(const int32_t *f, int want, long long limit, int32_t *err)
{
    for (long long it = 0; flag_load(f) < want; it++) {
        if (it >= limit) {
            atomicExch(err, 2);
            break;
        }
    }
}

// Zeroes the per-box flags of the persistent passes (a kernel, not a memset,
// so that it takes part in the programmatic launch chain).
__global__ void __launch_bounds__(256) k_clear_flags(int32_t *__restrict__ flag, int64_t n)
{
    griddep_wait();
    griddep_launch_dependents();
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        flag[i] = 0;
}

// -------------------------------------------------------------------------
// Double-float arithmetic for the shifts of the split path.  GB300 runs FP64
// at a small fraction of its FP32 rate, and the level passes are chains of
// small products whose every step waits for FP64 issue.  A value is carried
// as hi + lo (two FP32 numbers, about 48 significant bits); a product is made
// exact with an FMA and added by an error-free two-sum, the rounding errors
// gathering in lo.  Accuracy about 2^-46 of the sum of |terms|, far inside the
// 2^-40 of the split products.  The explicitly rounded intrinsics keep the
// compiler from contracting the error-free steps.
// -------------------------------------------------------------------------
__device__ __forceinline__ float4 df4_of(double2 v)
{
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, __double2float_rn(v.x - double(rh)), ih, __double2float_rn(v.y - double(ih)));
}

// (sh, sl) += (xh + xl)(yh + yl)
__device__ __forceinline__ void df_mac(float &sh, float &sl, float xh, float xl, float yh, float yl)
{
    const float pr = __fmul_rn(xh, yh);
    const float e = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -pr)));
    const float t = __fadd_rn(sh, pr);
    const float v = __fsub_rn(t, sh);
    const float r = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, v)), __fsub_rn(pr, v));   // sh + pr = t + r
    sl = __fadd_rn(sl, __fadd_rn(r, e));
    sh = t;
}

// (re, im) += o * x for double-float complex numbers {Re hi, Re lo, Im hi, Im lo}
__device__ __forceinline__ void df_cmac(float &rh, float &rl, float &ih, float &il, float4 o, float4 x)
{
    df_mac(rh, rl, o.x, o.y, x.x, x.y);
    df_mac(rh, rl, -o.z, -o.w, x.z, x.w);
    df_mac(ih, il, o.x, o.y, x.z, x.w);
    df_mac(ih, il, o.z, o.w, x.x, x.y);
}

// Two double-float numbers (h0 + l0) + (h1 + l1), with the error of the hi
// sum kept (Knuth's two-sum) and the result renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float s = __fadd_rn(a.x, b.x);
    const float v = __fsub_rn(s, a.x);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b.x, v)), __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float4 df4_add(float4 a, float4 b)
{
    const float2 r = df_add(make_float2(a.x, a.y), make_float2(b.x, b.y));
    const float2 i = df_add(make_float2(a.z, a.w), make_float2(b.z, b.w));
    return make_float4(r.x, r.y, i.x, i.y);
}

// Dynamic shared memory of the upward pass: children, partial sums, the leaf
// values, and (double-float variant, schedule of T terms per lane) the
// scheduled operator entries, the partial-sum slots, the term codes and the
// per-output slot counts.
inline size_t up_smem_bytes(int NP, int P1, int T, int maxp)
{
    return sizeof(double2) * 8 * P1 + sizeof(double) * ((NP + 1) & ~1) +
           (T > 0 ? sizeof(float4) * (size_t(4) * T * 32 + size_t(4) * P1 * maxp) + sizeof(uint32_t) * T * 32 +
                        sizeof(int32_t) * ((P1 + 3) & ~3)
                  : 0);
}
// Dynamic shared memory of the downward pass: the parent expansion and the
// partial sums; the FP64 variant adds the factored shift's run sums and its
// schedule (coefficients, codes, slot counts).
inline size_t down_smem_bytes(int P1, int T, int maxp, bool df)
{
    return sizeof(double2) * (5 * P1 + 1) +
           (df ? 0 : sizeof(double2) * size_t(P1) * maxp + (sizeof(double) + sizeof(uint32_t)) * T * 32 +
                         sizeof(int32_t) * P1);
}
// The FP64 variant: children, partial sums, leaf values, then the factored
// shift's schedule (coefficients, codes, slot counts) and the four children's
// partial-sum slots.
inline size_t up_smem_bytes_f64(int NP, int P1, int T, int maxp)
{
    return sizeof(double2) * 8 * P1 + sizeof(double) * ((NP + 1) & ~1) + sizeof(double) * T * 32 +
           sizeof(double2) * size_t(4) * P1 * maxp + sizeof(uint32_t) * T * 32 + sizeof(int32_t) * ((P1 + 3) & ~3);
}

// -------------------------------------------------------------------------
// upward pass, one persistent launch:
//   leaves: ex[box(leaf)][l] = s * sum_j OpA[j][l] v[leaf][j]
//           forward (P2M): OpA = Q^T, s = r^2;  adjoint (L2P^H): OpA = E^H, s = 1
//           (OpA == nullptr: the leaf expansions are already in ex, split path)
//   then level by level, deepest first, each parent once its children are
//   published (per-box flags; a box whose subtree holds no point source, per
//   the optional mask `live`, publishes a zero expansion at once):
//   parent: ex[p][l] = sum_q sum_k Up_q[l][k] ex[child_q(p)][k]    (levels >= 2)
//           forward: M2M; adjoint: L2L^H
// Four warps per block: in the leaf step warp w sums over the w-th quarter of
// the nodes, in a parent step warp q applies the operator of child q; the four
// partial sums meet in shared memory.  The FP64 variant applies Up_q in
// factored form (ShiftFac: so_q[l] sum_k B[l][k] si_q[k]), B's terms on a
// schedule that gives the 32 lanes equal shares of the triangle; about a
// third of the FP64 instructions of the dense complex product.  The
// double-float variant runs the
// parent step on the term schedule (DfSched), keeps its sums in double-float
// until the one conversion of each result, and publishes every climbed
// expansion twice: ex in FP64 and exdf as double-float pairs, which the
// parent's step reads without conversion.
// -------------------------------------------------------------------------
template <bool ADJ, bool DF>
__global__ void __launch_bounds__(128)
k_up_levels(int64_t nleaf, const int32_t *__restrict__ order, const int32_t *__restrict__ leaf_box,
            const int32_t *__restrict__ leaf_level, const int64_t *__restrict__ level_start, int nlevels,
            const int32_t *__restrict__ box_child0, const double *__restrict__ vin,
            const double2 *__restrict__ OpA, const float4 *__restrict__ OpADF, DfSched us, ShiftFac uf, double2 *ex,
            float4 *exdf, int NP, int P1, const double *__restrict__ lvtab, bool climb, int32_t *flag,
            const uint8_t *__restrict__ active, long long limit, int32_t *err, const uint8_t *__restrict__ live)
{
    extern __shared__ double2 shu[];
    double2 *sc = shu;                                       // 4 * P1 children
    double2 *part = sc + 4 * P1;                             // [4][P1] partial sums
    double *sv = reinterpret_cast<double *>(part + 4 * P1);  // NP
    // the shift schedule in shared memory, copied while the preceding kernel
    // drains (every parent step reads it)
    // double-float path: scheduled operator entries of the four children
    const int T = us.T, SL = P1 * us.maxp;   // terms per lane, slots per child
    float4 *sops = reinterpret_cast<float4 *>(sv + ((NP + 1) & ~1));   // [4][T][32] (DF only)
    float4 *sslot = sops + 4 * T * 32;                                 // [4][SL]
    uint32_t *scode = reinterpret_cast<uint32_t *>(sslot + 4 * SL);    // [T][32]
    int32_t *snp = reinterpret_cast<int32_t *>(scode + T * 32);        // [P1]
    // FP64 path: the factored shift's coefficients and codes (ShiftFac)
    const int TF = uf.T, SLF = P1 * uf.maxp;
    double *fcoef = sv + ((NP + 1) & ~1);                              // [TF][32] (FP64 only)
    double2 *fslot = reinterpret_cast<double2 *>(fcoef + TF * 32);     // [4][SLF]
    uint32_t *fcode = reinterpret_cast<uint32_t *>(fslot + 4 * SLF);   // [TF][32]
    int32_t *fnp = reinterpret_cast<int32_t *>(fcode + TF * 32);       // [P1]
    __shared__ int s_leafc[4];   // which children of the current parent are leaves
    if (climb) {
        if constexpr (DF) {
            for (int i = threadIdx.x; i < 4 * T * 32; i += blockDim.x) sops[i] = __ldg(&us.ops[i]);
            for (int i = threadIdx.x; i < T * 32; i += blockDim.x) scode[i] = __ldg(&us.code[i]);
            for (int i = threadIdx.x; i < P1; i += blockDim.x) snp[i] = __ldg(&us.np[i]);
        } else {
            for (int i = threadIdx.x; i < TF * 32; i += blockDim.x) {
                fcoef[i] = __ldg(&uf.coef[i]);
                fcode[i] = __ldg(&uf.code[i]);
            }
            for (int i = threadIdx.x; i < P1; i += blockDim.x) fnp[i] = __ldg(&uf.np[i]);
        }
    }
    griddep_wait();
    griddep_launch_dependents();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // leaf step: warp w sums the nodes [j0, j1) (any number of nodes)
    const int nq = (NP + 3) / 4, j0 = min(NP, w * nq), j1 = min(NP, j0 + nq);
    for (int64_t li = blockIdx.x; OpA && li < nleaf; li += gridDim.x) {
        const int leaf = order[li];
        const int b = leaf_box[leaf];
        const double s = ADJ ? 1.0 : lvtab[leaf_level[leaf]];   // r^2
        // a discarded leaf of a truncated tree is no source: its expansion is zero
        const bool skip = active && !active[leaf];
        __syncthreads();
        if constexpr (DF) {
            // double-float: the leaf values as {hi, lo} pairs, OpA as pairs
            float2 *svf = reinterpret_cast<float2 *>(sv);
            for (int j = threadIdx.x; j < NP; j += blockDim.x) {
                const double v = vin[int64_t(leaf) * NP + j];
                const float h = __double2float_rn(v);
                svf[j] = make_float2(h, __double2float_rn(v - double(h)));
            }
            __syncthreads();
            for (int l = lane; l < P1; l += 32) {
                float r0h = 0.f, r0l = 0.f, i0h = 0.f, i0l = 0.f, r1h = 0.f, r1l = 0.f, i1h = 0.f, i1l = 0.f;
                for (int jb = j0; jb < j1; jb += 8) {   // 8 operator loads in flight, two chains
                    float4 o[8];
#pragma unroll
                    for (int u = 0; u < 8; u++)
                        o[u] = jb + u < j1 ? __ldg(&OpADF[(jb + u) * P1 + l]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        if (jb + u >= j1) break;
                        const float2 v0 = svf[jb + u];
                        df_mac(r0h, r0l, o[u].x, o[u].y, v0.x, v0.y);
                        df_mac(i0h, i0l, o[u].z, o[u].w, v0.x, v0.y);
                        if (jb + u + 1 < j1) {
                            const float2 v1 = svf[jb + u + 1];
                            df_mac(r1h, r1l, o[u + 1].x, o[u + 1].y, v1.x, v1.y);
                            df_mac(i1h, i1l, o[u + 1].z, o[u + 1].w, v1.x, v1.y);
                        }
                    }
                }
                part[w * P1 + l] = make_double2((double(r0h) + double(r1h)) + (double(r0l) + double(r1l)),
                                                (double(i0h) + double(i1h)) + (double(i0l) + double(i1l)));
            }
        } else {
        for (int j = threadIdx.x; j < NP; j += blockDim.x) sv[j] = vin[int64_t(leaf) * NP + j];
        __syncthreads();
        for (int l = lane; l < P1; l += 32) {
            double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
            int j = j0;
            for (; j + 1 < j1; j += 2) {
                double2 o0 = OpA[j * P1 + l], o1 = OpA[(j + 1) * P1 + l];
                re0 = fma(o0.x, sv[j], re0);
                im0 = fma(o0.y, sv[j], im0);
                re1 = fma(o1.x, sv[j + 1], re1);
                im1 = fma(o1.y, sv[j + 1], im1);
            }
            if (j < j1) {
                double2 o0 = OpA[j * P1 + l];
                re0 = fma(o0.x, sv[j], re0);
                im0 = fma(o0.y, sv[j], im0);
            }
            part[w * P1 + l] = make_double2(re0 + re1, im0 + im1);
        }
        }
        __syncthreads();
        for (int l = threadIdx.x; l < P1; l += blockDim.x) {
            const double2 a0 = part[l], a1 = part[P1 + l], a2 = part[2 * P1 + l], a3 = part[3 * P1 + l];
            ex[int64_t(b) * P1 + l] =
                skip ? make_double2(0.0, 0.0)
                     : make_double2(s * ((a0.x + a1.x) + (a2.x + a3.x)), s * ((a0.y + a1.y) + (a2.y + a3.y)));
        }
        flag_publish(&flag[b], 1);
    }
    if (!climb) return;
    for (int lv = nlevels - 2; lv >= 2; lv--) {
        for (int64_t p = level_start[lv] + blockIdx.x; p < level_start[lv + 1]; p += gridDim.x) {
            const int c0 = box_child0[p];
            if (c0 < 0) continue;   // a leaf (uniform over the block)
            if (live && !live[p]) {
                // no source below this box (point sources): its expansion is
                // zero, with nothing to wait for
                for (int i = threadIdx.x; i < P1; i += blockDim.x) {
                    ex[int64_t(p) * P1 + i] = make_double2(0.0, 0.0);
                    if (DF) exdf[int64_t(p) * P1 + i] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                flag_publish(&flag[p], 1);
                continue;
            }
            // children computed in this launch: every child above the leaves,
            // and the leaves too when their expansions come from the leaf step
            if (threadIdx.x < 4) {
                const bool leafc = box_child0[c0 + threadIdx.x] < 0;
                if (DF) s_leafc[threadIdx.x] = leafc;
                if (OpA || !leafc) flag_wait(&flag[c0 + threadIdx.x], 1, limit, err);
            }
            __syncthreads();
            if constexpr (DF) {
                // the children as double-float pairs: climbed ones from exdf,
                // leaves (expansions of the leaf products) from ex
                float4 *scf = reinterpret_cast<float4 *>(sc);
                for (int i = threadIdx.x; i < 4 * P1; i += blockDim.x) {
                    const int64_t g = int64_t(c0) * P1 + i;
                    scf[i] = s_leafc[i / P1] ? df4_of(__ldcg(&ex[g])) : __ldcg(&exdf[g]);
                }
                __syncthreads();
                // warp w: the terms of child w, each lane its run of the schedule
                const float4 *opw = sops + w * T * 32 + lane;
                const float4 *a = scf + w * P1;
                float4 *slot = sslot + w * SL;
                float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll 2
                for (int t = 0; t < T; t++) {
                    const uint32_t code = scode[t * 32 + lane];
                    df_cmac(rh, rl, ih, il, opw[t * 32], a[code & 255u]);
                    if (code >> 8) {   // the run leaves an output here
                        slot[(code >> 8) - 1u] = make_float4(rh, rl, ih, il);
                        rh = rl = ih = il = 0.f;
                    }
                }
                __syncwarp();
                // lane l: the partial sums of output l for child w
                float4 *pf = reinterpret_cast<float4 *>(part);   // [4][P1]
                for (int l = lane; l < P1; l += 32) {
                    float4 v = slot[l * us.maxp];
                    for (int j = 1; j < snp[l]; j++) v = df4_add(v, slot[l * us.maxp + j]);
                    pf[w * P1 + l] = v;
                }
                __syncthreads();
                // thread (l, Re or Im): the four children, one conversion to FP64
                const float2 *pf2 = reinterpret_cast<const float2 *>(pf);
                for (int i = threadIdx.x; i < 2 * P1; i += blockDim.x) {
                    float2 v = df_add(df_add(pf2[i], pf2[2 * P1 + i]), df_add(pf2[4 * P1 + i], pf2[6 * P1 + i]));
                    const int64_t g = int64_t(p) * P1 * 2 + i;
                    reinterpret_cast<double *>(ex)[g] = double(v.x) + double(v.y);
                    reinterpret_cast<float2 *>(exdf)[g] = v;
                }
                flag_publish(&flag[p], 1);
            } else {
            // factored FP64 shift (ShiftFac), warp w = child w: a = si_w * child
            // (lane k), then B's terms on the schedule, each output's partial
            // sums added and scaled by so_w, and the four children summed
            double2 *a = sc + w * P1;
            for (int k = lane; k < P1; k += 32) {
                const double2 A = __ldcg(&ex[int64_t(c0 + w) * P1 + k]), S = __ldg(&uf.si[w * P1 + k]);
                a[k] = make_double2(fma(A.x, S.x, -A.y * S.y), fma(A.x, S.y, A.y * S.x));
            }
            __syncwarp();
            double2 *slot = fslot + w * SLF;
            double re = 0.0, im = 0.0;
#pragma unroll 2
            for (int t = 0; t < TF; t++) {
                const uint32_t code = fcode[t * 32 + lane];
                const double cf = fcoef[t * 32 + lane];
                const double2 x = a[code & 255u];
                re = fma(cf, x.x, re);
                im = fma(cf, x.y, im);
                if (code >> 8) {   // the run leaves an output here
                    slot[(code >> 8) - 1u] = make_double2(re, im);
                    re = im = 0.0;
                }
            }
            __syncwarp();
            for (int l = lane; l < P1; l += 32) {
                double2 y = slot[l * uf.maxp];
                for (int j = 1; j < fnp[l]; j++) {
                    const double2 v = slot[l * uf.maxp + j];
                    y.x += v.x;
                    y.y += v.y;
                }
                const double2 S = __ldg(&uf.so[w * P1 + l]);
                part[w * P1 + l] = make_double2(fma(y.x, S.x, -y.y * S.y), fma(y.x, S.y, y.y * S.x));
            }
            __syncthreads();
            for (int l = threadIdx.x; l < P1; l += blockDim.x) {
                const double2 a0 = part[l], a1 = part[P1 + l], a2 = part[2 * P1 + l], a3 = part[3 * P1 + l];
                ex[int64_t(p) * P1 + l] = make_double2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
            }
            flag_publish(&flag[p], 1);
            }
        }
    }
}

// Level of box b from the level offsets (boxes are sorted by level).
__device__ __forceinline__ int lv_of(const int64_t *__restrict__ level_start, int nlevels, int64_t b)
{
    int lo = 0, hi = nlevels - 1;   // last lv with level_start[lv] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (level_start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// -------------------------------------------------------------------------
// Binomial table of the factored M2L, shared by every offset and every
// expansion order P + 1 <= 32 (entries depend only on the indices):
//   c_binom[k][o] = C(k + o - 1, o) for k >= 1, c_binom[0][o] = -1/o (o >= 1),
//   c_binom[0][0] = 0.
// Constant memory: in the unrolled loops below each entry is a DFMA operand.
// -------------------------------------------------------------------------
__constant__ double c_binom[32][32];
// its transpose, so that the adjoint kernels also read a row with the lanes
// (consecutive o) on consecutive addresses
__constant__ double c_binomT[32][32];

// -------------------------------------------------------------------------
// m2l_boxes: the whole V-list sum of one target box b per block, in FP64,
// written once:
//   out[b][o] = sum_{e in V(b)} [ W_c[o] sum_k B[k][o] a_k(e) + (o = 0) (log|d_c| + log r_b) a_0(e) ]
//   a_k(e) = S_c[k] in[s_e][k]
// with (forward) S_c[k] = (-1)^k d^-k, W_c[o] = d^-o, B = c_binom, and
// (adjoint, the conjugate transpose of the reversed pair) S_c[k] =
// (-1)^k conj(d)^-k, W_c[o] = conj(d)^-o, B = c_binom transposed.  The log
// r_b term is the level term of the box's own local expansion (r-scaled A_0
// of each source times log r_b).  Boxes without V entries get 0.  Since
// S_c[k] = (-1)^k W_c[k], the kernel reads the W table only and carries the
// sign (-1)^k in its binomial column.
// The block is NG groups of P1 threads: thread (g, o) owns output o of the
// pairs v0 + g, v0 + g + NG, ...; per pair the group first forms a(e) in
// shared memory (thread o its coefficient o), then every thread contracts it
// with its column of B, held in registers (constant-memory reads with a
// different index per lane would serialise).  The rows are double-buffered,
// so one barrier per pair suffices (3.2 KB of shared memory per block: four
// blocks still fit beside a two-buffer near-field CTA).  The sums stay in registers
// until the groups meet in shared memory at the end of the box.  Nearly every
// instruction is an FP64 FMA: 2 P1 per pair and thread, plus 8 for the two
// diagonal scalings; NG P1 is a multiple of 32 wherever possible so that no
// lane idles.
// -------------------------------------------------------------------------
template <bool ADJ, int PMAX>
__global__ void __launch_bounds__(256)
k_m2l_boxes(int64_t b0, int64_t b1, const int32_t *__restrict__ v_ptr, const int32_t *__restrict__ v_src,
            const int32_t *__restrict__ v_code, const int32_t *__restrict__ box_level,
            const double2 *__restrict__ dsig, const double2 *__restrict__ dpow, const double *__restrict__ logd,
            const double *__restrict__ lvtab, const double2 *__restrict__ in, double2 *__restrict__ out, int P1,
            int NG, int tri)
{
    extern __shared__ double2 sm2l[];   // [NG][2][P1 + 1]: a(e) of each group's pair, then the group sums
    const int t = threadIdx.x, g = t / P1, o = t - g * P1;
    const bool act = g < NG;
    const int ld = P1 + 1;   // padded row: the groups' rows start in different banks
    double bcol[PMAX];
#pragma unroll
    for (int k = 0; k < PMAX; k++) {
        // tri = 1 keeps only the terms with k + o <= P (and exactly their transpose)
        const bool keep = !tri || (ADJ ? (o == 0 || k + o < P1) : (k == 0 || k + o < P1));
        const double sg = (k & 1) ? -1.0 : 1.0;   // (-1)^k of S_c[k]
        bcol[k] = (act && k < P1 && keep) ? sg * (ADJ ? c_binomT[k][o] : c_binom[k][o]) : 0.0;
    }
    // The dependents (the persistent downward pass) are released only at the
    // end: released early, their resident blocks would take the SM space that
    // a near-field tensor CTA on the internal stream needs beside this kernel.
    griddep_wait();
    // two rows per group (double buffer): a pair's row is written while
    // other groups may still read the previous one, so one barrier per pair
    double2 *arow0 = sm2l + 2 * (act ? g : 0) * ld;
    for (int64_t b = b0 + blockIdx.x; b < b1; b += gridDim.x) {
        const int v0 = v_ptr[b], v1 = v_ptr[b + 1];
        const double lgb = lvtab[kLvTab + box_level[b]];
        double accr = 0.0, acci = 0.0;
        int buf = 0;
        for (int e0 = v0; e0 < v1; e0 += NG) {
            const int e = e0 + g;
            const bool live = act && e < v1;
            double2 *arow = arow0 + buf * ld;
            int c = 0;
            if (live) {
                c = v_code[e];
                // S_c[k] = (-1)^k W_c[k]: the sign is in bcol, so one table
                // serves both scalings
                const double2 A = in[int64_t(v_src[e]) * P1 + o], S = dpow[c * P1 + o];
                arow[o] = make_double2(fma(A.x, S.x, -A.y * S.y), fma(A.x, S.y, A.y * S.x));
            }
            __syncthreads();
            if (live) {
                const double2 W = dpow[c * P1 + o];
                double sr = 0.0, si = 0.0;
#pragma unroll
                for (int k = 0; k < PMAX; k++) {
                    if (k < P1) {
                        const double2 a = arow[k];
                        sr = fma(bcol[k], a.x, sr);
                        si = fma(bcol[k], a.y, si);
                    }
                }
                if (o == 0) {
                    const double c0 = logd[c] + lgb;
                    const double2 a = arow[0];
                    sr = fma(c0, a.x, sr);
                    si = fma(c0, a.y, si);
                }
                accr = fma(sr, W.x, fma(-si, W.y, accr));
                acci = fma(sr, W.y, fma(si, W.x, acci));
            }
            buf ^= 1;
        }
        __syncthreads();   // last rows read
        if (act) sm2l[g * ld + o] = make_double2(accr, acci);
        __syncthreads();
        if (t < P1) {
            double2 s = sm2l[t];
            for (int q = 1; q < NG; q++) {
                const double2 v = sm2l[q * ld + t];
                s.x += v.x;
                s.y += v.y;
            }
            out[b * P1 + t] = s;
        }
        __syncthreads();   // group sums read before the next box's rows
    }
    griddep_launch_dependents();
}

// -------------------------------------------------------------------------
// m2l_mma: the same V-list sums as k_m2l_boxes, with the binomial contraction
// on the FP64 tensor cores (mma.sync m8n8k4, f64): one warp per target box.
// For the pairs e of V(b) taken four at a time, the real matrix product
//     T[o][n] = sum_k B[o][k] X[k][n],   B[o][k] = the binomial entry of (k, o)
// has eight columns n: the real and imaginary parts of a(e) = S_c(e) . A_s(e)
// for the four pairs (column n: pair n / 2, part n % 2); B (P1 x P1, padded to
// 8 MT rows and 4 KS columns with zeros) sits in registers as the MMA's A
// fragments for the whole launch.  Lane layout of the m8n8k4 f64 fragments
// (g = lane / 4, t = lane % 4): A[g][t], B[t][g], D[g][2t], D[g][2t+1]; so a
// lane forms X at rows 4s + t of column g and receives T at row 8m + g for
// pair t, real (D[..][2t]) and imaginary (D[..][2t+1]) parts together, which
// it scales by W_c(e)[o] and adds to its running sums.  The four pairs' sums
// meet by two shuffles at the end of the box.  One MMA does 256 FMAs, so the
// FP64 pipe stays busy with one warp per SM sub-partition and no shared
// memory.  Pairs past the end of the list are zero columns.
// -------------------------------------------------------------------------
__device__ __forceinline__ void dmma_m8n8k4(double &d0, double &d1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

template <bool ADJ, int MT, int KS>
__global__ void __launch_bounds__(128)
k_m2l_mma(int64_t b0, int64_t b1, const int32_t *__restrict__ v_ptr, const int32_t *__restrict__ v_src,
          const int32_t *__restrict__ v_code, const int32_t *__restrict__ box_level,
          const double2 *__restrict__ dsig, const double2 *__restrict__ dpow, const double *__restrict__ logd,
          const double *__restrict__ lvtab, const double2 *__restrict__ in, double2 *__restrict__ out, int P1,
          int tri)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    double bf[MT][KS];   // B[8m + g][4s + t]
#pragma unroll
    for (int m = 0; m < MT; m++)
#pragma unroll
        for (int s = 0; s < KS; s++) {
            const int o = 8 * m + g, k = 4 * s + t;
            // tri = 1 keeps only the terms with k + o <= P (and exactly their transpose)
            const bool keep = !tri || (ADJ ? (o == 0 || k + o < P1) : (k == 0 || k + o < P1));
            bf[m][s] = (o < P1 && k < P1 && keep) ? (ADJ ? c_binom[o][k] : c_binom[k][o]) : 0.0;
        }
    // The dependents (the persistent downward pass) are released only at the
    // end, as in k_m2l_boxes.
    griddep_wait();
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t b = b0 + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); b < b1; b += nwarps) {
        const int v0 = v_ptr[b], v1 = v_ptr[b + 1];
        const double lgb = lvtab[kLvTab + box_level[b]];
        double ar[MT], ai[MT];   // sums for rows 8m + g, pairs of slot t
#pragma unroll
        for (int m = 0; m < MT; m++) ar[m] = ai[m] = 0.0;
        for (int e0 = v0; e0 < v1; e0 += 4) {
            // this lane's column of X: pair slot g / 2, part g % 2, rows 4s + t
            const int ex = e0 + (g >> 1);
            double xv[KS];
            if (ex < v1) {
                const int s_src = v_src[ex], c = v_code[ex];
#pragma unroll
                for (int s = 0; s < KS; s++) {
                    const int k = 4 * s + t;
                    xv[s] = 0.0;
                    if (k < P1) {
                        const double2 A = in[int64_t(s_src) * P1 + k], S = dsig[c * P1 + k];
                        xv[s] = (g & 1) ? fma(A.x, S.y, A.y * S.x) : fma(A.x, S.x, -A.y * S.y);
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < KS; s++) xv[s] = 0.0;
            }
            double dr[MT], di[MT];
#pragma unroll
            for (int m = 0; m < MT; m++) dr[m] = di[m] = 0.0;
#pragma unroll
            for (int s = 0; s < KS; s++)
#pragma unroll
                for (int m = 0; m < MT; m++) dmma_m8n8k4(dr[m], di[m], bf[m][s], xv[s]);
            // T for pair slot t at rows 8m + g: scale by W_c[o] and add
            const int eo = e0 + t;
            if (eo < v1) {
                const int c = v_code[eo];
#pragma unroll
                for (int m = 0; m < MT; m++) {
                    const int o = 8 * m + g;
                    if (o < P1) {
                        double tr = dr[m], ti = di[m];
                        if (o == 0) {   // the log term of the box's local expansion
                            const double2 A0 = in[int64_t(v_src[eo]) * P1];
                            const double c0 = logd[c] + lgb;
                            tr = fma(c0, A0.x, tr);
                            ti = fma(c0, A0.y, ti);
                        }
                        const double2 W = dpow[c * P1 + o];
                        ar[m] = fma(tr, W.x, fma(-ti, W.y, ar[m]));
                        ai[m] = fma(tr, W.y, fma(ti, W.x, ai[m]));
                    }
                }
            }
        }
        // the four pair slots (lanes 4g .. 4g + 3) meet
#pragma unroll
        for (int m = 0; m < MT; m++) {
            ar[m] += __shfl_xor_sync(0xffffffffu, ar[m], 1);
            ai[m] += __shfl_xor_sync(0xffffffffu, ai[m], 1);
            ar[m] += __shfl_xor_sync(0xffffffffu, ar[m], 2);
            ai[m] += __shfl_xor_sync(0xffffffffu, ai[m], 2);
        }
        if (t == 0) {
#pragma unroll
            for (int m = 0; m < MT; m++) {
                const int o = 8 * m + g;
                if (o < P1) out[b * P1 + o] = make_double2(ar[m], ai[m]);
            }
        }
    }
    griddep_launch_dependents();
}

// Groups per block of the M2L kernel: the smallest NG >= 4 with NG * P1 a
// multiple of 32 (no idle lane) and at most 256 threads, else 4.
inline int m2l_groups(int P1)
{
    for (int ng = 4; ng * P1 <= 256; ng++)
        if ((ng * P1) % 32 == 0) return ng;
    return 4;
}
inline int m2l_threads(int P1) { return (m2l_groups(P1) * P1 + 31) / 32 * 32; }

// -------------------------------------------------------------------------
// x_entries (FP64 path): the X-list products, one block per entry e (target
// box b, source leaf c at level lv_b - 1):
//   PX[e][l] = s1 * sum_j OpX[code][j][l] x[c][j]
//   forward (P2L): s1 = r_c^2;  adjoint (M2P^H): s1 = 1
// Four warps split the nodes; the partial sums meet in shared memory.
// -------------------------------------------------------------------------
template <bool ADJ>
__global__ void __launch_bounds__(128)
k_x_entries(int64_t nx, const int32_t *__restrict__ x_box, const int32_t *__restrict__ x_src,
            const int32_t *__restrict__ x_code, const int32_t *__restrict__ box_level,
            const double2 *__restrict__ OpX, const double *__restrict__ xvec, double2 *__restrict__ PX, int NP,
            int P1, const double *__restrict__ lvtab)
{
    griddep_wait();
    griddep_launch_dependents();
    extern __shared__ double2 shx[];
    double2 *part = shx;                                     // [4][P1]
    double *sv = reinterpret_cast<double *>(part + 4 * P1);  // NP
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = (NP + 3) / 4, j0 = min(NP, w * nq), j1 = min(NP, j0 + nq);   // warp w's nodes
    for (int64_t e = blockIdx.x; e < nx; e += gridDim.x) {
        const int c = x_src[e];
        const double2 *op = OpX + size_t(x_code[e]) * NP * P1;
        const double s1 = ADJ ? 1.0 : lvtab[box_level[x_box[e]] - 1];
        __syncthreads();
        for (int j = threadIdx.x; j < NP; j += blockDim.x) sv[j] = xvec[int64_t(c) * NP + j];
        __syncthreads();
        for (int l = lane; l < P1; l += 32) {
            double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
            int j = j0;
            for (; j + 1 < j1; j += 2) {
                double2 o0 = op[j * P1 + l], o1 = op[(j + 1) * P1 + l];
                re0 = fma(o0.x, sv[j], re0);
                im0 = fma(o0.y, sv[j], im0);
                re1 = fma(o1.x, sv[j + 1], re1);
                im1 = fma(o1.y, sv[j + 1], im1);
            }
            if (j < j1) {
                double2 o0 = op[j * P1 + l];
                re0 = fma(o0.x, sv[j], re0);
                im0 = fma(o0.y, sv[j], im0);
            }
            part[w * P1 + l] = make_double2(re0 + re1, im0 + im1);
        }
        __syncthreads();
        for (int l = threadIdx.x; l < P1; l += blockDim.x) {
            const double2 a0 = part[l], a1 = part[P1 + l], a2 = part[2 * P1 + l], a3 = part[3 * P1 + l];
            PX[e * P1 + l] = make_double2(s1 * ((a0.x + a1.x) + (a2.x + a3.x)), s1 * ((a0.y + a1.y) + (a2.y + a3.y)));
        }
    }
}

// -------------------------------------------------------------------------
// down_levels: the local expansion (adjoint: multipole) of every box at
// level >= 2, in one persistent launch:
//   the box's own sums:
//     out[b] = V(b) + sum_{x in X(b)} (PX[x] + log(r_c) A_0(c) e_0)
//   where V(b) is out[b] itself on entry (vsum: the whole V-list sum, written
//   by k_m2l_boxes) or sum_{e in V(b)} Pv[e] (one row per pair, from the
//   tensor cores)
//   then (levels 3, 4, ...; once the parent is published):
//     out[b] += Par_q out[parent(b)]      (forward L2L, adjoint M2M^H)
// A block takes its boxes in ascending index (so ascending level) and does
// both steps for one box before the next, then publishes the box: the sums of
// deep boxes overlap the chain of the shallower levels, and a box waits only
// for its parent, a box of smaller index (so every wait ends).
// The X-list log term uses coefficient 0 of the source leaf's own expansion
// from the upward pass (forward A_0 = r_c^2 (w.f)/2pi, adjoint B_0 = sum_j g_j).
// With v_lsrc non-null (M2L products from the tensor cores, which leave out
// the log term) the sums add it in FP64 as well:
//     out[b][0] += sum_{e in V(b)} (log|d_e| + log r_b) first[s_e][0]
// Four warps per block.  The sums run side by side: warp 0 the X list (its
// log term gathered one entry per lane), warp 1 the V-list log term (one pair
// per lane), warps 2 and 3 the V pairs (vsum: warp 2 reads the V sum).  In
// the shift warp w applies a quarter of the operator's columns, fetched into
// registers before the wait for the parent (the shift chain is the critical
// path).  The double-float variant keeps that chain free of FP64 work: a copy
// of the box's sums is converted to pairs before the wait, the parent is read
// as pairs (outdf), the shift and its sum with the copy are formed as pairs
// and published for the children; the FP64 result, read only by later
// kernels, is the FP64 sums plus the shift, stored after the box's flag.
// -------------------------------------------------------------------------
template <bool DF>
__global__ void __launch_bounds__(128)
k_down_levels(const int64_t *__restrict__ level_start, int nlevels, const int32_t *__restrict__ v_ptr,
              const double2 *__restrict__ Pv, const int32_t *__restrict__ x_ptr, const int32_t *__restrict__ x_src,
              const double2 *__restrict__ PX, int px_stride, const int32_t *__restrict__ leaf_box,
              const double2 *__restrict__ first, const int32_t *__restrict__ parent,
              const int32_t *__restrict__ box_ix, const int32_t *__restrict__ box_iy,
              const float4 *__restrict__ OpParDF, ShiftFac pf, double2 *out, float4 *outdf, int P1,
              const double *__restrict__ lvtab,
              const int32_t *__restrict__ v_lsrc, const int32_t *__restrict__ v_code,
              const double *__restrict__ logd, bool vsum, int32_t *flag, long long limit, int32_t *err)
{
    extern __shared__ double2 sdn[];
    double2 *se = sdn;             // [P1] parent expansion (FP64 variant: times si_q)
    double2 *part = sdn + P1;      // [4][P1] partial sums
    // FP64 variant: the factored shift's schedule (ShiftFac) and the partial
    // sums of its runs, staged before the wait for the preceding kernel
    const int TF = DF ? 0 : pf.T, SLF = DF ? 0 : P1 * pf.maxp;
    double2 *fslot = part + 4 * P1;                                    // [SLF]
    double *fcoef = reinterpret_cast<double *>(fslot + SLF);           // [TF][32]
    uint32_t *fcode = reinterpret_cast<uint32_t *>(fcoef + TF * 32);   // [TF][32]
    int32_t *fnp = reinterpret_cast<int32_t *>(fcode + TF * 32);       // [P1]
    if constexpr (!DF) {
        for (int i = threadIdx.x; i < TF * 32; i += blockDim.x) {
            fcoef[i] = __ldg(&pf.coef[i]);
            fcode[i] = __ldg(&pf.code[i]);
        }
        for (int i = threadIdx.x; i < P1; i += blockDim.x) fnp[i] = __ldg(&pf.np[i]);
    }
    griddep_wait();
    griddep_launch_dependents();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kq = (P1 + 3) / 4, k0 = w * kq, k1 = min(P1, k0 + kq);   // this warp's shift columns (<= 8)
    const int o = lane;   // coefficient of this lane (P1 <= 32)
    for (int64_t b = level_start[2] + blockIdx.x; b < level_start[nlevels]; b += gridDim.x) {
        const int lvb = lv_of(level_start, nlevels, b);
        const bool shift = lvb >= 3;
        const int pb = shift ? parent[b] : 0;
        const int q = (box_ix[b] & 1) + 2 * (box_iy[b] & 1);
        // the shift operator does not depend on the parent's values: fetched
        // before the wait for them (FP64: warp 0's diagonals si_q, so_q)
        float4 wf[8];
        double2 fsi = make_double2(0.0, 0.0), fso = make_double2(0.0, 0.0);
        if (shift && o < P1) {
            if constexpr (DF) {
#pragma unroll
                for (int u = 0; u < 8; u++)
                    wf[u] = k0 + u < k1 ? __ldg(&OpParDF[(size_t(q) * P1 + k0 + u) * P1 + o])
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            } else if (w == 0) {
                fsi = __ldg(&pf.si[q * P1 + o]);
                fso = __ldg(&pf.so[q * P1 + o]);
            }
        }
        // ---- the box's own sums, one kind per warp: warp 0 the X list and
        // its log term, warp 1 the log term of the V list (tensor-core M2L),
        // warps 2 and 3 the V pairs
        double re = 0.0, im = 0.0;
        if (w == 0) {
            const int x0 = x_ptr[b], x1 = x_ptr[b + 1];
            if (o < P1) {
#pragma unroll 4
                for (int x = x0; x < x1; x++) {
                    const double2 t = PX[int64_t(x) * px_stride + o];
                    re += t.x;
                    im += t.y;
                }
            }
            double lx = 0.0;
            for (int x = x0 + lane; x < x1; x += 32) lx += first[int64_t(leaf_box[x_src[x]]) * P1].x;
            for (int m = 16; m > 0; m >>= 1) lx += __shfl_xor_sync(0xffffffffu, lx, m);
            if (o == 0) re = fma(lvtab[kLvTab + lvb - 1], lx, re);
        } else if (w == 1) {
            if (v_lsrc) {
                const int v0 = v_ptr[b], v1 = v_ptr[b + 1];
                const double lgb = lvtab[kLvTab + lvb];
                double lr = 0.0, li = 0.0;
                for (int e = v0 + lane; e < v1; e += 32) {
                    const double2 a0 = first[int64_t(v_lsrc[e]) * P1];
                    const double c0 = logd[v_code[e]] + lgb;
                    lr = fma(c0, a0.x, lr);
                    li = fma(c0, a0.y, li);
                }
                for (int m = 16; m > 0; m >>= 1) {
                    lr += __shfl_xor_sync(0xffffffffu, lr, m);
                    li += __shfl_xor_sync(0xffffffffu, li, m);
                }
                if (o == 0) {
                    re = lr;
                    im = li;
                }
            }
        } else if (vsum) {
            if (w == 2 && o < P1) {
                const double2 t = out[b * P1 + o];
                re = t.x;
                im = t.y;
            }
        } else if (o < P1) {
            const int v0 = v_ptr[b], v1 = v_ptr[b + 1];
            double re1 = 0.0, im1 = 0.0;
            int e = v0 + (w - 2);
            for (; e + 2 < v1; e += 4) {   // two loads in flight per step
                const double2 t0 = Pv[int64_t(e) * P1 + o], t1 = Pv[int64_t(e + 2) * P1 + o];
                re += t0.x;
                im += t0.y;
                re1 += t1.x;
                im1 += t1.y;
            }
            if (e < v1) {
                const double2 t0 = Pv[int64_t(e) * P1 + o];
                re += t0.x;
                im += t0.y;
            }
            re += re1;
            im += im1;
        }
        if (o < P1) part[w * P1 + o] = make_double2(re, im);
        __syncthreads();
        double2 acc = make_double2(0.0, 0.0);   // meaningful in warp 0, lanes o < P1
        float4 accf = make_float4(0.f, 0.f, 0.f, 0.f);   // the same as double-float pairs (DF)
        float4 shf = make_float4(0.f, 0.f, 0.f, 0.f);    // the shifted parent (DF)
        if (w == 0 && o < P1) {
            const double2 a0 = part[o], a1 = part[P1 + o], a2 = part[2 * P1 + o], a3 = part[3 * P1 + o];
            acc = make_double2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
            if (DF) accf = df4_of(acc);   // before the wait for the parent
        }
        // ---- plus the parent's expansion shifted to this box (levels >= 3)
        if (shift) {
            if (threadIdx.x == 0) flag_wait(&flag[pb], 2, limit, err);
            __syncthreads();   // also: warp 0 has read its partial sums
            if constexpr (DF) {
                float4 *sef = reinterpret_cast<float4 *>(se);   // the parent's double-float pairs
                for (int i = threadIdx.x; i < P1; i += blockDim.x) sef[i] = __ldcg(&outdf[int64_t(pb) * P1 + i]);
                __syncthreads();
                if (o < P1) {
                    float r0h = 0.f, r0l = 0.f, i0h = 0.f, i0l = 0.f, r1h = 0.f, r1l = 0.f, i1h = 0.f, i1l = 0.f;
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {   // two chains
                        if (k0 + u >= k1) break;
                        df_cmac(r0h, r0l, i0h, i0l, wf[u], sef[k0 + u]);
                        if (k0 + u + 1 < k1) df_cmac(r1h, r1l, i1h, i1l, wf[u + 1], sef[k0 + u + 1]);
                    }
                    reinterpret_cast<float4 *>(part)[w * P1 + o] =
                        df4_add(make_float4(r0h, r0l, i0h, i0l), make_float4(r1h, r1l, i1h, i1l));
                }
            } else if (w == 0) {
                // factored FP64 shift (ShiftFac) by warp 0: a = si_q * parent
                // (lane k), B's terms on the schedule, each output's partial
                // sums added and scaled by so_q
                if (o < P1) {
                    const double2 A = __ldcg(&out[int64_t(pb) * P1 + o]);
                    se[o] = make_double2(fma(A.x, fsi.x, -A.y * fsi.y), fma(A.x, fsi.y, A.y * fsi.x));
                }
                __syncwarp();
                double re = 0.0, im = 0.0;
#pragma unroll 2
                for (int t = 0; t < TF; t++) {
                    const uint32_t code = fcode[t * 32 + lane];
                    const double cf = fcoef[t * 32 + lane];
                    const double2 x = se[code & 255u];
                    re = fma(cf, x.x, re);
                    im = fma(cf, x.y, im);
                    if (code >> 8) {   // the run leaves an output here
                        fslot[(code >> 8) - 1u] = make_double2(re, im);
                        re = im = 0.0;
                    }
                }
                __syncwarp();
                if (o < P1) {
                    double2 y = fslot[o * pf.maxp];
                    for (int j = 1; j < fnp[o]; j++) {
                        const double2 v = fslot[o * pf.maxp + j];
                        y.x += v.x;
                        y.y += v.y;
                    }
                    acc.x += fma(y.x, fso.x, -y.y * fso.y);
                    acc.y += fma(y.x, fso.y, y.y * fso.x);
                }
            }
            if constexpr (DF) {
                __syncthreads();
                if (w == 0 && o < P1) {
                    const float4 *pf4 = reinterpret_cast<const float4 *>(part);
                    shf = df4_add(pf4[o], df4_add(pf4[P1 + o], df4_add(pf4[2 * P1 + o], pf4[3 * P1 + o])));
                    accf = df4_add(accf, shf);
                }
            }
        }
        if constexpr (DF) {
            // the children read the pairs (the input of their shifts); the
            // FP64 result, read by the later kernels only, is the FP64 sums
            // plus the shifted parent, stored after the flag, off the chain
            if (w == 0 && o < P1) outdf[b * P1 + o] = accf;
            flag_publish(&flag[b], 2);   // its barrier also frees the shared buffers
            if (w == 0 && o < P1)
                out[b * P1 + o] = make_double2(acc.x + (double(shf.x) + double(shf.y)),
                                               acc.y + (double(shf.z) + double(shf.w)));
        } else {
            if (w == 0 && o < P1) out[b * P1 + o] = acc;
            flag_publish(&flag[b], 2);   // its barrier also frees the shared buffers
        }
    }
}

// -------------------------------------------------------------------------
// down_warps: the FP64 downward pass with one warp per box (the same result
// as k_down_levels<false>).  Warp g of the grid takes the boxes
// level_start[2] + g, + G, ... (G warps in all), in ascending order, and for
// each:
//   the box's own sums (lane o = coefficient o): the V-list sum (vsum: the
//     row k_m2l_boxes wrote into out[b]; else the rows Pv[e] of the pairs and
//     the V-list log term), the X-list rows PX[x] and the X-list log term;
//   then (levels >= 3), once the parent is published, the parent's expansion
//     shifted to this box in factored form (ShiftFac: so_q[l] sum_k B[l][k]
//     si_q[k] parent[k], B's terms on the 32-lane schedule);
//   the result is written to out[b] and published by flag[b] = 2.
// A box waits only for its parent, a box of smaller index, so every wait
// ends once every warp is resident (the grid comes from the occupancy
// calculator).  Each warp of a block sits on its own SM sub-partition, so the
// shifts of concurrently processed boxes use all four FP64 pipes.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_down_warps(const int64_t *__restrict__ level_start, int nlevels, const int32_t *__restrict__ v_ptr,
             const double2 *__restrict__ Pv, const int32_t *__restrict__ x_ptr, const int32_t *__restrict__ x_src,
             const double2 *__restrict__ PX, int px_stride, const int32_t *__restrict__ leaf_box,
             const double2 *__restrict__ first, const int32_t *__restrict__ parent,
             const int32_t *__restrict__ box_ix, const int32_t *__restrict__ box_iy, ShiftFac pf, double2 *out, int P1,
             const double *__restrict__ lvtab, const int32_t *__restrict__ v_lsrc,
             const int32_t *__restrict__ v_code, const double *__restrict__ logd, bool vsum, int32_t *flag,
             long long limit, int32_t *err)
{
    extern __shared__ double2 sdw[];
    const int TF = pf.T, SLF = P1 * pf.maxp;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double2 *se = sdw + w * (P1 + SLF);                                   // [P1] si_q * parent
    double2 *fslot = se + P1;                                             // [SLF] run sums
    double *fcoef = reinterpret_cast<double *>(sdw + nw * (P1 + SLF));    // [TF][32]
    uint32_t *fcode = reinterpret_cast<uint32_t *>(fcoef + TF * 32);      // [TF][32]
    int32_t *fnp = reinterpret_cast<int32_t *>(fcode + TF * 32);          // [P1]
    for (int i = threadIdx.x; i < TF * 32; i += blockDim.x) {
        fcoef[i] = __ldg(&pf.coef[i]);
        fcode[i] = __ldg(&pf.code[i]);
    }
    for (int i = threadIdx.x; i < P1; i += blockDim.x) fnp[i] = __ldg(&pf.np[i]);
    __syncthreads();
    griddep_wait();
    griddep_launch_dependents();
    const int o = lane;   // coefficient of this lane (P1 <= 32)
    const int64_t G = int64_t(gridDim.x) * nw;
    for (int64_t b = level_start[2] + int64_t(blockIdx.x) * nw + w; b < level_start[nlevels]; b += G) {
        const int lvb = lv_of(level_start, nlevels, b);
        const bool shift = lvb >= 3;
        const int pb = shift ? parent[b] : 0;
        const int q = (box_ix[b] & 1) + 2 * (box_iy[b] & 1);
        double2 fsi = make_double2(0.0, 0.0), fso = make_double2(0.0, 0.0);
        if (shift && o < P1) {   // the shift's diagonals do not depend on the parent's values
            fsi = __ldg(&pf.si[q * P1 + o]);
            fso = __ldg(&pf.so[q * P1 + o]);
        }
        // ---- the box's own sums
        double re = 0.0, im = 0.0;
        if (o < P1) {
            if (vsum) {
                const double2 t = out[b * P1 + o];
                re = t.x;
                im = t.y;
            } else {
                for (int e = v_ptr[b]; e < v_ptr[b + 1]; e++) {
                    const double2 t = Pv[int64_t(e) * P1 + o];
                    re += t.x;
                    im += t.y;
                }
            }
        }
        const int x0 = x_ptr[b], x1 = x_ptr[b + 1];
        if (o < P1) {
#pragma unroll 4
            for (int x = x0; x < x1; x++) {
                const double2 t = PX[int64_t(x) * px_stride + o];
                re += t.x;
                im += t.y;
            }
        }
        // log terms, one entry per lane: the X list (times log r of the
        // source level) and, for tensor-core M2L rows, the V list
        double lx = 0.0, lr = 0.0, li = 0.0;
        for (int x = x0 + lane; x < x1; x += 32) lx += first[int64_t(leaf_box[x_src[x]]) * P1].x;
        if (!vsum && v_lsrc) {
            const double lgb = lvtab[kLvTab + lvb];
            for (int e = v_ptr[b] + lane; e < v_ptr[b + 1]; e += 32) {
                const double2 a0 = first[int64_t(v_lsrc[e]) * P1];
                const double c0 = logd[v_code[e]] + lgb;
                lr = fma(c0, a0.x, lr);
                li = fma(c0, a0.y, li);
            }
        }
        for (int m = 16; m > 0; m >>= 1) {
            lx += __shfl_xor_sync(0xffffffffu, lx, m);
            lr += __shfl_xor_sync(0xffffffffu, lr, m);
            li += __shfl_xor_sync(0xffffffffu, li, m);
        }
        if (o == 0) {
            re = fma(lvtab[kLvTab + lvb - 1], lx, re + lr);
            im += li;
        }
        // ---- plus the parent's expansion shifted to this box (levels >= 3)
        if (shift) {
            if (lane == 0) flag_wait(&flag[pb], 2, limit, err);
            __syncwarp();
            if (o < P1) {
                const double2 A = __ldcg(&out[int64_t(pb) * P1 + o]);
                se[o] = make_double2(fma(A.x, fsi.x, -A.y * fsi.y), fma(A.x, fsi.y, A.y * fsi.x));
            }
            __syncwarp();
            double sr = 0.0, si = 0.0;
#pragma unroll 2
            for (int t = 0; t < TF; t++) {
                const uint32_t code = fcode[t * 32 + lane];
                const double cf = fcoef[t * 32 + lane];
                const double2 xv = se[code & 255u];
                sr = fma(cf, xv.x, sr);
                si = fma(cf, xv.y, si);
                if (code >> 8) {   // the run leaves an output here
                    fslot[(code >> 8) - 1u] = make_double2(sr, si);
                    sr = si = 0.0;
                }
            }
            __syncwarp();
            if (o < P1) {
                double2 y = fslot[o * pf.maxp];
                for (int j = 1; j < fnp[o]; j++) {
                    const double2 v = fslot[o * pf.maxp + j];
                    y.x += v.x;
                    y.y += v.y;
                }
                re += fma(y.x, fso.x, -y.y * fso.y);
                im += fma(y.x, fso.y, y.y * fso.x);
            }
        }
        if (o < P1) out[b * P1 + o] = make_double2(re, im);
        // the warp's writes are ordered before lane 0's release store; the
        // next box's shared-memory writes come after every lane's reads
        __syncwarp();
        if (lane == 0) asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(&flag[b]), "r"(2) : "memory");
    }
}

inline size_t down_warps_smem_bytes(int P1, int T, int maxp, int nwarps)
{
    return sizeof(double2) * size_t(nwarps) * (P1 + size_t(P1) * maxp) + (sizeof(double) + sizeof(uint32_t)) * T * 32 +
           sizeof(int32_t) * P1;
}

// -------------------------------------------------------------------------
// leafB: for every leaf o, node j
//   out[o][j] = sE * Re(sum_l OpE[l][j] own[box(o)][l])                  (level >= 2)
//             + sum_{w in W(o)} [ sW * Re(sum_k OpW[code][k][j] src[w][k]) + cW_j * Re(src[w][0]) ]
//             + sum_{s in near(o)} [ sN * sum_k T[tab][k][j] v[s][k] + cN_j * Re(aux[box(s)][0]) ]
//   forward: sE = 1, sW = 1, cW = log r_o, sN = r_s^2, cN = log r_s (aux = multipoles: A_0 = r^2 w.f / 2pi)
//   adjoint: sE = r_o^2, sW = r_o^2, cW = r_o^2 log r_o w_j / 2pi, sN = r_o^2,
//            cN = r_o^2 log r_o w_j / 2pi (aux = adjoint locals: B_0 = sum_i g_i)
// The log terms factor per leaf (cW_j, and in the adjoint cN_j, do not depend
// on the entry; in the forward apply cN = log r_s does not depend on j): the
// first warp sums them over the W and near lists, one entry per lane, so the
// products of the lists are plain streams of independent loads.
// -------------------------------------------------------------------------
// The log-term sums of each target leaf's W and near lists (one warp per
// leaf, one entry per lane), computed before the leaf output so that its
// blocks stream the partial rows without waiting on this gather:
//   logs[o].x = sum_W A_0(w),  logs[o].y = sum_near log(r_s) A_0(s)  (forward)
//                                          sum_near B_0(s)           (adjoint)
template <bool ADJ>
__global__ void __launch_bounds__(256)
k_leaf_logs(int64_t nleaf, const int32_t *__restrict__ leaf_box, const int32_t *__restrict__ leaf_level,
            const int32_t *__restrict__ w_ptr, const int32_t *__restrict__ w_src, const int32_t *__restrict__ n_ptr,
            const int32_t *__restrict__ n_src, const double2 *__restrict__ src, const double2 *__restrict__ aux,
            const double *__restrict__ lvtab, int P1, double2 *__restrict__ logs)
{
    griddep_wait();
    griddep_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t o = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5); o < nleaf; o += nw) {
        double lw = 0.0, ln = 0.0;
        for (int e = w_ptr[o] + lane; e < w_ptr[o + 1]; e += 32) lw += src[int64_t(w_src[e]) * P1].x;
        for (int e = n_ptr[o] + lane; e < n_ptr[o + 1]; e += 32) {
            const int s = n_src[e];
            const double a0 = aux[int64_t(leaf_box[s]) * P1].x;
            ln += ADJ ? a0 : lvtab[kLvTab + leaf_level[s]] * a0;
        }
        for (int m = 16; m > 0; m >>= 1) {
            lw += __shfl_xor_sync(0xffffffffu, lw, m);
            ln += __shfl_xor_sync(0xffffffffu, ln, m);
        }
        if (lane == 0) logs[o] = make_double2(lw, ln);
    }
}

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
                           const double *__restrict__ PW, const uint8_t *__restrict__ active,
                           const double2 *__restrict__ logs)
{
    griddep_wait();
    griddep_launch_dependents();
    extern __shared__ double2 sh[];
    double2 *se = sh;                                  // P1
    double *sv = reinterpret_cast<double *>(sh + P1);  // NP
    __shared__ double s_log[2];
    const int lane = threadIdx.x & 31;
    for (int64_t li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int o = order[li];
        if (active && !active[o]) {   // a discarded leaf of a truncated tree (uniform over the block)
            vout[int64_t(o) * NP + threadIdx.x] = 0.0;
            continue;
        }
        const int lvo = leaf_level[o];
        const double r2o = lvtab[lvo], lgo = lvtab[kLvTab + lvo];
        const int j = threadIdx.x;   // blockDim.x == NP
        const double wj = wvec[j];
        // adjoint log term of a target leaf o: r_o^2 log(r_o) w_j / (2 pi)
        const double cO = ADJ ? r2o * lgo * wj * kInvTwoPi : lgo;
        const int w0 = w_ptr[o], w1 = w_ptr[o + 1], n0 = n_ptr[o], n1 = n_ptr[o + 1];
        if (!logs) __syncthreads();   // s_log of the previous leaf has been read
        if (!logs && threadIdx.x < 32) {
            // The log terms of the W and near sources, gathered by the first
            // warp (one entry per lane) while the others start on the products:
            //   lw = sum_W A_0(w)              (times cO below)
            //   ln = sum_near log(r_s) A_0(s)  forward,  sum_near B_0(s) adjoint (times cO)
            double lw = 0.0, ln = 0.0;
            for (int e = w0 + lane; e < w1; e += 32) lw += src[int64_t(w_src[e]) * P1].x;
            for (int e = n0 + lane; e < n1; e += 32) {
                const int s = n_src[e];
                const double a0 = aux[int64_t(leaf_box[s]) * P1].x;
                ln += ADJ ? a0 : lvtab[kLvTab + leaf_level[s]] * a0;
            }
            for (int m = 16; m > 0; m >>= 1) {
                lw += __shfl_xor_sync(0xffffffffu, lw, m);
                ln += __shfl_xor_sync(0xffffffffu, ln, m);
            }
            if (lane == 0) {
                s_log[0] = lw;
                s_log[1] = ln;
            }
        }
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
        if (PW) {
#pragma unroll 4
            for (int e = w0; e < w1; e++) acc += PW[size_t(e) * NP + j];
        } else {
            for (int e = w0; e < w1; e++) {
                const double2 *op = OpW + size_t(w_code[e]) * P1 * NP;
                __syncthreads();
                for (int i = threadIdx.x; i < P1; i += blockDim.x) se[i] = src[int64_t(w_src[e]) * P1 + i];
                __syncthreads();
                double s = 0.0;
                for (int k = 0; k < P1; k++) {
                    double2 opk = op[k * NP + j], b = se[k];
                    s = fma(opk.x, b.x, fma(-opk.y, b.y, s));
                }
                acc = fma(sW, s, acc);
            }
        }
        if (Pnear) {
            // split-precision results of the entries, scale already applied
#pragma unroll 4
            for (int e = n0; e < n1; e++) acc += Pnear[size_t(e) * NP + j];
        } else {
            for (int e = n0; e < n1; e++) {
                const int s = n_src[e];
                const double *tb = T + size_t(n_tab[e]) * NP * NP;
                __syncthreads();
                for (int i = threadIdx.x; i < NP; i += blockDim.x) sv[i] = vnear[int64_t(s) * NP + i];
                __syncthreads();
                double t = 0.0;
                for (int k = 0; k < NP; k++) t = fma(tb[k * NP + j], sv[k], t);
                acc = fma(ADJ ? r2o : lvtab[leaf_level[s]], t, acc);
            }
        }
        double l0, l1;
        if (logs) {
            const double2 lg = logs[o];
            l0 = lg.x;
            l1 = lg.y;
        } else {
            __syncthreads();   // s_log written
            l0 = s_log[0];
            l1 = s_log[1];
        }
        acc = fma(cO, l0, acc);
        acc = ADJ ? fma(cO, l1, acc) : acc + l1;
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

// -------------------------------------------------------------------------
// Value and gradient of the leaf interpolant at points (v_bulk and its
// gradient off the grid, as the glue step needs them on the fictitious curve):
// the point's leaf is found as in k_eval_points; with xi its reference
// coordinate, l_j the barycentric Lagrange basis (weights lam_j) and
// w_j = lam_j / (xi - x_j), S = sum w_j, T = sum w_j / (xi - x_j):
//     l_j = w_j / S,   l'_j = l_j (T/S - 1/(xi - x_j))   (j not the nearest node m)
//     l'_m = l_m sum_{k != m} lam_k (x_k - x_m) / (xi - x_k)^2 / (lam_m + d sum_{k != m} w_k),
// d = xi - x_m, which is the same quantity without the cancellation of
// T/S - 1/d as the point nears x_m; at a node the differentiation matrix
// D_mj = (lam_j / lam_m) / (x_m - x_j), D_mm = -sum_{j != m} D_mj.
// grad u = (1/r) (sum l_jy sum l'_jx u, sum l'_jy sum l_jx u).
// -------------------------------------------------------------------------
__device__ void bary_with_derivative(int p, double xi, double *l, double *dl)
{
    const double pi = 3.14159265358979323846;
    double xn[kMaxP], lam[kMaxP];
    int m = 0;
    for (int k = 0; k < p; k++) {
        const double th = (2.0 * k + 1.0) * pi / (2.0 * p);
        xn[k] = -cos(th);
        lam[k] = ((k & 1) ? -1.0 : 1.0) * sin(th);
        if (fabs(xi - xn[k]) < fabs(xi - xn[m])) m = k;
    }
    const double d = xi - xn[m];
    if (fabs(d) < 1e-250) {   // at the node (closer than any w_k could be formed without overflow)
        double dmm = 0.0;
        for (int j = 0; j < p; j++) {
            l[j] = j == m ? 1.0 : 0.0;
            if (j == m) continue;
            dl[j] = (lam[j] / lam[m]) / (xn[m] - xn[j]);
            dmm -= dl[j];
        }
        dl[m] = dmm;
        return;
    }
    double S = 0.0, T = 0.0, Sr = 0.0, Q = 0.0;   // Sr = sum_{k != m} w_k, Q = sum_{k != m} lam_k (x_k - x_m)/(xi - x_k)^2
    for (int k = 0; k < p; k++) {
        const double e = xi - xn[k], w = lam[k] / e;
        S += w;
        T += w / e;
        if (k != m) {
            Sr += w;
            Q += lam[k] * (xn[k] - xn[m]) / (e * e);
        }
    }
    for (int j = 0; j < p; j++) {
        l[j] = (lam[j] / (xi - xn[j])) / S;
        dl[j] = j == m ? l[j] * Q / (lam[m] + d * Sr) : l[j] * (T / S - 1.0 / (xi - xn[j]));
    }
}

__global__ void k_eval_points_grad(int64_t n, const double *__restrict__ xy, const double *__restrict__ u,
                                   const int32_t *__restrict__ child0, const int32_t *__restrict__ box_leaf,
                                   const int32_t *__restrict__ box_level, const int32_t *__restrict__ box_ix,
                                   const int32_t *__restrict__ box_iy, double x0, double y0, double L, int p,
                                   double *__restrict__ val, double *__restrict__ grad)
{
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double x = xy[2 * k], y = xy[2 * k + 1];
        if (!(x >= x0 && x <= x0 + L && y >= y0 && y <= y0 + L)) {
            val[k] = grad[2 * k] = grad[2 * k + 1] = nan("");
            continue;
        }
        int b = 0;
        while (box_leaf[b] < 0) {
            const int lv = box_level[b];
            const double h = ldexp(L, -lv);
            const double mx = x0 + (box_ix[b] + 0.5) * h, my = y0 + (box_iy[b] + 0.5) * h;
            b = child0[b] + (x >= mx ? 1 : 0) + (y >= my ? 2 : 0);
        }
        const int lv = box_level[b];
        const double h = ldexp(L, -lv), r = 0.5 * h;
        const double xi = (x - (x0 + (box_ix[b] + 0.5) * h)) / r, eta = (y - (y0 + (box_iy[b] + 0.5) * h)) / r;
        double lx[kMaxP], ly[kMaxP], dlx[kMaxP], dly[kMaxP];
        bary_with_derivative(p, xi, lx, dlx);
        bary_with_derivative(p, eta, ly, dly);
        const double *ub = u + int64_t(box_leaf[b]) * p * p;
        double v = 0.0, gx = 0.0, gy = 0.0;
        for (int jy = 0; jy < p; jy++) {
            double row = 0.0, drow = 0.0;
            for (int jx = 0; jx < p; jx++) {
                const double uv = ub[jy * p + jx];
                row = fma(lx[jx], uv, row);
                drow = fma(dlx[jx], uv, drow);
            }
            v = fma(ly[jy], row, v);
            gx = fma(ly[jy], drow, gx);
            gy = fma(dly[jy], row, gy);
        }
        val[k] = v;
        grad[2 * k] = gx / r;
        grad[2 * k + 1] = gy / r;
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
    const SideStream *sd = split ? split->side : nullptr;
    SplitGemm gv;   // tensor group V
    if (split) {
        gv.ops = sT->ops[0][dir]; gv.op_exp = sT->op_exp[0][dir];
        gv.dig = sp->vdig; gv.dexp = sp->vexp;
    }
    const bool leaf_tc = (parts & 2) != 0;
    // Late fork: with the M2L in FP64 (part 32 off) the internal stream's
    // tensor launches (X list, near field) start after the upward pass and run
    // beside the FP64 M2L, which leaves room for one tensor CTA per SM; the
    // upward pass runs alone before it.  Otherwise they start at once, beside
    // the level passes.
    const bool late = sd && !(parts & 32) && leaf_tc;
    // the internal stream's launches: X-list tiles (needed by the downward
    // pass, which waits for xdone), then the near field (joined before the
    // leaf output)
    auto side_launches = [&]() -> cudaError_t {
        cudaError_t e;
        if ((e = cudaEventRecord(sd->fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(sd->side, sd->fork, 0)) != cudaSuccess)
            return e;
        if (ev) cudaEventRecord(ev[8], sd->side);
        if (!leaf_tc) {
            e = launch_split_digits_vec(a.nleaf, vin, alpha0, sp->vdig, sp->vexp, sd->side, d.leaf_active,
                                            a.NP, sT->kv);
            if (e != cudaSuccess) return e;
        }
        SplitGemm g = gv;
        g.tiles = sp->tV[dir] + sp->ntA[dir]; g.cols = sp->cV[dir]; g.ntiles = sp->ntV[dir] - sp->ntA[dir];
        e = launch_split_gemm(g, sT->kv, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, sd->side, late);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(sd->xdone, sd->side)) != cudaSuccess) return e;
        if (late) {
            // the W list needs the multipoles only: their digits and the W
            // tiles here too, beside the FP64 M2L (the downward pass's group E
            // keeps the expansion-to-leaf tiles)
            const int64_t f0 = adj ? a.nbox : 0;
            e = launch_split_digits_exp(f0, f0 + a.nbox, a.nbox, d.expA, d.expB, P1, adj ? alpha0 : 1.0,
                                        sT->escale[dir], sp->edig, sp->eexp, sd->side);
            if (e != cudaSuccess) return e;
            SplitGemm gw;
            gw.tiles = sp->tE[dir] + sp->ntL[dir]; gw.cols = sp->cE[dir]; gw.ntiles = sp->ntE[dir] - sp->ntL[dir];
            gw.ops = sT->ops[1][dir]; gw.op_exp = sT->op_exp[1][dir];
            gw.dig = sp->edig; gw.dexp = sp->eexp;
            e = launch_split_gemm(gw, kSplitKE, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, sd->side,
                                  true);
            if (e != cudaSuccess) return e;
        }
        g.tiles = sp->tN[dir]; g.cols = sp->cN[dir]; g.ntiles = sp->ntN[dir];
        g.max_ctas = split->near_ctas;
        e = launch_split_gemm(g, sT->kv, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, sd->side, late);
        if (e != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[9], sd->side);
        return cudaEventRecord(sd->join, sd->side);
    };
    if (split) {
        // tensor group V: digits of alpha0 * vin; the near field into Pnear,
        // leafA (P2M / L2P^H, part 2) into `first` and the X list into PX, in
        // one launch, or (split_overlap) the leaf-to-expansion tiles in line
        // and the X list and the near field on the internal stream
        if (!sd) {
            // one launch: the near-field tiles (two jobs each) first, then the
            // leaf-to-expansion and X-list tiles
            ce = launch_split_digits_vec(a.nleaf, vin, alpha0, sp->vdig, sp->vexp, st, d.leaf_active, a.NP,
                                             sT->kv);
            if (ce != cudaSuccess) return ce;
            SplitGemm g = gv;
            g.tiles = sp->tVN[dir]; g.cols = sp->cVN[dir]; g.ntiles = sp->ntVN[dir];
            ce = launch_split_gemm(g, sT->kv, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, st);
            if (ce != cudaSuccess) return ce;
            if (ev) {
                cudaEventRecord(ev[8], st);
                cudaEventRecord(ev[9], st);
            }
        } else {
            // The upward pass needs the leaf-to-expansion step first: as
            // tensor tiles in line (part 2, after the digits), else in
            // double-float inside the upward pass, and then the digits run on
            // the internal stream too.
            if (leaf_tc) {
                ce = launch_split_digits_vec(a.nleaf, vin, alpha0, sp->vdig, sp->vexp, st, d.leaf_active, a.NP,
                                             sT->kv);
                if (ce != cudaSuccess) return ce;
            }
            if (!late && (ce = side_launches()) != cudaSuccess) return ce;
            if (leaf_tc) {
                SplitGemm g = gv;
                g.tiles = sp->tV[dir]; g.cols = sp->cV[dir]; g.ntiles = sp->ntA[dir];
                ce = launch_split_gemm(g, sT->kv, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, st);
                if (ce != cudaSuccess) return ce;
            }
        }
    } else if (ev) {
        cudaEventRecord(ev[8], st);
        cudaEventRecord(ev[9], st);
    }
    if (ev) cudaEventRecord(ev[1], st);
    // the per-box flags of the persistent passes start from zero
    {
        const int64_t nf = int64_t(h.box_level.size());
        ce = launch_pdl(k_clear_flags, grid_for((nf + 255) / 256, 152), 256, 0, st, d.flag, nf);
        if (ce != cudaSuccess) return ce;
    }
    if (ev) cudaEventRecord(ev[2], st);
    // flag polls go to L2 (several hundred cycles each): a sixteenth of the
    // mbarrier poll limit
    const long long glimit = std::max(1ll, a.wait_limit / 16);
    // leafA + upward pass in one persistent launch (leafA always runs: the
    // near-field log term reads coefficient 0 of its output; without the far
    // field no climb).  Split path: leafA came from the tensor cores.
    const int grid_leaf = grid_for(a.nleaf, 152 * (a.leaf_bps ? a.leaf_bps : 16));
    const double2 *opA = (parts & 2) ? nullptr : op.leafA;
    const bool climb = far && h.nlevels > 3;
    const bool dfp = (parts & 64) != 0;   // double-float shifts
    const size_t shU = dfp ? up_smem_bytes(NP, P1, op.up_s.T, op.up_s.maxp)
                           : up_smem_bytes_f64(NP, P1, op.up_f.T, op.up_f.maxp);
    if (opA || climb) {
#define BC_UP(A, D)                                                                                          \
    launch_pdl(k_up_levels<A, D>, a.up_blocks, 128, shU, st, a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level, \
               d.level_start, h.nlevels, d.box_child0, vin, opA, op.leafA_df, op.up_s, op.up_f, first, d.exdf, NP, \
               P1, d.lvtab, climb, d.flag, d.leaf_active, glimit, a.err, (const uint8_t *)nullptr)
        if (adj) ce = dfp ? BC_UP(true, true) : BC_UP(true, false);
        else ce = dfp ? BC_UP(false, true) : BC_UP(false, false);
#undef BC_UP
        if (ce != cudaSuccess) return ce;
    }
    if (late && (ce = side_launches()) != cudaSuccess) return ce;
    if (ev) cudaEventRecord(ev[3], st);
    bool first_digits = false;   // digits of `first` taken (tensor-core M2L)
    if (far && h.nlevels > 2) {
        // M2L: per V pair on the tensor cores (part 32; results one row per
        // pair, summed by the downward pass), else every box's V-list sum in
        // FP64, written into its row of `second`; then (FP64) the X-list
        // products, then the level-by-level sum
        const int64_t npairs = int64_t(h.v_src.size());
        if (npairs > 0 && (parts & 32)) {
            // tensor group M: digits of `first` (times alpha0 in the adjoint),
            // then every pair's translation but its log term
            const int64_t f0 = adj ? a.nbox : 0;
            ce = launch_split_digits_exp(f0, f0 + a.nbox, a.nbox, d.expA, d.expB, P1, adj ? alpha0 : 1.0,
                                         sT->escale[dir], sp->edig, sp->eexp, st);
            if (ce != cudaSuccess) return ce;
            first_digits = true;
            SplitGemm g;
            g.tiles = sp->tM[dir]; g.cols = sp->cM[dir]; g.ntiles = sp->ntM[dir];
            g.ops = sT->ops[1][dir]; g.op_exp = sT->op_exp[1][dir];
            g.dig = sp->edig; g.dexp = sp->eexp;
            ce = launch_split_gemm(g, kSplitKE, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, st);
            if (ce != cudaSuccess) return ce;
        } else if (a.m2l_kind == 1) {
            // FP64 tensor cores, one warp per target box; beside the
            // near-field tensor CTAs (late fork) two warps per SM
            // sub-partition fit next to one of them (registers)
            const int64_t b0 = h.level_start[2], b1 = a.nbox;
            const int grid = grid_for((b1 - b0 + 3) / 4, 152 * (a.m2l_bps ? a.m2l_bps : (late ? 2 : 4)));
            const double2 *dsig = adj ? tb.dsig_a : tb.dsig_f, *dpw = adj ? tb.dpow_a : tb.dpow_f;
#define BC_M2LT(A, MT, KS)                                                                                      \
    ce = launch_pdl(k_m2l_mma<A, MT, KS>, grid, 128, 0, st, b0, b1, d.v_ptr, d.v_src, d.v_code, d.box_level, dsig, \
                    dpw, tb.logd, d.lvtab, first, second, P1, m2l_tri)
#define BC_M2LD(MT, KS) { if (adj) BC_M2LT(true, MT, KS); else BC_M2LT(false, MT, KS); }
            switch ((P1 + 3) / 4) {
            case 1: BC_M2LD(1, 1) break;
            case 2: BC_M2LD(1, 2) break;
            case 3: BC_M2LD(2, 3) break;
            case 4: BC_M2LD(2, 4) break;
            case 5: BC_M2LD(3, 5) break;
            case 6: BC_M2LD(3, 6) break;
            case 7: BC_M2LD(4, 7) break;
            default: BC_M2LD(4, 8) break;
            }
#undef BC_M2LD
#undef BC_M2LT
            if (ce != cudaSuccess) return ce;
        } else {
            const int64_t b0 = h.level_start[2], b1 = a.nbox;
            const int ng = m2l_groups(P1), nth = m2l_threads(P1);
            const size_t shM = sizeof(double2) * 2 * ng * (P1 + 1);
            // beside the near-field tensor CTAs (late fork): 4 blocks per SM
            // fit next to one of them (registers per sub-partition, and the
            // shared memory the two-buffer tensor launch leaves)
            const int grid = grid_for(b1 - b0, 152 * (a.m2l_bps ? a.m2l_bps : (late ? 4 : 8)));
            const double2 *dsig = adj ? tb.dsig_a : tb.dsig_f, *dpw = adj ? tb.dpow_a : tb.dpow_f;
#define BC_M2L(A, PM)                                                                                           \
    ce = launch_pdl(k_m2l_boxes<A, PM>, grid, nth, shM, st, b0, b1, d.v_ptr, d.v_src, d.v_code, d.box_level, dsig, \
                    dpw, tb.logd, d.lvtab, first, second, P1, ng, m2l_tri)
            if (P1 <= 16) { if (adj) BC_M2L(true, 16); else BC_M2L(false, 16); }
            else if (P1 <= 24) { if (adj) BC_M2L(true, 24); else BC_M2L(false, 24); }
            else { if (adj) BC_M2L(true, 32); else BC_M2L(false, 32); }
#undef BC_M2L
            if (ce != cudaSuccess) return ce;
        }
        const double2 *PX = nullptr;
        int px_stride = P1;
        if (parts & 4) {
            PX = reinterpret_cast<const double2 *>(sp->PX);
            px_stride = kSplitKE / 2;
        } else if (!h.x_src.empty()) {
            const int64_t nx = int64_t(h.x_src.size());
            const size_t shX = sizeof(double2) * 4 * P1 + sizeof(double) * NP;
            if (adj)
                ce = launch_pdl(k_x_entries<true>, grid_for(nx, 152 * 16), 128, shX, st, nx, d.x_box, d.x_src,
                                d.x_code, d.box_level, op.x, vin, d.PX, NP, P1, d.lvtab);
            else
                ce = launch_pdl(k_x_entries<false>, grid_for(nx, 152 * 16), 128, shX, st, nx, d.x_box, d.x_src,
                                d.x_code, d.box_level, op.x, vin, d.PX, NP, P1, d.lvtab);
            if (ce != cudaSuccess) return ce;
            PX = d.PX;
        }
        if (ev) cudaEventRecord(ev[4], st);
        // the X-list products come from the internal stream
        if (split && split->side && (ce = cudaStreamWaitEvent(st, split->side->xdone, 0)) != cudaSuccess) return ce;
        if (dfp)
            ce = launch_pdl(k_down_levels<true>, a.shift_blocks, 128, down_smem_bytes(P1, 0, 0, true), st,
                            d.level_start, h.nlevels, d.v_ptr, d.Pv, d.x_ptr, d.x_src, PX, px_stride, d.leaf_box,
                            first, d.box_parent, d.box_ix, d.box_iy, op.par_df, op.par_f, second, d.exdf, P1, d.lvtab,
                            first_digits ? d.v_src : nullptr, d.v_code, tb.logd, !first_digits, d.flag, glimit,
                            a.err);
        else
            ce = launch_pdl(k_down_warps, a.down_blocks, 128, down_warps_smem_bytes(P1, op.par_f.T, op.par_f.maxp, 4),
                            st, d.level_start, h.nlevels, d.v_ptr, d.Pv, d.x_ptr, d.x_src, PX, px_stride,
                            d.leaf_box, first, d.box_parent, d.box_ix, d.box_iy, op.par_f, second, P1, d.lvtab,
                            first_digits ? d.v_src : nullptr, d.v_code, tb.logd, !first_digits, d.flag, glimit,
                            a.err);
        if (ce != cudaSuccess) return ce;
    } else if (ev) {
        cudaEventRecord(ev[4], st);
    }
    if (ev) cudaEventRecord(ev[5], st);
    if (split && far) {
        // tensor group E: digits of both expansion arrays (times alpha0 in the
        // adjoint; those of `first` already taken for the M2L or, late fork,
        // on the internal stream), then L2P (P2M^H) of `second` into PE and
        // the W list of `first` into PW (late fork: L2P only)
        const bool first_done = first_digits || late;
        const int64_t s0 = first_done ? (adj ? 0 : a.nbox) : 0, s1 = first_done ? s0 + a.nbox : 2 * a.nbox;
        ce = launch_split_digits_exp(s0, s1, a.nbox, d.expA, d.expB, P1, adj ? alpha0 : 1.0, sT->escale[dir],
                                     sp->edig, sp->eexp, st);
        if (ce != cudaSuccess) return ce;
        SplitGemm g;
        g.tiles = sp->tE[dir]; g.cols = sp->cE[dir]; g.ntiles = late ? sp->ntL[dir] : sp->ntE[dir];
        g.ops = sT->ops[1][dir]; g.op_exp = sT->op_exp[1][dir];
        g.dig = sp->edig; g.dexp = sp->eexp;
        ce = launch_split_gemm(g, kSplitKE, 1.0 / alpha0, sp->err, sT->wait_limit, sT->withhold_copy, st);
        if (ce != cudaSuccess) return ce;
    }
    // the log-term sums of every leaf's W and near lists (they read `first`
    // only), before the join: they run while the near field finishes
    {
        const int32_t *wl = far ? d.w_ptr : d.zero_ptr, *nl = near ? d.near_ptr : d.zero_ptr;
        const int lgrid = grid_for((a.nleaf + 7) / 8, 152 * 8);
        ce = adj ? launch_pdl(k_leaf_logs<true>, lgrid, 256, 0, st, a.nleaf, d.leaf_box, d.leaf_level, wl, d.w_src,
                              nl, d.near_src, first, first, d.lvtab, P1, d.leaf_logs)
                 : launch_pdl(k_leaf_logs<false>, lgrid, 256, 0, st, a.nleaf, d.leaf_box, d.leaf_level, wl, d.w_src,
                              nl, d.near_src, first, first, d.lvtab, P1, d.leaf_logs);
        if (ce != cudaSuccess) return ce;
    }
    if (ev) cudaEventRecord(ev[6], st);
    if (split && split->side && (ce = cudaStreamWaitEvent(st, split->side->join, 0)) != cudaSuccess) return ce;
    // leafB: own expansion = second (local / adjoint multipole), W sources and
    // near log aux = first (multipole / adjoint local)
    size_t shD = sizeof(double2) * P1 + sizeof(double) * NP;
    const int32_t *wp = far ? d.w_ptr : d.zero_ptr, *np_ = near ? d.near_ptr : d.zero_ptr;
    const double *Pnear = (parts & 1) ? sp->Pnear : nullptr, *PE = (parts & 8) ? sp->PE : nullptr,
                 *PW = (parts & 16) ? sp->PW : nullptr;
    if (adj)
        ce = launch_pdl(k_leaf_out<true>, grid_leaf, NP, shD, st, a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                        wp, d.w_src, d.w_code, np_, d.near_src, d.near_tab, op.e, op.w, op.t, tb.wvec, second, first,
                        first, vin, vout, NP, P1, d.lvtab, far, Pnear, PE, PW, d.leaf_active, d.leaf_logs);
    else
        ce = launch_pdl(k_leaf_out<false>, grid_leaf, NP, shD, st, a.nleaf, d.leaf_order, d.leaf_box, d.leaf_level,
                        wp, d.w_src, d.w_code, np_, d.near_src, d.near_tab, op.e, op.w, op.t, tb.wvec, second, first,
                        first, vin, vout, NP, P1, d.lvtab, far, Pnear, PE, PW, d.leaf_active, d.leaf_logs);
    if (ce != cudaSuccess) return ce;
    if (ev) cudaEventRecord(ev[7], st);
    return cudaGetLastError();
}

cudaError_t launch_far_points(const PassArgs &a, const HostTree &h, const DevTree &d, const DevTables &tb,
                              const FarLists &fl, cudaStream_t st)
{
    const int P1 = a.P1, NP = a.NP;
    const OpSet &op = tb.fwd;
    cudaError_t ce;
    const int64_t nf = int64_t(h.box_level.size());
    ce = launch_pdl(k_clear_flags, grid_for((nf + 255) / 256, 152), 256, 0, st, d.flag, nf);
    if (ce != cudaSuccess) return ce;
    if (h.nlevels <= 2) return cudaSuccess;
    const long long glimit = std::max(1ll, a.wait_limit / 16);
    if (h.nlevels > 3) {
        // climb only: the leaf expansions were written by the caller
        const size_t shU = up_smem_bytes_f64(NP, P1, op.up_f.T, op.up_f.maxp);
        ce = launch_pdl(k_up_levels<false, false>, a.up_blocks, 128, shU, st, a.nleaf, d.leaf_order, d.leaf_box,
                        d.leaf_level, d.level_start, h.nlevels, d.box_child0, (const double *)nullptr,
                        (const double2 *)nullptr, op.leafA_df, op.up_s, op.up_f, d.expA, d.exdf, NP, P1, d.lvtab,
                        true, d.flag, (const uint8_t *)nullptr, glimit, a.err, fl.live);
        if (ce != cudaSuccess) return ce;
    }
    {
        const int64_t b0 = h.level_start[2], b1 = a.nbox;
        const int ng = m2l_groups(P1), nth = m2l_threads(P1);
        const size_t shM = sizeof(double2) * 2 * ng * (P1 + 1);
        const int grid = grid_for(b1 - b0, 152 * (a.m2l_bps ? a.m2l_bps : 8));
#define BC_M2LP(PM)                                                                                             \
    ce = launch_pdl(k_m2l_boxes<false, PM>, grid, nth, shM, st, b0, b1, fl.v_ptr, fl.v_src, fl.v_code,          \
                    d.box_level, (const double2 *)nullptr, tb.dpow_f, tb.logd, d.lvtab, d.expA, d.expB, P1, ng, 0)
        if (P1 <= 16) BC_M2LP(16);
        else if (P1 <= 24) BC_M2LP(24);
        else BC_M2LP(32);
#undef BC_M2LP
        if (ce != cudaSuccess) return ce;
    }
    return launch_pdl(k_down_warps, a.down_blocks, 128, down_warps_smem_bytes(P1, op.par_f.T, op.par_f.maxp, 4), st,
                      d.level_start, h.nlevels, fl.v_ptr, d.Pv, fl.x_ptr, fl.x_src, fl.PX, P1, d.leaf_box, d.expA,
                      d.box_parent, d.box_ix, d.box_iy, op.par_f, d.expB, P1, d.lvtab, (const int32_t *)nullptr,
                      fl.v_code, tb.logd, true, d.flag, glimit, a.err);
}

cudaError_t fp64_prepare(int NP, int P1, int df_T, int df_maxp, int f_T, int f_maxp, int up_per_sm, int down_per_sm,
                         int *up_blocks, int *shift_blocks, int *down_blocks)
{
    {
        // binomial table of the factored M2L (see c_binom)
        double tab[32][32];
        for (int k = 0; k < 32; k++)
            for (int o = 0; o < 32; o++) {
                if (k == 0) {
                    tab[k][o] = o == 0 ? 0.0 : -1.0 / o;
                    continue;
                }
                long double c = 1.0L;   // C(k + o - 1, o)
                const int n = k + o - 1, m = std::min(o, n - o);
                for (int t = 1; t <= m; t++) c = c * (n - m + t) / t;
                tab[k][o] = double(c);
            }
        double tabT[32][32];
        for (int k = 0; k < 32; k++)
            for (int o = 0; o < 32; o++) tabT[k][o] = tab[o][k];
        cudaError_t e = cudaMemcpyToSymbol(c_binom, tab, sizeof(tab));
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_binomT, tabT, sizeof(tabT));
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, bu0 = 0, bu1 = 0, bs = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t shU = up_smem_bytes_f64(NP, P1, f_T, f_maxp), shUd = up_smem_bytes(NP, P1, df_T, df_maxp);
    const size_t shD = down_smem_bytes(P1, f_T, f_maxp, false), shDd = down_smem_bytes(P1, 0, 0, true);
    // the double-float variants hold the scheduled shift operators in shared
    // memory, beyond the default 48 KB at high orders; the limit is per
    // kernel, so it is only ever raised (contexts of different orders share
    // the kernels)
    for (const void *k : {(const void *)k_up_levels<false, true>, (const void *)k_up_levels<true, true>}) {
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
        if (e == cudaSuccess && size_t(fa.maxDynamicSharedSizeBytes) < shUd)
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shUd));
    }
    // The kernels that run before and beside the near-field tensor launch
    // prefer the largest shared-memory carveout: an SM's split between L1 and
    // shared memory is fixed while any block is resident on it, and a smaller
    // one, set by these kernels' blocks, would keep the tensor CTA (about
    // 220 KB of shared memory) off that SM until they have all exited.
    for (const void *k : {(const void *)k_clear_flags, (const void *)k_up_levels<false, false>,
                          (const void *)k_up_levels<true, false>, (const void *)k_up_levels<false, true>,
                          (const void *)k_up_levels<true, true>, (const void *)k_m2l_boxes<false, 16>,
                          (const void *)k_m2l_boxes<true, 16>, (const void *)k_m2l_boxes<false, 24>,
                          (const void *)k_m2l_boxes<true, 24>, (const void *)k_m2l_boxes<false, 32>,
                          (const void *)k_m2l_boxes<true, 32>, (const void *)k_down_warps,
                          (const void *)k_down_levels<false>, (const void *)k_down_levels<true>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    // every block of a persistent pass must be resident: the smallest
    // occupancy over the variants that share the grid
    int bu2 = 0, bu3 = 0, bs2 = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu0, k_up_levels<false, false>, 128, shU);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu1, k_up_levels<true, false>, 128, shU);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu2, k_up_levels<false, true>, 128, shUd);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu3, k_up_levels<true, true>, 128, shUd);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, k_down_levels<false>, 128, shD);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs2, k_down_levels<true>, 128, shDd);
    int bw = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bw, k_down_warps, 128,
                                                          down_warps_smem_bytes(P1, f_T, f_maxp, 4));
    if (e != cudaSuccess) return e;
    const int bu = std::min(std::min(bu0, bu1), std::min(bu2, bu3));
    bs = std::min(bs, bs2);
    if (bu < 1 || bs < 1 || bw < 1) return cudaErrorInvalidConfiguration;
    *up_blocks = sms * std::min(up_per_sm, bu);
    *shift_blocks = sms * std::min(down_per_sm, bs);
    *down_blocks = sms * std::min(down_per_sm, bw);
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

cudaError_t launch_eval_points_grad(const PassArgs &a, const DevTree &d, const double *u, const double *xy, int64_t n,
                                    double *val, double *grad, double x0, double y0, double L, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int grid = int(std::min<int64_t>((n + 127) / 128, 152 * 8));
    k_eval_points_grad<<<grid, 128, 0, st>>>(n, xy, u, d.box_child0, d.box_leaf, d.box_level, d.box_ix, d.box_iy,
                                             x0, y0, L, a.p, val, grad);
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
