// Split-precision operator products on the 5th-generation tensor cores
// (tcgen05), p = 16.
//
// Every fixed-operator product of the apply except the multipole-to-local
// translations -- the near-field tables, P2M, L2P, the W list (M2P) and the
// X list (P2L), and their adjoints -- is a dense real matrix (the operator)
// times many vectors (leaf values or expansion coefficients).  Each product
// is evaluated exactly in integer arithmetic on BF16 tensor cores:
//   * each FP64 operand row (operator row, input vector) is scaled by a power
//     of two 2^E so that its entries lie in (-1/2, 1/2), rounded to a 40-bit
//     fixed-point integer X and cut into five balanced base-256 digits,
//     X = sum_a theta_a 256^(5-a), |theta_a| <= 128; every digit is an integer
//     that BF16 holds exactly (Ozaki-style error-free splitting);
//   * A v = 2^(E_A + E_v - 48) * sum_g 256^(6-g) D_g,  D_g = sum_{a+b=g} theta_a . phi_b,
//     keeping the digit pairs a + b <= 6 (15 products; what is dropped is below
//     2^-38 relative to sum_k |A_ik v_k|);
//   * each D_g (g = 2..6) accumulates in its own FP32 TMEM accumulator: every
//     product is an integer of magnitude <= 2^14 and a level sums at most
//     4 x 256 of them for g <= 5, so the accumulation is exact (< 2^24);
//   * the five levels are combined in int64 and converted to FP64 once, by
//     integer operations on the bit pattern (the FP64 pipe stays free).
//
// Work decomposition: a tile is one operator times up to 48 columns.
//   B operand: the columns' digits, gathered into shared memory with 16-byte
//              asynchronous copies (cp.async), resident for the whole tile;
//   A operand: the operator's digits, 128 rows x KC columns per chunk, brought
//              in by bulk asynchronous copies through three buffers: the copy
//              of chunk i+2 starts when the MMAs of chunk i-1 are done and
//              overlaps those of chunks i and i+1;
//   D:         5 levels x 2 row halves x 48 columns of FP32 in TMEM.
// The gather of the next tile and its first operator chunks are issued before
// the epilogue of the current tile, so they overlap it.  All waits are bounded:
// a wait that runs out sets the error flag, waits (bounded) for the copies and
// MMAs in flight, frees TMEM and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "bc_internal.h"

namespace bc {

namespace {

constexpr int kS = kSplitSlices;   // 5 digits
constexpr int kN = kSplitTileN;    // 48 columns per tile
constexpr int kNBuf = 3;           // operator chunk buffers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// UMMA shared-memory descriptor, K-major, no swizzle: core matrices of 8 rows
// x 16 bytes; lbo = byte step between core matrices along K, sbo = byte step
// between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFFu) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;   // descriptor version for tcgen05
    return d;                 // base offset 0, absolute LBO, SWIZZLE_NONE
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait on an mbarrier phase by a whole warp; false when the limit ran
// out.  The result is uniform over the warp.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, long long limit)
{
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < limit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (__any_sync(0xffffffffu, ok)) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// MMA and commit executed by a whole (converged) warp: one elected lane
// issues them, so the operands stay warp-uniform.
__device__ __forceinline__ void umma_bf16_warp(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit_warp(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// S * 2^ex as an FP64 value (round to nearest even) by integer operations on
// the bit pattern, keeping the conversion off the FP64 pipe.  |S| < 2^62.
__device__ __forceinline__ double i64_scaled(long long S, int ex)
{
    if (S == 0) return 0.0;
    const unsigned long long sign = S < 0 ? (1ull << 63) : 0ull;
    const unsigned long long m = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
    const int lz = __clzll(m);
    const unsigned long long t = m << lz;                 // leading one at bit 63
    unsigned long long mant = t >> 11;                    // 53 bits with the leading one
    const unsigned long long rem = t & 0x7FFull;
    if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) mant++;
    const long long be = (long long)(63 - lz + ex) + 1023;   // biased exponent
    if (be <= 0) return 0.0;                              // below the normal range: negligible here
    const unsigned long long bits = ((unsigned long long)be << 52) + (mant - (1ull << 52));
    return __longlong_as_double((long long)(bits | sign));
}

// Five balanced base-256 digits (BF16 bit patterns) of round(x * 2^(40 - E)),
// |x| < 2^(E-1), from the FP64 bit pattern by integer operations; written to
// out[0], out[stride], ... (most significant first).
__device__ __forceinline__ void digits_of(long long bits, int E, uint16_t *out, int stride)
{
    const int e = int((bits >> 52) & 0x7FF);
    long long X = 0;
    if (e != 0) {
        const long long mant = (bits & ((1ll << 52) - 1)) | (1ll << 52);
        const int rs = -(e - 1075 + 40 - E);   // >= 14
        X = rs >= 62 ? 0 : (mant + (1ll << (rs - 1))) >> rs;
        if (bits < 0) X = -X;
    }
#pragma unroll
    for (int a = kS; a >= 2; a--) {
        int d = int(X & 255);
        if (d >= 128) d -= 256;
        X = (X - d) >> 8;
        out[(a - 1) * stride] = uint16_t(__float_as_uint(float(d)) >> 16);
    }
    out[0] = uint16_t(__float_as_uint(float(int(X))) >> 16);   // leading digit, |X| <= 128
}

// ---------------------------------------------------------------------------
// Digits of scale * (leaf vectors): dig[leaf][a][k], dexp[leaf] = E with
// max |scale v| < 2^(E-1).  One block of 256 threads per leaf.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_split_vec(int64_t nleaf, const double *__restrict__ v, double scale,
                                                   uint16_t *__restrict__ dig, int32_t *__restrict__ dexp)
{
    __shared__ int wmax[8];
    const int k = threadIdx.x;
    for (int64_t leaf = blockIdx.x; leaf < nleaf; leaf += gridDim.x) {
        const long long bits = __double_as_longlong(scale * v[leaf * 256 + k]);
        int m = int((bits >> 52) & 0x7FF);
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((k & 31) == 0) wmax[k >> 5] = m;
        __syncthreads();
        int emax = wmax[0];
        for (int w = 1; w < 8; w++) emax = max(emax, wmax[w]);
        __syncthreads();
        const int E = emax ? emax - 1023 + 2 : 0;
        digits_of(emax ? bits : 0ll, E, dig + leaf * (kS * 256) + k, 256);
        if (k == 0) dexp[leaf] = E;
    }
}

// Digits of scale * s_k * (expansion coefficient k): vector i < nbox is ea[i]
// with column scales escale[0..63], else eb[i - nbox] with escale[64..127];
// its 2*P1 reals (re, im interleaved) padded with zeros to 64.  One warp per
// vector: dig[i][a][64], dexp[i].
__global__ void __launch_bounds__(256) k_split_exp(int64_t nbox, const double *__restrict__ ea,
                                                   const double *__restrict__ eb, int nreal, double scale,
                                                   const double *__restrict__ escale, uint16_t *__restrict__ dig,
                                                   int32_t *__restrict__ dexp)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < 2 * nbox; i += nw) {
        const double *src = i < nbox ? ea + i * nreal : eb + (i - nbox) * nreal;
        const double *sc = escale + (i < nbox ? 0 : kSplitKE);
        const long long b0 = lane < nreal ? __double_as_longlong(scale * sc[lane] * src[lane]) : 0ll;
        const long long b1 =
            lane + 32 < nreal ? __double_as_longlong(scale * sc[lane + 32] * src[lane + 32]) : 0ll;
        int m = max(int((b0 >> 52) & 0x7FF), int((b1 >> 52) & 0x7FF));
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int E = m ? m - 1023 + 2 : 0;
        uint16_t *out = dig + i * (kS * kSplitKE);
        digits_of(m ? b0 : 0ll, E, out + lane, kSplitKE);
        digits_of(m ? b1 : 0ll, E, out + lane + 32, kSplitKE);
        if (lane == 0) dexp[i] = E;
    }
}

// ---------------------------------------------------------------------------
// Operator x columns on tcgen05.  KD = 256 (leaf vectors) or 64 (expansions).
// ---------------------------------------------------------------------------
struct ColMeta {
    double *out;
    int32_t exp;    // E_v + shift - 48
    int32_t flag;   // multiply by 1/alpha0
    int32_t vec;
    int32_t pad;
};

template <int KD>
struct GemmShape {
    static constexpr int KC = KD < 128 ? KD : 128;    // K columns per operator chunk
    static constexpr int NKC = KD / KC;
    static constexpr int kBSlice = kN * KD * 2;        // bytes of one B digit slice
    static constexpr int kChunk = 128 * KC * 2;        // bytes of one operator chunk
    static constexpr int kBSBO = (KD / 8) * 128;       // B: bytes between 8-row groups
    static constexpr int kASBO = (KC / 8) * 128;       // A: bytes between 8-row groups
    static constexpr size_t kSmem = size_t(kS) * kBSlice + size_t(kNBuf) * kChunk + 2 * kN * sizeof(ColMeta) +
                                    2 * kNBuf * sizeof(uint64_t) + 16;
};

constexpr int kGemmThreads = 256;   // 8 warps: warp 0 issues, all 8 run the epilogue

template <int KD>
__global__ void __launch_bounds__(kGemmThreads, 1)
k_split_gemm(SplitGemm gm, double inv_alpha0, int32_t *__restrict__ err, long long wait_limit, int withhold)
{
    using Sh = GemmShape<KD>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *Bs = smem;                                                      // kS x kBSlice
    uint8_t *As = smem + kS * Sh::kBSlice;                                   // kNBuf x kChunk
    ColMeta *meta = reinterpret_cast<ColMeta *>(As + kNBuf * Sh::kChunk);    // [2][kN]
    uint64_t *lbar = reinterpret_cast<uint64_t *>(meta + 2 * kN);            // [kNBuf] chunk loaded
    uint64_t *mbar = lbar + kNBuf;                                           // [kNBuf] MMAs on chunk done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + kNBuf);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kNBuf; i++) {
            mbar_init(&lbar[i], 1);
            mbar_init(&mbar[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = umma_idesc(128, kN);

    // Pipeline state, kept identically by every lane of warp 0 (lane 0 issues
    // the copies, MMAs and commits): chunk loads issued (global chunk index),
    // loads waited, and the last chunk whose MMAs were committed.
    long long n_issued = 0, n_waited = 0, last_commit = -1;
    const uint64_t adesc0 = umma_desc(smem_u32(As), 128, Sh::kASBO);
    const uint64_t bdesc0 = umma_desc(smem_u32(Bs), 128, Sh::kBSBO);
    bool failed = false;

    // Stage the metadata of tile t into meta[mb] and gather its B digits.
    auto stage = [&](int t, int mb) {
        const SplitTile tl = gm.tiles[t];
        ColMeta *M = meta + mb * kN;
        if (tid < tl.cnt) {
            const SplitCol c = gm.cols[tl.p0 + tid];
            ColMeta m;
            m.out = c.out;
            m.exp = gm.dexp[c.vec] + (c.ctl >> 1) - 48;
            m.flag = c.ctl & 1;
            m.vec = c.vec;
            m.pad = 0;
            M[tid] = m;
        }
        __syncthreads();
        constexpr int kItems = kS * (KD / 8);   // 16-byte pieces per column
        for (int item = tid; item < tl.cnt * kItems; item += blockDim.x) {
            const int c = item / kItems, r = item % kItems, b = r / (KD / 8), kg = r % (KD / 8);
            const uint16_t *src = gm.dig + (size_t(M[c].vec) * kS + b) * KD + kg * 8;
            cp_async16(Bs + b * Sh::kBSlice + ((c >> 3) * (KD / 8) + kg) * 128 + (c & 7) * 16, src);
        }
        cp_async_commit();
    };
    // Chunk g of tile tl: digit a, row half h, K chunk kc.
    auto issue_load = [&](const SplitTile &tl, int g) {
        const int mh = tl.rows > 128 ? 2 : 1;
        const int a = g / (mh * Sh::NKC), h = (g / Sh::NKC) % mh, kc = g % Sh::NKC;
        const int rows_h = min(128, tl.rows - 128 * h);
        const uint32_t bytes = uint32_t((rows_h + 7) / 8) * 8 * Sh::KC * 2;
        const uint8_t *src = gm.ops + tl.a_off + size_t((a * mh + h) * Sh::NKC + kc) * Sh::kChunk;
        const int buf = int(n_issued % kNBuf);
        if (!withhold) {
            if (lane == 0) {
                mbar_expect_tx(&lbar[buf], bytes);
                uint8_t *dst = As + buf * Sh::kChunk;
                for (uint32_t q = 0; q < bytes; q += 16384)
                    bulk_g2s(dst + q, src + q, min(16384u, bytes - q), &lbar[buf]);
            }
            n_issued++;
        }
    };

    int tile = blockIdx.x;
    if (tile < gm.ntiles) {
        stage(tile, 0);
        if (warp == 0) {
            const SplitTile tl = gm.tiles[tile];
            const int n = kS * (tl.rows > 128 ? 2 : 1) * Sh::NKC;
            for (int g = 0; g < 2 && g < n; g++) issue_load(tl, g);
        }
    }
    long long gbase = 0;   // global index of the current tile's first chunk
    for (int it = 0; tile < gm.ntiles; it++) {
        const SplitTile tl = gm.tiles[tile];
        const int mh = tl.rows > 128 ? 2 : 1;
        const int n = kS * mh * Sh::NKC;
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (warp == 0) {
            for (int g = 0; g < n; g++) {
                const long long G = gbase + g;
                const int buf = int(G % kNBuf);
                if (G >= n_issued || !mbar_wait_warp(&lbar[buf], uint32_t((G / kNBuf) & 1), wait_limit)) {
                    failed = true;
                    break;
                }
                n_waited = G + 1;
                tc_fence_after();
                const int a = g / (mh * Sh::NKC) + 1, h = (g / Sh::NKC) % mh, kc = g % Sh::NKC;
                // descriptors advance by 16 (= 256 bytes >> 4) per K step of 16
                const uint64_t ad = adesc0 + uint64_t(buf) * (Sh::kChunk >> 4);
                const uint32_t first = (a == 1 && kc == 0) ? 0u : 1u;
                for (int b = 1; b + a <= kS + 1; b++) {
                    const uint32_t dcol = tmem + uint32_t(((a + b - 2) * 2 + h) * kN);
                    const uint64_t bd =
                        bdesc0 + uint64_t(b - 1) * (Sh::kBSlice >> 4) + uint64_t(kc) * ((Sh::KC / 8) * 128 >> 4);
#pragma unroll
                    for (int j = 0; j < Sh::KC / 16; j++)
                        umma_bf16_warp(dcol, ad + 16 * j, bd + 16 * j, idesc, j == 0 ? first : 1u);
                }
                umma_commit_warp(&mbar[buf]);
                last_commit = G;
                if (g + 2 < n) {
                    // the buffer of chunk G + 2 was last read by the MMAs of chunk G + 2 - kNBuf
                    const long long P = G + 2 - kNBuf;
                    if (P >= 0 && !mbar_wait_warp(&mbar[int(P % kNBuf)], uint32_t((P / kNBuf) & 1), wait_limit)) {
                        failed = true;
                        break;
                    }
                    issue_load(tl, g + 2);
                }
            }
            if (!failed &&
                !mbar_wait_warp(&mbar[int(last_commit % kNBuf)], uint32_t((last_commit / kNBuf) & 1), wait_limit))
                failed = true;
            if (!failed) last_commit = -1;   // every committed MMA has completed
        }
        gbase += n;
        failed = __syncthreads_or(failed);
        if (failed) break;
        tc_fence_after();
        // next tile: metadata, B gather and first operator chunks, overlapping this epilogue
        const int next = tile + gridDim.x;
        if (next < gm.ntiles) {
            stage(next, (it + 1) & 1);
            if (warp == 0) {
                const SplitTile tn = gm.tiles[next];
                const int nn = kS * (tn.rows > 128 ? 2 : 1) * Sh::NKC;
                for (int g = 0; g < 2 && g < nn; g++) issue_load(tn, g);
            }
        }
        // epilogue: warp w owns TMEM lanes 32(w%4)..32(w%4)+31 (rows 32(w%4)+lane
        // of each half); the two warp groups take alternate (half, 16-column)
        // items
        const ColMeta *M = meta + (it & 1) * kN;
        const int wq = warp & 3, wg = warp >> 2;
        const int ncc = (tl.cnt + 15) / 16;
        for (int item = wg; item < mh * ncc; item += 2) {   // uniform over the warp
            const int h = item / ncc, cc = item % ncc;
            const int row = h * 128 + wq * 32 + lane;
            const bool live = row < tl.rows;
            const int ea = live ? gm.op_exp[tl.exp_off + row] : 0;
            {
                uint32_t d[kS][16];
#pragma unroll
                for (int g = 0; g < kS; g++)
                    tmem_ld16(tmem + (uint32_t(wq * 32) << 16) + uint32_t((g * 2 + h) * kN + cc * 16), d[g]);
                tmem_ld_wait();
                if (!live) continue;
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int c = cc * 16 + q;
                    if (c >= tl.cnt) continue;
                    long long S = 0;
#pragma unroll
                    for (int g = 0; g < kS; g++)
                        S += (long long)__float2int_rn(__uint_as_float(d[g][q])) << (8 * (kS - 1 - g));
                    double val = i64_scaled(S, ea + M[c].exp);
                    if (M[c].flag) val *= inv_alpha0;
                    M[c].out[row] = val;
                }
            }
        }
        tc_fence_before();
        tile = next;
    }
    if (failed && warp == 0) {
        if (lane == 0) atomicExch(err, 1);
        // wait (bounded) for the copies and MMAs still in flight before the
        // shared memory and TMEM are released
        for (long long G = n_waited; G < n_issued; G++)
            mbar_wait_warp(&lbar[int(G % kNBuf)], uint32_t((G / kNBuf) & 1), wait_limit);
        if (last_commit >= 0)
            mbar_wait_warp(&mbar[int(last_commit % kNBuf)], uint32_t((last_commit / kNBuf) & 1), wait_limit);
    }
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

int g_sms = 0;

}  // namespace

size_t split_smem_bytes(int kd) { return kd == 256 ? GemmShape<256>::kSmem : GemmShape<64>::kSmem; }

cudaError_t split_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_split_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(GemmShape<256>::kSmem));
    // The K = 64 kernel asks for more shared memory than it uses so that no
    // two CTAs of the tensor-core kernels share an SM (each holds all 512 TMEM
    // columns while it runs).
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_split_gemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 * 1024);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    return e;
}

cudaError_t launch_split_digits_vec(int64_t nleaf, const double *v, double scale, uint16_t *dig, int32_t *dexp,
                                    cudaStream_t st)
{
    if (nleaf <= 0) return cudaSuccess;
    k_split_vec<<<int(std::min<int64_t>(nleaf, 152 * 16)), 256, 0, st>>>(nleaf, v, scale, dig, dexp);
    return cudaGetLastError();
}

cudaError_t launch_split_digits_exp(int64_t nbox, const double2 *ea, const double2 *eb, int P1, double scale,
                                    const double *escale, uint16_t *dig, int32_t *dexp, cudaStream_t st)
{
    if (nbox <= 0) return cudaSuccess;
    const int grid = int(std::min<int64_t>((2 * nbox + 7) / 8, 152 * 16));
    k_split_exp<<<grid, 256, 0, st>>>(nbox, reinterpret_cast<const double *>(ea), reinterpret_cast<const double *>(eb),
                                      2 * P1, scale, escale, dig, dexp);
    return cudaGetLastError();
}

cudaError_t launch_split_gemm(const SplitGemm &g, int kd, double inv_alpha0, int32_t *err, long long wait_limit,
                              int withhold, cudaStream_t st)
{
    if (g.ntiles <= 0) return cudaSuccess;
    const int grid = std::min(g.ntiles, g_sms > 0 ? g_sms : 152);
    if (kd == 256)
        k_split_gemm<256><<<grid, kGemmThreads, GemmShape<256>::kSmem, st>>>(g, inv_alpha0, err, wait_limit, withhold);
    else
        k_split_gemm<64><<<grid, kGemmThreads, 120 * 1024, st>>>(g, inv_alpha0, err, wait_limit, withhold);
    return cudaGetLastError();
}

}  // namespace bc
