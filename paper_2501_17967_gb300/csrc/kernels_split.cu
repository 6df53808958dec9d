// Split-precision near field on the 5th-generation tensor cores (tcgen05),
// p = 16 (256 nodes per leaf).
//
// Every near-field product u_t += alpha * T f_s (T a 256x256 FP64 table) is
// evaluated exactly in integer arithmetic on BF16 tensor cores:
//   * each FP64 operand row is scaled by a power of two 2^E so that its entries
//     lie in (-1/2, 1/2), rounded to a 40-bit fixed-point integer X and cut into
//     five balanced base-256 digits, X = sum_a theta_a 256^(5-a), |theta_a| <= 128;
//     every digit is an integer that BF16 holds exactly (Ozaki-style splitting);
//   * T f = 2^(E_T + E_f - 48) * sum_g 256^(6-g) D_g,  D_g = sum_{a+b=g} theta_a . phi_b,
//     keeping the digit pairs a + b <= 6 (15 products; what is dropped is below
//     2^-38 relative to sum_k |T_ik f_k|);
//   * each D_g (g = 2..6) accumulates in its own FP32 TMEM accumulator: every
//     product is an integer of magnitude <= 2^14 and a level sums at most
//     4 x 256 of them for g <= 5, so the accumulation is exact (< 2^24);
//   * the five levels are combined in int64 and converted to FP64 once.
// Work decomposition: near entries are grouped by table; a CTA tile holds up to
// 48 entries of one table.  B operand = the gathered density digits of the 48
// entries (resident in shared memory), A operand = the table digits, 128 rows at
// a time, copied from global memory with bulk asynchronous copies.  The result
// of each entry (256 FP64 values, alpha included) goes to a scratch row that the
// leaf-output pass adds to the far field and the log term.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bc_internal.h"

namespace bc {

namespace {

constexpr int kNP = 256;                      // p = 16
constexpr int kS = kSplitSlices;              // 5 digits
constexpr int kN = kSplitTileN;               // 48 entries per tile
constexpr int kBSlice = kN * kNP * 2;         // bytes of one B digit slice (24 KB)
constexpr int kAChunk = 128 * kNP * 2;        // bytes of one A digit slice, 128 rows (64 KB)

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

// Bounded wait on an mbarrier phase; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit)
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
        if (ok) return true;
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

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
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

// ---------------------------------------------------------------------------
// Digits of the leaf vectors times alpha0: vsl[leaf][a][k] (BF16 bits),
// vexp[leaf] = E with max |alpha0 v| < 2^(E-1).  One FP64 multiply per value;
// the rest is integer arithmetic on the FP64 bit patterns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_split_vec(int64_t nleaf, const double *__restrict__ v, double alpha0,
                                                   uint16_t *__restrict__ vsl, int32_t *__restrict__ vexp)
{
    __shared__ int wmax[8];
    const int k = threadIdx.x;
    for (int64_t leaf = blockIdx.x; leaf < nleaf; leaf += gridDim.x) {
        const long long bits = __double_as_longlong(alpha0 * v[leaf * kNP + k]);
        const int e = int((bits >> 52) & 0x7FF);
        int m = e;
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((k & 31) == 0) wmax[k >> 5] = m;
        __syncthreads();
        int emax = wmax[0];
        for (int w = 1; w < 8; w++) emax = max(emax, wmax[w]);
        __syncthreads();
        const int E = emax ? emax - 1023 + 2 : 0;
        long long X = 0;
        if (e != 0 && emax != 0) {
            const long long mant = (bits & ((1ll << 52) - 1)) | (1ll << 52);
            const int rs = -(e - 1075 + 40 - E);   // >= 14
            X = rs >= 62 ? 0 : (mant + (1ll << (rs - 1))) >> rs;
            if (bits < 0) X = -X;
        }
        uint16_t *out = vsl + leaf * (kS * kNP) + k;
#pragma unroll
        for (int a = kS; a >= 2; a--) {
            int d = int(X & 255);
            if (d >= 128) d -= 256;
            X = (X - d) >> 8;
            out[(a - 1) * kNP] = uint16_t(__float_as_uint(float(d)) >> 16);
        }
        out[0] = uint16_t(__float_as_uint(float(int(X))) >> 16);   // leading digit, |X| <= 128
        if (k == 0) vexp[leaf] = E;
    }
}

// ---------------------------------------------------------------------------
// Near-field entries of one table per tile, on tcgen05.
// ---------------------------------------------------------------------------
struct TileArgs {
    const int32_t *tile_tab, *tile_p0, *tile_cnt;
    const int32_t *pair_vec, *pair_out, *pair_lvl;
    int ntiles;
};

__global__ void __launch_bounds__(128, 1)
k_near_mma(TileArgs T, const uint8_t *__restrict__ Asl, const int32_t *__restrict__ Aexp,
           const uint16_t *__restrict__ vsl, const int32_t *__restrict__ vexp, double *__restrict__ P,
           int32_t *__restrict__ err, long long wait_limit, int withhold)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *Bs = smem;                                            // kS * kBSlice
    uint8_t *As = smem + kS * kBSlice;                             // kAChunk
    uint64_t *bars = reinterpret_cast<uint64_t *>(As + kAChunk);   // [0] A load, [1] MMA done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phA = 0, phM = 0;
    bool failed = false;
    const uint32_t idesc = umma_idesc(128, kN);

    for (int tile = blockIdx.x; tile < T.ntiles && !failed; tile += gridDim.x) {
        const int tab = T.tile_tab[tile], p0 = T.tile_p0[tile], cnt = T.tile_cnt[tile];
        // B: digits of the tile's vectors, K-major core-matrix layout
        // [slice][row group][k group][8 rows][8 elements]
        for (int item = tid; item < cnt * kS * 32; item += blockDim.x) {
            const int c = item / (kS * 32), r = item % (kS * 32), b = r / 32, kg = r % 32;
            const uint4 val =
                *reinterpret_cast<const uint4 *>(vsl + (size_t(T.pair_vec[p0 + c]) * kS + b) * kNP + kg * 8);
            *reinterpret_cast<uint4 *>(Bs + b * kBSlice + ((c >> 3) * 32 + kg) * 128 + (c & 7) * 16) = val;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        for (int a = 1; a <= kS && !failed; a++)
            for (int h = 0; h < 2 && !failed; h++) {
                if (tid == 0) {
                    const uint8_t *src = Asl + (size_t((tab * kS + (a - 1)) * 2 + h)) * kAChunk;
                    if (!withhold) {
                        mbar_expect_tx(&bars[0], kAChunk);
                        for (int q = 0; q < 4; q++)
                            bulk_g2s(As + q * (kAChunk / 4), src + q * (kAChunk / 4), kAChunk / 4, &bars[0]);
                    }
                    bool ok = mbar_wait(&bars[0], phA, wait_limit);
                    if (ok) {
                        tc_fence_after();
                        for (int b = 1; b + a <= kS + 1; b++) {
                            const int acc = a + b - 2;                        // level g - 2
                            const uint32_t dcol = tmem + uint32_t((acc * 2 + h) * kN);
                            for (int j = 0; j < kNP / 16; j++) {
                                const uint64_t ad = umma_desc(smem_u32(As) + j * 256, 128, 4096);
                                const uint64_t bd = umma_desc(smem_u32(Bs + (b - 1) * kBSlice) + j * 256, 128, 4096);
                                umma_bf16(dcol, ad, bd, idesc, (a == 1 && j == 0) ? 0u : 1u);
                            }
                        }
                        umma_commit(&bars[1]);
                        ok = mbar_wait(&bars[1], phM, wait_limit);
                    }
                    if (!ok) {
                        atomicExch(err, 1);
                        failed = true;
                    }
                    phA ^= 1u;
                    phM ^= 1u;
                }
                __syncthreads();
                failed = __syncthreads_or(failed);
            }
        if (failed) break;
        tc_fence_after();
        // epilogue: warp w owns TMEM lanes 32w..32w+31 = rows 32w+lane of each half
        for (int h = 0; h < 2; h++) {
            const int row = h * 128 + warp * 32 + lane;
            const int ea = Aexp[tab * kNP + row];
            for (int cc = 0; cc < kN / 16; cc++) {
                uint32_t d[kS][16];
#pragma unroll
                for (int g = 0; g < kS; g++)
                    tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t((g * 2 + h) * kN + cc * 16), d[g]);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int c = cc * 16 + q;
                    if (c >= cnt) continue;
                    long long S = 0;
#pragma unroll
                    for (int g = 0; g < kS; g++)
                        S += (long long)__float2int_rn(__uint_as_float(d[g][q])) << (8 * (kS - 1 - g));
                    const int pv = T.pair_vec[p0 + c];
                    const int ex = ea + vexp[pv] - 48 - 2 * T.pair_lvl[p0 + c];
                    P[size_t(T.pair_out[p0 + c]) * kNP + row] = i64_scaled(S, ex);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

}  // namespace

size_t split_smem_bytes() { return size_t(kS) * kBSlice + kAChunk + 64; }

cudaError_t split_prepare()
{
    return cudaFuncSetAttribute(k_near_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, int(split_smem_bytes()));
}

cudaError_t launch_split_near(const PassArgs &a, const SplitTables &st, const SplitTree &sp, bool adj,
                              const double *vin, cudaStream_t stream)
{
    const int grid_v = int(std::min<int64_t>(a.nleaf, 152 * 16));
    k_split_vec<<<grid_v, 256, 0, stream>>>(a.nleaf, vin, a.half_L * a.half_L, sp.vsl, sp.vexp);
    if (sp.ntiles == 0) return cudaGetLastError();
    TileArgs T{sp.tile_tab, sp.tile_p0, sp.tile_cnt, sp.pair_vec, sp.pair_out, adj ? sp.pair_lvl_a : sp.pair_lvl_f,
               sp.ntiles};
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int grid = std::min(sp.ntiles, sms);
    k_near_mma<<<grid, 128, split_smem_bytes(), stream>>>(T, adj ? st.A[1] : st.A[0], adj ? st.Aexp[1] : st.Aexp[0],
                                                          sp.vsl, sp.vexp, sp.P, sp.err, st.wait_limit,
                                                          st.withhold_copy);
    return cudaGetLastError();
}

}  // namespace bc
