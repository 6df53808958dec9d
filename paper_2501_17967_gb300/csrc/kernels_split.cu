// Split-precision operator products on the 5th-generation tensor cores
// (tcgen05), p = 16.
//
// The fixed-operator products of a split-precision apply -- the near-field
// tables, P2M, L2P, the W list (M2P) and the X list (P2L), their adjoints,
// and in BC_SPLIT_BF16_ALL also the multipole-to-local translations -- are
// dense real matrices (the operators) times many vectors (leaf values or
// expansion coefficients).  Each product is evaluated exactly in integer
// arithmetic on BF16 tensor cores:
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
//   * the five levels are combined in int64 and converted to FP64 once (a
//     hardware conversion; the power-of-two scale is then added to the
//     exponent field of the bit pattern).
//
// Work decomposition: a tile is one operator times up to 48 columns, done as
// one job per 128-row half of the operator.
//   B operand: the columns' digits, gathered into shared memory slice by slice
//              with 16-byte asynchronous copies (cp.async), resident for the
//              tile; the next tile's slices are gathered as the current tile's
//              last job stops reading them;
//   A operand: the operator's digits, 128 rows x 128 columns per chunk (32 KB),
//              brought in by bulk asynchronous copies through three buffers
//              (two in the K = 256 launches beside the FP64 M2L);
//              a tile's first row-half job takes the operator digits in the
//              order 0, 4, 1, 3, 2 (long and short chunks alternate, so copies
//              keep up), its last job in the order 0..4 (B slices are freed
//              earliest);
//   D:         5 levels x 48 columns of FP32 per job, two TMEM buffers, so one
//              job's epilogue overlaps the next job's MMAs.
// One tcgen05.mma of 128 x 48 x 16 takes about as long as one of 128 x 16 x 16
// (a fixed cost per instruction), which the MMA warp now reaches.  All waits
// are bounded: a wait that runs out sets the error flag, every role stops at
// its next wait, copies and MMAs in flight are waited for (bounded), TMEM is
// freed and the kernel returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "bc_internal.h"
#include "pdl.h"

namespace bc {

namespace {

constexpr int kS = kSplitSlices;   // 5 digits
constexpr int kN = kSplitTileN;    // 48 columns per tile
constexpr int kNBuf = 3;           // operator chunk buffers (32 KB each)

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
// waits until at most n (0..4) of this thread's cp.async groups are pending
__device__ __forceinline__ void cp_async_wait_pending(int n)
{
    switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    }
}

// NK MMAs along K (16 columns each) issued from one elected lane of a
// converged warp: the descriptors advance by 16 (256 bytes) per step; the
// first MMA takes `first` as its accumulate flag, the others accumulate.
template <int NK>
__device__ __forceinline__ void umma_kchain_warp(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                 uint32_t first);
template <>
__device__ __forceinline__ void umma_kchain_warp<8>(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                    uint32_t first)
{
    asm volatile(
        "{\n\t.reg .pred p, q, e;\n\t.reg .b64 a, b;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "setp.eq.u32 q, 0, 0;\n\t"
        "mov.b64 a, %1;\n\t"
        "mov.b64 b, %2;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, p;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(first)
        : "memory");
}
template <>
__device__ __forceinline__ void umma_kchain_warp<4>(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                    uint32_t first)
{
    asm volatile(
        "{\n\t.reg .pred p, q, e;\n\t.reg .b64 a, b;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "setp.eq.u32 q, 0, 0;\n\t"
        "mov.b64 a, %1;\n\t"
        "mov.b64 b, %2;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, p;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n\t"
        "add.s64 a, a, 16;\n\t"
        "add.s64 b, b, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(first)
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait on an mbarrier phase by a whole warp that also gives up as soon
// as another role of the CTA has failed (*fail != 0); on running out it sets
// *fail.  The result is uniform over the warp.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, long long limit, volatile int *fail)
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
        if ((it & 31) == 31 && __any_sync(0xffffffffu, *fail != 0)) return false;
    }
    *fail = 1;
    return false;
}

// Named barrier over the gather warps (id 1); the _or form returns whether any
// of them passed a true predicate.
__device__ __forceinline__ void gather_sync(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
__device__ __forceinline__ bool gather_sync_or(int nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(uint32_t(pred)), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// S * 2^ex as an FP64 value: the conversion rounds S to nearest even and the
// scaling adds ex to the exponent field (exact; results below the normal
// range, negligible here, become zero).  |S| < 2^62.
__device__ __forceinline__ double i64_scaled(long long S, int ex)
{
    const long long b = __double_as_longlong(__ll2double_rn(S));
    const int e = int((b >> 52) & 0x7FF) + ex;
    return (S == 0 || e <= 0) ? 0.0 : __longlong_as_double(b + ((long long)ex << 52));
}

// The same value with integer operations only (bit for bit: S rounded to 53
// bits, nearest with ties to even).  The tensor launches that run beside the
// FP64 kernels use it, since the hardware conversion occupies the FP64 pipe,
// a small fraction of the FP32 rate on this GPU.  The magnitude is
// normalised so that its leading one is bit 63; its top 53 bits, rounded by
// the 11 below them, are the significand, whose leading one (and a carry from
// rounding up to 2^53) adds into the exponent field.
__device__ __forceinline__ double i64_scaled_int(long long S, int ex)
{
    if (S == 0) return 0.0;
    const unsigned long long sgn = static_cast<unsigned long long>(S) & 0x8000000000000000ull;
    unsigned long long m = S < 0 ? 0ull - static_cast<unsigned long long>(S) : static_cast<unsigned long long>(S);
    const int lz = __clzll(static_cast<long long>(m));
    m <<= lz;
    const unsigned long long rem = m & 0x7FFull, mant = m >> 11;
    const unsigned long long up = (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
    const int e = 63 - lz + ex + 1023;   // biased exponent of the leading one
    if (e <= 0) return 0.0;
    return __longlong_as_double(
        static_cast<long long>((sgn | (static_cast<unsigned long long>(e - 1) << 52)) + mant + up));
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
// max |scale v| < 2^(E-1).  One block of kv threads (kv = 64 or 256) per
// leaf; the np <= kv nodes of a leaf, then zero digits up to kv.
__global__ void __launch_bounds__(256) k_split_vec(int64_t nleaf, const double *__restrict__ v, double scale,
                                                   uint16_t *__restrict__ dig, int32_t *__restrict__ dexp,
                                                   const uint8_t *__restrict__ active, int np)
{
    griddep_wait();
    griddep_launch_dependents();
    __shared__ int wmax[8];
    const int k = threadIdx.x, kv = blockDim.x;
    for (int64_t leaf = blockIdx.x; leaf < nleaf; leaf += gridDim.x) {
        // a discarded leaf of a truncated tree is no source: zero digits
        const double x = (k >= np || (active && !active[leaf])) ? 0.0 : v[leaf * np + k];
        const long long bits = __double_as_longlong(scale * x);
        int m = int((bits >> 52) & 0x7FF);
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((k & 31) == 0) wmax[k >> 5] = m;
        __syncthreads();
        int emax = wmax[0];
        for (int w = 1; w < (kv >> 5); w++) emax = max(emax, wmax[w]);
        __syncthreads();
        const int E = emax ? emax - 1023 + 2 : 0;
        digits_of(emax ? bits : 0ll, E, dig + leaf * (kS * kv) + k, kv);
        if (k == 0) dexp[leaf] = E;
    }
}

// Digits of scale * s_k * (expansion coefficient k) for the vectors i in
// [i0, i1): vector i < nbox is ea[i] with column scales escale[0..63], else
// eb[i - nbox] with escale[64..127]; its 2*P1 reals (re, im interleaved)
// padded with zeros to 64.  One warp per vector: dig[i][a][64], dexp[i].
__global__ void __launch_bounds__(256) k_split_exp(int64_t i0, int64_t i1, int64_t nbox,
                                                   const double *__restrict__ ea, const double *__restrict__ eb,
                                                   int nreal, double scale, const double *__restrict__ escale,
                                                   uint16_t *__restrict__ dig, int32_t *__restrict__ dexp)
{
    griddep_wait();
    griddep_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = i0 + ((blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5); i < i1; i += nw) {
        const int64_t box = i < nbox ? i : i - nbox;
        const double *src = (i < nbox ? ea : eb) + box * nreal;
        const double *sc = escale + (i < nbox ? 0 : kSplitKE);
        const double v0 = lane < nreal ? src[lane] : 0.0, v1 = lane + 32 < nreal ? src[lane + 32] : 0.0;
        const long long b0 = __double_as_longlong(scale * sc[lane] * v0);
        const long long b1 = __double_as_longlong(scale * sc[lane + 32] * v1);
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

// Operator digit of the p-th chunk group of a job: the order 0, 4, 1, 3, 2
// alternates long and short MMA runs (a tile's first row-half job); 0..4 frees
// the B slices earliest (a tile's last job).
__device__ __forceinline__ int chunk_digit(int p, bool interleave)
{
    return interleave ? ((0x23140 >> (4 * p)) & 0xF) : p;
}

template <int KD, int NB = kNBuf>
struct GemmShape {
    static constexpr int KC = KD < kSplitKC ? KD : kSplitKC;   // K columns per operator chunk
    static constexpr int NKC = KD / KC;
    static constexpr int kChunksPerJob = kS * NKC;     // digit x K chunk
    static constexpr int kBSlice = kN * KD * 2;        // bytes of one B digit slice
    static constexpr int kChunk = 128 * KC * 2;        // bytes of one operator chunk
    static constexpr int kBSBO = (KD / 8) * 128;       // B: bytes between 8-row groups
    static constexpr int kASBO = (KC / 8) * 128;       // A: bytes between 8-row groups
    // B buffers: two for K = 64 (the next tile is gathered while this one's
    // MMAs run), one for K = 256 (120 KB)
    static constexpr int kBBuf = KD <= 64 ? 2 : 1;
    static constexpr int kBTile = kS * kBSlice;         // bytes of one tile's B
    static constexpr size_t kSmem = size_t(kBBuf) * kBTile + size_t(NB) * kChunk + 2 * kN * sizeof(ColMeta) +
                                    64 * sizeof(uint64_t);
};

// Roles (16 warps): warp 0 issues the MMAs; warp 1 copies the operator chunks;
// warps 2-7 stage each tile's column metadata and gather its B digits, slice by
// slice; warps 8-15 run the epilogues (two warps per TMEM lane quarter, 24
// columns each).
constexpr int kGemmThreads = 512;
constexpr int kGatherWarp0 = 2;
constexpr int kGatherThreads = 192;
constexpr int kEpiWarp0 = 8;
constexpr int kEpiWarps = 8;
constexpr int kTmemBuf = 256;        // TMEM columns per job buffer (5 levels x 48 used)
constexpr int kNoExp = 0x7FFFFFFF;   // 1/alpha0 is not a power of two

// Barriers (mbarriers in shared memory); counts in brackets:
//   lbar[b] (1)        operator chunk in buffer b has landed (bulk-copy bytes)
//   mbar[b] (1)        the MMAs reading buffer b have completed (commit)
//   job_full[r] (1)    the MMAs of the job in TMEM buffer r have completed (commit)
//   job_empty[r] (8)   the epilogue warps have read TMEM buffer r
//   b_full[t][s] (1)   B digit slice s (and the metadata) of tile parity t is ready
//   b_empty[u][s] (1)  no MMA of the tile last held in B buffer u reads slice s any more (commit)
//   meta_empty[t] (8)  the epilogue warps are done with metadata buffer t
// Digit slice s (0-based) of B is read by the chunks of operator digit a <= 4 - s,
// so in a tile's last job it is free after those chunks; the next tile's B is
// gathered slice by slice from s = 4 down to 0 and its first chunk issues its
// MMAs from slice 4 down, so with one B buffer only slice 0 is waited for at
// the tile change.  Tile k uses B buffer k % kBBuf.
struct GemmBars {
    uint64_t lbar[kNBuf], mbar[kNBuf], job_full[2], job_empty[2], b_full[2][kS], b_empty[2][kS], meta_empty[2];
    uint32_t tslot;
    int fail;
};

// The second launch bound caps the registers at 64 per thread: 16 warps x 64
// leave room, in each SM sub-partition's register file, for the FP64 M2L
// blocks that run beside a near-field CTA.  Two CTAs never share an SM (shared
// memory allows one).
template <int KD, bool ICVT>
__global__ void __launch_bounds__(kGemmThreads, 2)
k_split_gemm(SplitGemm gm, double inv_alpha0, int inv_alpha_exp, int32_t *__restrict__ err, long long wait_limit,
             int withhold)
{
    // the K = 256 launches beside the FP64 M2L (ICVT) keep two operator
    // buffers: 32 KB less shared memory makes room for a fourth M2L block
    constexpr int NB = (KD == 256 && ICVT) ? 2 : kNBuf;
    using Sh = GemmShape<KD, NB>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *Bs = smem;                                                      // kBBuf x kS x kBSlice
    uint8_t *As = smem + Sh::kBBuf * Sh::kBTile;                             // NB x kChunk
    ColMeta *meta = reinterpret_cast<ColMeta *>(As + NB * Sh::kChunk);       // [2][kN]
    GemmBars *bars = reinterpret_cast<GemmBars *>(meta + 2 * kN);
    volatile int *fail = &bars->fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < NB; i++) {
            mbar_init(&bars->lbar[i], 1);
            mbar_init(&bars->mbar[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&bars->job_full[i], 1);
            mbar_init(&bars->job_empty[i], kEpiWarps);
            mbar_init(&bars->meta_empty[i], kEpiWarps);
            for (int sl = 0; sl < kS; sl++) mbar_init(&bars->b_full[i][sl], 1);
        }
        for (int u = 0; u < 2; u++)
            for (int sl = 0; sl < kS; sl++) mbar_init(&bars->b_empty[u][sl], 1);
        bars->fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tslot;
    // tensor memory and barriers are set up: now wait for the inputs
    griddep_wait();
    griddep_launch_dependents();

    if (warp == 0) {
        // ---------------- MMAs ----------------
        const uint64_t adesc0 = umma_desc(smem_u32(As), 128, Sh::kASBO);
        const uint64_t bdesc0 = umma_desc(smem_u32(Bs), 128, Sh::kBSBO);
        long long G = 0, last_commit = -1;   // chunks consumed
        int job = 0, k = 0;
        bool failed = false;
        for (int tile = blockIdx.x; tile < gm.ntiles && !failed; tile += gridDim.x, k++) {
            const SplitTile tl = gm.tiles[tile];
            const int mh = tl.rows > 128 ? 2 : 1;
            uint32_t ready = 0;   // B slices of this tile known to be gathered
            for (int h = 0; h < mh && !failed; h++, job++) {
                const int r = job & 1;
                const bool last_job = h == mh - 1;
                if (job >= 2 && !wait_bar(&bars->job_empty[r], uint32_t(((job - 2) >> 1) & 1), wait_limit, fail)) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                for (int g = 0; g < Sh::kChunksPerJob; g++, G++) {
                    const int buf = int(G % NB);
                    if (!wait_bar(&bars->lbar[buf], uint32_t((G / NB) & 1), wait_limit, fail)) {
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    const int a = chunk_digit(g / Sh::NKC, !last_job), kc = g % Sh::NKC;   // 0-based digit of A
                    const uint64_t ad = adesc0 + uint64_t(buf) * (Sh::kChunk >> 4);
                    const uint32_t first = (a == 0 && kc == 0) ? 0u : 1u;
                    for (int b = kS - 1 - a; b >= 0; b--) {   // B digit slices 0 .. kS-1-a present
                        if (!(ready >> b & 1u)) {
                            if (!wait_bar(&bars->b_full[k & 1][b], uint32_t((k >> 1) & 1), wait_limit, fail)) {
                                failed = true;
                                break;
                            }
                            tc_fence_after();
                            ready |= 1u << b;
                        }
                    }
                    if (failed) break;
                    // slices 0 .. kS-1-a lie one after another (a (kS-a) kN-row B
                    // operand) and feed levels a .. kS-1, adjacent TMEM column
                    // blocks: one MMA chain of N = (kS - a) kN per chunk
                    const uint32_t dcol = tmem + uint32_t(r * kTmemBuf + a * kN);
                    const uint64_t bd = bdesc0 + uint64_t(k % Sh::kBBuf) * (Sh::kBTile >> 4) +
                                        uint64_t(kc) * ((Sh::KC / 8) * 128 >> 4);
                    umma_kchain_warp<Sh::KC / 16>(dcol, ad, bd, umma_idesc(128, (kS - a) * kN), first);
                    umma_commit_warp(&bars->mbar[buf]);
                    last_commit = G;
                    // in the tile's last job, slice kS-1-a is read by no later chunk
                    if (last_job && kc == Sh::NKC - 1) umma_commit_warp(&bars->b_empty[k % Sh::kBBuf][kS - 1 - a]);
                }
                if (failed) break;
                umma_commit_warp(&bars->job_full[r]);
            }
        }
        if (failed) {
            *fail = 1;
            int dummy = 0;   // bounded wait, without the failure shortcut
            if (last_commit >= 0)
                wait_bar(&bars->mbar[int(last_commit % NB)], uint32_t((last_commit / NB) & 1), wait_limit,
                         &dummy);
        }
    } else if (warp == 1) {
        // ---------------- operator chunk copies ----------------
        long long n = 0;   // chunks issued
        bool failed = false;
        for (int tile = blockIdx.x; tile < gm.ntiles && !failed; tile += gridDim.x) {
            const SplitTile tl = gm.tiles[tile];
            const int mh = tl.rows > 128 ? 2 : 1;
            for (int h = 0; h < mh && !failed; h++)
                for (int g = 0; g < Sh::kChunksPerJob; g++, n++) {
                    const int buf = int(n % NB);
                    // buffer free once the MMAs of chunk n - NB have completed
                    if (n >= NB &&
                        !wait_bar(&bars->mbar[buf], uint32_t(((n - NB) / NB) & 1), wait_limit, fail)) {
                        failed = true;
                        break;
                    }
                    if (withhold) continue;   // diagnostics: the MMA warp's first wait runs out
                    const int a = chunk_digit(g / Sh::NKC, h < mh - 1), kc = g % Sh::NKC;
                    const int rows_h = min(128, tl.rows - 128 * h);
                    const uint32_t bytes = uint32_t((rows_h + 7) / 8) * 8 * Sh::KC * 2;
                    const uint8_t *src = gm.ops + tl.a_off + size_t((a * mh + h) * Sh::NKC + kc) * Sh::kChunk;
                    // an operator of at most 64 rows is copied twice, to rows 0-63
                    // and 64-127, so that every TMEM lane quarter holds a result
                    const int copies = tl.rows <= 64 ? 2 : 1;
                    if (lane == 0) {
                        mbar_expect_tx(&bars->lbar[buf], bytes * copies);
                        for (int cp = 0; cp < copies; cp++) {
                            uint8_t *dst = As + buf * Sh::kChunk + cp * (Sh::kChunk / 2);
                            for (uint32_t q = 0; q < bytes; q += 16384)
                                bulk_g2s(dst + q, src + q, min(16384u, bytes - q), &bars->lbar[buf]);
                        }
                    }
                    __syncwarp();
                }
        }
        if (failed && !withhold) {
            // copies still in flight: at most the last NB issued
            int dummy = 0;
            for (long long q = n > NB ? n - NB : 0; q < n; q++)
                wait_bar(&bars->lbar[int(q % NB)], uint32_t((q / NB) & 1), wait_limit, &dummy);
        }
    } else if (warp < kEpiWarp0) {
        // ---------------- column metadata and B gather ----------------
        const int gt = tid - 32 * kGatherWarp0;
        constexpr int kPieces = KD / 8;   // 16-byte pieces per column and slice
        // two B buffers: the next tile's record, this thread's column of it and
        // the column's digit exponent are fetched while the current tile's
        // slices are in flight
        SplitTile ntl{};
        SplitCol ncol{};
        int nexp = 0;
        bool have = false;
        int k = 0;
        bool stop = false;
        for (int tile = blockIdx.x; tile < gm.ntiles && !stop; tile += gridDim.x, k++) {
            bool ok = true;
            // the epilogues of tile k - 2 no longer read this metadata buffer
            if (k >= 2) ok = wait_bar(&bars->meta_empty[k & 1], uint32_t(((k - 2) >> 1) & 1), wait_limit, fail);
            if (gather_sync_or(kGatherThreads, !ok)) break;   // uniform over the gather warps
            const SplitTile tl = have ? ntl : gm.tiles[tile];
            ColMeta *M = meta + (k & 1) * kN;
            if (gt < tl.cnt) {
                const SplitCol c = have ? ncol : gm.cols[tl.p0 + gt];
                ColMeta m;
                m.out = c.out;
                m.exp = (have ? nexp : gm.dexp[c.vec]) + (c.ctl >> 1) - 48;
                m.flag = c.ctl & 1;
                if (m.flag && inv_alpha_exp != kNoExp) {   // 1/alpha0 a power of two: an exponent shift
                    m.exp += inv_alpha_exp;
                    m.flag = 0;
                }
                m.vec = c.vec;
                m.pad = 0;
                M[gt] = m;
            }
            have = false;
            gather_sync(kGatherThreads);
            uint8_t *Bt = Bs + (k % Sh::kBBuf) * Sh::kBTile;
            if constexpr (Sh::kBBuf == 2) {
                // every slice at once: tile k - 2, the last one in this buffer,
                // has released all of them
                bool ok2 = true;
                if (k >= 2)
                    for (int sl = 0; sl < kS && ok2; sl++)
                        ok2 = wait_bar(&bars->b_empty[k & 1][sl], uint32_t(((k - 2) >> 1) & 1), wait_limit, fail);
                if (gather_sync_or(kGatherThreads, !ok2)) break;
                for (int sl = kS - 1; sl >= 0; sl--) {
                    for (int item = gt; item < tl.cnt * kPieces; item += kGatherThreads) {
                        const int c = item / kPieces, kg = item % kPieces;
                        const uint16_t *src = gm.dig + (size_t(M[c].vec) * kS + sl) * KD + kg * 8;
                        cp_async16(Bt + sl * Sh::kBSlice + ((c >> 3) * kPieces + kg) * 128 + (c & 7) * 16, src);
                    }
                    cp_async_commit();
                }
                const int nt = tile + gridDim.x;
#pragma unroll
                for (int j = 0; j < kS; j++) {
                    cp_async_wait_pending(kS - 1 - j);   // slices kS-1 .. kS-1-j have landed
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    gather_sync(kGatherThreads);
                    if (gt == 0) mbar_arrive(&bars->b_full[k & 1][kS - 1 - j]);
                    // one step of the next tile's metadata chain per slice
                    if (nt < gm.ntiles) {
                        if (j == 0) {
                            ntl = gm.tiles[nt];
                        } else if (j == 1) {
                            if (gt < ntl.cnt) ncol = gm.cols[ntl.p0 + gt];
                        } else if (j == 2) {
                            if (gt < ntl.cnt) nexp = gm.dexp[ncol.vec];
                            have = true;
                        }
                    }
                }
            } else {
                // one B buffer: two slices in flight, each issued once the
                // previous tile's MMAs have released it; complete slice sl + 1
                for (int sl = kS - 1; sl >= -1; sl--) {
                    if (sl >= 0) {
                        bool ok2 = true;
                        if (k >= 1) ok2 = wait_bar(&bars->b_empty[0][sl], uint32_t((k - 1) & 1), wait_limit, fail);
                        if (gather_sync_or(kGatherThreads, !ok2)) {
                            stop = true;
                            break;
                        }
                        for (int item = gt; item < tl.cnt * kPieces; item += kGatherThreads) {
                            const int c = item / kPieces, kg = item % kPieces;
                            const uint16_t *src = gm.dig + (size_t(M[c].vec) * kS + sl) * KD + kg * 8;
                            cp_async16(Bt + sl * Sh::kBSlice + ((c >> 3) * kPieces + kg) * 128 + (c & 7) * 16, src);
                        }
                        cp_async_commit();
                    }
                    if (sl + 1 <= kS - 1) {
                        cp_async_wait_pending(sl >= 0 ? 1 : 0);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        gather_sync(kGatherThreads);
                        if (gt == 0) mbar_arrive(&bars->b_full[k & 1][sl + 1]);
                    }
                }
            }
        }
        cp_async_wait_all();
    } else {
        // ---------------- epilogues ----------------
        // warp w reads TMEM lanes 32(w%4)..32(w%4)+31.  Operators of more
        // than 64 rows: rows 32(w%4)+lane of the job's row half, warps 8-11
        // columns 0-23, warps 12-15 columns 24-47.  Up to 64 rows (held twice):
        // rows 32(w%2)+lane, lane quarters 0-1 columns 0-23 and 2-3 columns
        // 24-47, split 12 + 12 between the two warps of a quarter.
        const int wq = warp & 3, half = (warp - kEpiWarp0) >> 2;
        int job = 0, k = 0;
        bool failed = false;
        for (int tile = blockIdx.x; tile < gm.ntiles && !failed; tile += gridDim.x, k++) {
            // the metadata is staged before the first slice (kS - 1) is gathered
            if (!wait_bar(&bars->b_full[k & 1][kS - 1], uint32_t((k >> 1) & 1), wait_limit, fail)) break;
            const SplitTile tl = gm.tiles[tile];
            const int mh = tl.rows > 128 ? 2 : 1;
            const ColMeta *M = meta + (k & 1) * kN;
            for (int h = 0; h < mh; h++, job++) {
                const int r = job & 1;
                if (!wait_bar(&bars->job_full[r], uint32_t((job >> 1) & 1), wait_limit, fail)) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                const bool small = tl.rows <= 64;
                const int row = small ? (wq & 1) * 32 + lane : h * 128 + wq * 32 + lane;
                const bool live = row < tl.rows;
                const int ea = live ? gm.op_exp[tl.exp_off + row] : 0;
                const int cb = small ? (wq >> 1) * 24 + half * 12 : half * 24;
                const int ce = min(tl.cnt, cb + (small ? 12 : 24));
                for (int c0 = cb; c0 < ce; c0 += 8) {   // uniform over the warp
                    uint32_t d[kS][8];
#pragma unroll
                    for (int g = 0; g < kS; g++)
                        tmem_ld8(tmem + (uint32_t(wq * 32) << 16) + uint32_t(r * kTmemBuf + g * kN + c0), d[g]);
                    tmem_ld_wait();
                    if (!live) continue;
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int c = c0 + q;
                        if (c >= ce) continue;
                        long long S = 0;
#pragma unroll
                        for (int g = 0; g < kS; g++)
                            S += (long long)__float2int_rn(__uint_as_float(d[g][q])) << (8 * (kS - 1 - g));
                        double val = ICVT ? i64_scaled_int(S, ea + M[c].exp) : i64_scaled(S, ea + M[c].exp);
                        if (M[c].flag) val *= inv_alpha0;
                        M[c].out[row] = val;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars->job_empty[r]);
            }
            if (failed) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars->meta_empty[k & 1]);
        }
    }
    if (*fail && tid == 0) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

int g_sms = 0;
// The K = 64 kernel asks for more shared memory than it uses so that no two
// CTAs of the tensor-core kernels share an SM (each holds all 512 TMEM columns
// while it runs): 2 x 130 KB and 130 KB + the K = 256 kernel's both exceed an SM.
constexpr int kSmem64 = 130 * 1024;
static_assert(GemmShape<64>::kSmem <= size_t(kSmem64), "K = 64 shared memory");

}  // namespace

size_t split_smem_bytes(int kd) { return kd == 256 ? GemmShape<256>::kSmem : GemmShape<64>::kSmem; }

cudaError_t split_prepare()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_split_gemm<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(GemmShape<256>::kSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_split_gemm<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(GemmShape<256, 2>::kSmem));
    for (const void *k : {(const void *)k_split_gemm<64, false>, (const void *)k_split_gemm<64, true>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem64);
    // the digit kernels run before and beside the tensor launches: the
    // largest shared-memory carveout (see fp64_prepare)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_split_vec, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_split_exp, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    return e;
}

int split_sm_count() { return g_sms > 0 ? g_sms : 152; }

cudaError_t launch_split_digits_vec(int64_t nleaf, const double *v, double scale, uint16_t *dig, int32_t *dexp,
                                    cudaStream_t st, const uint8_t *active, int np, int kv)
{
    if (nleaf <= 0) return cudaSuccess;
    if ((kv != 64 && kv != 256) || np < 1 || np > kv) return cudaErrorInvalidValue;
    return launch_pdl(k_split_vec, int(std::min<int64_t>(nleaf, 152 * 16)), kv, 0, st, nleaf, v, scale, dig, dexp,
                      active, np);
}

cudaError_t launch_split_digits_exp(int64_t i0, int64_t i1, int64_t nbox, const double2 *ea, const double2 *eb,
                                    int P1, double scale, const double *escale, uint16_t *dig, int32_t *dexp,
                                    cudaStream_t st)
{
    if (i1 <= i0) return cudaSuccess;
    const int grid = int(std::min<int64_t>((i1 - i0 + 7) / 8, 152 * 16));
    return launch_pdl(k_split_exp, grid, 256, 0, st, i0, i1, nbox, reinterpret_cast<const double *>(ea),
                      reinterpret_cast<const double *>(eb), 2 * P1, scale, escale, dig, dexp);
}

cudaError_t launch_split_gemm(const SplitGemm &g, int kd, double inv_alpha0, int32_t *err, long long wait_limit,
                              int withhold, cudaStream_t st, bool intcvt)
{
    if (g.ntiles <= 0) return cudaSuccess;
    const int sms = g_sms > 0 ? g_sms : 152;
    const int grid = std::min(g.ntiles, g.max_ctas > 0 ? std::min(g.max_ctas, sms) : sms);
    int ie = 0;
    const int inv_alpha_exp = std::frexp(inv_alpha0, &ie) == 0.5 ? ie - 1 : kNoExp;
    if (kd == 256)
        return launch_pdl(intcvt ? k_split_gemm<256, true> : k_split_gemm<256, false>, grid, kGemmThreads,
                          intcvt ? GemmShape<256, 2>::kSmem : GemmShape<256>::kSmem, st, g, inv_alpha0, inv_alpha_exp,
                          err, wait_limit, withhold);
    return launch_pdl(intcvt ? k_split_gemm<64, true> : k_split_gemm<64, false>, grid, kGemmThreads, size_t(kSmem64),
                      st, g, inv_alpha0, inv_alpha_exp, err, wait_limit, withhold);
}

}  // namespace bc
