// Internal declarations shared by the host code (tree, tables, API) and the
// CUDA kernels of the box code.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/boxcode.h"

namespace bc {

constexpr int kMaxP = 16;
constexpr int kNumNear = 41;   // near-table slots (33 used; see near_table_geometry)
constexpr int kNumV = 49;      // V offsets on the 7x7 grid (40 used)
constexpr int kNumWX = 36;     // W/X offsets on the 6x6 half-integer grid (20 used)
constexpr int kDefaultNterms = 30;
constexpr int kLvTab = 32;     // levels in the per-level constant tables (tree levels <= 24)

void set_error(const char *fmt, ...);

// ---------------------------------------------------------------------------
// Host tree
// ---------------------------------------------------------------------------
struct HostTree {
    double x0 = 0, y0 = 0, L = 1;
    int p = 0;
    int64_t nleaf = 0;
    std::vector<int32_t> leaf_level, leaf_ix, leaf_iy;   // caller order
    // boxes sorted by (level, Morton key); children of a box are contiguous
    // and ordered q = qx + 2*qy
    int nlevels = 0;                                      // max level + 1
    std::vector<int32_t> box_level, box_ix, box_iy, box_parent, box_child0, box_leaf;
    std::vector<int64_t> level_start;                     // [nlevels + 1]
    std::vector<int32_t> leaf_box;                        // caller leaf -> box
    std::vector<int32_t> leaf_order;                      // leaves in Morton order of their boxes
    // CSR lists (ptr has one extra entry)
    std::vector<int32_t> near_ptr, near_src, near_tab;    // per leaf: source leaf, table id
    std::vector<int32_t> v_ptr, v_src, v_code;            // per box: source box, V code
    std::vector<int32_t> w_ptr, w_src, w_code;            // per leaf: source box, W code
    std::vector<int32_t> x_ptr, x_src, x_code;            // per box: source leaf, X code
    int64_t n_nonleaf = 0, n_down = 0;
    // truncated trees (Alg. 2 with a domain): the domain's boundary polygon
    // and each leaf's class, 0 outside the domain (discarded: no source, zero
    // output), 1 cut by its boundary, 2 inside (empty: no truncation)
    std::vector<double> gamma;
    std::vector<int8_t> leaf_class;
};
void drop_inactive(HostTree &t, const std::vector<uint8_t> &active);

// Builds boxes and lists from explicit leaves; returns BC_OK or BC_ERR_TREE /
// BC_ERR_ARG with the message set.
bc_status build_host_tree(HostTree &t, double x0, double y0, double L, int p, int64_t nleaf,
                          const int32_t *level, const int32_t *ix, const int32_t *iy);
// A closed polygon (vertices xy[2n], the last joined to the first).
struct Polygon {
    const double *xy = nullptr;
    int64_t n = 0;
};
// The truncation of Alg. 2: the domain Omega bounded by gamma, the bulk region
// Omega_B bounded by gamma_b (inside Omega); the strip is Omega \ Omega_B.
struct Truncation {
    Polygon gamma, gamma_b;
};
enum class BoxSide { Inside, Outside, Cut };
BoxSide box_side(const Polygon &P, double x0, double x1, double y0, double y1);
bool polygon_contains(const Polygon &P, double x, double y);
bool truncation_split(const Truncation &tr, double cx, double cy, double r);
// Alg. 2 followed by 2:1 balancing; fills the leaf arrays (level/ix/iy)
// only.  Without a truncation only the function-resolution criterion
// applies; with one, f is extended by zero outside Omega, the resolution
// criterion applies to boxes inside Omega and the separation criterion to
// every box.
bc_status refine_leaves(int p, double x0, double y0, double L, bc_density_fn fn, void *user,
                        double eps, int max_level, std::vector<int32_t> &lv,
                        std::vector<int32_t> &ix, std::vector<int32_t> &iy, const Truncation *tr = nullptr);

// ---------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------
// Geometry of near table k: target nodes in the source's reference square are
// g + rho * node.  valid == false for unused slots.
struct NearGeom {
    bool valid;
    double gx, gy, rho;
    int rev;  // table of the reversed pair (target <-> source)
};
NearGeom near_table_geometry(int k);
int near_code_same(int gx2, int gy2);     // g = (c_t - c_s)/r in {-2,0,2}: pass g
int near_code_coarse(int g2x, int g2y);   // source one level coarser: pass 2g in {-3..3}
int near_code_fine(int gx, int gy);       // source one level finer: pass g in {-3..3} odd
int v_code(int dx, int dy);               // dx = ix_s - ix_t in [-3,3]
int wx_code(int d2x, int d2y);            // 2*offset in {-5,-3,-1,1,3,5}

struct HostTables {
    int p = 0, P1 = 0, NP = 0;
    std::vector<double> nodes;       // p
    std::vector<double> w;           // NP tensor quadrature weights (int of Lagrange basis)
    std::vector<double> T;           // [kNumNear][NP target][NP source] near tables (1/2pi included)
    // far field (complex as interleaved re,im)
    std::vector<double> Q;           // [P1][NP] P2M (scale r^2 at run time)
    std::vector<double> E;           // [NP][P1] L2P
    std::vector<double> M2M;         // [4][P1][P1]  A_par[l] = sum_k M2M[q][l][k] A_child[k]
    std::vector<double> L2L;         // [4][P1][P1]  B_child[m] = sum_l L2L[q][m][l] B_par[l]
    std::vector<double> M2L;         // [kNumV][P1][P1]  B[l] = sum_k M2L[c][l][k] A[k]
    std::vector<double> M2P;         // [kNumWX][NP][P1] W list
    std::vector<double> P2L;         // [kNumWX][P1][NP] X list (scale r_c^2)
};
bc_status build_tables(HostTables &ht, int p, int P1, const char *cache_dir);

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------
// One operator set drives one direction (forward or adjoint) of the apply.
// Every complex operator is stored so that the kernel computes
// out[l] = sum_k Op[k*P1 + l] * in[k]  ("element (l,k) at [k][l]").
// Term schedule of the double-float upward shift.  The nonzero terms
// (output l, input k) of the four child operators (the shift is triangular:
// k <= l) are taken output by output and cut into 32 runs of T terms, one
// run per lane, so that the lanes share the triangle evenly; each lane ends a
// partial sum where its run leaves an output, and the partial sums of an
// output (np[l] of them, consecutive lanes) are added afterwards.
struct DfSched {
    const uint32_t *code = nullptr;   // [T][32] input k (bits 0-7); (slot + 1) << 8 where a partial sum ends
    const float4 *ops = nullptr;      // [4][T][32] the operator entry of each term, per child, {Re hi, lo, Im hi, lo}
    const int32_t *np = nullptr;      // [P1] partial sums per output; output l owns slots l * maxp + [0, np[l])
    int T = 0, maxp = 0;
};

// FP64 shift in factored form (kernels compute the same operator as `up` /
// `par`): for child q,
//     out[l] = so[q][l] * sum_k B[l][k] * (si[q][k] * in[k])
// with B real and triangular (binomial coefficients, the same for the four
// children) and si, so complex diagonals (powers of the child offset delta_q
// = +-1 +- i or of delta_q / 2).  B's nonzero terms, taken output by output,
// are cut into 32 runs of T terms, one run per lane of a warp (the scheme of
// DfSched); each lane ends a partial sum where its run leaves an output.
struct ShiftFac {
    const double2 *si = nullptr, *so = nullptr;   // [4][P1]
    const uint32_t *code = nullptr;   // [T][32] input k (bits 0-7); (slot + 1) << 8 where a partial sum ends
    const double *coef = nullptr;     // [T][32] B[l][k] of each term (0 for padding)
    const int32_t *np = nullptr;      // [P1] partial sums per output; output l owns slots l * maxp + [0, np[l])
    int T = 0, maxp = 0;
};

struct OpSet {
    const double2 *leafA = nullptr;   // [NP][P1]        leaf vector -> box expansion
    const double2 *up = nullptr;      // [4][P1][P1]     child -> parent
    const double2 *par = nullptr;     // [4][P1][P1]     parent -> child
    const double2 *v = nullptr;       // [kNumV][P1][P1] V-list translation
    const double2 *x = nullptr;       // [kNumWX][NP][P1] leaf vector -> expansion (X list)
    const double2 *e = nullptr;       // [P1][NP]        expansion -> leaf nodes (real part)
    const double2 *w = nullptr;       // [kNumWX][P1][NP] expansion -> leaf nodes (W list)
    const double *t = nullptr;        // [kNumNear][NP][NP] near tables, element (j,k) at [k][j]
    // par as double-float pairs {Re hi, Re lo, Im hi, Im lo} (each entry the
    // sum of two FP32 numbers, about 48 significant bits)
    const float4 *par_df = nullptr;
    const float4 *leafA_df = nullptr;   // leafA as double-float pairs
    DfSched up_s;                       // up, scheduled for the double-float climb
    ShiftFac up_f, par_f;               // up and par in factored form (FP64 level passes)
};

struct DevTables {
    OpSet fwd, adj;
    double *wvec = nullptr;           // [NP]
    // M2L in factored form: d^-k (forward) / conj(d)^-k (adjoint) per V code,
    // the same with the sign (-1)^k, and log|d| per code (the binomial table
    // is a constant-memory table of the kernels).
    double2 *dpow_f = nullptr, *dpow_a = nullptr;   // [kNumV][P1]
    double2 *dsig_f = nullptr, *dsig_a = nullptr;   // [kNumV][P1]
    double *logd = nullptr;                          // [kNumV]
    std::vector<void *> allocs;
};

struct DevTree {
    int32_t *leaf_box = nullptr, *leaf_level = nullptr, *leaf_order = nullptr;
    int32_t *box_parent = nullptr, *box_child0 = nullptr, *box_level = nullptr, *box_ix = nullptr,
            *box_iy = nullptr, *box_leaf = nullptr;
    int32_t *near_ptr = nullptr, *near_src = nullptr, *near_tab = nullptr;
    int32_t *v_ptr = nullptr, *v_src = nullptr, *v_code = nullptr;
    int32_t *w_ptr = nullptr, *w_src = nullptr, *w_code = nullptr;
    int32_t *x_ptr = nullptr, *x_src = nullptr, *x_code = nullptr;
    int32_t *v_box = nullptr, *x_box = nullptr;       // target box of each V / X entry
    double2 *Pv = nullptr;                             // [n_v][P1] M2L of each V pair (tensor-core M2L only; split set-up)
    double2 *PX = nullptr;                             // [n_x][P1] X-list product of each entry (FP64 path)
    double2 *expA = nullptr, *expB = nullptr;  // [nbox][P1] workspaces
    int32_t *zero_ptr = nullptr;               // [nleaf+1] zeros: empty lists (diagnostic pass masks)
    double2 *leaf_logs = nullptr;              // [nleaf] the W and near lists' log-term sums of each target leaf
    double *lvtab = nullptr;                   // [2][kLvTab]: r^2 and log r per level
    int64_t *level_start = nullptr;            // [nlevels + 1] first box of each level
    int32_t *flag = nullptr;                   // [nbox] completion flags of the persistent level passes
    float4 *exdf = nullptr;                    // [nbox][P1] double-float upward expansions of the climb
    double *stage_in = nullptr, *stage_out = nullptr; // host-pointer staging [nleaf*NP]
    const uint8_t *leaf_active = nullptr;      // [nleaf] truncated trees: 0 = discarded leaf (zero output); null: all
    std::vector<void *> allocs;
};

// Split precision (p = 16 only).  The fixed-operator products of the apply
// run on the tensor cores as exact BF16 digit products (kernels_split.cu):
//   group V (K = 256, input = leaf vectors): near tables, P2M (adjoint L2P^H),
//            X list (adjoint M2P^H)
//   group E (K = 64, input = expansions, 2*P1 reals padded to 64): L2P
//            (adjoint P2M^H), W list (adjoint P2L^H)
//   group M (K = 64, BC_SPLIT_BF16_ALL only): the V-list translations, one
//            operator per offset
// An operator is a real matrix of `rows` <= 256 rows; its BF16 digits are
// stored as chunks [digit a][row half h][K chunk kc] of 128 rows x KC
// columns (KC = min(K, kSplitKC)) in the canonical K-major core-matrix layout.
constexpr int kSplitSlices = 5;
constexpr int kSplitTileN = 48;
constexpr int kSplitKE = 64;                 // K of group E (expansion reals, padded)
constexpr int kSplitKC = 128;                // K columns per operator chunk (one bulk copy)
struct SplitOp {
    int64_t a_off = 0;     // byte offset of the operator's first chunk
    int32_t rows = 0;      // valid rows
    int32_t exp_off = 0;   // index of the operator's first row exponent
};
struct SplitTables {
    // [group V, group E][forward, adjoint]
    const uint8_t *ops[2][2] = {};
    const int32_t *op_exp[2][2] = {};
    std::vector<SplitOp> near_op[2], x_op[2], w_op[2];   // [dir][code]
    std::vector<SplitOp> m2l_op[2];                       // [dir][V code] (group E, 2 P1 rows)
    SplitOp leafA_op[2], e_op[2];
    // group E column scales (powers of two) per direction: [expA][64], [expB][64].
    // Coefficient k of an expansion is multiplied by s_k before its digits are
    // taken and column k of the operator is divided by s_k (exact rescaling
    // that balances the fixed-point rounding of operator and input).
    const double *escale[2] = {nullptr, nullptr};
    // group V's inner dimension: the p^2 leaf nodes, zero-padded to one of
    // the tensor kernel's K (64 for p = 8, 256 for p = 12 and 16)
    int np = 256, kv = 256;
    long long wait_limit = 1ll << 26;            // polls of a bounded mbarrier wait
    int withhold_copy = 0;                       // diagnostics: never start the operator copies (forces a timeout)
};
// One tile = one operator times up to kSplitTileN columns.
struct SplitTile {
    int64_t a_off;
    int32_t rows, exp_off;
    int32_t p0, cnt;       // columns [p0, p0 + cnt)
};
// One column = one input vector and where its result rows go.
struct SplitCol {
    int32_t vec;           // digit-vector index
    int32_t ctl;           // (power-of-two exponent shift << 1) | (multiply by 1/alpha0)
    double *out;           // result row r goes to out[r]
};
struct SplitGemm {
    const SplitTile *tiles = nullptr;
    const SplitCol *cols = nullptr;
    int ntiles = 0;
    const uint8_t *ops = nullptr;
    const int32_t *op_exp = nullptr;
    const uint16_t *dig = nullptr;     // [nvec][5][K] BF16 digit bits
    const int32_t *dexp = nullptr;     // [nvec]
    int max_ctas = 0;                  // CTAs of the launch at most (0: one per SM)
};
struct SplitTree {
    // [forward, adjoint]; group V as far part (leafA, X list: needed by the
    // upward and downward passes) and near part (needed at the leaf output),
    // launched apart when the near part runs on the side stream, and as one
    // list (near tiles first: two jobs each) otherwise; group E (L2P / P2M^H,
    // W list); group M: the V-list translations (M2L) by offset code
    SplitTile *tV[2] = {}, *tN[2] = {}, *tVN[2] = {}, *tE[2] = {}, *tM[2] = {};
    SplitCol *cV[2] = {}, *cN[2] = {}, *cVN[2] = {}, *cE[2] = {}, *cM[2] = {};
    int ntV[2] = {}, ntN[2] = {}, ntVN[2] = {}, ntE[2] = {}, ntM[2] = {};
    int ntA[2] = {};   // the first ntA tiles of tV: leaf-to-expansion (the rest: X list)
    int ntL[2] = {};   // the first ntL tiles of tE: expansion-to-leaf (the rest: W list)
    double *Pnear = nullptr;      // [n_near][256] near-field result per entry (scale included)
    double *PX = nullptr;         // [n_x][64] X-list result per entry
    double *PE = nullptr;         // [nleaf][256] L2P (adjoint P2M^H) result per leaf
    double *PW = nullptr;         // [n_w][256] W-list result per entry
    uint16_t *vdig = nullptr;     // [nleaf][5][256] digits of the leaf vectors
    int32_t *vexp = nullptr;      // [nleaf]
    uint16_t *edig = nullptr;     // [2 nbox][5][64] digits of expA (first nbox) and expB
    int32_t *eexp = nullptr;      // [2 nbox]
    int32_t *err = nullptr;       // device error flag (bounded waits)
};
size_t split_smem_bytes(int kd);
cudaError_t split_prepare();   // kernel attributes of the split path (before any capture)
int split_sm_count();          // SMs of the device (after split_prepare)
// parts: which products take the tensor-core results (bits: 1 near field,
// 2 leafA, 4 X list, 8 L2P / P2M^H, 16 W list, 32 M2L); the others run in FP64.
// Bit 64: the shifts of the two level passes in double-float arithmetic on
// the FP32 units instead of FP64, and, with bit 2 off, the leaf-to-expansion
// step too (inside the upward pass; then the input digits run on the side
// stream; on the 20-Gaussian workload the leaf step in the upward pass
// doubles that pass, since each block streams the 98 KB operator for its ~4
// leaves before it can climb).
// BC_SPLIT_BF16 takes the fixed-operator products (bits 1-16: the M2L, the
// shifts, the log terms and the sums stay FP64), BC_SPLIT_BF16_ALL every part.
constexpr int kSplitAllParts = 127;
constexpr int kSplitTableParts = 31;
inline bool is_split(int prec) { return prec == BC_SPLIT_BF16 || prec == BC_SPLIT_BF16_ALL; }
// parts of a split apply: the mode's set, or the diagnostic override (>= 0)
inline int split_parts_for(int prec, int override_parts)
{
    return override_parts >= 0 ? override_parts : (prec == BC_SPLIT_BF16_ALL ? kSplitAllParts : kSplitTableParts);
}
struct SplitLaunch {
    const SplitTables *tables;
    const SplitTree *tree;
    int parts = kSplitTableParts;
    const struct SideStream *side = nullptr;   // null: the near-field launch stays on the apply's stream
    int near_ctas = 0;                          // CTAs of the near-field launch on the side stream (0: all SMs)
};
// Digits of the leaf vectors (times scale), of the two expansion arrays
// (times scale), and the tensor-core operator products of one group.
// (np nodes per leaf, digits zero-padded to kv per slice)
cudaError_t launch_split_digits_vec(int64_t nleaf, const double *v, double scale, uint16_t *dig, int32_t *dexp,
                                    cudaStream_t st, const uint8_t *active, int np, int kv);
// Expansion digits of vectors [i0, i1) of the pair (expA: 0..nbox-1, expB:
// nbox..2 nbox-1).
cudaError_t launch_split_digits_exp(int64_t i0, int64_t i1, int64_t nbox, const double2 *ea, const double2 *eb,
                                    int P1, double scale, const double *escale, uint16_t *dig, int32_t *dexp,
                                    cudaStream_t st);
// intcvt: the epilogue converts its integer sums to FP64 with integer
// operations only (same bits), for launches that run beside FP64 kernels.
cudaError_t launch_split_gemm(const SplitGemm &g, int kd, double inv_alpha0, int32_t *err, long long wait_limit,
                              int withhold, cudaStream_t st, bool intcvt = false);

// Launch parameters common to the passes.  leaf_bps / m2l_bps: resident
// blocks per SM used to size the grids of the leaf kernels and of the M2L
// kernel (tunable; 0 = default).
struct PassArgs {
    int p, NP, P1;
    double half_L;        // r at level 0
    int64_t nleaf, nbox;
    int leaf_bps = 0, m2l_bps = 0;
    int m2l_kind = 0;     // FP64 M2L: 0 by FMAs (k_m2l_boxes), 1 on the FP64 tensor cores (k_m2l_mma)
    // persistent level-synchronous passes: resident blocks of the upward and
    // shift kernels (all blocks must be resident), bounded barrier waits
    int up_blocks = 0, shift_blocks = 0, down_blocks = 0;   // down_blocks: the one-warp-per-box FP64 pass
    long long wait_limit = 1ll << 26;
    int32_t *err = nullptr;
};
// Launch parameters of an apply of `t` on the context (grids, limits, flags).
PassArgs pass_args(const bc_ctx *ctx, const bc_tree *t);
// Largest grids of the persistent FP64 passes whose blocks are all resident
// (occupancy calculator), capped at `per_sm` blocks per SM.
// (df_T, df_maxp: the double-float climb's schedule; f_T, f_maxp: the largest
// factored FP64 shift schedule of the context.)
cudaError_t fp64_prepare(int NP, int P1, int df_T, int df_maxp, int f_T, int f_maxp, int up_per_sm, int down_per_sm,
                         int *up_blocks, int *shift_blocks, int *down_blocks);

// Disjoint union of trees (batched applies): leaves and boxes renumbered,
// boxes sorted by (level, tree, Morton order), lists concatenated.
bc_status merge_host_trees(const std::vector<const HostTree *> &trees, HostTree &out,
                           std::vector<int64_t> &leaf_offset);

// Forward (adj = false) or adjoint (adj = true) apply on `stream`.
// vin: f (forward) or g (adjoint); vout: u or h.  Device pointers.
// Stage boundaries recorded when timing is on (events 0..7 on the apply's
// stream): tensor group V | barrier reset | upward | M2L pairs (and the FP64
// X-list products) | downward level pass | tensor group E | leaf output;
// events 8, 9 bracket the near-field tensor launch on the side stream (stage
// 7, overlapping stages 1-4; empty when the near field is part of the single
// group-V launch of stage 0).  The FP64 path leaves the tensor stages empty.
constexpr int kNumStages = 8;
constexpr int kNumEvents = 10;
// pass_mask bit 0: near field, bit 1: far field.  ev: kNumStages+1 events or null.
// m2l_tri: triangular truncation of the M2L series (k + l <= P).
cudaError_t launch_apply(const PassArgs &a, const HostTree &h, const DevTree &d, const DevTables &tb,
                         bool adj, const double *vin, double *vout, cudaStream_t stream, int pass_mask,
                         cudaEvent_t *ev, int m2l_tri, const struct SplitLaunch *split);
// Fork/join resources of the split path: the near-field tensor launch runs on
// `side` between the events.
struct SideStream {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t xdone = nullptr;   // the X-list tiles (first on the side stream) are done
};
// Far-field passes for point sources on a tree (the glue layer potential):
// the caller has written every leaf box's multipole into d.expA and the X-list
// rows into fl.PX; this clears the flags, climbs (M2M), runs the M2L over the
// given V lists into d.expB and the downward pass (L2L + X rows) in place.
// FP64, forward only.
struct FarLists {
    const int32_t *v_ptr = nullptr, *v_src = nullptr, *v_code = nullptr;   // per box
    const int32_t *x_ptr = nullptr, *x_src = nullptr;                        // per box
    const double2 *PX = nullptr;                                             // [n_x][P1]
    const uint8_t *live = nullptr;   // [nbox] 1 where the subtree holds sources (null: every box)
};
cudaError_t launch_far_points(const PassArgs &a, const HostTree &h, const DevTree &d, const DevTables &tb,
                              const FarLists &fl, cudaStream_t stream);
// Point sources of the glue layer potential on a tree (device side): the
// sources sorted by leaf, their permutation, the scaled strengths, and the
// tree's lists kept only where the source side holds sources (V: source box
// with sources in its subtree; W: the same; X: source leaf with sources; near:
// leaves with sources).
struct LayerDev {
    int64_t n = 0, nx = 0;
    const int32_t *order = nullptr;     // [nleaf] leaf output order (heaviest near work first)
    const int32_t *src_ptr = nullptr;   // [nleaf + 1] caller-leaf CSR into the sorted sources
    const int32_t *perm = nullptr;      // [n] sorted -> caller order
    const double2 *sxy = nullptr;       // [n]
    double *cq = nullptr;               // [n] -q / (2 pi), sorted
    double2 *cm = nullptr;              // [n] -m / (2 pi), sorted
    const int32_t *v_ptr = nullptr, *v_src = nullptr, *v_code = nullptr;
    const int32_t *x_ptr = nullptr, *x_src = nullptr, *x_box = nullptr;
    const int32_t *w_ptr = nullptr, *w_src = nullptr, *w_code = nullptr;
    const int32_t *n_ptr = nullptr, *n_src = nullptr;
    double2 *PX = nullptr;              // [nx][P1]
    const uint8_t *live = nullptr;      // [nbox] 1 where the box's subtree holds sources
};
// u at every leaf node (device pointers: q [n], m [n][2] caller order, u [nleaf][NP]).
// With split (tables and the tree's tiles), the L2P at every leaf runs as the
// forward group-E tiles of the volume apply (expansion digits of the locals,
// then the tensor products into the tree's PE rows); otherwise in FP64.
cudaError_t launch_layer(const PassArgs &a, const HostTree &h, const DevTree &d, const DevTables &tb,
                         const LayerDev &ly, const double *q, const double *m, double *u, cudaStream_t stream,
                         const struct SplitLaunch *split = nullptr);
// The near sums' logarithm and reciprocal: table upload (before the first
// layer launch on a device) and a check launch (x, lg, inv device arrays).
cudaError_t layer_log_init();
cudaError_t launch_log_inv_check(const double *x, int64_t n, double *lg, double *inv, cudaStream_t st);
// The split path's tiles of a tree (built on first use; api.cpp).
bc_status prepare_split_tree(struct bc_tree *t);
// Strip solve (kernels_strip.cu): nsys block-cyclic-tridiagonal systems,
// one warp each; workspace strip_work_doubles(N, m, r) per system.
size_t strip_work_doubles(int64_t N, int m, int r);
size_t strip_smem_bytes(int m, int r);
cudaError_t launch_strip(int64_t nsys, int64_t N, int m, int r, const double *A, const double *B, const double *C,
                         const double *b, double *x, double *work, int32_t *status, cudaStream_t stream);
// large blocks (m > 32): the pieces of the blocked LU, launched by strip.cpp
int strip_panel_width();
// shared-memory limit of the panel kernel for panels of up to nmax rows (before any capture)
cudaError_t strip_prepare(int nmax);
cudaError_t launch_strip_aug(int64_t N, int m, int r, int64_t k, const double *A, const double *B, const double *C,
                             const double *b, double *aug, int Wc, cudaStream_t stream);
cudaError_t launch_strip_panel(double *M, int n, int ld, int j0, int jb, int32_t *piv, int32_t *status,
                               cudaStream_t stream);
// the row exchanges of the panel at j0 on columns [c0, c1)
cudaError_t launch_strip_swap(double *M, int ld, int j0, int jb, const int32_t *piv, int c0, int c1,
                              cudaStream_t stream);
cudaError_t launch_strip_border(int64_t N, int m, int r, const double *A, const double *B, const double *C,
                                const double *b, double *S, cudaStream_t stream);
// rows [j0, j0 + jb) of columns [c0, c1) := L11^-1 (unit lower, upper = false)
// or U11^-1 (upper = true) times themselves
cudaError_t launch_strip_trsm(double *M, int ld, int j0, int jb, bool upper, int c0, int c1, cudaStream_t stream);
// Batched applies: copy the per-tree arrays into / out of the union's vectors.
constexpr int kBatchChunk = 96;   // trees per gather/scatter launch (pointer tables go by value)
struct BatchPtrs {
    const double *in[kBatchChunk];
    double *out[kBatchChunk];
    int64_t off[kBatchChunk + 1];   // first union leaf of each tree in this chunk (+ end)
    int n;
};
cudaError_t launch_batch_copy(const BatchPtrs &bp, bool gather, double *union_buf, int NP, cudaStream_t st);
cudaError_t launch_eval_points_grad(const PassArgs &a, const DevTree &d, const double *u, const double *xy,
                                    int64_t n, double *val, double *grad, double x0, double y0, double L,
                                    cudaStream_t stream);
cudaError_t launch_eval_points(const PassArgs &a, const DevTree &d, const double *u, const double *xy,
                               int64_t n, double *out, double x0, double y0, double L,
                               cudaStream_t stream);

}  // namespace bc

struct bc_ctx {
    bc_config cfg{};
    int device = 0;
    int p = 0, NP = 0, P1 = 0;
    bool tables_ready = false;
    int pass_mask = 3;          // diagnostics: bit 0 near field, bit 1 far field
    int m2l_tri = 0;            // 1: keep only M2L terms with k + l <= P (triangular truncation)
    int split_parts = -1;       // diagnostics: split-precision products in use (-1: the precision mode's set)
    int split_overlap = 1;      // near-field tensor launch on the side stream (1) or inline (0)
    int overlap_ctas = 0;       // CTAs of that launch (0: by arrangement, see near_ctas_for)
    int m2l_bps = 0;            // resident blocks per SM of the FP64 M2L kernel (0: by arrangement)
    int m2l_kind = 0;           // FP64 M2L kernel: 0 FMA, 1 tensor-core MMA (see PassArgs)
    bool timing = false;        // record CUDA events around each stage
    cudaEvent_t ev[2][bc::kNumEvents] = {};   // [forward, adjoint]
    bc::SideStream side;
    bc::HostTables ht;
    bc::DevTables dt;
    bc::SplitTables split;
    std::vector<void *> split_allocs;
    bool split_ready = false;
    int32_t *dev_err = nullptr;   // device flag set by kernels whose bounded waits gave up
    int up_blocks = 0, shift_blocks = 0, down_blocks = 0;   // grids of the persistent passes
    // launch shapes chosen by the autotuner: key = precision*1024 + adjoint*512 + log2(nleaf)
    std::vector<std::pair<int, std::pair<int, int>>> tuned;
    std::mutex mu;
};

struct bc_tree {
    bc_ctx *ctx = nullptr;
    bool is_union = false;   // the union tree of a batch
    bc::HostTree h;
    bc::DevTree d;
    bc::SplitTree sp;
    bool split_ready = false;
    bool m2l_ready = false;   // tensor-core M2L tiles and rows (BC_SPLIT_BF16_ALL)
};
