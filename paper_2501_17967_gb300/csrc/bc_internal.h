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
};

// Builds boxes and lists from explicit leaves; returns BC_OK or BC_ERR_TREE /
// BC_ERR_ARG with the message set.
bc_status build_host_tree(HostTree &t, double x0, double y0, double L, int p, int64_t nleaf,
                          const int32_t *level, const int32_t *ix, const int32_t *iy);
// Alg. 2 (function-resolution criterion) followed by 2:1 balancing; fills the
// leaf arrays (level/ix/iy) only.
bc_status refine_leaves(int p, double x0, double y0, double L, bc_density_fn fn, void *user,
                        double eps, int max_level, std::vector<int32_t> &lv,
                        std::vector<int32_t> &ix, std::vector<int32_t> &iy);

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
struct OpSet {
    const double2 *leafA = nullptr;   // [NP][P1]        leaf vector -> box expansion
    const double2 *up = nullptr;      // [4][P1][P1]     child -> parent
    const double2 *par = nullptr;     // [4][P1][P1]     parent -> child
    const double2 *v = nullptr;       // [kNumV][P1][P1] V-list translation
    const double2 *x = nullptr;       // [kNumWX][NP][P1] leaf vector -> expansion (X list)
    const double2 *e = nullptr;       // [P1][NP]        expansion -> leaf nodes (real part)
    const double2 *w = nullptr;       // [kNumWX][P1][NP] expansion -> leaf nodes (W list)
    const double *t = nullptr;        // [kNumNear][NP][NP] near tables, element (j,k) at [k][j]
};

struct DevTables {
    OpSet fwd, adj;
    double *wvec = nullptr;           // [NP]
    // M2L in factored form: d^-k (forward) / conj(d)^-k (adjoint) per V code,
    // log|d| per code, and the binomial table C(i+j-1, j) at [i][j] (row
    // stride P1 + 1) shared by every offset.
    double2 *dpow_f = nullptr, *dpow_a = nullptr;   // [kNumV][P1]
    double *logd = nullptr;                          // [kNumV]
    double *binom = nullptr;                         // [P1][P1 + 1]
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
    double2 *expA = nullptr, *expB = nullptr;  // [nbox][P1] workspaces
    int32_t *zero_ptr = nullptr;               // [nleaf+1] zeros: empty lists (diagnostic pass masks)
    int32_t *cnt = nullptr;                    // [2][nbox] arrival counters (upward, downward passes)
    double *stage_in = nullptr, *stage_out = nullptr; // host-pointer staging [nleaf*NP]
    std::vector<void *> allocs;
};

// Split-precision near field (p = 16 only): BF16 digit slices of the tables
// (per context) and the entry tiles, digit buffers and result scratch (per tree).
constexpr int kSplitSlices = 5;
constexpr int kSplitTileN = 48;
struct SplitTables {
    const uint8_t *A[2] = {nullptr, nullptr};    // [kNumNear][5][2][128 x 256 canonical] fwd, adj
    const int32_t *Aexp[2] = {nullptr, nullptr}; // [kNumNear][256] row exponents
    long long wait_limit = 1ll << 26;            // polls of a bounded mbarrier wait
    int withhold_copy = 0;                       // diagnostics: never start the table copy (forces a timeout)
};
struct SplitTree {
    int ntiles = 0;
    int32_t *tile_tab = nullptr, *tile_p0 = nullptr, *tile_cnt = nullptr;
    int32_t *pair_vec = nullptr, *pair_out = nullptr, *pair_lvl_f = nullptr, *pair_lvl_a = nullptr;
    double *P = nullptr;          // [n_near][256] near-field result per entry
    uint16_t *vsl = nullptr;      // [nleaf][5][256] digits of the input vector (BF16 bits)
    int32_t *vexp = nullptr;      // [nleaf]
    int32_t *err = nullptr;       // device error flag (bounded waits)
};
size_t split_smem_bytes();
cudaError_t split_prepare();   // kernel attributes of the split path (before any capture)
// Split near field of one apply (null: FP64 near field).
struct SplitLaunch {
    const SplitTables *tables;
    const SplitTree *tree;
};

// Launch parameters common to the passes.  leaf_bps / m2l_bps: resident
// blocks per SM used to size the grids of the leaf kernels and of the M2L
// kernel (tunable; 0 = default).
struct PassArgs {
    int p, NP, P1;
    double half_L;        // r at level 0
    int64_t nleaf, nbox;
    int leaf_bps = 0, m2l_bps = 0;
};

// Disjoint union of trees (batched applies): leaves and boxes renumbered,
// boxes sorted by (level, tree, Morton order), lists concatenated.
bc_status merge_host_trees(const std::vector<const HostTree *> &trees, HostTree &out,
                           std::vector<int64_t> &leaf_offset);

// Forward (adj = false) or adjoint (adj = true) apply on `stream`.
// vin: f (forward) or g (adjoint); vout: u or h.  Device pointers.
// Stage boundaries recorded when timing is on:
// split near field | leafA | up | down | leafB.
constexpr int kNumStages = 5;
// pass_mask bit 0: near field, bit 1: far field.  ev: kNumStages+1 events or null.
// m2l_tri: triangular truncation of the M2L series (k + l <= P).
cudaError_t launch_apply(const PassArgs &a, const HostTree &h, const DevTree &d, const DevTables &tb,
                         bool adj, const double *vin, double *vout, cudaStream_t stream, int pass_mask,
                         cudaEvent_t *ev, int m2l_tri, const struct SplitLaunch *split);
// Split near field: digits of vin, then every near entry's 256 results into sp.P.
cudaError_t launch_split_near(const PassArgs &a, const SplitTables &st, const SplitTree &sp, bool adj,
                              const double *vin, cudaStream_t stream);
// Batched applies: copy the per-tree arrays into / out of the union's vectors.
constexpr int kBatchChunk = 96;   // trees per gather/scatter launch (pointer tables go by value)
struct BatchPtrs {
    const double *in[kBatchChunk];
    double *out[kBatchChunk];
    int64_t off[kBatchChunk + 1];   // first union leaf of each tree in this chunk (+ end)
    int n;
};
cudaError_t launch_batch_copy(const BatchPtrs &bp, bool gather, double *union_buf, int NP, cudaStream_t st);
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
    bool timing = false;        // record CUDA events around each stage
    cudaEvent_t ev[2][bc::kNumStages + 1] = {};   // [forward, adjoint]
    bc::HostTables ht;
    bc::DevTables dt;
    bc::SplitTables split;
    std::vector<void *> split_allocs;
    bool split_ready = false;
    int32_t *dev_err = nullptr;   // device flag set by kernels whose bounded waits gave up
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
};
