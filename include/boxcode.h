/*
 * boxcode.h -- C ABI of the GB300 machine code: the free-space 2D Laplace volume
 * potential on an adaptive quadtree of p x p Chebyshev leaf boxes.
 *
 * The operation (paper Sec. 3.2, eq. (vbulk), with Phi from Sec. 2):
 *
 *     u(x_i) = (1/2pi) * sum_{leaves B} int_B log|x_i - y| f_B(y) dy
 *
 * i.e. u = v_bulk = -int_{Omega_B} Phi(x,y) f(y) dy with Omega_B the union of
 * the leaves, so that Laplace(u) = f.  f_B is the tensor-product polynomial of
 * degree p-1 per variable interpolating the leaf's node values (Sec. 3.2.1).
 * The x_i are the nodes of all leaves.  Leaves form a 2:1-balanced quadtree
 * (Sec. 3.2.1, last paragraph): leaves that touch, across an edge or a
 * corner, differ by at most one level.
 *
 * Conventions shared by every call:
 *   - Nodes: first-kind Chebyshev points x_j = -cos((2j+1) pi / (2p)),
 *     j = 0..p-1 (ascending), scaled to each leaf.  A leaf's values are p*p
 *     doubles, row-major with the x index fastest: v[jy*p + jx].
 *   - Arrays of leaf values are [nleaf][p][p] FP64, contiguous, with leaves in
 *     the order the caller gave when creating the tree.
 *   - Ownership: the context owns the tables, a tree owns its lists and its
 *     workspaces; the caller owns every array it passes and the library never
 *     frees or retains caller memory beyond the call (asynchronous calls read
 *     and write it in stream order).
 *   - Errors: every call returns a bc_status; nothing aborts.  The message of
 *     the last failure on the calling thread is bc_last_error().  Work queued
 *     on a stream reports device-side failures at the next synchronising
 *     call on that tree or context (bc_sync).
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Device calls are ordered on it.
 *   - Results are overwritten, never accumulated.
 *   - Thread safety: calls on different trees may run concurrently; calls on
 *     the same tree must be serialised by the caller (a tree's workspaces are
 *     shared by its applies).
 */
#ifndef BOXCODE_H
#define BOXCODE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bc_ctx bc_ctx;   /* opaque: device, order p, tables */
typedef struct bc_tree bc_tree; /* opaque: leaves, interaction lists, workspaces */

typedef enum {
    BC_OK = 0,
    BC_ERR_ARG = -1,         /* invalid argument (NULL, size, range) */
    BC_ERR_TREE = -2,        /* leaves overlap, leave gaps, or are not 2:1 balanced */
    BC_ERR_CUDA = -3,        /* a CUDA runtime error; message names it */
    BC_ERR_OOM = -4,         /* host or device allocation failed */
    BC_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    BC_ERR_UNSUPPORTED = -6, /* valid request this build does not provide */
    BC_ERR_STATE = -7        /* call order violated (e.g. apply before tables) */
} bc_status;

/* Arithmetic of an apply.  "BF16 digits" means: each FP64 operand row (an
 * operator row, an input vector) is scaled by a power of two, rounded to a
 * 40-bit fixed-point integer and cut into five BF16 digits; the digit
 * products run on the tensor cores (tcgen05, FP32 accumulation, exact), and
 * the recombination is integer/FP64.  The rounding of the operands to 40 bits
 * is the only error (about 2^-40 of sum |A_ik v_k| per output). */
typedef enum {
    BC_FP64 = 0,           /* every step in native FP64 */
    BC_SPLIT_BF16 = 1,     /* BF16 digits for the fixed-operator products: the
                              near-field tables, P2M, L2P, the W list (M2P) and
                              the X list (P2L), and their adjoints.  Native FP64
                              for the multipole-to-local translations, the
                              M2M and L2L shifts, every log-kernel scaling
                              term and every sum of partial results
                              (p = 8, 12 and 16, nterms <= 32; other orders
                              BC_ERR_UNSUPPORTED) */
    BC_SPLIT_BF16_ALL = 2  /* BC_SPLIT_BF16 plus the multipole-to-local
                              translations on BF16 digits (their log terms
                              stay FP64) and the M2M / L2L shifts in
                              double-float arithmetic (pairs of FP32 numbers,
                              about 48 bits, on the FP32 units); the V- and
                              X-list sums and the local expansions handed to
                              later steps stay FP64 (p = 8, 12, 16) */
} bc_precision;

typedef struct {
    int p;            /* nodes per side, 4..16 (paper uses 16) */
    int nterms;       /* far-field expansion terms P+1, 4..32; 0 = default 30 */
    int node_kind;    /* 1 = first-kind Chebyshev (the only kind provided); 0 = default */
    int split_slices; /* BF16 slices per operand for BC_SPLIT_BF16; 0 = default */
    int autotune;     /* 1 = time tile shapes on first batched apply; 0 = fixed */
} bc_config;

/* Counts describing a tree, for flop and byte accounting. */
typedef struct {
    int64_t nleaf, nbox, nlevels;  /* nlevels = max leaf level + 1 */
    int64_t n_near;  /* near-field (leaf,leaf) slots, self included */
    int64_t n_v;     /* M2L translations (V lists) */
    int64_t n_w;     /* multipole-to-node evaluations (W lists, "list 3") */
    int64_t n_x;     /* node-density-to-local conversions (X lists, "list 4") */
    int64_t n_nonleaf; /* boxes at level >= 2 with children (M2M/L2L work) */
    int64_t n_down;  /* boxes at level >= 2 (local expansions) */
} bc_tree_stats;

/* Create a context on CUDA device `device` for order cfg->p.  Allocates
 * nothing on the device until bc_tables_build.  device = -1 gives a host-only
 * context: tables and trees are built on the host (for inspection and tests)
 * and every device call returns BC_ERR_STATE. */
bc_status bc_create(const bc_config *cfg, int device, bc_ctx **out);
void bc_destroy(bc_ctx *ctx);

/* Message of the last failed call on this thread ("" if none). */
const char *bc_last_error(void);

/* Precompute and upload every table (near-field tables for the 33 relative
 * positions a 2:1-balanced tree allows, far-field translation operators, the
 * BF16 digits of the split-precision operators).  Not in the paper: these are
 * the internals of the box code it calls as a black box (Sec. 3.2.1, last
 * paragraph); every table is a quadrature of the kernel of eq. (vbulk) or a
 * translation of its multipole / local expansions.  Host FP64 quadrature;
 * cached in `cache_dir` (NULL: no cache) in a file keyed by (p, nterms, node
 * kind, format version) with a checksum.  The factored forms of the level
 * shifts are checked against the dense operators here (BC_ERR_STATE if they
 * differ). */
bc_status bc_tables_build(bc_ctx *ctx, const char *cache_dir);

/* Tree from explicit leaves of the root box [x0, x0+L] x [y0, y0+L] (the
 * quadtree of Sec. 3.2.1, 2:1 balanced as in its last paragraph): leaf k is
 * the dyadic box (level[k], ix[k], iy[k]) with 0 <= ix,iy < 2^level, level <= 24.
 * Validates that the leaves are disjoint, cover the root and are 2:1 balanced
 * (BC_ERR_TREE otherwise); builds the interaction lists on the host and
 * uploads them.  Host arrays, read during the call only. */
bc_status bc_tree_create(bc_ctx *ctx, double x0, double y0, double L, int64_t nleaf,
                         const int32_t *level, const int32_t *ix, const int32_t *iy,
                         bc_tree **out);

/* Density callback: out[k] = f(xy[2k], xy[2k+1]) for k < n. */
typedef void (*bc_density_fn)(const double *xy, int64_t n, double *out, void *user);

/* Adaptive tree (paper Alg. 2, function-resolution criterion, then 2:1
 * balance): a box is split while max |c_ab| over the Chebyshev coefficients
 * with a >= p-2 or b >= p-2 exceeds eps * vscale (vscale = largest |f| at the
 * root box's nodes, or 1 if f vanishes there) and its level is below
 * max_level. */
bc_status bc_tree_refine(bc_ctx *ctx, double x0, double y0, double L, bc_density_fn fn,
                         void *user, double eps, int max_level, bc_tree **out);

/* Truncated adaptive tree (paper Alg. 2 with both criteria, Sec. 3.2.1): the
 * domain Omega is bounded by the closed polygon gamma (n_gamma vertices
 * [x, y], the last joined to the first), the bulk region Omega_B by the
 * closed polygon gamma_b (inside Omega); the strip is Omega \ Omega_B.  f is
 * evaluated at the nodes inside Omega only and extended by zero outside it.
 * A box is split (below max_level) if it lies inside Omega and its
 * coefficients are not resolved to eps (as in bc_tree_refine); if it meets
 * both Omega_B and the outside of Omega; or if it meets the strip and its
 * diagonal exceeds half the local strip width s, s the distance between the
 * vertices of gamma and of gamma_b nearest to the box centre.  Then 2:1
 * balance.  Leaves outside Omega are discarded: they are no source and their
 * output is zero (bc_apply / bc_apply_adjoint); leaves cut by gamma keep the
 * zero-extended f (the paper's remark on cut boxes).  The density passed to
 * the applies should be the zero extension (bc_tree_node_mask).  Both curves
 * are simple polygons; gamma lies in the root box; BC_ERR_ARG otherwise. */
bc_status bc_tree_refine_truncated(bc_ctx *ctx, double x0, double y0, double L, bc_density_fn fn, void *user,
                                   double eps, int max_level, const double *gamma, int64_t n_gamma,
                                   const double *gamma_b, int64_t n_gamma_b, bc_tree **out);
/* Leaf classes (host array of nleaf): 0 outside the domain (discarded), 1 cut
 * by its boundary, 2 inside (every leaf of a tree without truncation). */
bc_status bc_tree_leaf_class(const bc_tree *tree, int8_t *cls);
/* Node mask of the zero extension (host array [nleaf][p*p]): 1 where the
 * node lies inside the domain (every node of a tree without truncation). */
bc_status bc_tree_node_mask(const bc_tree *tree, uint8_t *mask);

int64_t bc_tree_nleaf(const bc_tree *tree);
/* Leaves in caller order (host arrays of nleaf entries). */
bc_status bc_tree_leaves(const bc_tree *tree, int32_t *level, int32_t *ix, int32_t *iy);
/* Physical node coordinates, host array [nleaf][p*p][2]. */
bc_status bc_tree_nodes(const bc_tree *tree, double *xy);
bc_status bc_tree_stats_get(const bc_tree *tree, bc_tree_stats *out);
/* Interaction lists, for inspection and tests.  kind: 0 near (per leaf: leaf,
 * table id), 1 V (per box: box, offset code), 2 W (per leaf: box, code),
 * 3 X (per box: leaf, code).  Two-call protocol: pass NULL arrays to get the
 * sizes in *nrows / *nnz, then arrays of that size: ptr[nrows+1], idx[nnz],
 * code[nnz].  Boxes are numbered as in bc_tree_boxes. */
bc_status bc_tree_lists(const bc_tree *tree, int kind, int64_t *nrows, int64_t *nnz,
                        int64_t *ptr, int64_t *idx, int32_t *code);
/* Box table (host arrays of nbox entries): level, ix, iy, parent (-1 root),
 * leaf (caller leaf index or -1). */
bc_status bc_tree_boxes(const bc_tree *tree, int32_t *level, int32_t *ix, int32_t *iy,
                        int32_t *parent, int32_t *leaf);
void bc_tree_destroy(bc_tree *tree);

/* u = A f: the volume potential v_bulk at every leaf node (eq. (vbulk) of
 * Sec. 3.2, definition above), in the arithmetic `prec` names (bc_precision).
 * f, u: [nleaf][p][p] FP64.  Device pointers are used in place and the call
 * is asynchronous on `stream`.  Host pointers are staged through the tree's
 * device buffers, except pinned (page-locked) ones on the split paths, which
 * the kernels read and write in place; with host pointers the call returns
 * after u is written.  u must not alias f. */
bc_status bc_apply(bc_ctx *ctx, const bc_tree *tree, const double *f, double *u,
                   bc_precision prec, void *stream);

/* h = A^T g: the exact transpose of the discrete operator applied by
 * bc_apply (same passes, every operator transposed; the gradient of a loss of
 * u with respect to f).  Not in the paper, whose solver needs the forward
 * operator only.  Same layout, pointer and stream rules as bc_apply. */
bc_status bc_apply_adjoint(bc_ctx *ctx, const bc_tree *tree, const double *g, double *h,
                           bc_precision prec, void *stream);

/* out[k] = interpolant of the leaf-node values u at point xy[k]: v_bulk off
 * the grid, as the glue step needs it on the fictitious curve (Sec. 3.4)
 * (barycentric Chebyshev interpolation on the leaf containing the point; a point on a
 * shared edge belongs to the leaf on its +x / +y side, the root's far edges to
 * the last leaf).  Points outside the root give BC_ERR_ARG on the host path;
 * on the device path they produce NaN.  u, xy, out: device or host (all of the
 * same kind). */
bc_status bc_eval_points(bc_ctx *ctx, const bc_tree *tree, const double *u, const double *xy,
                         int64_t n, double *out, void *stream);

/* Value and gradient at points: val[k] as in bc_eval_points and
 * grad[2k], grad[2k+1] = the x and y derivatives of the same leaf
 * interpolant at xy[k] (barycentric differentiation, free of cancellation as
 * a point nears a node).  The glue step of Sec. 3.4 needs v_bulk and its
 * normal derivative n . grad v_bulk on the fictitious curve (the jumps tau
 * and sigma of Alg. 1).  u, xy, val, grad: device or host (all of the same
 * kind); points outside the root: BC_ERR_ARG on the host path, NaN on the
 * device path. */
bc_status bc_eval_points_grad(bc_ctx *ctx, const bc_tree *tree, const double *u, const double *xy, int64_t n,
                              double *val, double *grad, void *stream);

/* Glue layer potential (Sec. 3.4): v_glue = S[sigma] - D[tau] on the
 * fictitious curve, with S[s](x) = int Phi(x,y) s(y) dy, D[t](x) = int
 * dPhi(x,y)/dn_y t(y) dy and Phi = (1/2pi) log(1/|x-y|), evaluated by the
 * fast multipole method at every leaf node of a tree (the step that, with the
 * box code, gives the particular solution at the nodes; Sec. 4.1 times it).
 * The curve is discretised by quadrature nodes y_j (weights w_j, unit normals
 * n_j); with q_j = w_j sigma(y_j) and m_j = w_j tau(y_j) n_j (a vector):
 *
 *     u(x_i) = -(1/2pi) sum_j [ q_j log|x_i - y_j| + m_j . (x_i - y_j) / |x_i - y_j|^2 ]
 *
 * at every leaf node x_i ([nleaf][p][p], as the applies).  A source that
 * coincides with a node contributes nothing there.  The far field uses the
 * tree's expansions and lists (error of the expansion order, as the volume
 * apply), the near field is summed directly, in FP64.  precision BC_FP64: all
 * of it in FP64; BC_SPLIT_BF16 (p = 8, 12, 16, nterms <= 32, else
 * BC_ERR_UNSUPPORTED): the local-to-node evaluation (L2P) at every leaf runs
 * on the BF16 tensor cores as exact digit products (the volume apply's
 * split-precision L2P), the rest in FP64; other values BC_ERR_ARG.
 *
 * bc_layer_create: the sources xy[n][2] (host, read during the call), inside
 * the root box (else BC_ERR_ARG), are sorted into the tree's leaves, and the
 * tree's lists are kept only where the source side holds sources.  The layer
 * keeps the tree (destroy the layer first) and shares its workspaces: an
 * apply of any kind on the same tree must not overlap a layer apply.
 * bc_layer_apply: q[n], m[n][2] in the order of xy, u[nleaf*p*p]; device
 * pointers (ordered on `stream`) or host pointers (staged, synchronous), all
 * of one kind.
 * bc_layer_info: counts[6] = sources, V pairs, W pairs, X entries,
 * (target leaf, near source) pairs, leaves holding sources. */
typedef struct bc_layer bc_layer;
bc_status bc_layer_create(bc_tree *tree, const double *xy, int64_t n, bc_layer **out);
bc_status bc_layer_apply(bc_ctx *ctx, bc_layer *layer, const double *q, const double *m, double *u,
                         bc_precision precision, void *stream);
bc_status bc_layer_info(const bc_layer *layer, int64_t *counts);
void bc_layer_destroy(bc_layer *layer);

/* Strip solve (Sec. 3.3): the spectral-collocation system of the strip
 * couples each element only to its two neighbours around the closed strip,
 * so it is block tridiagonal with two corner blocks from the periodicity:
 *
 *     C[k] x[k-1] + A[k] x[k] + B[k] x[k+1] = b[k],   k = 0..N-1, indices mod N
 *
 * (with N = 1 or 2 the blocks meeting at one position add).  Solved as the
 * paper does: block LU of the tridiagonal part, then the Woodbury identity
 * for the corner blocks C[0] and B[N-1] (O(m^3 N) per system).  Batched over
 * nsys independent systems: blocks up to 32 x 32 one warp per system, all
 * systems at once; larger blocks (the paper's elements, 16 x 24 = 384 nodes)
 * one system after another, each step a blocked LU over the whole GPU (rank
 * updates as cuBLAS DGEMMs).  Layout, all FP64 row-major device arrays: A, B,
 * C [nsys][N][m][m]; b, x [nsys][N][m][r].  Shapes: N >= 1, 1 <= m <= 448,
 * 1 <= r <= 32.  work: device scratch of
 * bc_strip_workspace() bytes, owned by the caller.  status: NULL or device
 * int32 [nsys], set to 1 where a pivot of the block LU (every diagonal block
 * D_k and the 2m x 2m capacitance matrix are factored with partial pivoting)
 * was zero or not finite, else 0; no pivoting across blocks, so the systems
 * should be block diagonally dominant, as collocation strips with their
 * continuity rows are.  Host pointers: BC_ERR_ARG.  Stream-ordered. */
bc_status bc_strip_workspace(int64_t nsys, int64_t N, int m, int r, int64_t *bytes);
bc_status bc_strip_solve(int64_t nsys, int64_t N, int m, int r, const double *A, const double *B, const double *C,
                         const double *b, double *x, void *work, int32_t *status, void *stream);

/* Batched applies: many independent densities on different trees (all of
 * this context's p and root side L) in one launch per pass.  Not in the
 * paper (its solver applies one box code at a time).  A batch is the
 * disjoint union of its trees (leaves and boxes renumbered, lists
 * concatenated), uploaded once; every pass of an apply then covers all trees
 * in a single kernel launch, and the whole pass sequence is captured once per
 * (precision, direction) as a CUDA graph and replayed.  The trees must stay
 * alive while the batch exists.  bc_batch_create allocates the union's lists,
 * workspaces and input/output buffers. */
typedef struct bc_batch bc_batch;
bc_status bc_batch_create(bc_ctx *ctx, const bc_tree *const *trees, int n, bc_batch **out);
void bc_batch_destroy(bc_batch *batch);
int64_t bc_batch_nleaf(const bc_batch *batch);   /* total leaves */
/* in[k] -> out[k] for tree k (device arrays [nleaf_k][p][p]); adjoint != 0
 * applies A^T.  Ordered on `stream`: gather into the union's buffer, replay of
 * the captured graph, scatter to out[k].  The first run of a (precision,
 * direction) captures the graph (with the context's autotune flag set it
 * first runs bc_batch_autotune). */
bc_status bc_batch_run(bc_ctx *ctx, bc_batch *batch, const double *const *in, double *const *out,
                       bc_precision prec, int adjoint, void *stream);
/* Times a few launch shapes (resident blocks per SM of the leaf kernels and
 * of the M2L kernel) for both directions on `stream`, keeps the fastest graph
 * and records the choice in the context, keyed by precision, direction and
 * log2 of the batch's leaf count, for later batches of that size.  The batch
 * buffers' contents are overwritten. */
bc_status bc_batch_autotune(bc_ctx *ctx, bc_batch *batch, bc_precision prec, void *stream);
/* The launch shape in use for (precision, adjoint): 0 before the first run. */
bc_status bc_batch_shape(const bc_batch *batch, int precision, int adjoint, int *leaf_blocks_per_sm,
                         int *m2l_blocks_per_sm);

/* Copy a host table for inspection: which = 0 nodes[p], 1 w[p*p] (integrals
 * of the Lagrange basis), 2 near tables [41][p*p][p*p] (unused slots zero),
 * 3 P2M [P+1][p*p] complex, 4 L2P [p*p][P+1] complex, 5 M2M [4][P+1][P+1],
 * 6 L2L [4][P+1][P+1], 7 M2L [49][P+1][P+1], 8 M2P [36][p*p][P+1],
 * 9 P2L [36][P+1][p*p] (complex entries as interleaved re, im).  Pass
 * out = NULL to get *count (doubles). */
bc_status bc_table_export(const bc_ctx *ctx, int which, int64_t *count, double *out);

/* Runtime options of a context (none in the paper).
 *   "m2l_triangular" (0/1, default 0): keep only the terms with k + l <= P of
 *     each multipole-to-local translation (and exactly their transpose in the
 *     adjoint), which halves the M2L arithmetic but loses accuracy.
 *   "m2l_kernel" (0/1, default 0): the FP64 multipole-to-local kernel: 0 FP64
 *     FMAs, one block per target box; 1 the FP64 tensor cores (mma.sync f64
 *     tiles of the binomial matrix), one warp per target box.  Same results
 *     to rounding.
 *   "m2l_blocks_per_sm" (integer 0..32, default 0): resident blocks per SM of
 *     the FP64 M2L launch; 0 chooses by arrangement (3, or 2 for kernel 1,
 *     beside the near-field tensor launch, which fits beside them; 8 (4)
 *     otherwise).
 *   "wait_limit" (default 2^26): polls of each bounded device-side wait of the
 *     split-precision kernel before it gives up, records the failure (reported
 *     by bc_sync as BC_ERR_TIMEOUT), frees its tensor memory and returns; the
 *     level passes' box flags poll a sixteenth of it and report the same way.
 *   "split_overlap" (0..3, default 1): the X-list and near-field tensor-core
 *     launches of a split-precision apply run on an internal stream and are
 *     joined before the downward pass (X list) and the leaf output (near
 *     field) (1; 2 in the forward apply only, 3 in the adjoint only), or in
 *     line on the apply's stream (0).  With the M2L in FP64
 *     (BC_SPLIT_BF16) they start after the upward pass and run beside the
 *     FP64 M2L (they use the tensor cores, it the FP64 units); with the
 *     tensor-core M2L (BC_SPLIT_BF16_ALL) they start at once, beside the
 *     latency-bound level passes.
 *   "split_overlap_ctas" (integer >= 0, default 0): CTAs (one per SM) of
 *     that near-field launch; 0 takes every SM beside the FP64 M2L and three
 *     quarters of them beside the level passes.
 *   "debug_split_parts" (integer -1..127, default -1): diagnostics; which
 *     products of a split-precision apply use the tensor-core results (bits:
 *     1 near field, 2 leaf-to-expansion, 4 X list, 8 expansion-to-leaf,
 *     16 W list, 32 M2L translations); the others are evaluated in FP64.
 *     Bit 64: the shifts of the upward and downward level passes, and with
 *     bit 2 off the leaf-to-expansion step, in double-float arithmetic (pairs
 *     of FP32 numbers, about 48 bits) instead of FP64.  -1 takes the set of
 *     the precision mode: 31 for BC_SPLIT_BF16, 127 for BC_SPLIT_BF16_ALL.
   "debug_withhold_copy" (0/1, default 0): diagnostics; the split-precision
 *     kernel never starts its table copy, so its first wait runs out (tests of
 *     the timeout path).
 * Unknown names give BC_ERR_ARG. */
bc_status bc_set_option(bc_ctx *ctx, const char *name, double value);

/* Diagnostics.  pass_mask selects the parts of the operator an apply
 * evaluates: bit 0 the near field (leaf-to-leaf tables), bit 1 the far field
 * (expansions); 3 = the full operator (default).  timing != 0 records a CUDA
 * event at each stage boundary:
 *   0 tensor group V, far part (split precision: digits of the input,
 *     leaf-to-expansion; in line also the X list and the near field),
 *     1 flag clearing, 2 upward pass (FP64: with the leaf-to-expansion step),
 *     3 M2L (FP64 path: and the X-list products), 4 downward level pass (sums,
 *     shifts), 5 tensor group E (split precision: digits of the expansions,
 *     expansion-to-leaf and W list), 6 leaf output; 7 the X-list and
 *     near-field tensor launches when they run apart on the internal stream
 *     (split_overlap: beside stage 3 with the FP64 M2L, beside stages 1-4
 *     otherwise; in line stage 7 is empty);
 * bc_debug_stage_times then waits for the last events of the most recent
 * forward (adjoint = 0) or adjoint apply and writes the eight stage durations
 * in milliseconds to ms[8] (stages 0, 5 and 7 are empty for FP64 applies). */
bc_status bc_debug_set(bc_ctx *ctx, int pass_mask, int timing);
bc_status bc_debug_stage_times(bc_ctx *ctx, int adjoint, double *ms);
/* The term schedule of the double-float upward shift of BC_SPLIT_BF16_ALL, for
 * the forward (adjoint = 0: M2M) or adjoint (L2L^H) operator of a context
 * whose tables are built (host-only contexts too).  The nonzero terms
 * (output l, input k) of the four child operators, output by output, are cut
 * into 32 runs of *T terms, run i on lane i; a lane ends a partial sum where
 * its run leaves an output, in slot l * (*maxp) + (its place among the
 * output's lanes).  code: [T][32], input k in bits 0-7 and, where a partial
 * sum ends, slot + 1 from bit 8 (0 elsewhere, and for the zero terms that
 * pad the last runs); ops: [4][T][32][4], child q's entry of each term as
 * {Re hi, Re lo, Im hi, Im lo} (x = hi + lo, both FP32); np: [nterms], the
 * partial sums of each output.  With code, ops and np NULL only *T and
 * *maxp are written; otherwise each non-NULL array receives its full size.
 * BC_ERR_STATE before the tables are built. */
bc_status bc_debug_up_schedule(const bc_ctx *ctx, int adjoint, int32_t *T, int32_t *maxp, uint32_t *code,
                               float *ops, int32_t *np);
/* Measured FP64 FMA throughput of `device` in TFLOP/s (independent FMA chains,
 * 8 blocks per SM, best of three timed runs).  The roofline denominator of
 * the FP64 passes (diagnostics; not in the paper). */
bc_status bc_debug_fp64_peak(int device, double *tflops);
/* The layer potential's near-sum logarithm and reciprocal (a table-driven
 * logarithm after Tang, ACM TOMS 16, 1990, and the matching reciprocal
 * series) applied to x[n] > 0 (normal, 1/x normal): lg[i] = log x[i],
 * inv[i] = 1/x[i].  Device pointers, ordered on `stream`.  Diagnostics: the
 * tests compare it with the CUDA math library's log and division. */
bc_status bc_debug_log_inv(int device, const double *x, int64_t n, double *lg, double *inv, void *stream);

/* FP64 apply (adjoint = 0: u = A f; adjoint != 0: the transpose) that
 * allocates no memory during the call.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory at call
 * time, such as code running inside another framework whose memory pool owns
 * the device's free memory, or work recorded while allocation is forbidden.
 * The expansion workspaces come from one fixed 16 MiB array in the library's
 * device image (held by every device that loads the library, until exit)
 * instead of the tree's own buffers; the tree needs
 * 2 x boxes x nterms x 16 bytes of it, and larger trees give BC_ERR_ARG.
 * in/out: device arrays [nleaf][p][p] FP64, as in bc_apply.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) and so
 * should come before any stream capture.  All calls share the array and it
 * keeps what the last call left in it (nothing in it needs clearing); calls
 * that overlap on the GPU race with each other, so serialise them.  The call
 * also uses the tree's own per-box flags and X-list buffer, so it races with
 * an overlapping bc_apply or bc_apply_adjoint on the same tree as well: the
 * caller serialises every apply of one tree. */
bc_status bc_apply_noalloc(bc_ctx *ctx, const bc_tree *tree, const double *in, double *out, int adjoint,
                           void *stream);

/* Wait for the stream and report device-side failures recorded by earlier
 * calls on this context (BC_ERR_TIMEOUT, BC_ERR_CUDA). */
bc_status bc_sync(bc_ctx *ctx, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BOXCODE_H */
