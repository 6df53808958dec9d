// C ABI of the glue layer potential (include/boxcode.h, bc_layer_*): point
// sources on the fictitious curve, binned into the leaves of a tree, and the
// FMM evaluation of S[sigma] - D[tau] at every leaf node (Sec. 3.4).  The
// host side sorts the sources by leaf and keeps the tree's interaction lists
// only where the source side holds sources, so that the far field costs in
// proportion to the boxes the curve passes through; the kernels are in
// kernels_layer.cu and the level passes are the volume potential's.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bc_internal.h"

struct bc_layer {
    bc_tree *tree = nullptr;
    int64_t n = 0;
    bc::LayerDev d;
    int64_t counts[6] = {};   // sources, V pairs, W pairs, X entries, near (leaf, source) pairs, leaves with sources
    double *stage_q = nullptr, *stage_m = nullptr, *stage_u = nullptr;   // host-pointer staging
    std::vector<void *> allocs;
};

namespace bc {
namespace {

template <class T>
cudaError_t upload(std::vector<void *> &allocs, T **dst, const T *src, size_t n)
{
    *dst = nullptr;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    allocs.push_back(p);
    *dst = static_cast<T *>(p);
    if (src && n) return cudaMemcpy(p, src, n * sizeof(T), cudaMemcpyHostToDevice);
    return cudaMemset(p, 0, (n ? n : 1) * sizeof(T));
}

void release(std::vector<void *> &allocs)
{
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
}

bc_status fail(cudaError_t e, const char *what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA;
}

bool on_device(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The leaf (caller index) holding (x, y): descend from the root; a point on a
// shared edge goes to the +x / +y side, as for off-grid evaluation.
int64_t leaf_of(const HostTree &h, double x, double y)
{
    int b = 0;
    while (h.box_child0[b] >= 0) {
        const double hb = std::ldexp(h.L, -h.box_level[b]);
        const double mx = h.x0 + (h.box_ix[b] + 0.5) * hb, my = h.y0 + (h.box_iy[b] + 0.5) * hb;
        b = h.box_child0[b] + (x >= mx ? 1 : 0) + (y >= my ? 2 : 0);
    }
    return h.box_leaf[b];
}

}  // namespace
}  // namespace bc

using namespace bc;

bc_status bc_layer_create(bc_tree *tree, const double *xy, int64_t n, bc_layer **out)
{
    if (!tree || !out || n < 0 || (n > 0 && !xy)) {
        set_error("bc_layer_create: bad argument");
        return BC_ERR_ARG;
    }
    *out = nullptr;
    bc_ctx *ctx = tree->ctx;
    if (ctx->device < 0) { set_error("bc_layer_create: host-only context (device -1)"); return BC_ERR_STATE; }
    if (!ctx->tables_ready) { set_error("bc_layer_create: call bc_tables_build first"); return BC_ERR_STATE; }
    if (tree->is_union) { set_error("bc_layer_create: a batch's union tree takes no sources"); return BC_ERR_ARG; }
    if (n > INT32_MAX / 2) { set_error("bc_layer_create: too many sources"); return BC_ERR_ARG; }
    const HostTree &h = tree->h;
    // bin the sources by leaf
    std::vector<int64_t> leaf(static_cast<size_t>(n));
    for (int64_t k = 0; k < n; k++) {
        const double x = xy[2 * k], y = xy[2 * k + 1];
        if (!(x >= h.x0 && x <= h.x0 + h.L && y >= h.y0 && y <= h.y0 + h.L)) {
            set_error("bc_layer_create: source %lld outside the root box", (long long)k);
            return BC_ERR_ARG;
        }
        leaf[k] = leaf_of(h, x, y);
    }
    const int64_t nleaf = h.nleaf;
    std::vector<int32_t> src_ptr(static_cast<size_t>(nleaf) + 1, 0), perm(static_cast<size_t>(n));
    for (int64_t k = 0; k < n; k++) src_ptr[leaf[k] + 1]++;
    for (int64_t l = 0; l < nleaf; l++) src_ptr[l + 1] += src_ptr[l];
    {
        std::vector<int32_t> fill(src_ptr.begin(), src_ptr.end() - 1);
        for (int64_t k = 0; k < n; k++) perm[fill[leaf[k]]++] = int32_t(k);
    }
    std::vector<double2> sxy(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; i++) sxy[i] = make_double2(xy[2 * perm[i]], xy[2 * perm[i] + 1]);
    // sources per box (subtree), boxes sorted by level: children after parents
    const size_t nbox = h.box_level.size();
    std::vector<int64_t> cnt(nbox, 0);
    for (int64_t l = 0; l < nleaf; l++) cnt[h.leaf_box[l]] = src_ptr[l + 1] - src_ptr[l];
    for (size_t b = nbox; b-- > 1;) cnt[h.box_parent[b]] += cnt[b];
    // lists kept where the source side holds sources
    std::vector<int32_t> v_ptr(nbox + 1, 0), v_src, v_code, x_ptr(nbox + 1, 0), x_src, x_box;
    for (size_t b = 0; b < nbox; b++) {
        for (int e = h.v_ptr[b]; e < h.v_ptr[b + 1]; e++)
            if (cnt[h.v_src[e]] > 0) { v_src.push_back(h.v_src[e]); v_code.push_back(h.v_code[e]); }
        v_ptr[b + 1] = int32_t(v_src.size());
        for (int e = h.x_ptr[b]; e < h.x_ptr[b + 1]; e++)
            if (src_ptr[h.x_src[e] + 1] > src_ptr[h.x_src[e]]) { x_src.push_back(h.x_src[e]); x_box.push_back(int32_t(b)); }
        x_ptr[b + 1] = int32_t(x_src.size());
    }
    std::vector<int32_t> w_ptr(size_t(nleaf) + 1, 0), w_src, w_code, n_ptr(size_t(nleaf) + 1, 0), n_src;
    int64_t near_pairs = 0;
    for (int64_t o = 0; o < nleaf; o++) {
        for (int e = h.w_ptr[o]; e < h.w_ptr[o + 1]; e++)
            if (cnt[h.w_src[e]] > 0) { w_src.push_back(h.w_src[e]); w_code.push_back(h.w_code[e]); }
        w_ptr[o + 1] = int32_t(w_src.size());
        for (int e = h.near_ptr[o]; e < h.near_ptr[o + 1]; e++) {
            const int s = h.near_src[e];
            if (src_ptr[s + 1] > src_ptr[s]) {
                n_src.push_back(s);
                near_pairs += src_ptr[s + 1] - src_ptr[s];
            }
        }
        n_ptr[o + 1] = int32_t(n_src.size());
    }
    // output order: target leaves by descending near work (near sources x
    // nodes), the heavy ones first, so that the grid-stride loop of the leaf
    // output spreads them over every block
    std::vector<int64_t> work(static_cast<size_t>(nleaf), 0);
    for (int64_t o = 0; o < nleaf; o++)
        for (int e = n_ptr[o]; e < n_ptr[o + 1]; e++) work[o] += src_ptr[n_src[e] + 1] - src_ptr[n_src[e]];
    std::vector<int32_t> out_order(static_cast<size_t>(nleaf));
    for (int64_t o = 0; o < nleaf; o++) out_order[o] = int32_t(o);
    std::stable_sort(out_order.begin(), out_order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
    bc_layer *L = new bc_layer;
    L->tree = tree;
    L->n = n;
    L->counts[0] = n;
    L->counts[1] = int64_t(v_src.size());
    L->counts[2] = int64_t(w_src.size());
    L->counts[3] = int64_t(x_src.size());
    L->counts[4] = near_pairs;
    for (int64_t l = 0; l < nleaf; l++) L->counts[5] += src_ptr[l + 1] > src_ptr[l] ? 1 : 0;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = layer_log_init();   // the near sums' log table
    LayerDev &d = L->d;
    d.n = n;
    d.nx = int64_t(x_src.size());
    int32_t *p_order, *p_src_ptr, *p_perm, *p_v_ptr, *p_v_src, *p_v_code, *p_x_ptr, *p_x_src, *p_x_box, *p_w_ptr, *p_w_src,
        *p_w_code, *p_n_ptr, *p_n_src;
    double2 *p_sxy;
    if (e == cudaSuccess) e = upload(L->allocs, &p_order, out_order.data(), out_order.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_src_ptr, src_ptr.data(), src_ptr.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_perm, perm.data(), perm.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_sxy, sxy.data(), sxy.size());
    if (e == cudaSuccess) e = upload<double>(L->allocs, &d.cq, nullptr, size_t(n));
    if (e == cudaSuccess) e = upload<double2>(L->allocs, &d.cm, nullptr, size_t(n));
    if (e == cudaSuccess) e = upload(L->allocs, &p_v_ptr, v_ptr.data(), v_ptr.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_v_src, v_src.data(), v_src.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_v_code, v_code.data(), v_code.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_x_ptr, x_ptr.data(), x_ptr.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_x_src, x_src.data(), x_src.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_x_box, x_box.data(), x_box.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_w_ptr, w_ptr.data(), w_ptr.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_w_src, w_src.data(), w_src.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_w_code, w_code.data(), w_code.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_n_ptr, n_ptr.data(), n_ptr.size());
    if (e == cudaSuccess) e = upload(L->allocs, &p_n_src, n_src.data(), n_src.size());
    if (e == cudaSuccess) e = upload<double2>(L->allocs, &d.PX, nullptr, x_src.size() * size_t(ctx->P1));
    // boxes whose subtree holds sources (the climb gives the others zero)
    std::vector<uint8_t> live(nbox);
    for (size_t b = 0; b < nbox; b++) live[b] = cnt[b] > 0 ? 1 : 0;
    uint8_t *p_live = nullptr;
    if (e == cudaSuccess) e = upload(L->allocs, &p_live, live.data(), live.size());
    if (e != cudaSuccess) {
        release(L->allocs);
        delete L;
        return fail(e, "bc_layer_create");
    }
    d.order = p_order; d.src_ptr = p_src_ptr; d.perm = p_perm; d.sxy = p_sxy;
    d.v_ptr = p_v_ptr; d.v_src = p_v_src; d.v_code = p_v_code;
    d.x_ptr = p_x_ptr; d.x_src = p_x_src; d.x_box = p_x_box;
    d.w_ptr = p_w_ptr; d.w_src = p_w_src; d.w_code = p_w_code;
    d.n_ptr = p_n_ptr; d.n_src = p_n_src;
    d.live = p_live;
    *out = L;
    return BC_OK;
}

bc_status bc_layer_info(const bc_layer *layer, int64_t *counts)
{
    if (!layer || !counts) { set_error("bc_layer_info: NULL argument"); return BC_ERR_ARG; }
    std::memcpy(counts, layer->counts, sizeof(layer->counts));
    return BC_OK;
}

bc_status bc_layer_apply(bc_ctx *ctx, bc_layer *layer, const double *q, const double *m, double *u,
                         bc_precision prec, void *stream)
{
    if (!ctx || !layer || !u || (layer->n > 0 && (!q || !m))) {
        set_error("bc_layer_apply: bad argument");
        return BC_ERR_ARG;
    }
    if (layer->tree->ctx != ctx) { set_error("bc_layer_apply: layer belongs to another context"); return BC_ERR_ARG; }
    if (prec != BC_FP64 && prec != BC_SPLIT_BF16) {
        set_error("bc_layer_apply: precision must be BC_FP64 or BC_SPLIT_BF16");
        return BC_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bc_tree *tree = layer->tree;
    const PassArgs a = pass_args(ctx, tree);
    SplitLaunch sl{&ctx->split, nullptr};
    const SplitLaunch *split = nullptr;
    if (prec == BC_SPLIT_BF16) {
        if (!ctx->split_ready) {
            set_error("bc_layer_apply: split precision is provided for p = 16 with nterms <= 32 only");
            return BC_ERR_UNSUPPORTED;
        }
        const bc_status bs = prepare_split_tree(tree);
        if (bs != BC_OK) return bs;
        sl.tree = &tree->sp;
        split = &sl;
    }
    const size_t nu = size_t(tree->h.nleaf) * ctx->NP, n = size_t(layer->n);
    const bool dq = n == 0 || on_device(q), dm = n == 0 || on_device(m), du = on_device(u);
    if (dq && dm && du) {
        e = launch_layer(a, tree->h, tree->d, ctx->dt, layer->d, q, m, u, st, split);
        return e == cudaSuccess ? BC_OK : fail(e, "bc_layer_apply");
    }
    if ((n > 0 && (on_device(q) || on_device(m))) || du) {
        set_error("bc_layer_apply: q, m and u must all be device or all host memory");
        return BC_ERR_ARG;
    }
    // host arrays: staged through device buffers kept with the layer
    if (!layer->stage_u) {
        if ((e = upload<double>(layer->allocs, &layer->stage_q, nullptr, n)) != cudaSuccess ||
            (e = upload<double>(layer->allocs, &layer->stage_m, nullptr, 2 * n)) != cudaSuccess ||
            (e = upload<double>(layer->allocs, &layer->stage_u, nullptr, nu)) != cudaSuccess)
            return fail(e, "bc_layer_apply staging");
    }
    if (n > 0) {
        e = cudaMemcpyAsync(layer->stage_q, q, n * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(layer->stage_m, m, 2 * n * sizeof(double), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess)
        e = launch_layer(a, tree->h, tree->d, ctx->dt, layer->d, layer->stage_q, layer->stage_m, layer->stage_u, st,
                         split);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, layer->stage_u, nu * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? BC_OK : fail(e, "bc_layer_apply");
}

bc_status bc_debug_log_inv(int device, const double *x, int64_t n, double *lg, double *inv, void *stream)
{
    if (n < 0 || (n > 0 && (!x || !lg || !inv))) { set_error("bc_debug_log_inv: bad argument"); return BC_ERR_ARG; }
    if (n > 0 && (!on_device(x) || !on_device(lg) || !on_device(inv))) {
        set_error("bc_debug_log_inv: x, lg and inv must be device pointers");
        return BC_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = layer_log_init();
    if (e == cudaSuccess) e = launch_log_inv_check(x, n, lg, inv, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BC_OK : fail(e, "bc_debug_log_inv");
}

void bc_layer_destroy(bc_layer *layer)
{
    if (!layer) return;
    if (layer->tree->ctx->device >= 0) cudaSetDevice(layer->tree->ctx->device);
    release(layer->allocs);
    delete layer;
}
