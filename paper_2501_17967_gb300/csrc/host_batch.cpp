// Disjoint union of several quadtrees for batched applies.  Each tree keeps
// its own leaves, boxes and lists; the union renumbers them so that one
// launch of each pass covers every tree: leaves are concatenated tree by
// tree, boxes are sorted by (level, tree, position in the tree's own Morton
// order), which keeps the four children of a box contiguous and in q order.
#include <algorithm>
#include <numeric>

#include "bc_internal.h"

namespace bc {

bc_status merge_host_trees(const std::vector<const HostTree *> &trees, HostTree &out,
                           std::vector<int64_t> &leaf_offset)
{
    if (trees.empty()) { set_error("batch: no trees"); return BC_ERR_ARG; }
    const HostTree &t0 = *trees[0];
    out = HostTree();
    out.x0 = t0.x0; out.y0 = t0.y0; out.L = t0.L; out.p = t0.p;
    const size_t n = trees.size();
    leaf_offset.assign(n + 1, 0);
    std::vector<int64_t> box_offset(n + 1, 0);
    int nlevels = 0;
    for (size_t k = 0; k < n; k++) {
        const HostTree &t = *trees[k];
        if (t.L != t0.L || t.p != t0.p) {
            set_error("batch: every tree needs the same order p and root side L");
            return BC_ERR_ARG;
        }
        leaf_offset[k + 1] = leaf_offset[k] + t.nleaf;
        box_offset[k + 1] = box_offset[k] + int64_t(t.box_level.size());
        nlevels = std::max(nlevels, t.nlevels);
    }
    const int64_t nleaf = leaf_offset[n], nbox = box_offset[n];
    if (nleaf >= (int64_t(1) << 31) || nbox >= (int64_t(1) << 31)) { set_error("batch: too large"); return BC_ERR_ARG; }
    out.nleaf = nleaf;
    out.nlevels = nlevels;
    // new box order: (level, tree, original index)
    std::vector<int64_t> order(nbox);
    std::vector<int32_t> tree_of(nbox), lvl(nbox);
    for (size_t k = 0; k < n; k++)
        for (int64_t b = 0; b < int64_t(trees[k]->box_level.size()); b++) {
            int64_t g = box_offset[k] + b;
            order[g] = g;
            tree_of[g] = int32_t(k);
            lvl[g] = trees[k]->box_level[b];
        }
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return lvl[a] != lvl[b] ? lvl[a] < lvl[b] : a < b;   // a < b keeps (tree, original) order
    });
    std::vector<int32_t> newidx(nbox);
    for (int64_t i = 0; i < nbox; i++) newidx[order[i]] = int32_t(i);
    auto remap_box = [&](size_t k, int32_t b) -> int32_t { return b < 0 ? -1 : newidx[box_offset[k] + b]; };
    auto remap_leaf = [&](size_t k, int32_t l) -> int32_t { return l < 0 ? -1 : int32_t(leaf_offset[k] + l); };

    out.box_level.resize(nbox); out.box_ix.resize(nbox); out.box_iy.resize(nbox);
    out.box_parent.resize(nbox); out.box_child0.resize(nbox); out.box_leaf.resize(nbox);
    out.level_start.assign(nlevels + 1, 0);
    out.v_ptr.assign(nbox + 1, 0);
    out.x_ptr.assign(nbox + 1, 0);
    for (int64_t i = 0; i < nbox; i++) {
        const int64_t g = order[i];
        const size_t k = size_t(tree_of[g]);
        const HostTree &t = *trees[k];
        const int32_t b = int32_t(g - box_offset[k]);
        out.box_level[i] = t.box_level[b];
        out.box_ix[i] = t.box_ix[b];
        out.box_iy[i] = t.box_iy[b];
        out.box_parent[i] = remap_box(k, t.box_parent[b]);
        out.box_child0[i] = remap_box(k, t.box_child0[b]);
        out.box_leaf[i] = remap_leaf(k, t.box_leaf[b]);
        out.level_start[t.box_level[b] + 1] = i + 1;
        for (int32_t e = t.v_ptr[b]; e < t.v_ptr[b + 1]; e++) {
            out.v_src.push_back(remap_box(k, t.v_src[e]));
            out.v_code.push_back(t.v_code[e]);
        }
        for (int32_t e = t.x_ptr[b]; e < t.x_ptr[b + 1]; e++) {
            out.x_src.push_back(remap_leaf(k, t.x_src[e]));
            out.x_code.push_back(t.x_code[e]);
        }
        out.v_ptr[i + 1] = int32_t(out.v_src.size());
        out.x_ptr[i + 1] = int32_t(out.x_src.size());
    }
    for (int l = 1; l <= nlevels; l++) out.level_start[l] = std::max(out.level_start[l], out.level_start[l - 1]);
    out.near_ptr.assign(nleaf + 1, 0);
    out.w_ptr.assign(nleaf + 1, 0);
    bool any_class = false;   // truncated trees keep their leaf classes (discarded leaves: zero output)
    for (size_t k = 0; k < n; k++) any_class = any_class || !trees[k]->leaf_class.empty();
    for (size_t k = 0; k < n; k++) {
        const HostTree &t = *trees[k];
        for (int64_t l = 0; l < t.nleaf; l++) {
            const int64_t gl = leaf_offset[k] + l;
            if (any_class) out.leaf_class.push_back(t.leaf_class.empty() ? int8_t(2) : t.leaf_class[l]);
            out.leaf_level.push_back(t.leaf_level[l]);
            out.leaf_ix.push_back(t.leaf_ix[l]);
            out.leaf_iy.push_back(t.leaf_iy[l]);
            out.leaf_box.push_back(remap_box(k, t.leaf_box[l]));
            out.leaf_order.push_back(remap_leaf(k, t.leaf_order[l]));
            for (int32_t e = t.near_ptr[l]; e < t.near_ptr[l + 1]; e++) {
                out.near_src.push_back(remap_leaf(k, t.near_src[e]));
                out.near_tab.push_back(t.near_tab[e]);
            }
            for (int32_t e = t.w_ptr[l]; e < t.w_ptr[l + 1]; e++) {
                out.w_src.push_back(remap_box(k, t.w_src[e]));
                out.w_code.push_back(t.w_code[e]);
            }
            out.near_ptr[gl + 1] = int32_t(out.near_src.size());
            out.w_ptr[gl + 1] = int32_t(out.w_src.size());
        }
        out.n_nonleaf += t.n_nonleaf;
        out.n_down += t.n_down;
    }
    return BC_OK;
}

}  // namespace bc
