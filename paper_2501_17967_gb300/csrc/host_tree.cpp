// Host-side quadtree: validation of explicit leaves, the 2:1 balance check
// (paper Sec. 3.2.1: every box at most one level apart from its neighbours,
// edge and corner neighbours alike), the adaptive refinement of Alg. 2
// (function-resolution criterion), Morton ordering, and the interaction
// lists of the adaptive box code:
//   near (U) list : leaves touching the target leaf, and the leaf itself;
//   V list        : children of the parent's neighbours that do not touch the box;
//   W list        : children of a leaf's neighbours that do not touch the leaf;
//   X list        : the dual of W (leaf neighbours of the parent that do not
//                   touch the box).
// Every (target node, source leaf) pair is covered exactly once by near(t),
// the subtrees of W(t), X(a) and the subtrees of V(a) over the ancestors a of
// t (tests/test_tree_lists.py checks this by brute force).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <unordered_set>

#include "bc_internal.h"

namespace bc {

namespace {

constexpr int kMaxLevel = 24;

inline uint64_t key_of(int lv, int64_t ix, int64_t iy)
{
    return (uint64_t(lv) << 52) | (uint64_t(ix) << 26) | uint64_t(iy);
}

inline uint64_t morton(uint32_t x, uint32_t y)
{
    uint64_t k = 0;
    for (int b = 0; b < 26; b++) {
        k |= uint64_t((x >> b) & 1u) << (2 * b);
        k |= uint64_t((y >> b) & 1u) << (2 * b + 1);
    }
    return k;
}

// Closed boxes intersect but their interiors do not: the boxes share an edge
// or a corner.
bool touching(int la, int64_t ia, int64_t ja, int lb, int64_t ib, int64_t jb)
{
    int lf = std::max(la, lb);
    int64_t a0 = ia << (lf - la), a1 = (ia + 1) << (lf - la);
    int64_t c0 = ja << (lf - la), c1 = (ja + 1) << (lf - la);
    int64_t b0 = ib << (lf - lb), b1 = (ib + 1) << (lf - lb);
    int64_t d0 = jb << (lf - lb), d1 = (jb + 1) << (lf - lb);
    bool xo = a0 <= b1 && b0 <= a1, yo = c0 <= d1 && d0 <= c1;
    bool xi = a0 < b1 && b0 < a1, yi = c0 < d1 && d0 < c1;
    return xo && yo && !(xi && yi);
}

}  // namespace

// ---------------------------------------------------------------------------
// Relative-position codes.
// ---------------------------------------------------------------------------
int near_code_same(int gx, int gy) { return (gy / 2 + 1) * 3 + (gx / 2 + 1); }
int near_code_coarse(int g2x, int g2y) { return 9 + ((g2y + 3) / 2) * 4 + (g2x + 3) / 2; }
int near_code_fine(int gx, int gy) { return 25 + ((gy + 3) / 2) * 4 + (gx + 3) / 2; }
int v_code(int dx, int dy) { return (dy + 3) * 7 + (dx + 3); }
int wx_code(int d2x, int d2y) { return ((d2y + 5) / 2) * 6 + (d2x + 5) / 2; }

NearGeom near_table_geometry(int k)
{
    NearGeom g{false, 0, 0, 1, -1};
    if (k >= 0 && k < 9) {
        int gx = (k % 3 - 1) * 2, gy = (k / 3 - 1) * 2;
        g = {true, double(gx), double(gy), 1.0, near_code_same(-gx, -gy)};
    } else if (k >= 9 && k < 25) {
        int i = (k - 9) % 4, j = (k - 9) / 4;
        int g2x = 2 * i - 3, g2y = 2 * j - 3;     // 2g
        bool inner = std::abs(g2x) <= 1 && std::abs(g2y) <= 1;
        if (!inner)   // reversed pair: source one level finer, g' = -2g
            g = {true, 0.5 * g2x, 0.5 * g2y, 0.5, near_code_fine(-g2x, -g2y)};
    } else if (k >= 25 && k < 41) {
        int i = (k - 25) % 4, j = (k - 25) / 4;
        int gx = 2 * i - 3, gy = 2 * j - 3;
        bool inner = std::abs(gx) <= 1 && std::abs(gy) <= 1;
        if (!inner)   // reversed pair: source one level coarser, 2g' = -g
            g = {true, double(gx), double(gy), 2.0, near_code_coarse(-gx, -gy)};
    }
    return g;
}

// ---------------------------------------------------------------------------
// Tree construction from explicit leaves.
// ---------------------------------------------------------------------------
bc_status build_host_tree(HostTree &t, double x0, double y0, double L, int p, int64_t nleaf,
                          const int32_t *level, const int32_t *ix, const int32_t *iy)
{
    if (nleaf <= 0 || !level || !ix || !iy) { set_error("tree: need nleaf > 0 and leaf arrays"); return BC_ERR_ARG; }
    if (!(L > 0.0) || !std::isfinite(L) || !std::isfinite(x0) || !std::isfinite(y0)) {
        set_error("tree: root box must be finite with L > 0");
        return BC_ERR_ARG;
    }
    if (nleaf > (int64_t(1) << 30)) { set_error("tree: too many leaves"); return BC_ERR_ARG; }
    t = HostTree();
    t.x0 = x0; t.y0 = y0; t.L = L; t.p = p; t.nleaf = nleaf;
    t.leaf_level.assign(level, level + nleaf);
    t.leaf_ix.assign(ix, ix + nleaf);
    t.leaf_iy.assign(iy, iy + nleaf);

    std::unordered_map<uint64_t, int64_t> leaf_of;   // key -> caller leaf
    leaf_of.reserve(size_t(nleaf) * 2);
    const uint64_t full = uint64_t(1) << (2 * kMaxLevel);
    uint64_t area = 0;
    int maxlv = 0;
    for (int64_t k = 0; k < nleaf; k++) {
        int lv = level[k];
        if (lv < 0 || lv > kMaxLevel) { set_error("tree: leaf %lld has level %d outside [0,%d]", (long long)k, lv, kMaxLevel); return BC_ERR_TREE; }
        int64_t n = int64_t(1) << lv;
        if (ix[k] < 0 || iy[k] < 0 || ix[k] >= n || iy[k] >= n) { set_error("tree: leaf %lld index outside its level", (long long)k); return BC_ERR_TREE; }
        if (!leaf_of.emplace(key_of(lv, ix[k], iy[k]), k).second) { set_error("tree: leaf %lld duplicated", (long long)k); return BC_ERR_TREE; }
        area += uint64_t(1) << (2 * (kMaxLevel - lv));
        if (area > full) { set_error("tree: leaves overlap (area exceeds the root)"); return BC_ERR_TREE; }
        maxlv = std::max(maxlv, lv);
    }
    // no leaf inside another leaf
    for (int64_t k = 0; k < nleaf; k++)
        for (int l = level[k] - 1; l >= 0; l--) {
            int s = level[k] - l;
            if (leaf_of.count(key_of(l, ix[k] >> s, iy[k] >> s))) { set_error("tree: leaf %lld lies inside another leaf", (long long)k); return BC_ERR_TREE; }
        }
    if (area != full) { set_error("tree: leaves do not cover the root box"); return BC_ERR_TREE; }

    // all boxes = leaves and their ancestors
    struct B { int lv; int32_t ix, iy; uint64_t m; int64_t leaf; };
    std::unordered_map<uint64_t, int64_t> seen;
    std::vector<B> boxes;
    boxes.reserve(size_t(nleaf) * 2);
    for (int64_t k = 0; k < nleaf; k++) {
        for (int l = level[k]; l >= 0; l--) {
            int s = level[k] - l;
            int32_t a = ix[k] >> s, b = iy[k] >> s;
            uint64_t key = key_of(l, a, b);
            if (seen.count(key)) break;
            seen.emplace(key, 0);
            boxes.push_back({l, a, b, morton(a, b), l == level[k] ? k : -1});
        }
    }
    std::sort(boxes.begin(), boxes.end(), [](const B &a, const B &b) {
        return a.lv != b.lv ? a.lv < b.lv : a.m < b.m;
    });
    int64_t nbox = int64_t(boxes.size());
    t.nlevels = maxlv + 1;
    t.box_level.resize(nbox); t.box_ix.resize(nbox); t.box_iy.resize(nbox);
    t.box_parent.assign(nbox, -1); t.box_child0.assign(nbox, -1); t.box_leaf.resize(nbox);
    t.level_start.assign(t.nlevels + 1, 0);
    std::unordered_map<uint64_t, int32_t> box_of;
    box_of.reserve(size_t(nbox) * 2);
    for (int64_t b = 0; b < nbox; b++) {
        t.box_level[b] = boxes[b].lv; t.box_ix[b] = boxes[b].ix; t.box_iy[b] = boxes[b].iy;
        t.box_leaf[b] = int32_t(boxes[b].leaf);
        box_of[key_of(boxes[b].lv, boxes[b].ix, boxes[b].iy)] = int32_t(b);
        t.level_start[boxes[b].lv + 1] = b + 1;
    }
    for (int l = 1; l <= t.nlevels; l++) t.level_start[l] = std::max(t.level_start[l], t.level_start[l - 1]);
    t.leaf_box.assign(nleaf, -1);
    for (int64_t b = 0; b < nbox; b++) {
        if (t.box_leaf[b] >= 0) t.leaf_box[t.box_leaf[b]] = int32_t(b);
        if (boxes[b].lv > 0) {
            int32_t par = box_of.at(key_of(boxes[b].lv - 1, boxes[b].ix >> 1, boxes[b].iy >> 1));
            t.box_parent[b] = par;
            int q = (boxes[b].ix & 1) + 2 * (boxes[b].iy & 1);
            if (q == 0) t.box_child0[par] = int32_t(b);
        }
    }
    // children are contiguous: check
    for (int64_t b = 0; b < nbox; b++) {
        if (t.box_leaf[b] >= 0) continue;
        int32_t c0 = t.box_child0[b];
        if (c0 < 0 || c0 + 3 >= nbox) { set_error("tree: internal child layout"); return BC_ERR_TREE; }
        for (int q = 0; q < 4; q++)
            if (t.box_parent[c0 + q] != b || (t.box_ix[c0 + q] & 1) + 2 * (t.box_iy[c0 + q] & 1) != q) {
                set_error("tree: internal child layout");
                return BC_ERR_TREE;
            }
    }
    // leaf processing order: Morton order of the lower-left corners
    {
        std::vector<std::pair<uint64_t, int32_t>> ord(nleaf);
        for (int64_t k = 0; k < nleaf; k++) {
            int s = maxlv - level[k];
            ord[k] = {morton(uint32_t(ix[k]) << s, uint32_t(iy[k]) << s), int32_t(k)};
        }
        std::sort(ord.begin(), ord.end());
        t.leaf_order.resize(nleaf);
        for (int64_t k = 0; k < nleaf; k++) t.leaf_order[k] = ord[k].second;
    }

    auto find_box = [&](int lv, int64_t a, int64_t b) -> int32_t {
        if (lv < 0 || a < 0 || b < 0 || a >= (int64_t(1) << lv) || b >= (int64_t(1) << lv)) return -2;
        auto it = box_of.find(key_of(lv, a, b));
        return it == box_of.end() ? -1 : it->second;
    };

    // ---- near lists (and the 2:1 balance check) --------------------------
    t.near_ptr.assign(nleaf + 1, 0);
    t.w_ptr.assign(nleaf + 1, 0);
    for (int64_t k = 0; k < nleaf; k++) {
        int lv = level[k];
        int64_t a0 = ix[k], b0 = iy[k];
        int32_t coarse_seen[3];
        int ncoarse = 0;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int64_t a = a0 + dx, b = b0 + dy;
                int32_t nb = find_box(lv, a, b);
                if (nb == -2) continue;  // outside the root
                if (nb >= 0) {
                    if (t.box_leaf[nb] >= 0) {
                        t.near_src.push_back(t.box_leaf[nb]);
                        t.near_tab.push_back(near_code_same(int(2 * (a0 - a)), int(2 * (b0 - b))));
                    } else {
                        int32_t c0 = t.box_child0[nb];
                        for (int q = 0; q < 4; q++) {
                            int32_t c = c0 + q;
                            if (!touching(lv, a0, b0, lv + 1, t.box_ix[c], t.box_iy[c])) continue;
                            if (t.box_leaf[c] < 0) {
                                set_error("tree: not 2:1 balanced near leaf %lld (level %d)", (long long)k, lv);
                                return BC_ERR_TREE;
                            }
                            int gx = int(4 * a0 - 2 * t.box_ix[c] + 1), gy = int(4 * b0 - 2 * t.box_iy[c] + 1);
                            t.near_src.push_back(t.box_leaf[c]);
                            t.near_tab.push_back(near_code_fine(gx, gy));
                        }
                        // non-touching children of a touching neighbour: W list
                        if (dx != 0 || dy != 0)
                            for (int q = 0; q < 4; q++) {
                                int32_t c = c0 + q;
                                if (touching(lv, a0, b0, lv + 1, t.box_ix[c], t.box_iy[c])) continue;
                                t.w_src.push_back(c);
                                t.w_code.push_back(wx_code(int(2 * t.box_ix[c] - 4 * a0 - 1), int(2 * t.box_iy[c] - 4 * b0 - 1)));
                            }
                    }
                } else {
                    int32_t cb = find_box(lv - 1, a >> 1, b >> 1);
                    if (cb < 0 || t.box_leaf[cb] < 0) {
                        set_error("tree: not 2:1 balanced near leaf %lld (level %d)", (long long)k, lv);
                        return BC_ERR_TREE;
                    }
                    bool dup = false;
                    for (int s = 0; s < ncoarse; s++) dup |= coarse_seen[s] == cb;
                    if (dup) continue;
                    coarse_seen[ncoarse++] = cb;
                    int g2x = int(2 * a0 - 4 * t.box_ix[cb] - 1), g2y = int(2 * b0 - 4 * t.box_iy[cb] - 1);
                    t.near_src.push_back(t.box_leaf[cb]);
                    t.near_tab.push_back(near_code_coarse(g2x, g2y));
                }
            }
        t.near_ptr[k + 1] = int32_t(t.near_src.size());
        t.w_ptr[k + 1] = int32_t(t.w_src.size());
    }

    // ---- V and X lists ----------------------------------------------------
    t.v_ptr.assign(nbox + 1, 0);
    t.x_ptr.assign(nbox + 1, 0);
    for (int64_t b = 0; b < nbox; b++) {
        int lv = t.box_level[b];
        if (lv >= 2) {
            int64_t bx = t.box_ix[b], by = t.box_iy[b], px = bx >> 1, py = by >> 1;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    if (dx == 0 && dy == 0) continue;
                    int32_t Q = find_box(lv - 1, px + dx, py + dy);
                    if (Q == -2) continue;
                    if (Q < 0) { set_error("tree: not 2:1 balanced around box %lld", (long long)b); return BC_ERR_TREE; }
                    if (t.box_leaf[Q] < 0) {
                        int32_t c0 = t.box_child0[Q];
                        for (int q = 0; q < 4; q++) {
                            int32_t c = c0 + q;
                            if (touching(lv, bx, by, lv, t.box_ix[c], t.box_iy[c])) continue;
                            t.v_src.push_back(c);
                            t.v_code.push_back(v_code(int(t.box_ix[c] - bx), int(t.box_iy[c] - by)));
                        }
                    } else if (!touching(lv, bx, by, lv - 1, t.box_ix[Q], t.box_iy[Q])) {
                        t.x_src.push_back(t.box_leaf[Q]);
                        t.x_code.push_back(wx_code(int(2 * bx - 4 * t.box_ix[Q] - 1), int(2 * by - 4 * t.box_iy[Q] - 1)));
                    } else if (t.box_leaf[b] < 0) {
                        set_error("tree: not 2:1 balanced around box %lld", (long long)b);
                        return BC_ERR_TREE;
                    }
                }
            t.n_down++;
            if (t.box_leaf[b] < 0) t.n_nonleaf++;
        }
        t.v_ptr[b + 1] = int32_t(t.v_src.size());
        t.x_ptr[b + 1] = int32_t(t.x_src.size());
    }
    return BC_OK;
}

// ---------------------------------------------------------------------------
// Alg. 2 (function-resolution criterion) + 2:1 balance.
// ---------------------------------------------------------------------------
// Drops from the lists what a zero density or a discarded target makes void:
// near entries whose target or source is inactive, W entries of inactive
// targets, X entries of inactive sources (leaf-indexed active flags).
void drop_inactive(HostTree &t, const std::vector<uint8_t> &active)
{
    auto filter = [](std::vector<int32_t> &ptr, std::vector<int32_t> &src, std::vector<int32_t> &code,
                     auto keep) {
        std::vector<int32_t> nsrc, ncode;
        nsrc.reserve(src.size());
        ncode.reserve(code.size());
        int32_t w = 0;
        for (size_t r = 0; r + 1 < ptr.size(); r++) {
            const int32_t a = ptr[r], b = ptr[r + 1];
            ptr[r] = w;
            for (int32_t k = a; k < b; k++)
                if (keep(int64_t(r), src[k])) {
                    nsrc.push_back(src[k]);
                    ncode.push_back(code[k]);
                    w++;
                }
        }
        ptr.back() = w;
        src.swap(nsrc);
        code.swap(ncode);
    };
    filter(t.near_ptr, t.near_src, t.near_tab, [&](int64_t o, int32_t s) { return active[o] && active[s]; });
    filter(t.w_ptr, t.w_src, t.w_code, [&](int64_t o, int32_t) { return bool(active[o]); });
    filter(t.x_ptr, t.x_src, t.x_code, [&](int64_t, int32_t s) { return bool(active[s]); });
}

// ---------------------------------------------------------------------------
// Polygon geometry for the truncated tree (Alg. 2, separation criterion).
// A curve is a closed polygon: vertices v_0 .. v_{n-1}, edge v_{n-1} -> v_0.
// ---------------------------------------------------------------------------
namespace {

// even-odd crossing rule
bool point_in_polygon(const Polygon &P, double x, double y)
{
    bool in = false;
    for (int64_t i = 0, j = P.n - 1; i < P.n; j = i++) {
        const double xi = P.xy[2 * i], yi = P.xy[2 * i + 1], xj = P.xy[2 * j], yj = P.xy[2 * j + 1];
        if ((yi > y) != (yj > y) && x < (xj - xi) * (y - yi) / (yj - yi) + xi) in = !in;
    }
    return in;
}

// does the segment (ax,ay)-(bx,by) meet the closed box [x0,x1] x [y0,y1]?
// (Liang-Barsky clipping of the segment's parameter interval)
bool segment_meets_box(double ax, double ay, double bx, double by, double x0, double x1, double y0, double y1)
{
    double t0 = 0.0, t1 = 1.0;
    const double dx = bx - ax, dy = by - ay;
    const double pq[4][2] = {{-dx, ax - x0}, {dx, x1 - ax}, {-dy, ay - y0}, {dy, y1 - ay}};
    for (const auto &e : pq) {
        if (e[0] == 0.0) {
            if (e[1] < 0.0) return false;
        } else {
            const double t = e[1] / e[0];
            if (e[0] < 0.0) t0 = std::max(t0, t);
            else t1 = std::min(t1, t);
            if (t0 > t1) return false;
        }
    }
    return true;
}

}  // namespace

// Where a box lies relative to a polygon: the curve meets the box (cut), or
// the box lies wholly inside or wholly outside the region it bounds.
BoxSide box_side(const Polygon &P, double x0, double x1, double y0, double y1)
{
    for (int64_t i = 0, j = P.n - 1; i < P.n; j = i++)
        if (segment_meets_box(P.xy[2 * j], P.xy[2 * j + 1], P.xy[2 * i], P.xy[2 * i + 1], x0, x1, y0, y1))
            return BoxSide::Cut;
    // the curve misses the box: the box is on one side (its centre tells)
    return point_in_polygon(P, 0.5 * (x0 + x1), 0.5 * (y0 + y1)) ? BoxSide::Inside : BoxSide::Outside;
}

bool polygon_contains(const Polygon &P, double x, double y) { return point_in_polygon(P, x, y); }

// Distance from (x, y) to the nearest vertex of P, and that vertex.
static int64_t nearest_vertex(const Polygon &P, double x, double y)
{
    int64_t best = 0;
    double bd = 1e300;
    for (int64_t i = 0; i < P.n; i++) {
        const double d = (P.xy[2 * i] - x) * (P.xy[2 * i] - x) + (P.xy[2 * i + 1] - y) * (P.xy[2 * i + 1] - y);
        if (d < bd) { bd = d; best = i; }
    }
    return best;
}

// Alg. 2's separation criterion for box B (half side r, centre c): B must be
// split if it meets the bulk region and the outside of the domain, or if it
// meets the strip and its diagonal exceeds half the local strip width s, s
// the distance between the vertices of Gamma and of Gamma_b nearest to c.
bool truncation_split(const Truncation &tr, double cx, double cy, double r)
{
    const double x0 = cx - r, x1 = cx + r, y0 = cy - r, y1 = cy + r;
    const BoxSide so = box_side(tr.gamma, x0, x1, y0, y1), sb = box_side(tr.gamma_b, x0, x1, y0, y1);
    if (sb != BoxSide::Outside && so != BoxSide::Inside) return true;   // meets Omega_B and R^2 \ Omega
    if (so != BoxSide::Outside && sb != BoxSide::Inside) {              // meets the strip Omega \ Omega_B
        const int64_t a = nearest_vertex(tr.gamma, cx, cy), b = nearest_vertex(tr.gamma_b, cx, cy);
        const double s = std::hypot(tr.gamma.xy[2 * a] - tr.gamma_b.xy[2 * b],
                                    tr.gamma.xy[2 * a + 1] - tr.gamma_b.xy[2 * b + 1]);
        if (2.0 * std::sqrt(2.0) * r > 0.5 * s) return true;
    }
    return false;
}

bc_status refine_leaves(int p, double x0, double y0, double L, bc_density_fn fn, void *user,
                        double eps, int max_level, std::vector<int32_t> &lv_out,
                        std::vector<int32_t> &ix_out, std::vector<int32_t> &iy_out, const Truncation *tr)
{
    if (!fn || !(eps > 0.0) || max_level < 0 || max_level > kMaxLevel || !(L > 0.0)) {
        set_error("refine: need a callback, eps > 0, 0 <= max_level <= %d, L > 0", kMaxLevel);
        return BC_ERR_ARG;
    }
    const double pi = 3.14159265358979323846;
    std::vector<double> xn(p), Tm(p * p);   // Tm[m*p + a] = T_a(x_m)
    for (int m = 0; m < p; m++) {
        xn[m] = -std::cos((2.0 * m + 1.0) * pi / (2.0 * p));
        double t0 = 1.0, t1 = xn[m];
        Tm[m * p + 0] = 1.0;
        if (p > 1) Tm[m * p + 1] = t1;
        for (int a = 2; a < p; a++) {
            double t2 = 2.0 * xn[m] * t1 - t0;
            Tm[m * p + a] = t2;
            t0 = t1; t1 = t2;
        }
    }
    struct Bx { int lv; int32_t ix, iy; };
    std::vector<Bx> cur{{0, 0, 0}};
    std::unordered_set<uint64_t> leaves;
    double vscale = 0.0;
    const int NP = p * p;
    std::vector<double> xy, fv, tmp(NP);
    while (!cur.empty()) {
        size_t nb = cur.size();
        xy.resize(nb * NP * 2);
        fv.assign(nb * NP, 0.0);
        for (size_t k = 0; k < nb; k++) {
            double r = 0.5 * L / double(int64_t(1) << cur[k].lv);
            double cx = x0 + (2.0 * cur[k].ix + 1.0) * r, cy = y0 + (2.0 * cur[k].iy + 1.0) * r;
            for (int jy = 0; jy < p; jy++)
                for (int jx = 0; jx < p; jx++) {
                    xy[(k * NP + jy * p + jx) * 2] = cx + r * xn[jx];
                    xy[(k * NP + jy * p + jx) * 2 + 1] = cy + r * xn[jy];
                }
        }
        // with a truncation, f is evaluated at the nodes inside the domain
        // only and extended by zero outside it (Alg. 2; on cut boxes its
        // coefficients are kept, Sec. 3.2.1, remark on cut boxes)
        std::vector<BoxSide> side(nb, BoxSide::Inside);
        if (!tr) {
            fn(xy.data(), int64_t(nb * NP), fv.data(), user);
        } else {
            std::vector<double> xin;
            std::vector<int64_t> where;
            for (size_t k = 0; k < nb; k++) {
                const double r = 0.5 * L / double(int64_t(1) << cur[k].lv);
                const double cx = x0 + (2.0 * cur[k].ix + 1.0) * r, cy = y0 + (2.0 * cur[k].iy + 1.0) * r;
                side[k] = box_side(tr->gamma, cx - r, cx + r, cy - r, cy + r);
                if (side[k] == BoxSide::Outside) continue;
                for (int j = 0; j < NP; j++) {
                    const double px = xy[(k * NP + j) * 2], py = xy[(k * NP + j) * 2 + 1];
                    if (side[k] == BoxSide::Inside || point_in_polygon(tr->gamma, px, py)) {
                        xin.push_back(px);
                        xin.push_back(py);
                        where.push_back(int64_t(k * NP + j));
                    }
                }
            }
            std::vector<double> fin(where.size());
            if (!where.empty()) fn(xin.data(), int64_t(where.size()), fin.data(), user);
            for (size_t i = 0; i < where.size(); i++) fv[where[i]] = fin[i];
        }
        for (double v : fv)
            if (!std::isfinite(v)) { set_error("refine: density callback returned a non-finite value"); return BC_ERR_ARG; }
        if (cur.size() == 1 && cur[0].lv == 0) {
            // the scale of f is fixed once, from the root's nodes
            for (double v : fv) vscale = std::max(vscale, std::fabs(v));
            if (!(vscale > 0.0)) vscale = 1.0;
        }
        std::vector<Bx> next;
        for (size_t k = 0; k < nb; k++) {
            const double *f = &fv[k * NP];
            // c_ab = (2-[a=0])(2-[b=0])/p^2 sum_{m,n} f[n][m] T_a(x_m) T_b(x_n)
            for (int n = 0; n < p; n++)
                for (int a = 0; a < p; a++) {
                    double s = 0.0;
                    for (int m = 0; m < p; m++) s += f[n * p + m] * Tm[m * p + a];
                    tmp[n * p + a] = s * (a == 0 ? 1.0 : 2.0) / p;
                }
            double tail = 0.0;
            for (int b = 0; b < p; b++)
                for (int a = 0; a < p; a++) {
                    if (a < p - 2 && b < p - 2) continue;
                    double s = 0.0;
                    for (int n = 0; n < p; n++) s += tmp[n * p + a] * Tm[n * p + b];
                    tail = std::max(tail, std::fabs(s * (b == 0 ? 1.0 : 2.0) / p));
                }
            bool split = tail > eps * vscale && side[k] == BoxSide::Inside;   // function resolution
            if (tr && !split) {
                const double r = 0.5 * L / double(int64_t(1) << cur[k].lv);
                split = truncation_split(*tr, x0 + (2.0 * cur[k].ix + 1.0) * r, y0 + (2.0 * cur[k].iy + 1.0) * r, r);
            }
            if (split && cur[k].lv < max_level) {
                for (int q = 0; q < 4; q++)
                    next.push_back({cur[k].lv + 1, 2 * cur[k].ix + (q & 1), 2 * cur[k].iy + (q >> 1)});
            } else {
                leaves.insert(key_of(cur[k].lv, cur[k].ix, cur[k].iy));
            }
        }
        cur.swap(next);
    }
    // 2:1 balance: split any leaf that touches a leaf two or more levels finer
    auto covering = [&](int lv, int64_t a, int64_t b, int &clv) -> bool {
        for (int l = lv; l >= 0; l--) {
            int s = lv - l;
            if (leaves.count(key_of(l, a >> s, b >> s))) { clv = l; return true; }
        }
        return false;
    };
    bool changed = true;
    while (changed) {
        changed = false;
        std::vector<uint64_t> snapshot(leaves.begin(), leaves.end());
        std::sort(snapshot.begin(), snapshot.end(), [](uint64_t a, uint64_t b) { return (a >> 52) > (b >> 52); });
        for (uint64_t key : snapshot) {
            if (!leaves.count(key)) continue;
            int lv = int(key >> 52);
            int64_t a0 = int64_t((key >> 26) & ((1u << 26) - 1)), b0 = int64_t(key & ((1u << 26) - 1));
            int64_t n = int64_t(1) << lv;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    if (dx == 0 && dy == 0) continue;
                    int64_t a = a0 + dx, b = b0 + dy;
                    if (a < 0 || b < 0 || a >= n || b >= n) continue;
                    int clv;
                    if (covering(lv, a, b, clv) && clv < lv - 1) {
                        int s = lv - clv;
                        int64_t ca = a >> s, cb = b >> s;
                        leaves.erase(key_of(clv, ca, cb));
                        for (int q = 0; q < 4; q++) leaves.insert(key_of(clv + 1, 2 * ca + (q & 1), 2 * cb + (q >> 1)));
                        changed = true;
                    }
                }
        }
    }
    std::vector<uint64_t> all(leaves.begin(), leaves.end());
    std::sort(all.begin(), all.end());
    lv_out.resize(all.size()); ix_out.resize(all.size()); iy_out.resize(all.size());
    for (size_t k = 0; k < all.size(); k++) {
        lv_out[k] = int32_t(all[k] >> 52);
        ix_out[k] = int32_t((all[k] >> 26) & ((1u << 26) - 1));
        iy_out[k] = int32_t(all[k] & ((1u << 26) - 1));
    }
    return BC_OK;
}

}  // namespace bc
