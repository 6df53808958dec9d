// C ABI of the box code (declared in include/boxcode.h): contexts, tables,
// trees, applies.  Device memory is plain cudaMalloc; every entry point
// returns a bc_status and records a message for bc_last_error().
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "bc_internal.h"

namespace bc {

namespace {
thread_local char g_err[512] = "";

template <class T>
cudaError_t dev_upload(std::vector<void *> &allocs, T **dst, const T *src, size_t n)
{
    *dst = nullptr;
    const size_t nalloc = n ? n : 1;   // a valid pointer even for an empty list
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, nalloc * sizeof(T));
    if (e != cudaSuccess) return e;
    allocs.push_back(p);
    *dst = static_cast<T *>(p);
    if (src && n) return cudaMemcpy(p, src, n * sizeof(T), cudaMemcpyHostToDevice);
    return cudaMemset(p, 0, nalloc * sizeof(T));
}

void free_all(std::vector<void *> &allocs)
{
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
}

bc_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The device address of page-locked (pinned, mapped) host memory, else nullptr.
const void *pinned_device_ptr(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Operator layouts (see OpSet): element (l,k) of a complex operator at [k][l].
using cplx = std::complex<double>;
inline cplx at2(const std::vector<double> &v, size_t i) { return cplx(v[2 * i], v[2 * i + 1]); }

struct OpBuild {
    std::vector<double2> leafA, up, par, v, x, e, w;
    std::vector<double> t;
};

void build_opsets(const HostTables &ht, OpBuild &F, OpBuild &A)
{
    const int P1 = ht.P1, NP = ht.NP;
    auto d2 = [](cplx z) { return make_double2(z.real(), z.imag()); };
    auto cj = [](cplx z) { return std::conj(z); };
    // leafA: fwd element (l,j) = Q[l][j];  adj element (l,j) = conj(E[j][l])
    F.leafA.resize(size_t(NP) * P1); A.leafA.resize(size_t(NP) * P1);
    for (int j = 0; j < NP; j++)
        for (int l = 0; l < P1; l++) {
            F.leafA[size_t(j) * P1 + l] = d2(at2(ht.Q, size_t(l) * NP + j));
            A.leafA[size_t(j) * P1 + l] = d2(cj(at2(ht.E, size_t(j) * P1 + l)));
        }
    // up: fwd (l,k) = M2M_q[l][k];  adj (l,k) = conj(L2L_q[k][l])
    // par: fwd (l,k) = L2L_q[l][k]; adj (l,k) = conj(M2M_q[k][l])
    F.up.resize(size_t(4) * P1 * P1); A.up.resize(F.up.size());
    F.par.resize(F.up.size()); A.par.resize(F.up.size());
    for (int q = 0; q < 4; q++)
        for (int k = 0; k < P1; k++)
            for (int l = 0; l < P1; l++) {
                size_t dst = (size_t(q) * P1 + k) * P1 + l;
                size_t lk = (size_t(q) * P1 + l) * P1 + k, kl = (size_t(q) * P1 + k) * P1 + l;
                F.up[dst] = d2(at2(ht.M2M, lk));
                A.up[dst] = d2(cj(at2(ht.L2L, kl)));
                F.par[dst] = d2(at2(ht.L2L, lk));
                A.par[dst] = d2(cj(at2(ht.M2M, kl)));
            }
    // v: fwd (l,k) = M2L_c[l][k];  adj code c (offset d): (l,k) = conj(M2L_{-d}[k][l])
    F.v.resize(size_t(kNumV) * P1 * P1); A.v.resize(F.v.size());
    for (int c = 0; c < kNumV; c++) {
        int cr = kNumV - 1 - c;   // code of -d
        for (int k = 0; k < P1; k++)
            for (int l = 0; l < P1; l++) {
                size_t dst = (size_t(c) * P1 + k) * P1 + l;
                F.v[dst] = d2(at2(ht.M2L, (size_t(c) * P1 + l) * P1 + k));
                A.v[dst] = d2(cj(at2(ht.M2L, (size_t(cr) * P1 + k) * P1 + l)));
            }
    }
    // x: fwd (l,j) = P2L_c[l][j];  adj (l,j) = conj(M2P_c[j][l])
    // w: fwd (j,k) = M2P_c[j][k];  adj (j,k) = conj(P2L_c[k][j])
    F.x.resize(size_t(kNumWX) * NP * P1); A.x.resize(F.x.size());
    F.w.resize(size_t(kNumWX) * P1 * NP); A.w.resize(F.w.size());
    for (int c = 0; c < kNumWX; c++)
        for (int j = 0; j < NP; j++)
            for (int l = 0; l < P1; l++) {
                size_t xdst = (size_t(c) * NP + j) * P1 + l;      // [c][j][l]
                size_t wdst = (size_t(c) * P1 + l) * NP + j;      // [c][k=l][j]
                cplx p2l = at2(ht.P2L, (size_t(c) * P1 + l) * NP + j);
                cplx m2p = at2(ht.M2P, (size_t(c) * NP + j) * P1 + l);
                F.x[xdst] = d2(p2l);
                A.x[xdst] = d2(cj(m2p));
                F.w[wdst] = d2(m2p);
                A.w[wdst] = d2(cj(p2l));
            }
    // e: fwd (j,l) = E[j][l];  adj (j,l) = conj(Q[l][j]);  stored [l][j]
    F.e.resize(size_t(P1) * NP); A.e.resize(F.e.size());
    for (int l = 0; l < P1; l++)
        for (int j = 0; j < NP; j++) {
            F.e[size_t(l) * NP + j] = d2(at2(ht.E, size_t(j) * P1 + l));
            A.e[size_t(l) * NP + j] = d2(cj(at2(ht.Q, size_t(l) * NP + j)));
        }
    // t: fwd (j,k) = T_tab[j][k];  adj (j,k) = T_rev(tab)[k][j];  stored [tab][k][j]
    F.t.assign(size_t(kNumNear) * NP * NP, 0.0); A.t.assign(F.t.size(), 0.0);
    for (int tab = 0; tab < kNumNear; tab++) {
        NearGeom g = near_table_geometry(tab);
        if (!g.valid) continue;
        for (int k = 0; k < NP; k++)
            for (int j = 0; j < NP; j++) {
                F.t[(size_t(tab) * NP + k) * NP + j] = ht.T[(size_t(tab) * NP + j) * NP + k];
                A.t[(size_t(tab) * NP + k) * NP + j] = ht.T[(size_t(g.rev) * NP + k) * NP + j];
            }
    }
}

// Term schedule of the double-float upward shift (DfSched) from the operator
// of the four children, up[q][k][l] (output l, input k).  The k range of
// each output over the four children (exact zeros left out; an all-zero
// output keeps one zero term) gives the nonzero terms, taken output by
// output; they are cut into 32 runs of T, lane i taking run i.  A lane ends
// a partial sum (slot l * maxp + its place among the output's lanes) where
// its run leaves an output.  Entries are split as x = hi + lo, hi the FP32
// rounding of x and lo that of the remainder.
struct UpScheduleHost {
    int T = 0, maxp = 0;
    std::vector<uint32_t> code;   // [T][32]
    std::vector<float4> ops;      // [4][T][32]
    std::vector<int32_t> np;      // [P1]
};

UpScheduleHost build_up_schedule(const std::vector<double2> &up)
{
    int P1 = 0;   // up is [4][P1][P1]
    while (size_t(4) * (P1 + 1) * (P1 + 1) <= up.size()) P1++;
    auto dfs = [](double x) {
        const float h = float(x);
        return std::make_pair(h, float(x - double(h)));
    };
    std::vector<int> klo(P1, P1), khi(P1, -1);
    for (int q = 0; q < 4; q++)
        for (int k = 0; k < P1; k++)
            for (int l = 0; l < P1; l++) {
                const double2 o = up[(size_t(q) * P1 + k) * P1 + l];
                if (o.x != 0.0 || o.y != 0.0) {
                    klo[l] = std::min(klo[l], k);
                    khi[l] = std::max(khi[l], k);
                }
            }
    std::vector<std::pair<int, int>> terms;   // (l, k), output by output
    for (int l = 0; l < P1; l++) {
        if (khi[l] < klo[l]) klo[l] = khi[l] = 0;
        for (int k = klo[l]; k <= khi[l]; k++) terms.emplace_back(l, k);
    }
    UpScheduleHost r;
    const int N = int(terms.size());
    r.T = (N + 31) / 32;
    std::vector<int> lf(P1, -1);
    r.np.assign(P1, 0);
    for (int i = 0; i < N; i++) {
        const int l = terms[i].first, lane = i / r.T;
        if (lf[l] < 0) lf[l] = lane;
        r.np[l] = lane - lf[l] + 1;
    }
    r.maxp = P1 > 0 ? *std::max_element(r.np.begin(), r.np.end()) : 0;
    r.code.assign(size_t(r.T) * 32, 0u);
    r.ops.assign(size_t(4) * r.T * 32, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int i = 0; i < N; i++) {
        const int l = terms[i].first, k = terms[i].second, lane = i / r.T, t = i % r.T;
        const bool last = i + 1 == N || terms[i + 1].first != l || (i + 1) % r.T == 0;
        const uint32_t slot = uint32_t(l * r.maxp + lane - lf[l]);
        r.code[size_t(t) * 32 + lane] = uint32_t(k) | (last ? (slot + 1u) << 8 : 0u);
        for (int q = 0; q < 4; q++) {
            const double2 o = up[(size_t(q) * P1 + k) * P1 + l];
            const auto re = dfs(o.x), im = dfs(o.y);
            r.ops[(size_t(q) * r.T + t) * 32 + lane] = make_float4(re.first, re.second, im.first, im.second);
        }
    }
    return r;
}

// Factored FP64 shifts (ShiftFac).  With delta_q = (2qx - 1) + i (2qy - 1)
// the child's centre offset in child radii, the four shifts of the scaled
// expansions (host tables: M2M[l][k] = C(l-1,k-1) 2^-l delta^(l-k), M2M[l][0] =
// -(delta/2)^l / l, L2L[m][l] = C(l,m) 2^-l delta^(l-m)) factor as
//   forward up (M2M):     so = (delta/2)^l,        si = delta^-k,         B[l][k] = C(l-1,k-1), B[l][0] = -1/l
//   forward par (L2L):    so = delta^-m,           si = (delta/2)^l,      B[m][l] = C(l,m)
//   adjoint up (L2L^H):   so = (conj delta/2)^l,   si = conj(delta)^-k,   B[l][k] = C(l,k)
//   adjoint par (M2M^H):  so = conj(delta)^-l,     si = (conj delta/2)^k, B[l][k] = C(k-1,l-1), B[0][k] = -1/k
// (B[0][0] = 1 in the M2M cases).  The products are checked against the
// dense operators (`dense`, layout [q][k][l]) before they are used.
struct ShiftFacHost {
    int T = 0, maxp = 0;
    std::vector<double2> si, so;   // [4][P1]
    std::vector<uint32_t> code;    // [T][32]
    std::vector<double> coef;      // [T][32]
    std::vector<int32_t> np;       // [P1]
};

bc_status build_shift_fac(int P1, bool par, bool adj, const std::vector<double2> &dense, ShiftFacHost &r)
{
    using lcplx = std::complex<long double>;
    std::vector<long double> bin(size_t(2 * P1 + 2) * (2 * P1 + 2), 0.0L);
    auto C = [&](int n, int k) -> long double & { return bin[size_t(n) * (2 * P1 + 2) + k]; };
    for (int n = 0; n < 2 * P1 + 2; n++) {
        C(n, 0) = 1.0L;
        for (int k = 1; k <= n; k++) C(n, k) = C(n - 1, k - 1) + (k <= n - 1 ? C(n - 1, k) : 0.0L);
    }
    // B[l][k] (output l, input k)
    std::vector<long double> B(size_t(P1) * P1, 0.0L);
    for (int l = 0; l < P1; l++)
        for (int k = 0; k < P1; k++) {
            long double v = 0.0L;
            const bool m2m = par == adj;   // forward up and adjoint par come from M2M
            if (m2m) {
                const int o = adj ? k : l, i = adj ? l : k;   // M2M element (o, i), o >= i
                if (o == 0 && i == 0) v = 1.0L;
                else if (o >= 1 && i == 0) v = -1.0L / o;
                else if (i >= 1 && i <= o) v = C(o - 1, i - 1);
            } else {
                const int o = adj ? l : k, i = adj ? k : l;   // L2L element (m = i, l = o), o >= i
                if (o >= i) v = C(o, i);
            }
            B[size_t(l) * P1 + k] = v;
        }
    r.si.assign(size_t(4) * P1, make_double2(0, 0));
    r.so.assign(size_t(4) * P1, make_double2(0, 0));
    long double worst = 0.0L;
    for (int q = 0; q < 4; q++) {
        lcplx dl(2.0L * (q & 1) - 1.0L, 2.0L * (q >> 1) - 1.0L);
        if (adj) dl = std::conj(dl);
        std::vector<lcplx> si(P1), so(P1);
        lcplx ph = 1.0L, pinv = 1.0L;   // (delta/2)^n, delta^-n
        for (int n = 0; n < P1; n++) {
            // child -> parent: so = (delta/2)^l, si = delta^-k; parent -> child: the reverse
            if (!par) { so[n] = ph; si[n] = pinv; }
            else { so[n] = pinv; si[n] = ph; }
            ph *= dl / 2.0L;
            pinv /= dl;
        }
        for (int n = 0; n < P1; n++) {
            r.si[size_t(q) * P1 + n] = make_double2(double(si[n].real()), double(si[n].imag()));
            r.so[size_t(q) * P1 + n] = make_double2(double(so[n].real()), double(so[n].imag()));
        }
        // check against the dense operator, element by element, relative to
        // the largest entry of its output row
        for (int l = 0; l < P1; l++) {
            long double rowmax = 0.0L;
            for (int k = 0; k < P1; k++) {
                const double2 d = dense[(size_t(q) * P1 + k) * P1 + l];
                rowmax = std::max(rowmax, std::abs(lcplx(d.x, d.y)));
            }
            for (int k = 0; k < P1; k++) {
                const double2 d = dense[(size_t(q) * P1 + k) * P1 + l];
                const lcplx f = so[l] * B[size_t(l) * P1 + k] * si[k];
                const long double e = std::abs(f - lcplx(d.x, d.y)) / (rowmax > 0 ? rowmax : 1.0L);
                worst = std::max(worst, e);
            }
        }
    }
    if (!(worst < 1e-14L)) {
        set_error("tables: factored %s shift (%s) differs from the dense operator by %.3Le", par ? "parent" : "child",
                  adj ? "adjoint" : "forward", worst);
        return BC_ERR_STATE;
    }
    // term schedule over B's nonzeros, output by output, 32 runs
    std::vector<std::pair<int, int>> terms;
    for (int l = 0; l < P1; l++) {
        bool any = false;
        for (int k = 0; k < P1; k++)
            if (B[size_t(l) * P1 + k] != 0.0L) { terms.emplace_back(l, k); any = true; }
        if (!any) terms.emplace_back(l, 0);   // an all-zero output keeps one zero term
    }
    const int N = int(terms.size());
    r.T = (N + 31) / 32;
    std::vector<int> lf(P1, -1);
    r.np.assign(P1, 0);
    for (int i = 0; i < N; i++) {
        const int l = terms[i].first, lane = i / r.T;
        if (lf[l] < 0) lf[l] = lane;
        r.np[l] = lane - lf[l] + 1;
    }
    r.maxp = *std::max_element(r.np.begin(), r.np.end());
    r.code.assign(size_t(r.T) * 32, 0u);
    r.coef.assign(size_t(r.T) * 32, 0.0);
    for (int i = 0; i < N; i++) {
        const int l = terms[i].first, k = terms[i].second, lane = i / r.T, t = i % r.T;
        const bool last = i + 1 == N || terms[i + 1].first != l || (i + 1) % r.T == 0;
        const uint32_t slot = uint32_t(l * r.maxp + lane - lf[l]);
        r.code[size_t(t) * 32 + lane] = uint32_t(k) | (last ? (slot + 1u) << 8 : 0u);
        r.coef[size_t(t) * 32 + lane] = double(B[size_t(l) * P1 + k]);
    }
    return BC_OK;
}

bc_status upload_shift_fac(DevTables &dt, ShiftFac &f, const ShiftFacHost &h)
{
    double2 *psi = nullptr, *pso = nullptr;
    uint32_t *pc = nullptr;
    double *pf = nullptr;
    int32_t *pn = nullptr;
    cudaError_t e;
    if ((e = dev_upload(dt.allocs, &psi, h.si.data(), h.si.size())) != cudaSuccess ||
        (e = dev_upload(dt.allocs, &pso, h.so.data(), h.so.size())) != cudaSuccess ||
        (e = dev_upload(dt.allocs, &pc, h.code.data(), h.code.size())) != cudaSuccess ||
        (e = dev_upload(dt.allocs, &pf, h.coef.data(), h.coef.size())) != cudaSuccess ||
        (e = dev_upload(dt.allocs, &pn, h.np.data(), h.np.size())) != cudaSuccess)
        return cuda_fail(e, "tables upload");
    f.si = psi; f.so = pso; f.code = pc; f.coef = pf; f.np = pn;
    f.T = h.T; f.maxp = h.maxp;
    return BC_OK;
}

bc_status upload_opset(DevTables &dt, OpSet &os, const OpBuild &b, bool adj)
{
    cudaError_t e;
    double2 *p;
    double *q;
#define UP2(field)                                                              \
    e = dev_upload(dt.allocs, &p, b.field.data(), b.field.size());              \
    if (e != cudaSuccess) return cuda_fail(e, "tables upload");                  \
    os.field = p;
    UP2(leafA) UP2(up) UP2(par) UP2(v) UP2(x) UP2(e) UP2(w)
#undef UP2
    {
        // double-float copies of the shift operators: x = hi + lo, hi the FP32
        // rounding of x and lo that of the remainder
        auto dfs = [](double x) {
            const float h = float(x);
            return std::make_pair(h, float(x - double(h)));
        };
        for (int which = 1; which < 3; which++) {   // par, leafA (up: the schedule below)
            const std::vector<double2> &src = which == 2 ? b.leafA : b.par;
            std::vector<float4> f(src.size());
            for (size_t i = 0; i < src.size(); i++) {
                const auto re = dfs(src[i].x), im = dfs(src[i].y);
                f[i] = make_float4(re.first, re.second, im.first, im.second);
            }
            float4 *pf = nullptr;
            e = dev_upload(dt.allocs, &pf, f.data(), f.size());
            if (e != cudaSuccess) return cuda_fail(e, "tables upload");
            (which == 2 ? os.leafA_df : os.par_df) = pf;
        }
        // the term schedule of the double-float climb (DfSched)
        const UpScheduleHost us = build_up_schedule(b.up);
        uint32_t *pc = nullptr;
        float4 *po = nullptr;
        int32_t *pn = nullptr;
        if ((e = dev_upload(dt.allocs, &pc, us.code.data(), us.code.size())) != cudaSuccess ||
            (e = dev_upload(dt.allocs, &po, us.ops.data(), us.ops.size())) != cudaSuccess ||
            (e = dev_upload(dt.allocs, &pn, us.np.data(), us.np.size())) != cudaSuccess)
            return cuda_fail(e, "tables upload");
        os.up_s.code = pc;
        os.up_s.ops = po;
        os.up_s.np = pn;
        os.up_s.T = us.T;
        os.up_s.maxp = us.maxp;
    }
    {
        const int P1 = int(std::lround(std::sqrt(double(b.up.size() / 4))));
        ShiftFacHost fu, fp;
        bc_status s;
        if ((s = build_shift_fac(P1, false, adj, b.up, fu)) != BC_OK ||
            (s = build_shift_fac(P1, true, adj, b.par, fp)) != BC_OK ||
            (s = upload_shift_fac(dt, os.up_f, fu)) != BC_OK || (s = upload_shift_fac(dt, os.par_f, fp)) != BC_OK)
            return s;
    }
    e = dev_upload(dt.allocs, &q, b.t.data(), b.t.size());
    if (e != cudaSuccess) return cuda_fail(e, "tables upload");
    os.t = q;
    return BC_OK;
}

bc_status upload_tree(bc_tree *t)
{
    HostTree &h = t->h;
    DevTree &d = t->d;
    const int P1 = t->ctx->P1;
    cudaError_t e;
#define UPV(dst, vec)                                                           \
    e = dev_upload(d.allocs, &d.dst, vec.data(), vec.size());                   \
    if (e != cudaSuccess) return cuda_fail(e, "tree upload");
    UPV(leaf_box, h.leaf_box) UPV(leaf_level, h.leaf_level) UPV(leaf_order, h.leaf_order)
    UPV(box_parent, h.box_parent) UPV(box_child0, h.box_child0) UPV(box_level, h.box_level)
    UPV(box_ix, h.box_ix) UPV(box_iy, h.box_iy) UPV(box_leaf, h.box_leaf)
    UPV(near_ptr, h.near_ptr) UPV(near_src, h.near_src) UPV(near_tab, h.near_tab)
    UPV(v_ptr, h.v_ptr) UPV(v_src, h.v_src) UPV(v_code, h.v_code)
    UPV(w_ptr, h.w_ptr) UPV(w_src, h.w_src) UPV(w_code, h.w_code)
    UPV(x_ptr, h.x_ptr) UPV(x_src, h.x_src) UPV(x_code, h.x_code)
#undef UPV
    e = dev_upload<int32_t>(d.allocs, &d.zero_ptr, nullptr, size_t(h.nleaf) + 1);
    if (e != cudaSuccess) return cuda_fail(e, "tree upload");
    e = dev_upload<double2>(d.allocs, &d.leaf_logs, nullptr, size_t(h.nleaf));
    if (e != cudaSuccess) return cuda_fail(e, "tree upload");
    if (!h.leaf_class.empty()) {
        std::vector<uint8_t> act(h.nleaf);
        for (int64_t k = 0; k < h.nleaf; k++) act[k] = h.leaf_class[k] != 0;
        uint8_t *pa = nullptr;
        e = dev_upload(d.allocs, &pa, act.data(), act.size());
        if (e != cudaSuccess) return cuda_fail(e, "tree upload");
        d.leaf_active = pa;
    }
    // r^2 and log r per level, r = (L/2) 2^-lv
    std::vector<double> lt(2 * kLvTab, 0.0);
    for (int lv = 0; lv < kLvTab; lv++) {
        const double r = std::ldexp(0.5 * h.L, -lv);
        lt[lv] = r * r;
        lt[kLvTab + lv] = double(std::log((long double)(0.5 * h.L)) - (long double)lv * std::log(2.0L));
    }
    e = dev_upload(d.allocs, &d.lvtab, lt.data(), lt.size());
    if (e != cudaSuccess) return cuda_fail(e, "tree upload");
    {
        std::vector<int32_t> vb(h.v_src.size()), xb(h.x_src.size());
        for (size_t b = 0; b + 1 < h.v_ptr.size(); b++)
            for (int32_t k = h.v_ptr[b]; k < h.v_ptr[b + 1]; k++) vb[k] = int32_t(b);
        for (size_t b = 0; b + 1 < h.x_ptr.size(); b++)
            for (int32_t k = h.x_ptr[b]; k < h.x_ptr[b + 1]; k++) xb[k] = int32_t(b);
        if ((e = dev_upload(d.allocs, &d.v_box, vb.data(), vb.size())) != cudaSuccess ||
            (e = dev_upload(d.allocs, &d.x_box, xb.data(), xb.size())) != cudaSuccess ||
            (e = dev_upload<double2>(d.allocs, &d.PX, nullptr, h.x_src.size() * size_t(P1))) != cudaSuccess)
            return cuda_fail(e, "tree upload");
    }
    e = dev_upload(d.allocs, &d.level_start, h.level_start.data(), h.level_start.size());
    if (e != cudaSuccess) return cuda_fail(e, "tree upload");
    e = dev_upload<int32_t>(d.allocs, &d.flag, nullptr, h.box_level.size());
    if (e != cudaSuccess) return cuda_fail(e, "tree upload");
    size_t nexp = size_t(h.box_level.size()) * P1;
    e = dev_upload<float4>(d.allocs, &d.exdf, nullptr, nexp);
    if (e != cudaSuccess) return cuda_fail(e, "tree workspace");
    e = dev_upload<double2>(d.allocs, &d.expA, nullptr, nexp);
    if (e != cudaSuccess) return cuda_fail(e, "tree workspace");
    e = dev_upload<double2>(d.allocs, &d.expB, nullptr, nexp);
    if (e != cudaSuccess) return cuda_fail(e, "tree workspace");
    return BC_OK;
}

bc_status finish_tree(bc_ctx *ctx, bc_tree **out, bc_tree *t)
{
    if (ctx->device < 0) { *out = t; return BC_OK; }   // host-only context: no upload
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) { delete t; return cuda_fail(e, "cudaSetDevice"); }
    bc_status s = upload_tree(t);
    if (s != BC_OK) {
        free_all(t->d.allocs);
        delete t;
        return s;
    }
    *out = t;
    return BC_OK;
}

}  // namespace

PassArgs pass_args(const bc_ctx *ctx, const bc_tree *t)
{
    PassArgs a;
    a.p = ctx->p; a.NP = ctx->NP; a.P1 = ctx->P1;
    a.half_L = 0.5 * t->h.L;
    a.nleaf = t->h.nleaf;
    a.nbox = int64_t(t->h.box_level.size());
    a.up_blocks = ctx->up_blocks;
    a.shift_blocks = ctx->shift_blocks;
    a.down_blocks = ctx->down_blocks;
    a.m2l_bps = ctx->m2l_bps;
    a.m2l_kind = ctx->m2l_kind;
    a.wait_limit = ctx->split.wait_limit;
    a.err = ctx->dev_err;
    return a;
}

namespace {

// Digits of one FP64 matrix row for the split near field: row scaled by 2^-E
// into (-1/2, 1/2), rounded to a 40-bit integer, five balanced base-256 digits.
int split_row(const double *row, int n, int16_t *digits /*[5][n]*/)
{
    double mx = 0.0;
    for (int k = 0; k < n; k++) mx = std::max(mx, std::fabs(row[k]));
    if (mx == 0.0) {
        std::fill(digits, digits + size_t(kSplitSlices) * n, int16_t(0));
        return 0;
    }
    int e = 0;
    std::frexp(mx, &e);            // mx < 2^e
    const int E = e + 1;           // mx < 2^(E-1)
    for (int k = 0; k < n; k++) {
        long long X = std::llround(std::ldexp(row[k], 40 - E));   // |X| < 2^39
        for (int a = kSplitSlices; a >= 2; a--) {
            int d = int(X & 255);
            if (d >= 128) d -= 256;
            X = (X - d) >> 8;
            digits[(a - 1) * n + k] = int16_t(d);
        }
        digits[k] = int16_t(X);   // leading digit, |X| <= 128
    }
    return E;
}

uint16_t bf16_of_int(int d)
{
    float f = float(d);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return uint16_t(u >> 16);
}

// Appends the BF16 digits of a real operator (rows x K, row-major) to `dig`
// in the chunk layout [digit a][row half h][K chunk kc] x (128 rows x KC) of
// canonical K-major core matrices, and its row exponents to `ex`.
SplitOp add_split_op(std::vector<uint16_t> &dig, std::vector<int32_t> &ex, const std::vector<double> &m, int rows,
                     int K)
{
    const int KC = std::min(K, kSplitKC), nkc = K / KC, mh = rows > 128 ? 2 : 1;
    const size_t chunk = size_t(128) * KC;   // elements per chunk
    SplitOp op;
    op.a_off = int64_t(dig.size()) * int64_t(sizeof(uint16_t));
    op.rows = rows;
    op.exp_off = int32_t(ex.size());
    const size_t base = dig.size();
    dig.resize(base + size_t(kSplitSlices) * mh * nkc * chunk, 0);
    ex.resize(ex.size() + size_t(mh) * 128, 0);
    std::vector<int16_t> dg(size_t(kSplitSlices) * K);
    for (int i = 0; i < rows; i++) {
        ex[size_t(op.exp_off) + i] = split_row(&m[size_t(i) * K], K, dg.data());
        const int h = i / 128, rg = (i % 128) / 8, r = i % 8;
        for (int a = 0; a < kSplitSlices; a++)
            for (int k = 0; k < K; k++) {
                const int kc = k / KC, kg = (k % KC) / 8, e = k % 8;
                const size_t off = base + ((size_t(a) * mh + h) * nkc + kc) * chunk +
                                   (size_t(rg) * (KC / 8) + kg) * 64 + size_t(r) * 8 + e;
                dig[off] = bf16_of_int(dg[size_t(a) * K + k]);
            }
    }
    return op;
}

// Real operators of the split path, direction dir (0 forward, 1 adjoint):
//   group V, K = KV (the p^2 leaf nodes, zero columns up to 64 for p = 8 and
//     to 256 for p = 12, 16): near tables (p^2 rows), leafA (2 P1 rows: P2M /
//     L2P^H), X list per code (2 P1 rows: P2L / M2P^H); output rows 2l, 2l+1 =
//     Re, Im of coefficient l;
//   group E, K = 64 (coefficient l at columns 2l, 2l+1 = Re, Im): L2P / P2M^H
//     and the W list per code (M2P / P2L^H), p^2 rows, output = real part.
bc_status build_split_tables(bc_ctx *ctx)
{
    // split path: p = 8, 12 or 16, P1 <= 32
    if ((ctx->p != 8 && ctx->p != 12 && ctx->p != 16) || ctx->device < 0 || 2 * ctx->P1 > kSplitKE) return BC_OK;
    const HostTables &ht = ctx->ht;
    const int NP = ctx->NP, KV = NP <= 64 ? 64 : 256, P1 = ctx->P1, R = 2 * P1, KE = kSplitKE;
    SplitTables &T = ctx->split;
    T.np = NP;
    T.kv = KV;
    for (int dir = 0; dir < 2; dir++) {
        std::vector<uint16_t> dv, de;
        std::vector<int32_t> xv, xe;
        std::vector<double> m;
        // group V
        T.near_op[dir].assign(kNumNear, SplitOp());
        m.assign(size_t(NP) * KV, 0.0);
        for (int tab = 0; tab < kNumNear; tab++) {
            NearGeom g = near_table_geometry(tab);
            if (!g.valid) continue;
            for (int i = 0; i < NP; i++)
                for (int k = 0; k < NP; k++)
                    m[size_t(i) * KV + k] = dir == 0 ? ht.T[(size_t(tab) * NP + i) * NP + k]
                                                     : ht.T[(size_t(g.rev) * NP + k) * NP + i];
            T.near_op[dir][tab] = add_split_op(dv, xv, m, NP, KV);
        }
        m.assign(size_t(R) * KV, 0.0);
        for (int l = 0; l < P1; l++)
            for (int j = 0; j < NP; j++) {
                cplx z = dir == 0 ? at2(ht.Q, size_t(l) * NP + j) : std::conj(at2(ht.E, size_t(j) * P1 + l));
                m[size_t(2 * l) * KV + j] = z.real();
                m[size_t(2 * l + 1) * KV + j] = z.imag();
            }
        T.leafA_op[dir] = add_split_op(dv, xv, m, R, KV);
        T.x_op[dir].assign(kNumWX, SplitOp());
        for (int c = 0; c < kNumWX; c++) {
            for (int l = 0; l < P1; l++)
                for (int j = 0; j < NP; j++) {
                    cplx z = dir == 0 ? at2(ht.P2L, (size_t(c) * P1 + l) * NP + j)
                                      : std::conj(at2(ht.M2P, (size_t(c) * NP + j) * P1 + l));
                    m[size_t(2 * l) * KV + j] = z.real();
                    m[size_t(2 * l + 1) * KV + j] = z.imag();
                }
            T.x_op[dir][c] = add_split_op(dv, xv, m, R, KV);
        }
        // group E: out_j = Re(sum_l Op(j,l) b_l) = sum_l Re Op(j,l) Re b_l - Im Op(j,l) Im b_l;
        // columns rescaled by powers of two (the expansion digits carry the inverse scale)
        std::vector<double> me(size_t(NP) * KE, 0.0);
        std::vector<std::vector<double>> mw(kNumWX, std::vector<double>(size_t(NP) * KE, 0.0));
        for (int j = 0; j < NP; j++)
            for (int l = 0; l < P1; l++) {
                cplx z = dir == 0 ? at2(ht.E, size_t(j) * P1 + l) : std::conj(at2(ht.Q, size_t(l) * NP + j));
                me[size_t(j) * KE + 2 * l] = z.real();
                me[size_t(j) * KE + 2 * l + 1] = -z.imag();
                for (int c = 0; c < kNumWX; c++) {
                    cplx w = dir == 0 ? at2(ht.M2P, (size_t(c) * NP + j) * P1 + l)
                                      : std::conj(at2(ht.P2L, (size_t(c) * P1 + l) * NP + j));
                    mw[c][size_t(j) * KE + 2 * l] = w.real();
                    mw[c][size_t(j) * KE + 2 * l + 1] = -w.imag();
                }
            }
        // Column scales.  The rounding error of output j is about
        // 2^-40 (max_k |A'_jk| sum_k |x'_k| + max_k |x'_k| sum_k |A'_jk|) with
        // A' = A / s, x' = s x; it is smallest for s_k = sqrt(alpha_k / beta_k),
        // alpha_k ~ |A_jk| and beta_k ~ |x_k| the profiles of coefficient k.
        // Expansion-to-leaf (L2P, P2M^H): the operator grows like (sqrt 2)^l
        // (nodes up to a corner of the box) and its inputs (local coefficients,
        // adjoint multipoles) decay at least like 3^-l (sources two box widths
        // away), so s = 2^l; the W list (M2P, P2L^H): operator ~ 3^-l, inputs
        // (multipoles, adjoint locals) ~ (sqrt 2)^l, so s = 2^-l.
        std::vector<double> se(KE), sw(KE);
        for (int k = 0; k < KE; k++) {
            se[k] = std::ldexp(1.0, k / 2);
            sw[k] = std::ldexp(1.0, -(k / 2));
            for (int j = 0; j < NP; j++) {
                me[size_t(j) * KE + k] /= se[k];
                for (int c = 0; c < kNumWX; c++) mw[c][size_t(j) * KE + k] /= sw[k];
            }
        }
        T.e_op[dir] = add_split_op(de, xe, me, NP, KE);
        T.w_op[dir].assign(kNumWX, SplitOp());
        for (int c = 0; c < kNumWX; c++) T.w_op[dir][c] = add_split_op(de, xe, mw[c], NP, KE);
        // Group M: M2L per V code in real form (rows 2l, 2l+1 = Re, Im of
        // output coefficient l; column 2k, 2k+1 = Re, Im of input k):
        //   forward (l,k) = M2L_c[l][k];  adjoint (l,k) = conj(M2L_{-d}[k][l]),
        // without the log term of (0,0): (log|d| + log r) A_0 stays in FP64
        // (downward pass), like every log term of the method.  The input is
        // the `first` array with the W-list scales 2^-k: the translation of a
        // source two box widths away decays like C(k+l-1, k-1) 4^-(k+l) and
        // its input grows at most like (sqrt 2)^k, so the rescaled rows stay
        // within a few powers of two.
        T.m2l_op[dir].assign(kNumV, SplitOp());
        {
            std::vector<double> mm(size_t(R) * KE, 0.0);
            for (int c = 0; c < kNumV; c++) {
                const int dx = c % 7 - 3, dy = c / 7 - 3, cr = kNumV - 1 - c;
                if (std::max(std::abs(dx), std::abs(dy)) < 2) continue;
                std::fill(mm.begin(), mm.end(), 0.0);
                for (int l = 0; l < P1; l++)
                    for (int k = 0; k < P1; k++) {
                        cplx z = dir == 0 ? at2(ht.M2L, (size_t(c) * P1 + l) * P1 + k)
                                          : std::conj(at2(ht.M2L, (size_t(cr) * P1 + k) * P1 + l));
                        if (l == 0 && k == 0) z = 0.0;
                        mm[size_t(2 * l) * KE + 2 * k] = z.real() / sw[2 * k];
                        mm[size_t(2 * l) * KE + 2 * k + 1] = -z.imag() / sw[2 * k + 1];
                        mm[size_t(2 * l + 1) * KE + 2 * k] = z.imag() / sw[2 * k];
                        mm[size_t(2 * l + 1) * KE + 2 * k + 1] = z.real() / sw[2 * k + 1];
                    }
                T.m2l_op[dir][c] = add_split_op(de, xe, mm, R, KE);
            }
        }
        // expA is the W source (first) in the forward apply and the P2M^H input
        // (second) in the adjoint; expB the other way round
        std::vector<double> scl(2 * KE);
        for (int k = 0; k < KE; k++) {
            scl[k] = dir == 0 ? sw[k] : se[k];
            scl[KE + k] = dir == 0 ? se[k] : sw[k];
        }
        double *dsc = nullptr;
        uint16_t *d0 = nullptr, *d1 = nullptr;
        int32_t *e0 = nullptr, *e1 = nullptr;
        cudaError_t e;
        if ((e = dev_upload(ctx->split_allocs, &d0, dv.data(), dv.size())) != cudaSuccess ||
            (e = dev_upload(ctx->split_allocs, &e0, xv.data(), xv.size())) != cudaSuccess ||
            (e = dev_upload(ctx->split_allocs, &d1, de.data(), de.size())) != cudaSuccess ||
            (e = dev_upload(ctx->split_allocs, &e1, xe.data(), xe.size())) != cudaSuccess ||
            (e = dev_upload(ctx->split_allocs, &dsc, scl.data(), scl.size())) != cudaSuccess)
            return cuda_fail(e, "split tables upload");
        T.escale[dir] = dsc;
        T.ops[0][dir] = reinterpret_cast<const uint8_t *>(d0);
        T.op_exp[0][dir] = e0;
        T.ops[1][dir] = reinterpret_cast<const uint8_t *>(d1);
        T.op_exp[1][dir] = e1;
    }
    cudaError_t e = split_prepare();
    if (e != cudaSuccess) return cuda_fail(e, "split kernel attributes");
    if (!ctx->side.side) {
        if ((e = cudaStreamCreateWithFlags(&ctx->side.side, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ctx->side.fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ctx->side.join, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ctx->side.xdone, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "split side stream");
    }
    ctx->split_ready = true;
    return BC_OK;
}

// Column lists of the split path for one tree.  Tiles hold up to
// kSplitTileN columns that share one operator; tiles of 256-row operators
// come first (longest work first).
struct TileBuilder {
    std::vector<SplitTile> tiles;
    std::vector<SplitCol> cols;
    // one operator, its columns given in order
    void add(const SplitOp &op, const std::vector<SplitCol> &c)
    {
        for (size_t i = 0; i < c.size(); i += kSplitTileN) {
            SplitTile t;
            t.a_off = op.a_off;
            t.rows = op.rows;
            t.exp_off = op.exp_off;
            t.p0 = int32_t(cols.size());
            t.cnt = int32_t(std::min<size_t>(kSplitTileN, c.size() - i));
            cols.insert(cols.end(), c.begin() + i, c.begin() + i + t.cnt);
            tiles.push_back(t);
        }
    }
};

inline int32_t col_ctl(int shift, bool inv_alpha) { return int32_t(shift * 2 + (inv_alpha ? 1 : 0)); }

bc_status build_split_tree(bc_tree *t)
{
    if (t->split_ready) return BC_OK;
    const HostTree &h = t->h;
    const SplitTables &T = t->ctx->split;
    const int P1 = t->ctx->P1;
    const int64_t nn = int64_t(h.near_src.size()), nx = int64_t(h.x_src.size()), nw = int64_t(h.w_src.size());
    const int64_t nbox = int64_t(h.box_level.size());
    SplitTree &s = t->sp;
    std::vector<void *> &al = t->d.allocs;
    cudaError_t e;
    const size_t NP = size_t(T.np), KV = size_t(T.kv);   // nodes per leaf, group-V K
    if ((e = dev_upload<double>(al, &s.Pnear, nullptr, size_t(nn) * NP)) != cudaSuccess ||
        (e = dev_upload<double>(al, &s.PX, nullptr, size_t(nx) * kSplitKE)) != cudaSuccess ||
        (e = dev_upload<double>(al, &s.PE, nullptr, size_t(h.nleaf) * NP)) != cudaSuccess ||
        (e = dev_upload<double>(al, &s.PW, nullptr, size_t(nw) * NP)) != cudaSuccess ||
        (e = dev_upload<uint16_t>(al, &s.vdig, nullptr, size_t(h.nleaf) * kSplitSlices * KV)) != cudaSuccess ||
        (e = dev_upload<int32_t>(al, &s.vexp, nullptr, size_t(h.nleaf))) != cudaSuccess ||
        (e = dev_upload<uint16_t>(al, &s.edig, nullptr, size_t(2 * nbox) * kSplitSlices * kSplitKE)) != cudaSuccess ||
        (e = dev_upload<int32_t>(al, &s.eexp, nullptr, size_t(2 * nbox))) != cudaSuccess)
        return cuda_fail(e, "split tree upload");
    // owners of the near and W entries, box of each X entry
    std::vector<int32_t> near_owner(nn), w_owner(nw), x_box(nx);
    for (int64_t o = 0; o < h.nleaf; o++) {
        for (int32_t k = h.near_ptr[o]; k < h.near_ptr[o + 1]; k++) near_owner[k] = int32_t(o);
        for (int32_t k = h.w_ptr[o]; k < h.w_ptr[o + 1]; k++) w_owner[k] = int32_t(o);
    }
    for (int64_t b = 0; b < nbox; b++)
        for (int32_t k = h.x_ptr[b]; k < h.x_ptr[b + 1]; k++) x_box[k] = int32_t(b);
    for (int dir = 0; dir < 2; dir++) {
        const bool adj = dir == 1;
        double2 *first = adj ? t->d.expB : t->d.expA;
        const int first_which = adj ? 1 : 0, second_which = adj ? 0 : 1;   // expA = 0, expB = 1
        TileBuilder V, NV, E;
        // near entries, by table
        std::vector<std::vector<SplitCol>> by_tab(kNumNear);
        for (int64_t k = 0; k < nn; k++) {
            const int32_t src = h.near_src[k], own = near_owner[k];
            SplitCol c;
            c.vec = src;
            c.ctl = col_ctl(-2 * (adj ? h.leaf_level[own] : h.leaf_level[src]), false);
            c.out = s.Pnear + size_t(k) * NP;
            by_tab[h.near_tab[k]].push_back(c);
        }
        for (int tab = 0; tab < kNumNear; tab++)
            if (!by_tab[tab].empty()) NV.add(T.near_op[dir][tab], by_tab[tab]);
        // leafA of every leaf (Morton order), then the X entries by code
        std::vector<SplitCol> cl;
        for (int64_t i = 0; i < h.nleaf; i++) {
            const int32_t o = h.leaf_order[i];
            SplitCol c;
            c.vec = o;
            c.ctl = adj ? col_ctl(0, true) : col_ctl(-2 * h.leaf_level[o], false);
            c.out = reinterpret_cast<double *>(first + size_t(h.leaf_box[o]) * P1);
            cl.push_back(c);
        }
        V.add(T.leafA_op[dir], cl);
        s.ntA[dir] = int(V.tiles.size());
        std::vector<std::vector<SplitCol>> by_code(kNumWX);
        for (int64_t k = 0; k < nx; k++) {
            SplitCol c;
            c.vec = h.x_src[k];
            c.ctl = adj ? col_ctl(0, true) : col_ctl(-2 * (h.box_level[x_box[k]] - 1), false);
            c.out = s.PX + size_t(k) * kSplitKE;
            by_code[h.x_code[k]].push_back(c);
        }
        for (int c = 0; c < kNumWX; c++)
            if (!by_code[c].empty()) V.add(T.x_op[dir][c], by_code[c]);
        // group E: L2P of the leaves at level >= 2, then the W entries by code
        cl.clear();
        for (int64_t i = 0; i < h.nleaf; i++) {
            const int32_t o = h.leaf_order[i];
            if (h.leaf_level[o] < 2) continue;
            SplitCol c;
            c.vec = int32_t(second_which * nbox + h.leaf_box[o]);
            c.ctl = col_ctl(adj ? -2 * h.leaf_level[o] : 0, false);
            c.out = s.PE + size_t(o) * NP;
            cl.push_back(c);
        }
        E.add(T.e_op[dir], cl);
        s.ntL[dir] = int(E.tiles.size());
        for (auto &v : by_code) v.clear();
        for (int64_t k = 0; k < nw; k++) {
            SplitCol c;
            c.vec = int32_t(first_which * nbox + h.w_src[k]);
            c.ctl = col_ctl(adj ? -2 * h.leaf_level[w_owner[k]] : 0, false);
            c.out = s.PW + size_t(k) * NP;
            by_code[h.w_code[k]].push_back(c);
        }
        for (int c = 0; c < kNumWX; c++)
            if (!by_code[c].empty()) E.add(T.w_op[dir][c], by_code[c]);
        TileBuilder VN = NV;   // near tiles first (longest), then the far ones
        for (SplitTile tl : V.tiles) {
            tl.p0 += int32_t(NV.cols.size());
            VN.tiles.push_back(tl);
        }
        VN.cols.insert(VN.cols.end(), V.cols.begin(), V.cols.end());
        if ((e = dev_upload(al, &s.tVN[dir], VN.tiles.data(), VN.tiles.size())) != cudaSuccess ||
            (e = dev_upload(al, &s.cVN[dir], VN.cols.data(), VN.cols.size())) != cudaSuccess)
            return cuda_fail(e, "split tree upload");
        s.ntVN[dir] = int(VN.tiles.size());
        if ((e = dev_upload(al, &s.tV[dir], V.tiles.data(), V.tiles.size())) != cudaSuccess ||
            (e = dev_upload(al, &s.cV[dir], V.cols.data(), V.cols.size())) != cudaSuccess ||
            (e = dev_upload(al, &s.tN[dir], NV.tiles.data(), NV.tiles.size())) != cudaSuccess ||
            (e = dev_upload(al, &s.cN[dir], NV.cols.data(), NV.cols.size())) != cudaSuccess ||
            (e = dev_upload(al, &s.tE[dir], E.tiles.data(), E.tiles.size())) != cudaSuccess ||
            (e = dev_upload(al, &s.cE[dir], E.cols.data(), E.cols.size())) != cudaSuccess)
            return cuda_fail(e, "split tree upload");
        s.ntV[dir] = int(V.tiles.size());
        s.ntN[dir] = int(NV.tiles.size());
        s.ntE[dir] = int(E.tiles.size());
    }
    s.err = t->ctx->dev_err;
    t->split_ready = true;
    return BC_OK;
}

// Tensor-core M2L (part 32, BC_SPLIT_BF16_ALL): one column per V pair
// (source box digits, the result row into Pv, allocated here on first use:
// n_v x nterms x 16 bytes; the adjoint digits carry alpha0).
bc_status build_split_m2l(bc_tree *t)
{
    if (t->m2l_ready) return BC_OK;
    const HostTree &h = t->h;
    const SplitTables &T = t->ctx->split;
    const int P1 = t->ctx->P1;
    const int64_t nbox = int64_t(h.box_level.size());
    SplitTree &s = t->sp;
    std::vector<void *> &al = t->d.allocs;
    cudaError_t e = dev_upload<double2>(al, &t->d.Pv, nullptr, h.v_src.size() * size_t(P1));
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core M2L rows");
    for (int dir = 0; dir < 2; dir++) {
        const int first_which = dir == 1 ? 1 : 0;   // expA = 0, expB = 1
        TileBuilder M;
        std::vector<std::vector<SplitCol>> by_v(kNumV);
        for (size_t k = 0; k < h.v_src.size(); k++) {
            SplitCol c;
            c.vec = int32_t(first_which * nbox + h.v_src[k]);
            c.ctl = col_ctl(0, dir == 1);
            c.out = reinterpret_cast<double *>(t->d.Pv + k * size_t(P1));
            by_v[h.v_code[k]].push_back(c);
        }
        for (int c = 0; c < kNumV; c++)
            if (!by_v[c].empty()) M.add(T.m2l_op[dir][c], by_v[c]);
        if ((e = dev_upload(al, &s.tM[dir], M.tiles.data(), M.tiles.size())) != cudaSuccess ||
            (e = dev_upload(al, &s.cM[dir], M.cols.data(), M.cols.size())) != cudaSuccess)
            return cuda_fail(e, "tensor-core M2L tiles");
        s.ntM[dir] = int(M.tiles.size());
    }
    t->m2l_ready = true;
    return BC_OK;
}

// CTAs of the near-field launch on the internal stream: the option, else all
// SMs when it runs beside the FP64 M2L (one tensor CTA per SM next to the M2L
// blocks), three quarters of them when it runs beside the level passes
int near_ctas_for(const bc_ctx *ctx, int parts)
{
    if (ctx->overlap_ctas > 0) return ctx->overlap_ctas;
    return (parts & 32) ? std::max(1, 3 * split_sm_count() / 4) : split_sm_count();
}

bc_status check_apply_args(bc_ctx *ctx, const bc_tree *tree, const void *in, const void *out, bc_precision prec)
{
    if (!ctx || !tree || !in || !out) { set_error("apply: NULL argument"); return BC_ERR_ARG; }
    if (tree->ctx != ctx) { set_error("apply: tree belongs to another context"); return BC_ERR_ARG; }
    if (ctx->device < 0) { set_error("apply: host-only context (device -1) cannot apply"); return BC_ERR_STATE; }
    if (!ctx->tables_ready) { set_error("apply: call bc_tables_build first"); return BC_ERR_STATE; }
    if (in == out) { set_error("apply: output must not alias input"); return BC_ERR_ARG; }
    if (prec != BC_FP64 && !is_split(prec)) { set_error("apply: unknown precision %d", int(prec)); return BC_ERR_ARG; }
    return BC_OK;
}

bc_status apply_impl(bc_ctx *ctx, const bc_tree *tree, const double *vin, double *vout, bc_precision prec,
                     void *stream, bool adj)
{
    bc_status s = check_apply_args(ctx, tree, vin, vout, prec);
    if (s != BC_OK) return s;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PassArgs a = pass_args(ctx, tree);
    bool din = is_device_ptr(vin), dout = is_device_ptr(vout);
    if (din != dout) { set_error("apply: input and output must both be device or both host memory"); return BC_ERR_ARG; }
    const int parts = split_parts_for(int(prec), ctx->split_parts);
    // split_overlap: 1 both directions beside the far field, 2 the forward
    // apply only, 3 the adjoint only, 0 neither
    const int ov = ctx->split_overlap;
    const bool side = ov == 1 || (ov == 2 && !adj) || (ov == 3 && adj);
    SplitLaunch sl{&ctx->split, nullptr, parts, side ? &ctx->side : nullptr, near_ctas_for(ctx, parts)};
    const SplitLaunch *split = nullptr;
    bc_tree *tw = const_cast<bc_tree *>(tree);
    if (is_split(prec)) {
        if (!ctx->split_ready) {
            set_error("apply: split precision is provided for p = 8, 12 and 16 with nterms <= 32 only");
            return BC_ERR_UNSUPPORTED;
        }
        s = build_split_tree(tw);
        if (s == BC_OK && (parts & 32)) s = build_split_m2l(tw);
        if (s != BC_OK) return s;
        sl.tree = &tw->sp;
        split = &sl;
    }
    if (din) {
        e = launch_apply(a, tree->h, tree->d, ctx->dt, adj, vin, vout, st, ctx->pass_mask, ctx->timing ? ctx->ev[adj ? 1 : 0] : nullptr, ctx->m2l_tri, split);
        if (e != cudaSuccess) return cuda_fail(e, "apply launch");
        return BC_OK;
    }
    // Host arrays.  Pinned ones are read and written in place by the kernels
    // when only the first kernel reads the input: the split path with the
    // near field, leaf-to-expansion and X list on the tensor cores (parts 1, 2
    // and 4), where the input digits (k_split_vec) read it and the leaf output
    // writes the result, so that no copy stands between the calls' kernels.
    // Otherwise they are staged through the tree's device buffers.
    const double *pin_in = static_cast<const double *>(pinned_device_ptr(vin));
    double *pin_out = static_cast<double *>(const_cast<void *>(pinned_device_ptr(vout)));
    if (split && (parts & 7) == 7 && pin_in && pin_out) {
        e = launch_apply(a, tree->h, tree->d, ctx->dt, adj, pin_in, pin_out, st, ctx->pass_mask,
                         ctx->timing ? ctx->ev[adj ? 1 : 0] : nullptr, ctx->m2l_tri, split);
        if (e != cudaSuccess) return cuda_fail(e, "apply launch");
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "apply sync");
        return BC_OK;
    }
    bc_tree *t = const_cast<bc_tree *>(tree);
    size_t n = size_t(a.nleaf) * a.NP;
    if (!t->d.stage_in) {
        e = dev_upload<double>(t->d.allocs, &t->d.stage_in, nullptr, n);
        if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
        e = dev_upload<double>(t->d.allocs, &t->d.stage_out, nullptr, n);
        if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
    }
    e = cudaMemcpyAsync(t->d.stage_in, vin, n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "apply H2D");
    e = launch_apply(a, tree->h, tree->d, ctx->dt, adj, t->d.stage_in, t->d.stage_out, st, ctx->pass_mask, ctx->timing ? ctx->ev[adj ? 1 : 0] : nullptr, ctx->m2l_tri, split);
    if (e != cudaSuccess) return cuda_fail(e, "apply launch");
    e = cudaMemcpyAsync(vout, t->d.stage_out, n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "apply D2H");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "apply sync");
    return BC_OK;
}

}  // namespace

bc_status prepare_split_tree(bc_tree *t) { return build_split_tree(t); }

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

}  // namespace bc

struct bc_batch {
    bc_ctx *ctx = nullptr;
    std::vector<const bc_tree *> trees;
    std::vector<int64_t> leaf_offset;
    bc_tree *u = nullptr;
    double *in_buf = nullptr, *out_buf = nullptr;
    cudaStream_t cap = nullptr;
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        int leaf_bps = 0, m2l_bps = 0;
    } g[3][2];   // [precision][adjoint]
    std::vector<void *> allocs;
};

namespace bc {
namespace {

int tune_key(int prec, int adj, int64_t nleaf)
{
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= nleaf) lg++;
    return prec * 1024 + adj * 512 + lg;
}

bc_status batch_capture(bc_batch *b, int prec, int adj, int leaf_bps, int m2l_bps, cudaGraphExec_t *out)
{
    bc_ctx *ctx = b->ctx;
    PassArgs a = pass_args(ctx, b->u);
    a.leaf_bps = leaf_bps;
    if (m2l_bps) a.m2l_bps = m2l_bps;
    const int parts = split_parts_for(prec, ctx->split_parts);
    const int ov = ctx->split_overlap;
    const bool side = ov == 1 || (ov == 2 && !adj) || (ov == 3 && adj);
    SplitLaunch sl{&ctx->split, &b->u->sp, parts, side ? &ctx->side : nullptr, near_ctas_for(ctx, parts)};
    if (is_split(prec) && (parts & 32)) {   // before the capture: it allocates
        bc_status s = build_split_m2l(b->u);
        if (s != BC_OK) return s;
    }
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "batch: begin capture");
    cudaError_t le = launch_apply(a, b->u->h, b->u->d, ctx->dt, adj != 0, b->in_buf, b->out_buf, b->cap, 3, nullptr,
                                  ctx->m2l_tri, is_split(prec) ? &sl : nullptr);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le, "batch: capture launch");
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch: end capture");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return e == cudaSuccess ? BC_OK : cuda_fail(e, "batch: instantiate");
}

bc_status batch_copy(bc_batch *b, const double *const *in, double *const *out, bool gather, cudaStream_t st)
{
    const int n = int(b->trees.size());
    for (int k0 = 0; k0 < n; k0 += kBatchChunk) {
        BatchPtrs bp{};
        bp.n = std::min(kBatchChunk, n - k0);
        for (int i = 0; i < bp.n; i++) {
            bp.in[i] = gather ? in[k0 + i] : nullptr;
            bp.out[i] = gather ? nullptr : out[k0 + i];
            bp.off[i] = b->leaf_offset[k0 + i];
        }
        bp.off[bp.n] = b->leaf_offset[k0 + bp.n];
        cudaError_t e = launch_batch_copy(bp, gather, gather ? b->in_buf : b->out_buf, b->ctx->NP, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch: copy launch");
    }
    return BC_OK;
}

}  // namespace
}  // namespace bc

using namespace bc;

extern "C" {

const char *bc_last_error(void) { return g_err; }

bc_status bc_create(const bc_config *cfg, int device, bc_ctx **out)
{
    if (!cfg || !out) { set_error("bc_create: NULL argument"); return BC_ERR_ARG; }
    *out = nullptr;
    if (cfg->p < 4 || cfg->p > kMaxP) { set_error("bc_create: p must be in [4, %d]", kMaxP); return BC_ERR_ARG; }
    int nterms = cfg->nterms ? cfg->nterms : kDefaultNterms;
    if (nterms < 4 || nterms > 32) { set_error("bc_create: nterms must be in [4, 32]"); return BC_ERR_ARG; }
    if (cfg->node_kind != 0 && cfg->node_kind != 1) { set_error("bc_create: only first-kind Chebyshev nodes (node_kind 1) are provided"); return BC_ERR_UNSUPPORTED; }
    if (cfg->split_slices < 0 || cfg->split_slices > 8) { set_error("bc_create: split_slices must be in [0, 8]"); return BC_ERR_ARG; }
    if (device != -1) {
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess) return cuda_fail(e, "bc_create: cudaGetDeviceCount");
        if (device < 0 || device >= ndev) { set_error("bc_create: device %d not present (%d devices)", device, ndev); return BC_ERR_ARG; }
    }
    bc_ctx *c = new (std::nothrow) bc_ctx();
    if (!c) { set_error("bc_create: out of host memory"); return BC_ERR_OOM; }
    c->cfg = *cfg;
    c->cfg.nterms = nterms;
    c->cfg.node_kind = 1;
    c->device = device;
    c->p = cfg->p;
    c->NP = cfg->p * cfg->p;
    c->P1 = nterms;
    *out = c;
    return BC_OK;
}

void bc_destroy(bc_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->device >= 0) cudaSetDevice(ctx->device);
    for (auto &dir : ctx->ev)
        for (auto &e : dir)
            if (e) cudaEventDestroy(e);
    if (ctx->side.fork) cudaEventDestroy(ctx->side.fork);
    if (ctx->side.join) cudaEventDestroy(ctx->side.join);
    if (ctx->side.xdone) cudaEventDestroy(ctx->side.xdone);
    if (ctx->side.side) cudaStreamDestroy(ctx->side.side);
    free_all(ctx->dt.allocs);
    free_all(ctx->split_allocs);
    delete ctx;
}

bc_status bc_tables_build(bc_ctx *ctx, const char *cache_dir)
{
    if (!ctx) { set_error("bc_tables_build: NULL context"); return BC_ERR_ARG; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->tables_ready) return BC_OK;
    bc_status s = build_tables(ctx->ht, ctx->p, ctx->P1, cache_dir);
    if (s != BC_OK) return s;
    OpBuild F, A;
    build_opsets(ctx->ht, F, A);
    if (ctx->device < 0) {
        // host-only: the factored shifts are built and checked against the
        // dense operators all the same (nothing is uploaded)
        for (int adj = 0; adj < 2; adj++) {
            ShiftFacHost fu, fp;
            const OpBuild &b = adj ? A : F;
            if ((s = build_shift_fac(ctx->P1, false, adj != 0, b.up, fu)) != BC_OK ||
                (s = build_shift_fac(ctx->P1, true, adj != 0, b.par, fp)) != BC_OK)
                return s;
        }
        ctx->tables_ready = true;
        return BC_OK;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if ((s = upload_opset(ctx->dt, ctx->dt.fwd, F, false)) != BC_OK) return s;
    if ((s = upload_opset(ctx->dt, ctx->dt.adj, A, true)) != BC_OK) return s;
    e = dev_upload(ctx->dt.allocs, &ctx->dt.wvec, ctx->ht.w.data(), ctx->ht.w.size());
    if (e != cudaSuccess) return cuda_fail(e, "tables upload");
    {
        // factored M2L: d = 2(dx + i dy) per code
        const int P1 = ctx->P1;
        std::vector<double2> df(size_t(kNumV) * P1, make_double2(0, 0)), da(df.size(), make_double2(0, 0));
        std::vector<double2> sf(df.size(), make_double2(0, 0)), sa(df.size(), make_double2(0, 0));
        std::vector<double> ld(kNumV, 0.0);
        for (int c = 0; c < kNumV; c++) {
            int dx = c % 7 - 3, dy = c / 7 - 3;
            if (std::max(std::abs(dx), std::abs(dy)) < 2) continue;
            std::complex<long double> d(2.0L * dx, 2.0L * dy), inv = 1.0L / d, pw = 1.0L;
            ld[c] = std::log(std::abs(std::complex<double>(2.0 * dx, 2.0 * dy)));
            for (int k = 0; k < P1; k++) {
                const double sg = (k & 1) ? -1.0 : 1.0;
                df[size_t(c) * P1 + k] = make_double2(double(pw.real()), double(pw.imag()));
                da[size_t(c) * P1 + k] = make_double2(double(pw.real()), -double(pw.imag()));
                sf[size_t(c) * P1 + k] = make_double2(sg * double(pw.real()), sg * double(pw.imag()));
                sa[size_t(c) * P1 + k] = make_double2(sg * double(pw.real()), -sg * double(pw.imag()));
                pw *= inv;
            }
        }
        if ((e = dev_upload(ctx->dt.allocs, &ctx->dt.dpow_f, df.data(), df.size())) != cudaSuccess ||
            (e = dev_upload(ctx->dt.allocs, &ctx->dt.dpow_a, da.data(), da.size())) != cudaSuccess ||
            (e = dev_upload(ctx->dt.allocs, &ctx->dt.dsig_f, sf.data(), sf.size())) != cudaSuccess ||
            (e = dev_upload(ctx->dt.allocs, &ctx->dt.dsig_a, sa.data(), sa.size())) != cudaSuccess ||
            (e = dev_upload(ctx->dt.allocs, &ctx->dt.logd, ld.data(), ld.size())) != cudaSuccess)
            return cuda_fail(e, "tables upload");
    }
    e = dev_upload<int32_t>(ctx->dt.allocs, &ctx->dev_err, nullptr, 1);
    if (e != cudaSuccess) return cuda_fail(e, "error flag");
    // two upward blocks per SM leave room for a tensor-core CTA beside them
    {
        const OpSet &F = ctx->dt.fwd, &A = ctx->dt.adj;
        const int fT = std::max(std::max(F.up_f.T, A.up_f.T), std::max(F.par_f.T, A.par_f.T));
        const int fm = std::max(std::max(F.up_f.maxp, A.up_f.maxp), std::max(F.par_f.maxp, A.par_f.maxp));
        e = fp64_prepare(ctx->NP, ctx->P1, std::max(F.up_s.T, A.up_s.T), std::max(F.up_s.maxp, A.up_s.maxp), fT, fm,
                         2, 4, &ctx->up_blocks, &ctx->shift_blocks, &ctx->down_blocks);
    }
    if (e != cudaSuccess) return cuda_fail(e, "FP64 kernel occupancy");
    s = build_split_tables(ctx);
    if (s != BC_OK) return s;
    ctx->tables_ready = true;
    return BC_OK;
}

bc_status bc_tree_create(bc_ctx *ctx, double x0, double y0, double L, int64_t nleaf, const int32_t *level,
                         const int32_t *ix, const int32_t *iy, bc_tree **out)
{
    if (!ctx || !out) { set_error("bc_tree_create: NULL argument"); return BC_ERR_ARG; }
    *out = nullptr;
    bc_tree *t = new (std::nothrow) bc_tree();
    if (!t) { set_error("bc_tree_create: out of host memory"); return BC_ERR_OOM; }
    t->ctx = ctx;
    bc_status s = build_host_tree(t->h, x0, y0, L, ctx->p, nleaf, level, ix, iy);
    if (s != BC_OK) { delete t; return s; }
    return finish_tree(ctx, out, t);
}

bc_status bc_tree_refine(bc_ctx *ctx, double x0, double y0, double L, bc_density_fn fn, void *user, double eps,
                         int max_level, bc_tree **out)
{
    if (!ctx || !out) { set_error("bc_tree_refine: NULL argument"); return BC_ERR_ARG; }
    *out = nullptr;
    std::vector<int32_t> lv, ix, iy;
    bc_status s = refine_leaves(ctx->p, x0, y0, L, fn, user, eps, max_level, lv, ix, iy);
    if (s != BC_OK) return s;
    return bc_tree_create(ctx, x0, y0, L, int64_t(lv.size()), lv.data(), ix.data(), iy.data(), out);
}

bc_status bc_tree_refine_truncated(bc_ctx *ctx, double x0, double y0, double L, bc_density_fn fn, void *user,
                                   double eps, int max_level, const double *gamma, int64_t n_gamma,
                                   const double *gamma_b, int64_t n_gamma_b, bc_tree **out)
{
    if (!ctx || !out || !gamma || !gamma_b) { set_error("bc_tree_refine_truncated: NULL argument"); return BC_ERR_ARG; }
    *out = nullptr;
    if (n_gamma < 3 || n_gamma_b < 3 || n_gamma > (int64_t(1) << 24) || n_gamma_b > (int64_t(1) << 24)) {
        set_error("bc_tree_refine_truncated: each curve needs 3 .. 2^24 vertices");
        return BC_ERR_ARG;
    }
    for (int64_t i = 0; i < 2 * n_gamma; i++)
        if (!std::isfinite(gamma[i])) { set_error("bc_tree_refine_truncated: non-finite vertex"); return BC_ERR_ARG; }
    for (int64_t i = 0; i < 2 * n_gamma_b; i++)
        if (!std::isfinite(gamma_b[i])) { set_error("bc_tree_refine_truncated: non-finite vertex"); return BC_ERR_ARG; }
    Truncation tr;
    tr.gamma = Polygon{gamma, n_gamma};
    tr.gamma_b = Polygon{gamma_b, n_gamma_b};
    for (int64_t i = 0; i < n_gamma_b; i++)
        if (!polygon_contains(tr.gamma, gamma_b[2 * i], gamma_b[2 * i + 1])) {
            set_error("bc_tree_refine_truncated: vertex %lld of the bulk curve lies outside the domain",
                      (long long)i);
            return BC_ERR_ARG;
        }
    for (int64_t i = 0; i < n_gamma; i++)
        if (!(gamma[2 * i] >= x0 && gamma[2 * i] <= x0 + L && gamma[2 * i + 1] >= y0 && gamma[2 * i + 1] <= y0 + L)) {
            set_error("bc_tree_refine_truncated: the domain must lie in the root box");
            return BC_ERR_ARG;
        }
    std::vector<int32_t> lv, ix, iy;
    bc_status s = refine_leaves(ctx->p, x0, y0, L, fn, user, eps, max_level, lv, ix, iy, &tr);
    if (s != BC_OK) return s;
    bc_tree *t = new bc_tree;
    t->ctx = ctx;
    s = build_host_tree(t->h, x0, y0, L, ctx->p, int64_t(lv.size()), lv.data(), ix.data(), iy.data());
    if (s != BC_OK) { delete t; return s; }
    // each leaf's class; leaves outside the domain are discarded (Alg. 2)
    HostTree &h = t->h;
    h.gamma.assign(gamma, gamma + 2 * n_gamma);
    h.leaf_class.resize(h.nleaf);
    std::vector<uint8_t> act(h.nleaf);
    for (int64_t k = 0; k < h.nleaf; k++) {
        const double r = 0.5 * L / double(int64_t(1) << h.leaf_level[k]);
        const double cx = x0 + (2.0 * h.leaf_ix[k] + 1.0) * r, cy = y0 + (2.0 * h.leaf_iy[k] + 1.0) * r;
        const BoxSide sd = box_side(tr.gamma, cx - r, cx + r, cy - r, cy + r);
        h.leaf_class[k] = sd == BoxSide::Outside ? 0 : sd == BoxSide::Cut ? 1 : 2;
        act[k] = h.leaf_class[k] != 0;
    }
    drop_inactive(h, act);
    return finish_tree(ctx, out, t);
}

bc_status bc_tree_leaf_class(const bc_tree *tree, int8_t *cls)
{
    if (!tree || !cls) { set_error("bc_tree_leaf_class: NULL argument"); return BC_ERR_ARG; }
    for (int64_t k = 0; k < tree->h.nleaf; k++) cls[k] = tree->h.leaf_class.empty() ? 2 : tree->h.leaf_class[k];
    return BC_OK;
}

bc_status bc_tree_node_mask(const bc_tree *tree, uint8_t *mask)
{
    if (!tree || !mask) { set_error("bc_tree_node_mask: NULL argument"); return BC_ERR_ARG; }
    const HostTree &h = tree->h;
    const int p = h.p, NP = p * p;
    std::vector<double> xy(size_t(h.nleaf) * NP * 2);
    bc_status s = bc_tree_nodes(tree, xy.data());
    if (s != BC_OK) return s;
    const Polygon G{h.gamma.data(), int64_t(h.gamma.size() / 2)};
    for (int64_t k = 0; k < h.nleaf; k++) {
        const int c = h.leaf_class.empty() ? 2 : h.leaf_class[k];
        for (int j = 0; j < NP; j++) {
            const size_t i = size_t(k) * NP + j;
            mask[i] = c == 2 ? 1 : c == 0 ? 0 : uint8_t(polygon_contains(G, xy[2 * i], xy[2 * i + 1]));
        }
    }
    return BC_OK;
}

int64_t bc_tree_nleaf(const bc_tree *tree) { return tree ? tree->h.nleaf : 0; }

bc_status bc_tree_leaves(const bc_tree *tree, int32_t *level, int32_t *ix, int32_t *iy)
{
    if (!tree || !level || !ix || !iy) { set_error("bc_tree_leaves: NULL argument"); return BC_ERR_ARG; }
    std::copy(tree->h.leaf_level.begin(), tree->h.leaf_level.end(), level);
    std::copy(tree->h.leaf_ix.begin(), tree->h.leaf_ix.end(), ix);
    std::copy(tree->h.leaf_iy.begin(), tree->h.leaf_iy.end(), iy);
    return BC_OK;
}

bc_status bc_tree_nodes(const bc_tree *tree, double *xy)
{
    if (!tree || !xy) { set_error("bc_tree_nodes: NULL argument"); return BC_ERR_ARG; }
    const HostTree &h = tree->h;
    const int p = h.p;
    const double pi = 3.14159265358979323846;
    std::vector<double> xn(p);
    for (int m = 0; m < p; m++) xn[m] = -std::cos((2.0 * m + 1.0) * pi / (2.0 * p));
    for (int64_t k = 0; k < h.nleaf; k++) {
        double r = 0.5 * h.L / double(int64_t(1) << h.leaf_level[k]);
        double cx = h.x0 + (2.0 * h.leaf_ix[k] + 1.0) * r, cy = h.y0 + (2.0 * h.leaf_iy[k] + 1.0) * r;
        for (int jy = 0; jy < p; jy++)
            for (int jx = 0; jx < p; jx++) {
                size_t o = (size_t(k) * p * p + jy * p + jx) * 2;
                xy[o] = cx + r * xn[jx];
                xy[o + 1] = cy + r * xn[jy];
            }
    }
    return BC_OK;
}

bc_status bc_tree_stats_get(const bc_tree *tree, bc_tree_stats *out)
{
    if (!tree || !out) { set_error("bc_tree_stats_get: NULL argument"); return BC_ERR_ARG; }
    const HostTree &h = tree->h;
    out->nleaf = h.nleaf;
    out->nbox = int64_t(h.box_level.size());
    out->nlevels = h.nlevels;
    out->n_near = int64_t(h.near_src.size());
    out->n_v = int64_t(h.v_src.size());
    out->n_w = int64_t(h.w_src.size());
    out->n_x = int64_t(h.x_src.size());
    out->n_nonleaf = h.n_nonleaf;
    out->n_down = h.n_down;
    return BC_OK;
}

bc_status bc_tree_lists(const bc_tree *tree, int kind, int64_t *nrows, int64_t *nnz, int64_t *ptr, int64_t *idx,
                        int32_t *code)
{
    if (!tree || !nrows || !nnz) { set_error("bc_tree_lists: NULL argument"); return BC_ERR_ARG; }
    const HostTree &h = tree->h;
    const std::vector<int32_t> *P, *I, *C;
    switch (kind) {
    case 0: P = &h.near_ptr; I = &h.near_src; C = &h.near_tab; break;
    case 1: P = &h.v_ptr; I = &h.v_src; C = &h.v_code; break;
    case 2: P = &h.w_ptr; I = &h.w_src; C = &h.w_code; break;
    case 3: P = &h.x_ptr; I = &h.x_src; C = &h.x_code; break;
    default: set_error("bc_tree_lists: kind must be 0..3"); return BC_ERR_ARG;
    }
    *nrows = int64_t(P->size()) - 1;
    *nnz = int64_t(I->size());
    if (ptr) for (size_t i = 0; i < P->size(); i++) ptr[i] = (*P)[i];
    if (idx) for (size_t i = 0; i < I->size(); i++) idx[i] = (*I)[i];
    if (code) for (size_t i = 0; i < C->size(); i++) code[i] = (*C)[i];
    return BC_OK;
}

bc_status bc_tree_boxes(const bc_tree *tree, int32_t *level, int32_t *ix, int32_t *iy, int32_t *parent,
                        int32_t *leaf)
{
    if (!tree) { set_error("bc_tree_boxes: NULL tree"); return BC_ERR_ARG; }
    const HostTree &h = tree->h;
    if (level) std::copy(h.box_level.begin(), h.box_level.end(), level);
    if (ix) std::copy(h.box_ix.begin(), h.box_ix.end(), ix);
    if (iy) std::copy(h.box_iy.begin(), h.box_iy.end(), iy);
    if (parent) std::copy(h.box_parent.begin(), h.box_parent.end(), parent);
    if (leaf) std::copy(h.box_leaf.begin(), h.box_leaf.end(), leaf);
    return BC_OK;
}

void bc_tree_destroy(bc_tree *tree)
{
    if (!tree) return;
    if (tree->ctx->device >= 0) cudaSetDevice(tree->ctx->device);
    free_all(tree->d.allocs);
    delete tree;
}

bc_status bc_apply(bc_ctx *ctx, const bc_tree *tree, const double *f, double *u, bc_precision prec, void *stream)
{
    return apply_impl(ctx, tree, f, u, prec, stream, false);
}

bc_status bc_apply_adjoint(bc_ctx *ctx, const bc_tree *tree, const double *g, double *h, bc_precision prec,
                           void *stream)
{
    return apply_impl(ctx, tree, g, h, prec, stream, true);
}

bc_status bc_eval_points_grad(bc_ctx *ctx, const bc_tree *tree, const double *u, const double *xy, int64_t n,
                              double *val, double *grad, void *stream)
{
    if (!ctx || !tree || (n > 0 && (!u || !xy || !val || !grad)) || n < 0) {
        set_error("bc_eval_points_grad: bad argument");
        return BC_ERR_ARG;
    }
    if (tree->ctx != ctx) { set_error("bc_eval_points_grad: tree belongs to another context"); return BC_ERR_ARG; }
    if (ctx->device < 0) { set_error("bc_eval_points_grad: host-only context (device -1)"); return BC_ERR_STATE; }
    if (n == 0) return BC_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PassArgs a = pass_args(ctx, tree);
    const HostTree &h = tree->h;
    const bool du = is_device_ptr(u), dx = is_device_ptr(xy), dv = is_device_ptr(val), dg = is_device_ptr(grad);
    if (du && dx && dv && dg) {
        e = launch_eval_points_grad(a, tree->d, u, xy, n, val, grad, h.x0, h.y0, h.L, st);
        return e == cudaSuccess ? BC_OK : cuda_fail(e, "eval launch");
    }
    if (du || dx || dv || dg) {
        set_error("bc_eval_points_grad: u, xy, val and grad must all be device or all host memory");
        return BC_ERR_ARG;
    }
    for (int64_t k = 0; k < n; k++) {
        const double x = xy[2 * k], y = xy[2 * k + 1];
        if (!(x >= h.x0 && x <= h.x0 + h.L && y >= h.y0 && y <= h.y0 + h.L)) {
            set_error("bc_eval_points_grad: point %lld outside the root box", (long long)k);
            return BC_ERR_ARG;
        }
    }
    const size_t nu = size_t(h.nleaf) * ctx->NP;
    double *du_ = nullptr, *dxy = nullptr, *dval = nullptr, *dgrad = nullptr;
    std::vector<void *> tmp;
    if ((e = dev_upload(tmp, &du_, u, nu)) != cudaSuccess || (e = dev_upload(tmp, &dxy, xy, size_t(2 * n))) != cudaSuccess ||
        (e = dev_upload<double>(tmp, &dval, nullptr, size_t(n))) != cudaSuccess ||
        (e = dev_upload<double>(tmp, &dgrad, nullptr, size_t(2 * n))) != cudaSuccess) {
        free_all(tmp);
        return cuda_fail(e, "eval staging");
    }
    e = launch_eval_points_grad(a, tree->d, du_, dxy, n, dval, dgrad, h.x0, h.y0, h.L, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(val, dval, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, dgrad, size_t(2 * n) * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free_all(tmp);
    return e == cudaSuccess ? BC_OK : cuda_fail(e, "eval");
}

bc_status bc_eval_points(bc_ctx *ctx, const bc_tree *tree, const double *u, const double *xy, int64_t n,
                         double *out, void *stream)
{
    if (!ctx || !tree || (n > 0 && (!u || !xy || !out)) || n < 0) { set_error("bc_eval_points: bad argument"); return BC_ERR_ARG; }
    if (tree->ctx != ctx) { set_error("bc_eval_points: tree belongs to another context"); return BC_ERR_ARG; }
    if (ctx->device < 0) { set_error("bc_eval_points: host-only context (device -1)"); return BC_ERR_STATE; }
    if (n == 0) return BC_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PassArgs a = pass_args(ctx, tree);
    const HostTree &h = tree->h;
    bool du = is_device_ptr(u), dx = is_device_ptr(xy), dout = is_device_ptr(out);
    if (du && dx && dout) {
        e = launch_eval_points(a, tree->d, u, xy, n, out, h.x0, h.y0, h.L, st);
        return e == cudaSuccess ? BC_OK : cuda_fail(e, "eval launch");
    }
    if (du || dx || dout) { set_error("bc_eval_points: u, xy and out must all be device or all host memory"); return BC_ERR_ARG; }
    for (int64_t k = 0; k < n; k++) {
        double x = xy[2 * k], y = xy[2 * k + 1];
        if (!(x >= h.x0 && x <= h.x0 + h.L && y >= h.y0 && y <= h.y0 + h.L)) {
            set_error("bc_eval_points: point %lld outside the root box", (long long)k);
            return BC_ERR_ARG;
        }
    }
    size_t nu = size_t(h.nleaf) * ctx->NP;
    double *du_ = nullptr, *dxy = nullptr, *dout_ = nullptr;
    std::vector<void *> tmp;
    if ((e = dev_upload(tmp, &du_, u, nu)) != cudaSuccess ||
        (e = dev_upload(tmp, &dxy, xy, size_t(2 * n))) != cudaSuccess ||
        (e = dev_upload<double>(tmp, &dout_, nullptr, size_t(n))) != cudaSuccess) {
        free_all(tmp);
        return cuda_fail(e, "eval staging");
    }
    e = launch_eval_points(a, tree->d, du_, dxy, n, dout_, h.x0, h.y0, h.L, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout_, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free_all(tmp);
    return e == cudaSuccess ? BC_OK : cuda_fail(e, "eval");
}

bc_status bc_batch_create(bc_ctx *ctx, const bc_tree *const *trees, int n, bc_batch **out)
{
    if (!ctx || !trees || n <= 0 || !out) { set_error("bc_batch_create: bad argument"); return BC_ERR_ARG; }
    *out = nullptr;
    if (ctx->device < 0) { set_error("bc_batch_create: host-only context"); return BC_ERR_STATE; }
    if (!ctx->tables_ready) { set_error("bc_batch_create: call bc_tables_build first"); return BC_ERR_STATE; }
    std::vector<const HostTree *> hs;
    for (int k = 0; k < n; k++) {
        if (!trees[k] || trees[k]->ctx != ctx) { set_error("bc_batch_create: tree %d missing or from another context", k); return BC_ERR_ARG; }
        hs.push_back(&trees[k]->h);
    }
    bc_batch *b = new (std::nothrow) bc_batch();
    if (!b) { set_error("bc_batch_create: out of host memory"); return BC_ERR_OOM; }
    b->ctx = ctx;
    b->trees.assign(trees, trees + n);
    b->u = new (std::nothrow) bc_tree();
    if (!b->u) { delete b; set_error("bc_batch_create: out of host memory"); return BC_ERR_OOM; }
    b->u->ctx = ctx;
    b->u->is_union = true;
    bc_status s = merge_host_trees(hs, b->u->h, b->leaf_offset);
    cudaError_t e = cudaSuccess;
    if (s == BC_OK) {
        e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaSetDevice");
    }
    if (s == BC_OK) s = upload_tree(b->u);
    const size_t nv = size_t(b->u->h.nleaf) * ctx->NP;
    if (s == BC_OK && ((e = dev_upload<double>(b->allocs, &b->in_buf, nullptr, nv)) != cudaSuccess ||
                       (e = dev_upload<double>(b->allocs, &b->out_buf, nullptr, nv)) != cudaSuccess))
        s = cuda_fail(e, "batch buffers");
    if (s == BC_OK && ctx->split_ready) s = build_split_tree(b->u);
    if (s == BC_OK && (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
        s = cuda_fail(e, "batch stream");
    if (s != BC_OK) {
        bc_batch_destroy(b);
        return s;
    }
    *out = b;
    return BC_OK;
}

void bc_batch_destroy(bc_batch *b)
{
    if (!b) return;
    if (b->ctx && b->ctx->device >= 0) cudaSetDevice(b->ctx->device);
    for (auto &row : b->g)
        for (auto &gr : row)
            if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->u) {
        free_all(b->u->d.allocs);
        delete b->u;
    }
    free_all(b->allocs);
    delete b;
}

bc_status bc_batch_autotune(bc_ctx *ctx, bc_batch *b, bc_precision prec, void *stream)
{
    if (!ctx || !b || b->ctx != ctx) { set_error("bc_batch_autotune: bad argument"); return BC_ERR_ARG; }
    if (prec != BC_FP64 && !is_split(prec)) { set_error("bc_batch_autotune: unknown precision"); return BC_ERR_ARG; }
    if (is_split(prec) && !ctx->split_ready) { set_error("bc_batch_autotune: split precision needs p = 8, 12 or 16"); return BC_ERR_UNSUPPORTED; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    static const int cand[][2] = {{16, 12}, {8, 8}, {4, 4}, {16, 16}, {8, 12}, {32, 12}, {16, 6}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int adj = 0; adj < 2; adj++) {
        float best = 1e30f;
        cudaGraphExec_t best_exec = nullptr;
        int bl = 0, bm = 0;
        for (const auto &c : cand) {
            cudaGraphExec_t ex = nullptr;
            bc_status s = batch_capture(b, int(prec), adj, c[0], c[1], &ex);
            if (s != BC_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
            float ms = 1e30f;
            for (int rep = 0; rep < 4; rep++) {
                cudaEventRecord(e0, st);
                cudaGraphLaunch(ex, st);
                cudaEventRecord(e1, st);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) { cudaGraphExecDestroy(ex); cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_fail(e, "bc_batch_autotune"); }
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms = std::min(ms, t);
            }
            if (ms < best) {
                if (best_exec) cudaGraphExecDestroy(best_exec);
                best = ms; best_exec = ex; bl = c[0]; bm = c[1];
            } else {
                cudaGraphExecDestroy(ex);
            }
        }
        auto &g = b->g[int(prec)][adj];
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = best_exec; g.leaf_bps = bl; g.m2l_bps = bm;
        const int key = tune_key(int(prec), adj, b->u->h.nleaf);
        bool found = false;
        for (auto &kv : ctx->tuned)
            if (kv.first == key) { kv.second = {bl, bm}; found = true; }
        if (!found) ctx->tuned.push_back({key, {bl, bm}});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return BC_OK;
}

bc_status bc_batch_run(bc_ctx *ctx, bc_batch *b, const double *const *in, double *const *out, bc_precision prec,
                       int adjoint, void *stream)
{
    if (!ctx || !b || b->ctx != ctx || !in || !out) { set_error("bc_batch_run: bad argument"); return BC_ERR_ARG; }
    if (prec != BC_FP64 && !is_split(prec)) { set_error("bc_batch_run: unknown precision"); return BC_ERR_ARG; }
    if (is_split(prec) && !ctx->split_ready) { set_error("bc_batch_run: split precision needs p = 8, 12 or 16"); return BC_ERR_UNSUPPORTED; }
    const int n = int(b->trees.size());
    for (int k = 0; k < n; k++)
        if (!in[k] || !out[k] || !is_device_ptr(in[k]) || !is_device_ptr(out[k]) || in[k] == out[k]) {
            set_error("bc_batch_run: array %d must be distinct device memory", k);
            return BC_ERR_ARG;
        }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int adj = adjoint != 0;
    auto &g = b->g[int(prec)][adj];
    if (!g.exec) {
        if (ctx->cfg.autotune) {
            bc_status s = bc_batch_autotune(ctx, b, prec, stream);
            if (s != BC_OK) return s;
        } else {
            int lb = 0, mb = 0;
            const int key = tune_key(int(prec), adj, b->u->h.nleaf);
            for (auto &kv : ctx->tuned)
                if (kv.first == key) { lb = kv.second.first; mb = kv.second.second; }
            bc_status s = batch_capture(b, int(prec), adj, lb, mb, &g.exec);
            if (s != BC_OK) return s;
            g.leaf_bps = lb; g.m2l_bps = mb;
        }
    }
    bc_status s = batch_copy(b, in, nullptr, true, st);
    if (s != BC_OK) return s;
    e = cudaGraphLaunch(g.exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "bc_batch_run: graph launch");
    return batch_copy(b, nullptr, out, false, st);
}

int64_t bc_batch_nleaf(const bc_batch *b) { return b ? b->u->h.nleaf : 0; }

bc_status bc_batch_shape(const bc_batch *b, int precision, int adjoint, int *leaf_blocks_per_sm, int *m2l_blocks_per_sm)
{
    if (!b || precision < 0 || precision > 2 || !leaf_blocks_per_sm || !m2l_blocks_per_sm) { set_error("bc_batch_shape: bad argument"); return BC_ERR_ARG; }
    const auto &g = b->g[precision][adjoint != 0];
    *leaf_blocks_per_sm = g.leaf_bps;
    *m2l_blocks_per_sm = g.m2l_bps;
    return BC_OK;
}

bc_status bc_table_export(const bc_ctx *ctx, int which, int64_t *count, double *out)
{
    if (!ctx || !count) { set_error("bc_table_export: NULL argument"); return BC_ERR_ARG; }
    if (!ctx->tables_ready) { set_error("bc_table_export: tables not built"); return BC_ERR_STATE; }
    const HostTables &h = ctx->ht;
    const std::vector<double> *v[] = {&h.nodes, &h.w, &h.T, &h.Q, &h.E, &h.M2M, &h.L2L, &h.M2L, &h.M2P, &h.P2L};
    if (which < 0 || which >= int(sizeof(v) / sizeof(v[0]))) { set_error("bc_table_export: which must be 0..9"); return BC_ERR_ARG; }
    *count = int64_t(v[which]->size());
    if (out) std::copy(v[which]->begin(), v[which]->end(), out);
    return BC_OK;
}

bc_status bc_debug_up_schedule(const bc_ctx *ctx, int adjoint, int32_t *T, int32_t *maxp, uint32_t *code,
                               float *ops, int32_t *np)
{
    if (!ctx || !T || !maxp) { set_error("bc_debug_up_schedule: NULL argument"); return BC_ERR_ARG; }
    if (!ctx->tables_ready) { set_error("bc_debug_up_schedule: tables not built"); return BC_ERR_STATE; }
    OpBuild F, A;
    build_opsets(ctx->ht, F, A);
    const UpScheduleHost us = build_up_schedule(adjoint ? A.up : F.up);
    *T = us.T;
    *maxp = us.maxp;
    if (code) std::copy(us.code.begin(), us.code.end(), code);
    if (ops)
        for (size_t i = 0; i < us.ops.size(); i++) {
            ops[4 * i] = us.ops[i].x;
            ops[4 * i + 1] = us.ops[i].y;
            ops[4 * i + 2] = us.ops[i].z;
            ops[4 * i + 3] = us.ops[i].w;
        }
    if (np) std::copy(us.np.begin(), us.np.end(), np);
    return BC_OK;
}

bc_status bc_debug_set(bc_ctx *ctx, int pass_mask, int timing)
{
    if (!ctx || pass_mask < 0 || pass_mask > 3) { set_error("bc_debug_set: bad argument"); return BC_ERR_ARG; }
    if (ctx->device < 0) { set_error("bc_debug_set: host-only context"); return BC_ERR_STATE; }
    ctx->pass_mask = pass_mask;
    if (timing && !ctx->ev[0][0]) {
        cudaError_t e = cudaSetDevice(ctx->device);
        for (int d = 0; d < 2; d++)
            for (int i = 0; e == cudaSuccess && i < kNumEvents; i++) e = cudaEventCreate(&ctx->ev[d][i]);
        if (e != cudaSuccess) return cuda_fail(e, "bc_debug_set: events");
    }
    ctx->timing = timing != 0;
    return BC_OK;
}

bc_status bc_set_option(bc_ctx *ctx, const char *name, double value)
{
    if (!ctx || !name) { set_error("bc_set_option: NULL argument"); return BC_ERR_ARG; }
    if (std::strcmp(name, "m2l_triangular") == 0) {
        ctx->m2l_tri = value != 0.0;
        return BC_OK;
    }
    if (std::strcmp(name, "wait_limit") == 0) {
        if (!(value >= 1.0 && value <= 1e15)) { set_error("bc_set_option: wait_limit must be in [1, 1e15]"); return BC_ERR_ARG; }
        ctx->split.wait_limit = (long long)value;
        return BC_OK;
    }
    if (std::strcmp(name, "split_overlap") == 0) {
        if (!(value >= 0.0 && value <= 3.0) || value != std::floor(value)) {
            set_error("bc_set_option: split_overlap must be 0, 1, 2 or 3");
            return BC_ERR_ARG;
        }
        ctx->split_overlap = int(value);
        return BC_OK;
    }
    if (std::strcmp(name, "split_overlap_ctas") == 0) {
        if (!(value >= 0.0 && value <= 65536.0) || value != std::floor(value)) {
            set_error("bc_set_option: split_overlap_ctas must be an integer in [0, 65536]");
            return BC_ERR_ARG;
        }
        ctx->overlap_ctas = int(value);
        return BC_OK;
    }
    if (std::strcmp(name, "m2l_kernel") == 0) {
        if (value != 0.0 && value != 1.0) {
            set_error("bc_set_option: m2l_kernel must be 0 (FP64 FMA) or 1 (FP64 tensor cores)");
            return BC_ERR_ARG;
        }
        ctx->m2l_kind = int(value);
        return BC_OK;
    }
    if (std::strcmp(name, "m2l_blocks_per_sm") == 0) {
        if (!(value >= 0.0 && value <= 32.0) || value != std::floor(value)) {
            set_error("bc_set_option: m2l_blocks_per_sm must be an integer in [0, 32]");
            return BC_ERR_ARG;
        }
        ctx->m2l_bps = int(value);
        return BC_OK;
    }
    if (std::strcmp(name, "debug_split_parts") == 0) {
        if (!(value >= -1.0 && value <= double(kSplitAllParts)) || value != std::floor(value)) {
            set_error("bc_set_option: debug_split_parts must be an integer in [-1, %d]", kSplitAllParts);
            return BC_ERR_ARG;
        }
        ctx->split_parts = int(value);
        return BC_OK;
    }
    if (std::strcmp(name, "debug_withhold_copy") == 0) {
        ctx->split.withhold_copy = value != 0.0;
        return BC_OK;
    }
    set_error("bc_set_option: unknown option '%s'", name);
    return BC_ERR_ARG;
}

bc_status bc_debug_stage_times(bc_ctx *ctx, int adjoint, double *ms)
{
    if (!ctx || !ms) { set_error("bc_debug_stage_times: NULL argument"); return BC_ERR_ARG; }
    if (!ctx->timing) { set_error("bc_debug_stage_times: timing is off"); return BC_ERR_STATE; }
    cudaEvent_t *ev = ctx->ev[adjoint ? 1 : 0];
    cudaError_t e = cudaEventSynchronize(ev[7]);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[9]);
    for (int i = 0; e == cudaSuccess && i < kNumStages; i++) {
        float t = 0.0f;
        e = i < 7 ? cudaEventElapsedTime(&t, ev[i], ev[i + 1]) : cudaEventElapsedTime(&t, ev[8], ev[9]);
        ms[i] = t;
    }
    return e == cudaSuccess ? BC_OK : cuda_fail(e, "bc_debug_stage_times");
}

bc_status bc_sync(bc_ctx *ctx, void *stream)
{
    if (!ctx) { set_error("bc_sync: NULL context"); return BC_ERR_ARG; }
    if (ctx->device < 0) return BC_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "bc_sync");
    if (ctx->dev_err) {
        int32_t flag = 0;
        e = cudaMemcpy(&flag, ctx->dev_err, sizeof(flag), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "bc_sync");
        if (flag) {
            cudaMemset(ctx->dev_err, 0, sizeof(int32_t));
            // 1: tensor-core operand copy, 2: level-pass box flag
            static const char *what[] = {"", " (tensor-core operand copy)", " (level-pass box flag)"};
            set_error("bc_sync: a bounded device-side wait gave up%s", what[flag >= 1 && flag <= 2 ? flag : 0]);
            return BC_ERR_TIMEOUT;
        }
    }
    return BC_OK;
}

}  // extern "C"
