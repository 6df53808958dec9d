// Host FP64 precompute of every table the box code applies.
//
// Near field.  For a source leaf with centre c and half-side r, and a target
// x = c + r*xi (paper Sec. 3.2, eq. (vbulk); Phi from Sec. 2):
//   (1/2pi) int_B log|x-y| f_B(y) dy
//      = r^2 * [ sum_j T(xi)_j f_j  +  log(r)/(2pi) * sum_j w_j f_j ],
//   T(xi)_j = (1/2pi) int_{[-1,1]^2} log|xi - eta| l_j(eta) d eta,
// l_j the tensor Lagrange basis of the first-kind nodes and w_j = int l_j.
// Under 2:1 balance the target leaf sits at one of 33 positions relative to
// a touching (or identical) source leaf, so T is tabulated at the nodes of
// those 33 target boxes.  Each entry is integrated directly against the
// Lagrange basis (barycentric form) by recursive subdivision of the square: a rectangle R is
// integrated with a 20x20 Gauss-Legendre rule once dist(xi,R) >= diam(R),
// otherwise split in four; rectangles of diameter < 1e-9 next to xi are
// dropped (|contribution| <= diam^2 |log diam| < 1e-16).
//
// Far field.  Complex-variable Laplace expansions in scaled form (box
// half-side r as the unit), so that every translation operator is the same
// at every level and only the log(r) terms depend on the level:
//   multipole  phi(z) = A_0 log(z-c) + sum_{k>=1} A_k (r/(z-c))^k,
//              A_0 = (1/2pi) int f,  A_k = -(1/(2pi k)) int ((y-c)/r)^k f
//   local      psi(z) = sum_l B_l ((z-c)/r)^l, potential = Re psi.
// M2M/L2L between a box and its children (child centre c + r_c*delta,
// delta = +-1 +- i), M2L between same-level boxes at offset d = (c_s-c_t)/r,
// the W-list evaluation of a finer box's multipole at leaf nodes (M2P) and the
// X-list conversion of a coarser leaf's density to a local expansion (P2L).
// The k = 0 / l = 0 log terms use log|.| (the imaginary parts of A_0 and B_0
// never reach Re psi).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>

#include "bc_internal.h"

namespace bc {

namespace {

using cplx = std::complex<double>;
constexpr double kPi = 3.14159265358979323846264338327950288;

struct Rule { std::vector<double> x, w; };

Rule gauss_legendre(int n)
{
    Rule g;
    g.x.resize(n); g.w.resize(n);
    for (int i = 0; i < n; i++) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; k++) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        g.x[n - 1 - i] = z;
        g.w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return g;
}

inline void chebT(int n, double x, double *T)
{
    T[0] = 1.0;
    if (n > 1) T[1] = x;
    for (int k = 2; k < n; k++) T[k] = 2.0 * x * T[k - 1] - T[k - 2];
}

// Node-value -> Chebyshev-coefficient map of the first-kind grid:
// c_a = sum_m C1[a*p + m] v_m.
std::vector<double> coef_map(int p, const std::vector<double> &xn)
{
    std::vector<double> C1(p * p), T(p);
    for (int m = 0; m < p; m++) {
        chebT(p, xn[m], T.data());
        for (int a = 0; a < p; a++) C1[a * p + m] = (a == 0 ? 1.0 : 2.0) / p * T[a];
    }
    return C1;
}

// First-kind barycentric weights (-1)^m sin(theta_m) for the ascending nodes.
struct Bary {
    int p;
    std::vector<double> x, lam;
};

// l_m(x) for all m by the barycentric formula (stable on Chebyshev grids).
void lagrange_bary(const Bary &B, double x, double *l)
{
    int hit = -1;
    double den = 0.0;
    for (int m = 0; m < B.p; m++) {
        double d = x - B.x[m];
        if (d == 0.0) { hit = m; break; }
        l[m] = B.lam[m] / d;
        den += l[m];
    }
    for (int m = 0; m < B.p; m++) l[m] = hit >= 0 ? (m == hit ? 1.0 : 0.0) : l[m] / den;
}

struct MomentCtx {
    const Bary *B;
    const Rule *g;
    double xi, eta;
    double *Trow;   // [jy*p + jx]: int log|xi - eta| l_jx(eta_1) l_jy(eta_2)
};

void moments_rect(const MomentCtx &c, double x0, double x1, double y0, double y1)
{
    const int p = c.B->p, n = int(c.g->x.size());
    double hx = 0.5 * (x1 - x0), hy = 0.5 * (y1 - y0);
    std::vector<double> Lu(n * p), Lv(n * p), v(n), S(p);
    for (int r = 0; r < n; r++) {
        v[r] = y0 + hy * (c.g->x[r] + 1.0);
        lagrange_bary(*c.B, v[r], &Lv[r * p]);
    }
    for (int q = 0; q < n; q++) {
        double u = x0 + hx * (c.g->x[q] + 1.0);
        lagrange_bary(*c.B, u, &Lu[q * p]);
        std::fill(S.begin(), S.end(), 0.0);
        double du = u - c.xi;
        for (int r = 0; r < n; r++) {
            double dv = v[r] - c.eta;
            double lg = 0.5 * std::log(du * du + dv * dv) * c.g->w[r] * hy;
            for (int b = 0; b < p; b++) S[b] += lg * Lv[r * p + b];
        }
        double wq = c.g->w[q] * hx;
        for (int b = 0; b < p; b++) {
            double sb = wq * S[b];
            for (int a = 0; a < p; a++) c.Trow[b * p + a] += sb * Lu[q * p + a];
        }
    }
}

void moments_rec(const MomentCtx &c, double x0, double x1, double y0, double y1)
{
    double diam = std::hypot(x1 - x0, y1 - y0);
    double dx = c.xi < x0 ? x0 - c.xi : (c.xi > x1 ? c.xi - x1 : 0.0);
    double dy = c.eta < y0 ? y0 - c.eta : (c.eta > y1 ? c.eta - y1 : 0.0);
    double dist = std::hypot(dx, dy);
    if (dist >= diam) { moments_rect(c, x0, x1, y0, y1); return; }
    if (diam < 1e-9) return;
    double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1);
    moments_rec(c, x0, xm, y0, ym);
    moments_rec(c, xm, x1, y0, ym);
    moments_rec(c, x0, xm, ym, y1);
    moments_rec(c, xm, x1, ym, y1);
}

template <class F>
void parallel_for(int64_t n, F fn)
{
    unsigned nt = std::max(1u, std::thread::hardware_concurrency());
    nt = std::min<unsigned>(nt, 64);
    std::vector<std::thread> th;
    std::atomic<int64_t> next{0};
    for (unsigned t = 0; t < nt; t++)
        th.emplace_back([&]() {
            for (;;) {
                int64_t i = next.fetch_add(1);
                if (i >= n) break;
                fn(i);
            }
        });
    for (auto &x : th) x.join();
}

uint64_t fnv1a(const void *data, size_t n, uint64_t h)
{
    const unsigned char *b = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; i++) { h ^= b[i]; h *= 1099511628211ull; }
    return h;
}

constexpr uint32_t kCacheVersion = 4;

std::vector<std::vector<double> *> table_fields(HostTables &ht)
{
    return {&ht.nodes, &ht.w, &ht.T, &ht.Q, &ht.E, &ht.M2M, &ht.L2L, &ht.M2L, &ht.M2P, &ht.P2L};
}

std::string cache_path(const char *dir, int p, int P1)
{
    char name[128];
    std::snprintf(name, sizeof(name), "/boxcode_tables_p%d_n%d_k1_v%u.bin", p, P1, kCacheVersion);
    return std::string(dir) + name;
}

bool cache_load(HostTables &ht, const char *dir)
{
    if (!dir) return false;
    FILE *fp = std::fopen(cache_path(dir, ht.p, ht.P1).c_str(), "rb");
    if (!fp) return false;
    bool ok = true;
    uint64_t h = 14695981039346656037ull;
    uint32_t hdr[4];
    ok = std::fread(hdr, sizeof(hdr), 1, fp) == 1 && hdr[0] == 0x42435431u && hdr[1] == kCacheVersion &&
         int(hdr[2]) == ht.p && int(hdr[3]) == ht.P1;
    for (auto *v : table_fields(ht)) {
        if (!ok) break;
        uint64_t n = 0;
        ok = std::fread(&n, sizeof(n), 1, fp) == 1 && n < (uint64_t(1) << 32);
        if (!ok) break;
        v->resize(n);
        ok = std::fread(v->data(), sizeof(double), n, fp) == n;
        h = fnv1a(v->data(), n * sizeof(double), h);
    }
    uint64_t hs = 0;
    ok = ok && std::fread(&hs, sizeof(hs), 1, fp) == 1 && hs == h;
    std::fclose(fp);
    return ok;
}

void cache_store(HostTables &ht, const char *dir)
{
    if (!dir) return;
    std::string path = cache_path(dir, ht.p, ht.P1);
    std::string tmp = path + ".tmp" + std::to_string(uint64_t(std::hash<std::thread::id>()(std::this_thread::get_id())));
    FILE *fp = std::fopen(tmp.c_str(), "wb");
    if (!fp) return;
    uint32_t hdr[4] = {0x42435431u, kCacheVersion, uint32_t(ht.p), uint32_t(ht.P1)};
    bool ok = std::fwrite(hdr, sizeof(hdr), 1, fp) == 1;
    uint64_t h = 14695981039346656037ull;
    for (auto *v : table_fields(ht)) {
        uint64_t n = v->size();
        ok = ok && std::fwrite(&n, sizeof(n), 1, fp) == 1;
        ok = ok && std::fwrite(v->data(), sizeof(double), n, fp) == n;
        h = fnv1a(v->data(), n * sizeof(double), h);
    }
    ok = ok && std::fwrite(&h, sizeof(h), 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    if (ok) std::rename(tmp.c_str(), path.c_str());
    else std::remove(tmp.c_str());
}

}  // namespace

bc_status build_tables(HostTables &ht, int p, int P1, const char *cache_dir)
{
    if (p < 4 || p > kMaxP || P1 < 4 || P1 > 64) {
        set_error("tables: p must be in [4,%d] and nterms in [4,64]", kMaxP);
        return BC_ERR_ARG;
    }
    ht = HostTables();
    ht.p = p; ht.P1 = P1; ht.NP = p * p;
    if (cache_load(ht, cache_dir)) return BC_OK;
    ht.p = p; ht.P1 = P1; ht.NP = p * p;
    const int NP = p * p;

    ht.nodes.resize(p);
    for (int m = 0; m < p; m++) ht.nodes[m] = -std::cos((2.0 * m + 1.0) * kPi / (2.0 * p));
    std::vector<double> C1 = coef_map(p, ht.nodes);
    // w_m = int l_m = sum_{a even} C1[a][m] * 2/(1-a^2)
    std::vector<double> w1(p, 0.0);
    for (int m = 0; m < p; m++)
        for (int a = 0; a < p; a += 2) w1[m] += C1[a * p + m] * 2.0 / (1.0 - double(a) * a);
    ht.w.resize(NP);
    for (int jy = 0; jy < p; jy++)
        for (int jx = 0; jx < p; jx++) ht.w[jy * p + jx] = w1[jx] * w1[jy];

    // ---------------- near tables ----------------
    ht.T.assign(size_t(kNumNear) * NP * NP, 0.0);
    const Rule g20 = gauss_legendre(20);
    Bary bary{p, ht.nodes, std::vector<double>(p)};
    for (int m = 0; m < p; m++) {
        double th = (2.0 * m + 1.0) * kPi / (2.0 * p);
        bary.lam[m] = ((m & 1) ? -1.0 : 1.0) * std::sin(th);
    }
    parallel_for(int64_t(kNumNear) * NP, [&](int64_t item) {
        int k = int(item / NP), i = int(item % NP);
        NearGeom geo = near_table_geometry(k);
        if (!geo.valid) return;
        double xi = geo.gx + geo.rho * ht.nodes[i % p];
        double eta = geo.gy + geo.rho * ht.nodes[i / p];
        double *row = &ht.T[(size_t(k) * NP + i) * NP];
        MomentCtx c{&bary, &g20, xi, eta, row};
        moments_rec(c, -1.0, 1.0, -1.0, 1.0);
        for (int j = 0; j < NP; j++) row[j] /= 2.0 * kPi;
    });

    // ---------------- far field ----------------
    std::vector<double> binom((2 * P1 + 2) * (2 * P1 + 2), 0.0);
    auto Bn = [&](int n, int k) -> double & { return binom[n * (2 * P1 + 2) + k]; };
    for (int n = 0; n < 2 * P1 + 2; n++) {
        Bn(n, 0) = 1.0;
        for (int k = 1; k <= n; k++) Bn(n, k) = Bn(n - 1, k - 1) + (k <= n - 1 ? Bn(n - 1, k) : 0.0);
    }
    auto put = [](std::vector<double> &v, size_t idx, cplx z) { v[2 * idx] = z.real(); v[2 * idx + 1] = z.imag(); };

    // P2M: Q[k][j] = int eta^k l_j (times -1/(2pi k), or w_j/(2pi) for k = 0)
    {
        const Rule g = gauss_legendre(64);
        const int n = 64;
        std::vector<double> L(n * p);   // L[q][m] = l_m(x_q)
        for (int q = 0; q < n; q++) lagrange_bary(bary, g.x[q], &L[q * p]);
        ht.Q.assign(size_t(2) * P1 * NP, 0.0);
        std::vector<cplx> S(size_t(n) * p * P1);   // S[q][jy][k] = sum_r w_r l_jy(y_r) z^k
        for (int q = 0; q < n; q++)
            for (int r = 0; r < n; r++) {
                cplx z(g.x[q], g.x[r]), zk(1.0, 0.0);
                for (int k = 0; k < P1; k++) {
                    for (int jy = 0; jy < p; jy++) S[(size_t(q) * p + jy) * P1 + k] += g.w[r] * L[r * p + jy] * zk;
                    zk *= z;
                }
            }
        for (int k = 0; k < P1; k++)
            for (int jy = 0; jy < p; jy++)
                for (int jx = 0; jx < p; jx++) {
                    cplx s = 0.0;
                    for (int q = 0; q < n; q++) s += g.w[q] * L[q * p + jx] * S[(size_t(q) * p + jy) * P1 + k];
                    cplx val = (k == 0) ? cplx(ht.w[jy * p + jx] / (2.0 * kPi), 0.0) : -s / (2.0 * kPi * k);
                    put(ht.Q, size_t(k) * NP + jy * p + jx, val);
                }
    }
    // L2P: E[j][l] = xi_j^l
    ht.E.assign(size_t(2) * NP * P1, 0.0);
    for (int j = 0; j < NP; j++) {
        cplx z(ht.nodes[j % p], ht.nodes[j / p]), zl(1.0, 0.0);
        for (int l = 0; l < P1; l++) { put(ht.E, size_t(j) * P1 + l, zl); zl *= z; }
    }
    // M2M and L2L for the four children q = qx + 2 qy, delta = (2qx-1) + i(2qy-1)
    ht.M2M.assign(size_t(2) * 4 * P1 * P1, 0.0);
    ht.L2L.assign(size_t(2) * 4 * P1 * P1, 0.0);
    for (int q = 0; q < 4; q++) {
        cplx delta(2.0 * (q & 1) - 1.0, 2.0 * (q >> 1) - 1.0);
        std::vector<cplx> dp(2 * P1 + 2), hp(2 * P1 + 2);   // delta^n, (delta/2)^n
        dp[0] = hp[0] = 1.0;
        for (int n = 1; n < 2 * P1 + 2; n++) { dp[n] = dp[n - 1] * delta; hp[n] = hp[n - 1] * (delta * 0.5); }
        size_t base = size_t(q) * P1 * P1;
        put(ht.M2M, base + 0, 1.0);
        for (int l = 1; l < P1; l++) {
            put(ht.M2M, base + size_t(l) * P1 + 0, -hp[l] / double(l));
            for (int k = 1; k <= l; k++)
                put(ht.M2M, base + size_t(l) * P1 + k, Bn(l - 1, k - 1) * std::ldexp(1.0, -l) * dp[l - k]);
        }
        for (int m = 0; m < P1; m++)
            for (int l = m; l < P1; l++)
                put(ht.L2L, base + size_t(m) * P1 + l, Bn(l, m) * std::ldexp(1.0, -l) * dp[l - m]);
    }
    // M2L for same-level offsets d = 2(dx + i dy), max(|dx|,|dy|) >= 2
    ht.M2L.assign(size_t(2) * kNumV * P1 * P1, 0.0);
    for (int dy = -3; dy <= 3; dy++)
        for (int dx = -3; dx <= 3; dx++) {
            if (std::max(std::abs(dx), std::abs(dy)) < 2) continue;
            cplx d(2.0 * dx, 2.0 * dy);
            size_t base = size_t(v_code(dx, dy)) * P1 * P1;
            std::vector<cplx> dinv(2 * P1 + 2);
            dinv[0] = 1.0;
            for (int n = 1; n < 2 * P1 + 2; n++) dinv[n] = dinv[n - 1] / d;
            put(ht.M2L, base + 0, std::log(std::abs(d)));
            for (int k = 1; k < P1; k++) put(ht.M2L, base + k, ((k & 1) ? -1.0 : 1.0) * dinv[k]);
            for (int l = 1; l < P1; l++) {
                put(ht.M2L, base + size_t(l) * P1 + 0, -dinv[l] / double(l));
                for (int k = 1; k < P1; k++)
                    put(ht.M2L, base + size_t(l) * P1 + k, ((k & 1) ? -1.0 : 1.0) * Bn(k + l - 1, l) * dinv[k + l]);
            }
        }
    // M2P (W list): node j of the target leaf, finer source box at offset d = (c_w-c_t)/r_t
    ht.M2P.assign(size_t(2) * kNumWX * NP * P1, 0.0);
    // P2L (X list): coarser source leaf, target box at offset e = (c_b-c_c)/r_c
    ht.P2L.assign(size_t(2) * kNumWX * P1 * NP, 0.0);
    const Rule g48 = gauss_legendre(48);
    std::vector<double> L48(48 * p);
    for (int q = 0; q < 48; q++) lagrange_bary(bary, g48.x[q], &L48[q * p]);
    for (int cy = 0; cy < 6; cy++)
        for (int cx = 0; cx < 6; cx++) {
            int d2x = 2 * cx - 5, d2y = 2 * cy - 5;
            if (std::max(std::abs(d2x), std::abs(d2y)) != 5) continue;
            int code = wx_code(d2x, d2y);
            cplx d(0.5 * d2x, 0.5 * d2y);
            for (int j = 0; j < NP; j++) {
                cplx z = cplx(ht.nodes[j % p], ht.nodes[j / p]) - d;
                cplx inv = 1.0 / (2.0 * z), pw = 1.0;
                size_t base = (size_t(code) * NP + j) * P1;
                put(ht.M2P, base, std::log(std::abs(z)));
                for (int k = 1; k < P1; k++) { pw *= inv; put(ht.M2P, base + k, pw); }
            }
            // P2L[l][j] = (1/2pi) int l_j(eta) g_l(eta), g_0 = log|e-eta|,
            // g_l = ((-1)^(l+1)/l) (2(e-eta))^(-l)
            std::vector<cplx> S(size_t(48) * p * P1, 0.0);   // S[q][jy][l]
            for (int q = 0; q < 48; q++)
                for (int r = 0; r < 48; r++) {
                    cplx z = d - cplx(g48.x[q], g48.x[r]);
                    cplx inv = 1.0 / (2.0 * z), pw = 1.0;
                    std::vector<cplx> gl(P1);
                    gl[0] = std::log(std::abs(z));
                    for (int l = 1; l < P1; l++) { pw *= inv; gl[l] = ((l & 1) ? 1.0 : -1.0) / double(l) * pw; }
                    for (int jy = 0; jy < p; jy++) {
                        double wl = g48.w[r] * L48[r * p + jy];
                        for (int l = 0; l < P1; l++) S[(size_t(q) * p + jy) * P1 + l] += wl * gl[l];
                    }
                }
            for (int l = 0; l < P1; l++)
                for (int jy = 0; jy < p; jy++)
                    for (int jx = 0; jx < p; jx++) {
                        cplx s = 0.0;
                        for (int q = 0; q < 48; q++) s += g48.w[q] * L48[q * p + jx] * S[(size_t(q) * p + jy) * P1 + l];
                        put(ht.P2L, (size_t(code) * P1 + l) * NP + jy * p + jx, s / (2.0 * kPi));
                    }
        }
    cache_store(ht, cache_dir);
    return BC_OK;
}

}  // namespace bc
