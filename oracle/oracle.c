/*
 * oracle.c -- plain, slow CPU FP64 oracle for the 2D free-space volume
 * potential on a quadtree of p x p Chebyshev leaves.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code
 * with the CUDA path (no headers, helpers or tables) and never calls it.
 *
 * What it computes (paper Sec. 3.2, eq. (vbulk) with the fundamental solution
 * Phi of Sec. 2):  v_bulk(x) = -int_{Omega_B} Phi(x,y) f(y) dy with
 * Phi(x,y) = (1/2pi) log(1/|x-y|), i.e.
 *
 *     u(x) = (1/2pi) * sum_{leaves B} int_B log|x - y| f_B(y) dy        (1)
 *
 * so that Laplace(u) = f.  Omega_B is the union of the leaves; f_B is the
 * tensor-product polynomial of degree p-1 in each variable that interpolates
 * the leaf's p x p node values (paper Sec. 3.2.1: order-p Chebyshev
 * approximation on every leaf box).  Nodes are first-kind Chebyshev points
 * x_j = -cos((2j+1) pi / (2p)), j = 0..p-1 (ascending); values are stored
 * [leaf][jy][jx] (x fastest).
 *
 * How each term of (1) is evaluated, per (target x, leaf B), in the leaf's
 * reference square [-1,1]^2 (y = c + r*eta):
 *     int_B log|x-y| f_B = r^2 [ log(r) * int f + int log|xi - eta| f(eta) deta ]
 *  * xi inside the closed square: the square is cut into four triangles with
 *    apex xi (one per edge) and each triangle is mapped by the Duffy map
 *    eta = xi + s (e(t) - xi), e(t) on the edge, Jacobian 2*Area*s.  Then
 *    log|xi-eta| = log s + log|e(t)-xi| and f along the ray is a polynomial
 *    of degree <= 2(p-1) in s, so the s-integral is done exactly (up to
 *    rounding) by a product rule for the weight s*log(s) on 2p nodes plus
 *    Gauss-Legendre for s*poly.  The t-integral is Gauss-Legendre on panels
 *    graded geometrically toward the foot of the perpendicular from xi.
 *  * xi outside the square: recursive subdivision; a rectangle R is
 *    integrated by a 16x16 tensor Gauss-Legendre rule once
 *    dist(xi,R) >= diam(R), else split in four.
 *
 * Sums over leaves are compensated (Neumaier).  Threads: pthreads over
 * targets.  Accuracy target ~1e-14 relative; see the pins in tests/.
 *
 * oracle_layer (at the end) is the glue layer potential of Sec. 3.4 on a
 * discretised curve, by direct summation.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_MAXP 32
#define OR_NQ 16      /* tensor Gauss-Legendre order on admissible rectangles */
#define OR_NT 32      /* Gauss-Legendre order on each t panel of a Duffy triangle */
#define OR_MAXS 64    /* max number of s nodes (2p) */

static const double OR_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights on [-1,1] (Newton on P_n).         */
/* ------------------------------------------------------------------ */
static void gl_rule(int n, double *x, double *w)
{
    for (int i = 0; i < n; i++) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p0 = 1.0; p1 = z; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Chebyshev T_0..T_{n-1} at x by the three-term recurrence. */
static inline void cheb_T(int n, double x, double *T)
{
    T[0] = 1.0;
    if (n > 1) T[1] = x;
    for (int k = 2; k < n; k++) T[k] = 2.0 * x * T[k - 1] - T[k - 2];
}

/* ------------------------------------------------------------------ */
/* Fixed rules, built once.                                            */
/* ------------------------------------------------------------------ */
static double g_q[OR_NQ], g_wq[OR_NQ];           /* GL16 on [-1,1] */
static double g_t[OR_NT], g_wt[OR_NT];           /* GL32 on [-1,1] */
static int g_ns_cached = 0;                      /* s rule built for this count */
static double g_s[OR_MAXS], g_wreg[OR_MAXS], g_wlog[OR_MAXS];
static pthread_mutex_t g_rule_mu = PTHREAD_MUTEX_INITIALIZER;
static int g_fixed_ready = 0;

/*
 * s-rule on [0,1] with ns Gauss-Legendre nodes s_m:
 *   wreg_m = GL weight * s_m           (int_0^1 s g(s) ds, exact deg(g) <= 2ns-2)
 *   wlog_m = int_0^1 s log(s) l_m(s) ds (l_m = Lagrange basis on the s_m;
 *            exact for deg(g) <= ns-1)
 * wlog is computed by composite Gauss-Legendre on the dyadic panels
 * [2^-(j+1), 2^-j], j = 0..120, where s log s is analytic on each panel.
 */
static void build_s_rule(int ns)
{
    double x[OR_MAXS], w[OR_MAXS];
    gl_rule(ns, x, w);
    for (int m = 0; m < ns; m++) {
        g_s[m] = 0.5 * (x[m] + 1.0);
        g_wreg[m] = 0.5 * w[m] * g_s[m];
    }
    /* barycentric weights of the s nodes */
    double lam[OR_MAXS];
    for (int m = 0; m < ns; m++) {
        double prod = 1.0;
        for (int k = 0; k < ns; k++)
            if (k != m) prod *= (g_s[m] - g_s[k]);
        lam[m] = 1.0 / prod;
    }
    double acc[OR_MAXS], comp[OR_MAXS];
    for (int m = 0; m < ns; m++) acc[m] = comp[m] = 0.0;
    for (int j = 0; j <= 120; j++) {
        double hi = ldexp(1.0, -j), lo = ldexp(1.0, -(j + 1));
        for (int q = 0; q < ns; q++) {
            double s = lo + (hi - lo) * 0.5 * (x[q] + 1.0);
            double wq = (hi - lo) * 0.5 * w[q] * s * log(s);
            /* l_m(s) = (lam_m/(s - s_m)) / sum_k lam_k/(s - s_k) */
            double den = 0.0;
            int hit = -1;
            for (int k = 0; k < ns; k++) {
                double d = s - g_s[k];
                if (d == 0.0) { hit = k; break; }
                den += lam[k] / d;
            }
            for (int m = 0; m < ns; m++) {
                double lm;
                if (hit >= 0) lm = (m == hit) ? 1.0 : 0.0;
                else lm = (lam[m] / (s - g_s[m])) / den;
                double y = wq * lm - comp[m];
                double t = acc[m] + y;
                comp[m] = (t - acc[m]) - y;
                acc[m] = t;
            }
        }
    }
    for (int m = 0; m < ns; m++) g_wlog[m] = acc[m];
    g_ns_cached = ns;
}

static void ensure_rules(int ns)
{
    pthread_mutex_lock(&g_rule_mu);
    if (!g_fixed_ready) {
        gl_rule(OR_NQ, g_q, g_wq);
        gl_rule(OR_NT, g_t, g_wt);
        g_fixed_ready = 1;
    }
    if (g_ns_cached != ns) build_s_rule(ns);
    pthread_mutex_unlock(&g_rule_mu);
}

/* ------------------------------------------------------------------ */
/* Per-leaf polynomial data.                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    int p;
    double *c;       /* p*p Chebyshev coefficients c[b*p + a], a: x-degree */
    double mass;     /* int_{[-1,1]^2} f */
    double *fgrid;   /* f at the GL16 x GL16 grid of [-1,1]^2, [qx][qy] */
} leaf_poly;

/* Node values -> Chebyshev coefficients by the discrete cosine sums of the
 * first-kind grid: c_a = (2 - [a==0])/p * sum_m f(x_m) T_a(x_m). */
static void leaf_coeffs(int p, const double *f, leaf_poly *L)
{
    double Tm[OR_MAXP][OR_MAXP]; /* Tm[m][a] = T_a(x_m) */
    for (int m = 0; m < p; m++) {
        double xm = -cos((2.0 * m + 1.0) * OR_PI / (2.0 * p));
        cheb_T(p, xm, Tm[m]);
    }
    double tmp[OR_MAXP * OR_MAXP]; /* tmp[n*p + a] = sum_m f[n][m] T_a(x_m) */
    for (int n = 0; n < p; n++)
        for (int a = 0; a < p; a++) {
            double s = 0.0;
            for (int m = 0; m < p; m++) s += f[n * p + m] * Tm[m][a];
            tmp[n * p + a] = s * (a == 0 ? 1.0 : 2.0) / p;
        }
    for (int b = 0; b < p; b++)
        for (int a = 0; a < p; a++) {
            double s = 0.0;
            for (int n = 0; n < p; n++) s += tmp[n * p + a] * Tm[n][b];
            L->c[b * p + a] = s * (b == 0 ? 1.0 : 2.0) / p;
        }
    L->p = p;
    /* int_{-1}^{1} T_a = 2/(1-a^2) for even a, 0 for odd a */
    double mass = 0.0;
    for (int b = 0; b < p; b += 2)
        for (int a = 0; a < p; a += 2)
            mass += L->c[b * p + a] * (2.0 / (1.0 - (double)a * a)) * (2.0 / (1.0 - (double)b * b));
    L->mass = mass;
    /* f on the GL16 grid of the whole square */
    double Tq[OR_NQ][OR_MAXP];
    for (int q = 0; q < OR_NQ; q++) cheb_T(p, g_q[q], Tq[q]);
    for (int qy = 0; qy < OR_NQ; qy++) {
        double row[OR_MAXP];
        for (int a = 0; a < p; a++) {
            double s = 0.0;
            for (int b = 0; b < p; b++) s += L->c[b * p + a] * Tq[qy][b];
            row[a] = s;
        }
        for (int qx = 0; qx < OR_NQ; qx++) {
            double s = 0.0;
            for (int a = 0; a < p; a++) s += row[a] * Tq[qx][a];
            L->fgrid[qx * OR_NQ + qy] = s;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Target outside the reference square: adaptive subdivision.         */
/* ------------------------------------------------------------------ */
static double rect_dist(double x, double y, double x0, double x1, double y0, double y1)
{
    double dx = x < x0 ? x0 - x : (x > x1 ? x - x1 : 0.0);
    double dy = y < y0 ? y0 - y : (y > y1 ? y - y1 : 0.0);
    return sqrt(dx * dx + dy * dy);
}

/* int_R log|xi - eta| f(eta) deta, 16x16 tensor GL with f evaluated by the
 * tensor form sum_a T_a(u) [sum_b c_ab T_b(v)]. */
static double rect_gl(const leaf_poly *L, double xi, double eta, double x0, double x1, double y0, double y1)
{
    int p = L->p;
    double hx = 0.5 * (x1 - x0), hy = 0.5 * (y1 - y0);
    double u[OR_NQ], v[OR_NQ];
    double Tu[OR_NQ][OR_MAXP], Tv[OR_NQ][OR_MAXP];
    for (int q = 0; q < OR_NQ; q++) {
        u[q] = x0 + hx * (g_q[q] + 1.0);
        v[q] = y0 + hy * (g_q[q] + 1.0);
        cheb_T(p, u[q], Tu[q]);
        cheb_T(p, v[q], Tv[q]);
    }
    double total = 0.0;
    for (int r = 0; r < OR_NQ; r++) {
        double row[OR_MAXP];
        for (int a = 0; a < p; a++) {
            double s = 0.0;
            for (int b = 0; b < p; b++) s += L->c[b * p + a] * Tv[r][b];
            row[a] = s;
        }
        double dy = v[r] - eta;
        double acc = 0.0;
        for (int q = 0; q < OR_NQ; q++) {
            double fv = 0.0;
            for (int a = 0; a < p; a++) fv += row[a] * Tu[q][a];
            double dx = u[q] - xi;
            acc += g_wq[q] * 0.5 * log(dx * dx + dy * dy) * fv;
        }
        total += g_wq[r] * acc;
    }
    return total * hx * hy;
}

static double subdiv(const leaf_poly *L, double xi, double eta, double x0, double x1, double y0, double y1)
{
    double diam = hypot(x1 - x0, y1 - y0);
    double dist = rect_dist(xi, eta, x0, x1, y0, y1);
    if (dist >= diam) return rect_gl(L, xi, eta, x0, x1, y0, y1);
    if (diam < 1e-13) return 0.0; /* |contribution| <= max|f| diam^2 |log diam| */
    double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1);
    return subdiv(L, xi, eta, x0, xm, y0, ym) + subdiv(L, xi, eta, xm, x1, y0, ym)
         + subdiv(L, xi, eta, x0, xm, ym, y1) + subdiv(L, xi, eta, xm, x1, ym, y1);
}

/* ------------------------------------------------------------------ */
/* Target inside the closed reference square: four Duffy triangles.   */
/* ------------------------------------------------------------------ */
#define OR_MAXPANEL 256

static int t_panels(double tf, double delta, double *br)
{
    /* breakpoints in [0,1] graded toward tf with smallest width delta */
    int n = 0;
    double left[OR_MAXPANEL], right[OR_MAXPANEL];
    int nl = 0, nr = 0;
    if (delta <= 0.0) delta = 1e-300;
    for (double d = delta; tf - d > 0.0 && nl < 120; d *= 2.0) left[nl++] = tf - d;
    for (double d = delta; tf + d < 1.0 && nr < 120; d *= 2.0) right[nr++] = tf + d;
    br[n++] = 0.0;
    for (int i = nl - 1; i >= 0; i--) br[n++] = left[i];
    if (tf > 0.0 && tf < 1.0) br[n++] = tf;
    for (int i = 0; i < nr; i++) br[n++] = right[i];
    br[n++] = 1.0;
    return n; /* number of breakpoints; panels = n - 1 */
}

static double duffy_square(const leaf_poly *L, double xi, double eta, int ns)
{
    static const double vx[5] = {-1.0, 1.0, 1.0, -1.0, -1.0};
    static const double vy[5] = {-1.0, -1.0, 1.0, 1.0, -1.0};
    int p = L->p;
    double total = 0.0;
    double *tk = (double *)malloc(sizeof(double) * OR_MAXPANEL * OR_NT * 3);
    double *wk = tk + OR_MAXPANEL * OR_NT;
    double *lk = wk + OR_MAXPANEL * OR_NT;
    for (int e = 0; e < 4; e++) {
        double ax = vx[e], ay = vy[e], bx = vx[e + 1], by = vy[e + 1];
        double ex = bx - ax, ey = by - ay;
        double le = hypot(ex, ey);
        double twoA = fabs((ax - xi) * ey - (ay - eta) * ex);
        if (twoA < 1e-300) continue;
        double d = twoA / le;
        double tf = ((xi - ax) * ex + (eta - ay) * ey) / (le * le);
        double br[2 * OR_MAXPANEL];
        int nb = t_panels(tf, d / le, br);
        int nt = 0;
        for (int k = 0; k + 1 < nb; k++) {
            double t0 = br[k], t1 = br[k + 1], h = 0.5 * (t1 - t0);
            for (int q = 0; q < OR_NT; q++) {
                double t = t0 + h * (g_t[q] + 1.0);
                tk[nt] = t;
                wk[nt] = h * g_wt[q];
                double px = ax + t * ex - xi, py = ay + t * ey - eta;
                lk[nt] = 0.5 * log(px * px + py * py);
                nt++;
            }
        }
        int horizontal = (ey == 0.0);
        double acc_tri = 0.0;
        for (int m = 0; m < ns; m++) {
            double s = g_s[m];
            double row[OR_MAXP], Tfix[OR_MAXP], Tvar[OR_MAXP];
            /* along t the coordinate orthogonal to the edge is fixed */
            if (horizontal) {
                double yfix = eta + s * (ay - eta);
                cheb_T(p, yfix, Tfix);
                for (int a = 0; a < p; a++) {
                    double acc = 0.0;
                    for (int b = 0; b < p; b++) acc += L->c[b * p + a] * Tfix[b];
                    row[a] = acc;
                }
            } else {
                double xfix = xi + s * (ax - xi);
                cheb_T(p, xfix, Tfix);
                for (int b = 0; b < p; b++) {
                    double acc = 0.0;
                    for (int a = 0; a < p; a++) acc += L->c[b * p + a] * Tfix[a];
                    row[b] = acc;
                }
            }
            double acc_s = 0.0;
            for (int k = 0; k < nt; k++) {
                double var = horizontal ? xi + s * (ax + tk[k] * ex - xi) : eta + s * (ay + tk[k] * ey - eta);
                cheb_T(p, var, Tvar);
                double g = 0.0;
                for (int a = 0; a < p; a++) g += row[a] * Tvar[a];
                acc_s += wk[k] * (g_wlog[m] + lk[k] * g_wreg[m]) * g;
            }
            acc_tri += acc_s;
        }
        total += twoA * acc_tri;
    }
    free(tk);
    return total;
}

/* int_{[-1,1]^2} log|xi - eta| f(eta) d eta for the leaf polynomial. */
static double ref_integral(const leaf_poly *L, double xi, double eta, int ns)
{
    if (fabs(xi) <= 1.0 && fabs(eta) <= 1.0) return duffy_square(L, xi, eta, ns);
    double dist = rect_dist(xi, eta, -1.0, 1.0, -1.0, 1.0);
    if (dist >= 2.0 * sqrt(2.0)) {
        /* whole leaf admissible: use the cached grid values */
        double total = 0.0;
        for (int qx = 0; qx < OR_NQ; qx++) {
            double dx = g_q[qx] - xi, acc = 0.0;
            for (int qy = 0; qy < OR_NQ; qy++) {
                double dy = g_q[qy] - eta;
                acc += g_wq[qy] * 0.5 * log(dx * dx + dy * dy) * L->fgrid[qx * OR_NQ + qy];
            }
            total += g_wq[qx] * acc;
        }
        return total;
    }
    return subdiv(L, xi, eta, -1.0, 1.0, -1.0, 1.0);
}

/* ------------------------------------------------------------------ */
/* Gradient kernel: int (xi - eta)/|xi - eta|^2 f(eta) d eta.          */
/* ------------------------------------------------------------------ */

/* the same on a rectangle by the 16x16 tensor GL rule (admissible) */
static void rect_gl_grad(const leaf_poly *L, double xi, double eta, double x0, double x1, double y0, double y1,
                         double *gx, double *gy)
{
    int p = L->p;
    double hx = 0.5 * (x1 - x0), hy = 0.5 * (y1 - y0);
    double u[OR_NQ], v[OR_NQ];
    double Tu[OR_NQ][OR_MAXP], Tv[OR_NQ][OR_MAXP];
    for (int q = 0; q < OR_NQ; q++) {
        u[q] = x0 + hx * (g_q[q] + 1.0);
        v[q] = y0 + hy * (g_q[q] + 1.0);
        cheb_T(p, u[q], Tu[q]);
        cheb_T(p, v[q], Tv[q]);
    }
    double sx = 0.0, sy = 0.0;
    for (int r = 0; r < OR_NQ; r++) {
        double row[OR_MAXP];
        for (int a = 0; a < p; a++) {
            double s = 0.0;
            for (int b = 0; b < p; b++) s += L->c[b * p + a] * Tv[r][b];
            row[a] = s;
        }
        double dy = eta - v[r];
        double ax = 0.0, ay = 0.0;
        for (int q = 0; q < OR_NQ; q++) {
            double fv = 0.0;
            for (int a = 0; a < p; a++) fv += row[a] * Tu[q][a];
            double dx = xi - u[q], d2 = dx * dx + dy * dy;
            ax += g_wq[q] * dx / d2 * fv;
            ay += g_wq[q] * dy / d2 * fv;
        }
        sx += g_wq[r] * ax;
        sy += g_wq[r] * ay;
    }
    *gx = sx * hx * hy;
    *gy = sy * hx * hy;
}

static void subdiv_grad(const leaf_poly *L, double xi, double eta, double x0, double x1, double y0, double y1,
                        double *gx, double *gy)
{
    double diam = hypot(x1 - x0, y1 - y0);
    double dist = rect_dist(xi, eta, x0, x1, y0, y1);
    if (dist >= diam) { rect_gl_grad(L, xi, eta, x0, x1, y0, y1, gx, gy); return; }
    *gx = *gy = 0.0;
    if (diam < 1e-14) return; /* |contribution| <= max|f| diam */
    double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1), ax, ay;
    subdiv_grad(L, xi, eta, x0, xm, y0, ym, &ax, &ay); *gx += ax; *gy += ay;
    subdiv_grad(L, xi, eta, xm, x1, y0, ym, &ax, &ay); *gx += ax; *gy += ay;
    subdiv_grad(L, xi, eta, x0, xm, ym, y1, &ax, &ay); *gx += ax; *gy += ay;
    subdiv_grad(L, xi, eta, xm, x1, ym, y1, &ax, &ay); *gx += ax; *gy += ay;
}

/* Target inside the closed square: the four Duffy triangles with apex xi.
 * On the ray eta = xi + s (e(t) - xi) the kernel is -(e - xi) / (s |e - xi|^2)
 * and the Jacobian twoA * s, so the s-integral of f is regular (plain
 * Gauss-Legendre on ns nodes, exact for the degree 2(p-1) of f along the ray)
 * and the t-integral of -(e - xi)/|e - xi|^2 is graded toward the foot of the
 * perpendicular from xi. */
static void duffy_square_grad(const leaf_poly *L, double xi, double eta, int ns, double *gx, double *gy)
{
    static const double vx[5] = {-1.0, 1.0, 1.0, -1.0, -1.0};
    static const double vy[5] = {-1.0, -1.0, 1.0, 1.0, -1.0};
    int p = L->p;
    double sn[OR_MAXS], sw[OR_MAXS];
    gl_rule(ns, sn, sw);
    for (int m = 0; m < ns; m++) { sn[m] = 0.5 * (sn[m] + 1.0); sw[m] *= 0.5; }
    double tx = 0.0, ty = 0.0;
    for (int e = 0; e < 4; e++) {
        double ax = vx[e], ay = vy[e], bx = vx[e + 1], by = vy[e + 1];
        double ex = bx - ax, ey = by - ay;
        double le = hypot(ex, ey);
        double twoA = fabs((ax - xi) * ey - (ay - eta) * ex);
        if (twoA < 1e-300) continue;
        double d = twoA / le;
        double tf = ((xi - ax) * ex + (eta - ay) * ey) / (le * le);
        double br[2 * OR_MAXPANEL];
        int nb = t_panels(tf, d / le, br);
        int horizontal = (ey == 0.0);
        for (int k = 0; k + 1 < nb; k++) {
            double t0 = br[k], t1 = br[k + 1], h = 0.5 * (t1 - t0);
            for (int q = 0; q < OR_NT; q++) {
                double t = t0 + h * (g_t[q] + 1.0), wt = h * g_wt[q];
                double px = ax + t * ex - xi, py = ay + t * ey - eta, d2 = px * px + py * py;
                /* int_0^1 f(xi + s (e(t) - xi)) ds */
                double fs = 0.0;
                for (int m = 0; m < ns; m++) {
                    double s = sn[m];
                    double X = xi + s * px, Y = eta + s * py;
                    double TX[OR_MAXP], TY[OR_MAXP];
                    cheb_T(p, X, TX);
                    cheb_T(p, Y, TY);
                    double fv = 0.0;
                    for (int b = 0; b < p; b++) {
                        double acc = 0.0;
                        for (int a = 0; a < p; a++) acc += L->c[b * p + a] * TX[a];
                        fv += acc * TY[b];
                    }
                    fs += sw[m] * fv;
                }
                (void)horizontal;
                tx -= wt * twoA * px / d2 * fs;
                ty -= wt * twoA * py / d2 * fs;
            }
        }
    }
    *gx = tx;
    *gy = ty;
}

/* int_{[-1,1]^2} (xi - eta)/|xi - eta|^2 f(eta) d eta for the leaf polynomial. */
static void ref_integral_grad(const leaf_poly *L, double xi, double eta, int ns, double *gx, double *gy)
{
    if (fabs(xi) <= 1.0 && fabs(eta) <= 1.0) { duffy_square_grad(L, xi, eta, ns, gx, gy); return; }
    double dist = rect_dist(xi, eta, -1.0, 1.0, -1.0, 1.0);
    if (dist >= 2.0 * sqrt(2.0)) {
        double sx = 0.0, sy = 0.0;
        for (int qx = 0; qx < OR_NQ; qx++) {
            double dx = xi - g_q[qx], ax = 0.0, ay = 0.0;
            for (int qy = 0; qy < OR_NQ; qy++) {
                double dy = eta - g_q[qy], d2 = dx * dx + dy * dy;
                double w = g_wq[qy] * L->fgrid[qx * OR_NQ + qy] / d2;
                ax += w * dx;
                ay += w * dy;
            }
            sx += g_wq[qx] * ax;
            sy += g_wq[qx] * ay;
        }
        *gx = sx;
        *gy = sy;
        return;
    }
    subdiv_grad(L, xi, eta, -1.0, 1.0, -1.0, 1.0, gx, gy);
}

/* ------------------------------------------------------------------ */
/* Driver.                                                             */
/* ------------------------------------------------------------------ */
typedef struct {
    int p, ns;
    int64_t nleaf, ntarget;
    const double *leaf;        /* [nleaf][3] cx, cy, r */
    const leaf_poly *poly;
    const double *txy;
    const int64_t *src_ptr, *src_idx;
    double *out;
    int64_t t0, t1;
    int grad;                  /* 1: out[2i], out[2i+1] = the gradient */
} or_job;

static void *or_worker(void *arg)
{
    or_job *J = (or_job *)arg;
    if (J->grad) {
        for (int64_t i = J->t0; i < J->t1; i++) {
            double X = J->txy[2 * i], Y = J->txy[2 * i + 1];
            double sx = 0.0, cx_ = 0.0, sy = 0.0, cy_ = 0.0;
            int64_t k0 = 0, k1 = J->nleaf;
            if (J->src_ptr) { k0 = J->src_ptr[i]; k1 = J->src_ptr[i + 1]; }
            for (int64_t k = k0; k < k1; k++) {
                int64_t b = J->src_ptr ? J->src_idx[k] : k;
                double cx = J->leaf[3 * b], cy = J->leaf[3 * b + 1], r = J->leaf[3 * b + 2];
                double gx, gy;
                ref_integral_grad(&J->poly[b], (X - cx) / r, (Y - cy) / r, J->ns, &gx, &gy);
                double vx = r * gx, vy = r * gy;
                double t = sx + vx;   /* Neumaier summation, per component */
                if (fabs(sx) >= fabs(vx)) cx_ += (sx - t) + vx; else cx_ += (vx - t) + sx;
                sx = t;
                t = sy + vy;
                if (fabs(sy) >= fabs(vy)) cy_ += (sy - t) + vy; else cy_ += (vy - t) + sy;
                sy = t;
            }
            J->out[2 * i] = (sx + cx_) / (2.0 * OR_PI);
            J->out[2 * i + 1] = (sy + cy_) / (2.0 * OR_PI);
        }
        return NULL;
    }
    for (int64_t i = J->t0; i < J->t1; i++) {
        double X = J->txy[2 * i], Y = J->txy[2 * i + 1];
        double sum = 0.0, comp = 0.0;
        int64_t k0 = 0, k1 = J->nleaf;
        if (J->src_ptr) { k0 = J->src_ptr[i]; k1 = J->src_ptr[i + 1]; }
        for (int64_t k = k0; k < k1; k++) {
            int64_t b = J->src_ptr ? J->src_idx[k] : k;
            double cx = J->leaf[3 * b], cy = J->leaf[3 * b + 1], r = J->leaf[3 * b + 2];
            const leaf_poly *L = &J->poly[b];
            double v = r * r * (log(r) * L->mass + ref_integral(L, (X - cx) / r, (Y - cy) / r, J->ns));
            /* Neumaier summation */
            double t = sum + v;
            if (fabs(sum) >= fabs(v)) comp += (sum - t) + v;
            else comp += (v - t) + sum;
            sum = t;
        }
        J->out[i] = (sum + comp) / (2.0 * OR_PI);
    }
    return NULL;
}

typedef struct {
    int p;
    const double *f;
    leaf_poly *poly;
    int64_t b0, b1;
} or_prep;

static void *or_prep_worker(void *arg)
{
    or_prep *J = (or_prep *)arg;
    for (int64_t b = J->b0; b < J->b1; b++) leaf_coeffs(J->p, J->f + b * J->p * J->p, &J->poly[b]);
    return NULL;
}

static int or_threads(int nthreads)
{
    if (nthreads <= 0) {
        long n = sysconf(_SC_NPROCESSORS_ONLN);
        nthreads = n > 0 ? (int)n : 1;
    }
    if (nthreads > 256) nthreads = 256;
    return nthreads;
}

/* static round-robin of target chunks over threads */
typedef struct {
    or_job *jobs;
    int64_t nchunks;
    int k, nt;
} or_rr;

static void *or_rr_worker(void *arg)
{
    or_rr *R = (or_rr *)arg;
    for (int64_t c = R->k; c < R->nchunks; c += R->nt) or_worker(&R->jobs[c]);
    return NULL;
}

/*
 * u[i] = (1/2pi) sum_{B in S(i)} int_B log|x_i - y| f_B(y) dy.
 * leaf:    [nleaf][3] = (cx, cy, r): centre and half-side of each leaf.
 * f:       [nleaf][p][p] node values, x fastest.
 * txy:     [ntarget][2] target points.
 * src_ptr/src_idx: optional CSR list S(i) of source leaves per target; NULL
 *          means every leaf.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
static int oracle_run(int p, int64_t nleaf, const double *leaf, const double *f, int64_t ntarget,
                      const double *txy, const int64_t *src_ptr, const int64_t *src_idx, double *out,
                      int nthreads, int grad);

int oracle_potential(int p, int64_t nleaf, const double *leaf, const double *f, int64_t ntarget,
                     const double *txy, const int64_t *src_ptr, const int64_t *src_idx, double *out,
                     int nthreads)
{
    return oracle_run(p, nleaf, leaf, f, ntarget, txy, src_ptr, src_idx, out, nthreads, 0);
}

/*
 * The gradient of the same potential at the targets:
 *   out[2i], out[2i+1] = (1/2pi) sum_{B in S(i)} int_B (x_i - y)/|x_i - y|^2 f_B(y) dy,
 * the derivative of eq. (vbulk) that the glue step needs on the fictitious
 * curve (normal derivative of v_bulk, Sec. 3.4).  Same arguments as
 * oracle_potential; out has 2 ntarget entries.
 */
int oracle_gradient(int p, int64_t nleaf, const double *leaf, const double *f, int64_t ntarget,
                    const double *txy, const int64_t *src_ptr, const int64_t *src_idx, double *out,
                    int nthreads)
{
    return oracle_run(p, nleaf, leaf, f, ntarget, txy, src_ptr, src_idx, out, nthreads, 1);
}

static int oracle_run(int p, int64_t nleaf, const double *leaf, const double *f, int64_t ntarget,
                      const double *txy, const int64_t *src_ptr, const int64_t *src_idx, double *out,
                      int nthreads, int grad)
{
    if (p < 2 || p > OR_MAXP || nleaf < 0 || ntarget < 0) return -1;
    if (ntarget == 0) return 0;
    int ns = 2 * p;
    ensure_rules(ns);
    size_t nl = (size_t)(nleaf > 0 ? nleaf : 1);
    leaf_poly *poly = (leaf_poly *)malloc(sizeof(leaf_poly) * nl);
    double *store = (double *)malloc(sizeof(double) * nl * (size_t)(p * p + OR_NQ * OR_NQ));
    if (!poly || !store) { free(poly); free(store); return -1; }
    for (size_t b = 0; b < (size_t)nleaf; b++) {
        poly[b].c = store + b * (size_t)(p * p + OR_NQ * OR_NQ);
        poly[b].fgrid = poly[b].c + p * p;
    }
    int nt = or_threads(nthreads);
    pthread_t th[256];
    {
        or_prep jobs[256];
        int used = 0;
        for (int k = 0; k < nt; k++) {
            jobs[k].p = p;
            jobs[k].f = f;
            jobs[k].poly = poly;
            jobs[k].b0 = nleaf * k / nt;
            jobs[k].b1 = nleaf * (k + 1) / nt;
            if (pthread_create(&th[k], NULL, or_prep_worker, &jobs[k]) != 0) {
                or_prep_worker(&jobs[k]);
                th[k] = 0;
            }
            used++;
        }
        for (int k = 0; k < used; k++)
            if (th[k]) pthread_join(th[k], NULL);
    }
    /* interleave targets over workers in small chunks for balance */
    int64_t chunk = 16;
    int64_t nchunks = (ntarget + chunk - 1) / chunk;
    or_job *jobs = (or_job *)malloc(sizeof(or_job) * (size_t)nchunks);
    if (!jobs) { free(poly); free(store); return -1; }
    for (int64_t c = 0; c < nchunks; c++) {
        or_job *J = &jobs[c];
        J->p = p; J->ns = ns; J->nleaf = nleaf; J->ntarget = ntarget;
        J->leaf = leaf; J->poly = poly; J->txy = txy;
        J->src_ptr = src_ptr; J->src_idx = src_idx; J->out = out; J->grad = grad;
        J->t0 = c * chunk;
        J->t1 = (c + 1) * chunk < ntarget ? (c + 1) * chunk : ntarget;
    }
    or_rr rr[256];
    for (int k = 0; k < nt; k++) { rr[k].jobs = jobs; rr[k].nchunks = nchunks; rr[k].k = k; rr[k].nt = nt; }
    for (int k = 0; k < nt; k++)
        if (pthread_create(&th[k], NULL, or_rr_worker, &rr[k]) != 0) { or_rr_worker(&rr[k]); th[k] = 0; }
    for (int k = 0; k < nt; k++)
        if (th[k]) pthread_join(th[k], NULL);
    free(jobs);
    free(poly);
    free(store);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Small helpers exposed for the pins.                                  */
/* ------------------------------------------------------------------ */

/* First-kind Chebyshev nodes, ascending. */
void oracle_nodes(int p, double *x)
{
    for (int j = 0; j < p; j++) x[j] = -cos((2.0 * j + 1.0) * OR_PI / (2.0 * p));
}

/* The s-rule used on Duffy rays: nodes, s-weights, s*log(s) product weights. */
int oracle_s_rule(int ns, double *s, double *wreg, double *wlog)
{
    if (ns < 1 || ns > OR_MAXS) return -1;
    ensure_rules(ns);
    pthread_mutex_lock(&g_rule_mu);
    if (g_ns_cached != ns) build_s_rule(ns);
    for (int m = 0; m < ns; m++) { s[m] = g_s[m]; wreg[m] = g_wreg[m]; wlog[m] = g_wlog[m]; }
    pthread_mutex_unlock(&g_rule_mu);
    return 0;
}

/* f_B at reference points (the interpolant), for pins of the coefficient map. */
int oracle_interp(int p, const double *f, int64_t n, const double *xy, double *out)
{
    if (p < 2 || p > OR_MAXP) return -1;
    ensure_rules(2 * p);
    double cbuf[OR_MAXP * OR_MAXP], gbuf[OR_NQ * OR_NQ];
    leaf_poly L;
    L.c = cbuf;
    L.fgrid = gbuf;
    leaf_coeffs(p, f, &L);
    for (int64_t i = 0; i < n; i++) {
        double Tx[OR_MAXP], Ty[OR_MAXP];
        cheb_T(p, xy[2 * i], Tx);
        cheb_T(p, xy[2 * i + 1], Ty);
        double s = 0.0;
        for (int b = 0; b < p; b++)
            for (int a = 0; a < p; a++) s += L.c[b * p + a] * Tx[a] * Ty[b];
        out[i] = s;
    }
    return 0;
}

/*
 * Glue layer potential by direct summation (Sec. 3.4: v_glue = S[sigma] -
 * D[tau] on the fictitious curve, with S[s](x) = int Phi(x,y) s(y) dy,
 * D[t](x) = int dPhi(x,y)/dn_y t(y) dy and Phi = (1/2pi) log(1/|x-y|)),
 * discretised by a quadrature on the curve: nodes y_j, weights w_j, unit
 * normals n_j, with q_j = w_j sigma(y_j) and m_j = w_j tau(y_j) n_j:
 *
 *   out[i] = -(1/2pi) sum_j [ q_j log|x_i - y_j| + m_j . (x_i - y_j) / |x_i - y_j|^2 ]
 *
 * since dPhi/dn_y = (1/2pi) (x - y).n_y / |x - y|^2.  A source that coincides
 * with a target contributes nothing.  Plain double loop, compensated
 * (Neumaier) per target; pthreads over targets.
 * src: [n][2] nodes; q: [n]; m: [n][2]; txy: [nt][2].  Returns 0 or -1.
 */
typedef struct {
    int64_t n, t0, t1;
    const double *src, *q, *m, *txy;
    double *out;
} lay_job;

static void *lay_worker(void *arg)
{
    const lay_job *J = (const lay_job *)arg;
    for (int64_t i = J->t0; i < J->t1; i++) {
        const double x = J->txy[2 * i], y = J->txy[2 * i + 1];
        double s = 0.0, c = 0.0;
        for (int64_t j = 0; j < J->n; j++) {
            const double dx = x - J->src[2 * j], dy = y - J->src[2 * j + 1];
            const double r2 = dx * dx + dy * dy;
            if (r2 == 0.0) continue;
            const double term = J->q[j] * 0.5 * log(r2) + (J->m[2 * j] * dx + J->m[2 * j + 1] * dy) / r2;
            const double t = s + term;
            c += fabs(s) >= fabs(term) ? (s - t) + term : (term - t) + s;
            s = t;
        }
        J->out[i] = -(s + c) / (2.0 * OR_PI);
    }
    return NULL;
}

int oracle_layer(int64_t n, const double *src, const double *q, const double *m, int64_t nt, const double *txy,
                 double *out, int nthreads)
{
    if (n < 0 || nt < 0 || (n > 0 && (!src || !q || !m)) || (nt > 0 && (!txy || !out))) return -1;
    int k = or_threads(nthreads);
    if (k > nt) k = nt > 0 ? (int)nt : 1;
    pthread_t th[256];
    lay_job jobs[256];
    int started[256];
    for (int i = 0; i < k; i++) {
        jobs[i].n = n; jobs[i].src = src; jobs[i].q = q; jobs[i].m = m; jobs[i].txy = txy; jobs[i].out = out;
        jobs[i].t0 = nt * i / k;
        jobs[i].t1 = nt * (i + 1) / k;
        started[i] = pthread_create(&th[i], NULL, lay_worker, &jobs[i]) == 0;
        if (!started[i]) lay_worker(&jobs[i]);
    }
    for (int i = 0; i < k; i++)
        if (started[i]) pthread_join(th[i], NULL);
    return 0;
}
