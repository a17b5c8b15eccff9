/*
 * iga_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, FP64 CPU oracle for the Galerkin stiffness matrix of the
 * pulled-back variable-coefficient diffusion operator on one mapped
 * tensor-product B-spline patch, as defined in Drzisga, Keith & Wohlmuth,
 * "The surrogate matrix methodology: low-cost assembly for isogeometric
 * analysis":
 *
 *   A_ij = a(B_j, B_i) = int_{(0,1)^n} grad B_i(x)^T K(x) grad B_j(x) dx,
 *   K(x) = kappa(phi(x)) |det Dphi(x)| Dphi(x)^{-1} Dphi(x)^{-T}
 *
 * (Sec. 3.2, eq. BilinearFormPoissonTensor and eq. ChangeOfVars; the factor
 * kappa is the diffusion coefficient of the workload, evaluated at the
 * physical point phi(x)).  The integral is taken with the (p+1)-point
 * Gauss-Legendre rule on every element in every direction, which is the
 * "exact" matrix the surrogate is compared with.
 *
 * The basis is the open uniform B-spline basis of Sec. 2.2: knots
 * 0 (p+1 times), k/n_el for k=1..n_el-1, 1 (p+1 times); m = n_el + p
 * functions per direction; global index colexicographic (Sec. 2.2):
 * i = i_0 + m_0 (i_1 + m_1 i_2), 0-based here.
 *
 * Rows are stored stencil-wise: out[r*S + s] is A_{i, i+delta_s}, where
 * slot s enumerates the offsets delta in {-p..p}^n colexicographically,
 * s = sum_d (delta_d + p)(2p+1)^d.  Offsets that leave the index range
 * give 0.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It shares no code, header or table with the CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXP 8

enum { ORC_MAP_IDENTITY = 0, ORC_MAP_AFFINE = 1, ORC_MAP_SINPROD = 2 };
enum { ORC_KAPPA_CONST = 0, ORC_KAPPA_SIN2D = 1, ORC_KAPPA_EXPSIN3D = 2, ORC_KAPPA_POLY = 3, ORC_KAPPA_BSPLINE3 = 4 };

/* Problem description (mirrored by a ctypes Structure in oracle/_lib.py). */
typedef struct {
    int32_t dim;          /* n = 2 or 3 */
    int32_t p;            /* spline degree */
    int32_t n_el[3];      /* elements per direction */
    int32_t map_kind;     /* ORC_MAP_* */
    int32_t kappa_kind;   /* ORC_KAPPA_* */
    int32_t kappa_deg;    /* degree per direction of the polynomial kappa */
    double map_amp;       /* amplitude of the sine-product map */
    double affine[12];    /* x = A xi + b: A row-major 3x3 in [0..8], b in [9..11] */
    double kappa_a;       /* constant / offset */
    double kappa_b;       /* amplitude */
    double kappa_poly[64];/* coef[a + (deg+1)(b + (deg+1)c)] of x^a y^b z^c */
    int32_t kappa_nctrl[3];      /* ORC_KAPPA_BSPLINE3: control values per direction (4..64) */
    const double* kappa_ctrl;    /* ORC_KAPPA_BSPLINE3: c[a + n0 (b + n1 c)], host memory */
} orc_problem;

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0,1]: Newton iteration on P_n.               */
/* ------------------------------------------------------------------ */
/* P_n(z) and P_{n-1}(z) by the three-term recurrence
 *   j P_j = (2j - 1) z P_{j-1} - (j - 1) P_{j-2},  P_0 = 1, P_1 = z. */
static void legendre_pair(int n, double z, double* pn, double* pnm1)
{
    double a = 1.0, b = z;          /* P_0, P_1 */
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int j = 2; j <= n; ++j) {
        double c = ((2.0 * j - 1.0) * z * b - (j - 1.0) * a) / j;
        a = b; b = c;
    }
    *pn = b; *pnm1 = a;
}

int orc_gauss_legendre(int n, double* x, double* w)
{
    if (n < 1 || n > 64) return -1;
    for (int k = 0; k < n; ++k) {
        /* starting guess for the (k+1)-th largest root of P_n */
        double z = cos(ORC_PI * (k + 0.75) / (n + 0.5));
        double pn, pm, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_pair(n, z, &pn, &pm);
            dp = n * (z * pn - pm) / (z * z - 1.0);   /* P_n'(z) */
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        legendre_pair(n, z, &pn, &pm);
        dp = n * (z * pn - pm) / (z * z - 1.0);
        /* weight on [-1,1]: 2 / ((1 - z^2) P_n'(z)^2); halved on [0,1] */
        x[n - 1 - k] = 0.5 * (1.0 + z);
        w[n - 1 - k] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Open uniform knot vector and Cox-de Boor recursion.                  */
/* ------------------------------------------------------------------ */
int orc_open_uniform_knots(int p, int n_el, double* t /* n_el + 2p + 1 */)
{
    int m = n_el + p;
    for (int k = 0; k <= p; ++k) t[k] = 0.0;
    for (int k = 1; k < n_el; ++k) t[p + k] = (double)k / (double)n_el;
    for (int k = m; k <= m + p; ++k) t[k] = 1.0;
    return 0;
}

/*
 * Values (and first derivatives) of all nb = nt - p - 1 B-splines of degree
 * p on the knot vector t[0..nt-1] at x, by the recursion
 *   N_{i,0} = 1 on [t_i, t_{i+1}),
 *   N_{i,k} = (x - t_i)/(t_{i+k} - t_i) N_{i,k-1}
 *           + (t_{i+k+1} - x)/(t_{i+k+1} - t_{i+1}) N_{i+1,k-1},
 *   N'_{i,k} = k/(t_{i+k} - t_i) N_{i,k-1} - k/(t_{i+k+1} - t_{i+1}) N_{i+1,k-1},
 * with 0/0 read as 0.  Intervals are half-open except that x equal to the
 * last knot belongs to the last non-empty interval.  der may be NULL.
 */
int orc_bspline_all(int p, int nt, const double* t, double x, double* val, double* der)
{
    int nb = nt - p - 1;
    if (nb < 1 || p < 0) return -1;
    double* N = (double*)calloc((size_t)nt, sizeof(double));
    double* Nprev = (double*)calloc((size_t)nt, sizeof(double));
    if (!N || !Nprev) { free(N); free(Nprev); return -2; }
    int last = -1;
    for (int i = 0; i + 1 < nt; ++i) if (t[i] < t[i + 1]) last = i;
    for (int i = 0; i + 1 < nt; ++i) {
        int inside = (t[i] <= x && x < t[i + 1]);
        if (i == last && x == t[i + 1]) inside = 1;
        N[i] = (t[i] < t[i + 1] && inside) ? 1.0 : 0.0;
    }
    for (int k = 1; k <= p; ++k) {
        memcpy(Nprev, N, sizeof(double) * (size_t)nt);
        for (int i = 0; i + k + 1 < nt; ++i) {
            double a = 0.0, b = 0.0;
            double d1 = t[i + k] - t[i], d2 = t[i + k + 1] - t[i + 1];
            if (d1 > 0.0) a = (x - t[i]) / d1 * Nprev[i];
            if (d2 > 0.0) b = (t[i + k + 1] - x) / d2 * Nprev[i + 1];
            N[i] = a + b;
        }
        for (int i = nt - k - 1; i < nt; ++i) if (i >= 0) N[i] = 0.0;
        if (k == p && der) {
            for (int i = 0; i < nb; ++i) {
                double a = 0.0, b = 0.0;
                double d1 = t[i + k] - t[i], d2 = t[i + k + 1] - t[i + 1];
                if (d1 > 0.0) a = k / d1 * Nprev[i];
                if (d2 > 0.0) b = k / d2 * Nprev[i + 1];
                der[i] = a - b;
            }
        }
    }
    if (p == 0 && der) for (int i = 0; i < nb; ++i) der[i] = 0.0;
    for (int i = 0; i < nb; ++i) val[i] = N[i];
    free(N); free(Nprev);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Geometry map, coefficient and the tensor K.                         */
/* ------------------------------------------------------------------ */
/* x = phi(xi), J[a*3+b] = d phi_a / d xi_b */
int orc_map(const orc_problem* P, const double* xi, double* x, double* J)
{
    int n = P->dim;
    for (int a = 0; a < 9; ++a) J[a] = 0.0;
    if (P->map_kind == ORC_MAP_IDENTITY) {
        for (int a = 0; a < n; ++a) { x[a] = xi[a]; J[a * 3 + a] = 1.0; }
    } else if (P->map_kind == ORC_MAP_AFFINE) {
        for (int a = 0; a < n; ++a) {
            x[a] = P->affine[9 + a];
            for (int b = 0; b < n; ++b) {
                x[a] += P->affine[a * 3 + b] * xi[b];
                J[a * 3 + b] = P->affine[a * 3 + b];
            }
        }
    } else if (P->map_kind == ORC_MAP_SINPROD) {
        /* x_a = xi_a + amp * prod_j sin(pi xi_j) */
        double s[3], c[3], prod = 1.0;
        for (int j = 0; j < n; ++j) { s[j] = sin(ORC_PI * xi[j]); c[j] = cos(ORC_PI * xi[j]); prod *= s[j]; }
        for (int a = 0; a < n; ++a) x[a] = xi[a] + P->map_amp * prod;
        for (int b = 0; b < n; ++b) {
            double dprod = ORC_PI * c[b];
            for (int j = 0; j < n; ++j) if (j != b) dprod *= s[j];
            for (int a = 0; a < n; ++a) J[a * 3 + b] = (a == b ? 1.0 : 0.0) + P->map_amp * dprod;
        }
    } else {
        return -1;
    }
    return 0;
}

double orc_kappa(const orc_problem* P, const double* x)
{
    int n = P->dim;
    switch (P->kappa_kind) {
    case ORC_KAPPA_CONST:
        return P->kappa_a;
    case ORC_KAPPA_SIN2D:
        return P->kappa_a + P->kappa_b * sin(2.0 * ORC_PI * x[0]) * sin(2.0 * ORC_PI * x[1]);
    case ORC_KAPPA_EXPSIN3D:
        return exp(P->kappa_b * sin(2.0 * ORC_PI * x[0]) * cos(2.0 * ORC_PI * x[1]) * sin(2.0 * ORC_PI * x[2]));
    case ORC_KAPPA_POLY: {
        int d = P->kappa_deg;
        double v = 0.0;
        int cmax = (n == 3) ? d : 0;
        for (int c = 0; c <= cmax; ++c)
            for (int b = 0; b <= d; ++b)
                for (int a = 0; a <= d; ++a) {
                    double term = P->kappa_poly[a + (d + 1) * (b + (d + 1) * c)];
                    term *= pow(x[0], a) * pow(x[1], b);
                    if (n == 3) term *= pow(x[2], c);
                    v += term;
                }
        return v;
    }
    case ORC_KAPPA_BSPLINE3: {
        /* cubic tensor-product B-spline on the physical unit cube, open uniform
           knots with nctrl_d - 3 elements per direction; points outside [0,1]
           are clamped onto it */
        double N[3][64], D[64];
        for (int d = 0; d < n; ++d) {
            const int nc = P->kappa_nctrl[d];
            if (nc < 4 || nc > 64) return NAN;
            double t[64 + 4];
            orc_open_uniform_knots(3, nc - 3, t);
            double xd = x[d] < 0.0 ? 0.0 : (x[d] > 1.0 ? 1.0 : x[d]);
            orc_bspline_all(3, nc + 4, t, xd, N[d], D);
        }
        double v = 0.0;
        const int n2 = (n == 3) ? P->kappa_nctrl[2] : 1;
        for (int c = 0; c < n2; ++c)
            for (int b = 0; b < P->kappa_nctrl[1]; ++b)
                for (int a = 0; a < P->kappa_nctrl[0]; ++a) {
                    double term = P->kappa_ctrl[a + P->kappa_nctrl[0] * (b + P->kappa_nctrl[1] * c)];
                    term *= N[0][a] * N[1][b];
                    if (n == 3) term *= N[2][c];
                    v += term;
                }
        return v;
    }
    default:
        return NAN;
    }
}

/* K = kappa(phi(xi)) |det J| J^{-1} J^{-T}, row-major n x n in K[3x3]. */
int orc_coefficient(const orc_problem* P, const double* xi, double* K)
{
    int n = P->dim;
    double x[3] = {0, 0, 0}, J[9];
    if (orc_map(P, xi, x, J)) return -1;
    double inv[9] = {0}, det;
    if (n == 2) {
        det = J[0] * J[4] - J[1] * J[3];
        inv[0] = J[4] / det;  inv[1] = -J[1] / det;
        inv[3] = -J[3] / det; inv[4] = J[0] / det;
    } else {
        /* inverse by cofactors: inv = adj(J) / det */
        double c00 = J[4] * J[8] - J[5] * J[7];
        double c01 = J[5] * J[6] - J[3] * J[8];
        double c02 = J[3] * J[7] - J[4] * J[6];
        det = J[0] * c00 + J[1] * c01 + J[2] * c02;
        inv[0] = c00 / det;
        inv[1] = (J[2] * J[7] - J[1] * J[8]) / det;
        inv[2] = (J[1] * J[5] - J[2] * J[4]) / det;
        inv[3] = c01 / det;
        inv[4] = (J[0] * J[8] - J[2] * J[6]) / det;
        inv[5] = (J[2] * J[3] - J[0] * J[5]) / det;
        inv[6] = c02 / det;
        inv[7] = (J[1] * J[6] - J[0] * J[7]) / det;
        inv[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    }
    double kap = orc_kappa(P, x);
    for (int a = 0; a < 9; ++a) K[a] = 0.0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double s = 0.0;
            for (int c = 0; c < n; ++c) s += inv[a * 3 + c] * inv[b * 3 + c];
            K[a * 3 + b] = kap * fabs(det) * s;
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 1-D tables at the Gauss points of every element.                    */
/* ------------------------------------------------------------------ */
typedef struct {
    int p, n_el, m, G;     /* G = n_el (p+1) Gauss points */
    double* xi;            /* [G] */
    double* wq;            /* [G] Gauss weight times element length */
    double* val;           /* [G][p+1]: value of basis e+a at point g of element e */
    double* der;           /* [G][p+1] */
} tab1d;

static void tab_free(tab1d* T) { free(T->xi); free(T->wq); free(T->val); free(T->der); }

static int tab_build(int p, int n_el, tab1d* T)
{
    int m = n_el + p, nt = m + p + 1;
    T->p = p; T->n_el = n_el; T->m = m; T->G = n_el * (p + 1);
    T->xi = (double*)malloc(sizeof(double) * T->G);
    T->wq = (double*)malloc(sizeof(double) * T->G);
    T->val = (double*)malloc(sizeof(double) * T->G * (p + 1));
    T->der = (double*)malloc(sizeof(double) * T->G * (p + 1));
    double* t = (double*)malloc(sizeof(double) * nt);
    double* v = (double*)malloc(sizeof(double) * m);
    double* d = (double*)malloc(sizeof(double) * m);
    double gx[ORC_MAXP + 1], gw[ORC_MAXP + 1];
    if (!T->xi || !T->wq || !T->val || !T->der || !t || !v || !d) { free(t); free(v); free(d); return -2; }
    orc_open_uniform_knots(p, n_el, t);
    orc_gauss_legendre(p + 1, gx, gw);
    double h = 1.0 / n_el;
    for (int e = 0; e < n_el; ++e)
        for (int r = 0; r <= p; ++r) {
            int g = e * (p + 1) + r;
            double x = (e + gx[r]) * h;
            T->xi[g] = x;
            T->wq[g] = gw[r] * h;
            orc_bspline_all(p, nt, t, x, v, d);
            for (int a = 0; a <= p; ++a) {
                T->val[g * (p + 1) + a] = v[e + a];
                T->der[g * (p + 1) + a] = d[e + a];
            }
        }
    free(t); free(v); free(d);
    return 0;
}

/* value (deriv=0) or derivative (deriv=1) of basis i at Gauss point g */
static inline double tab_get(const tab1d* T, int g, int i, int deriv)
{
    int e = g / (T->p + 1);
    int a = i - e;
    if (a < 0 || a > T->p) return 0.0;
    return deriv ? T->der[g * (T->p + 1) + a] : T->val[g * (T->p + 1) + a];
}

/* ------------------------------------------------------------------ */
/* Exact (Gauss) rows, computed row by row.                            */
/* ------------------------------------------------------------------ */
static int problem_ok(const orc_problem* P)
{
    if (P->dim < 2 || P->dim > 3) return 0;
    if (P->p < 1 || P->p > ORC_MAXP) return 0;
    for (int d = 0; d < P->dim; ++d) if (P->n_el[d] < 1) return 0;
    if (P->kappa_kind == ORC_KAPPA_BSPLINE3) {
        if (!P->kappa_ctrl) return 0;
        for (int d = 0; d < P->dim; ++d) if (P->kappa_nctrl[d] < 4 || P->kappa_nctrl[d] > 64) return 0;
    }
    return 1;
}

int64_t orc_num_dofs(const orc_problem* P)
{
    int64_t N = 1;
    for (int d = 0; d < P->dim; ++d) N *= (int64_t)(P->n_el[d] + P->p);
    return N;
}

int orc_num_slots(const orc_problem* P)
{
    int S = 1;
    for (int d = 0; d < P->dim; ++d) S *= 2 * P->p + 1;
    return S;
}

/* Row i: out[s] = sum over elements in supp(B_i), Gauss points x_g:
 *   w_g * grad B_i(x_g)^T K(x_g) grad B_j(x_g),  j = i + delta_s.          */
static void exact_row(const orc_problem* P, const tab1d* T, int64_t row, double* out)
{
    int n = P->dim, p = P->p, w = 2 * p + 1;
    int S = orc_num_slots(P);
    int m[3] = {1, 1, 1}, ii[3] = {0, 0, 0};
    for (int d = 0; d < n; ++d) m[d] = P->n_el[d] + p;
    int64_t rem = row;
    for (int d = 0; d < n; ++d) { ii[d] = (int)(rem % m[d]); rem /= m[d]; }
    for (int s = 0; s < S; ++s) out[s] = 0.0;

    int elo[3] = {0, 0, 0}, ehi[3] = {0, 0, 0};
    for (int d = 0; d < n; ++d) {
        elo[d] = ii[d] - p < 0 ? 0 : ii[d] - p;
        ehi[d] = ii[d] > P->n_el[d] - 1 ? P->n_el[d] - 1 : ii[d];
    }
    int e[3] = {0, 0, 0}, r[3] = {0, 0, 0};
    for (e[2] = (n == 3 ? elo[2] : 0); e[2] <= (n == 3 ? ehi[2] : 0); ++e[2])
    for (e[1] = elo[1]; e[1] <= ehi[1]; ++e[1])
    for (e[0] = elo[0]; e[0] <= ehi[0]; ++e[0])
    for (r[2] = 0; r[2] <= (n == 3 ? p : 0); ++r[2])
    for (r[1] = 0; r[1] <= p; ++r[1])
    for (r[0] = 0; r[0] <= p; ++r[0]) {
        int g[3] = {0, 0, 0};
        double xi[3] = {0, 0, 0}, wgt = 1.0;
        for (int d = 0; d < n; ++d) {
            g[d] = e[d] * (p + 1) + r[d];
            xi[d] = T[d].xi[g[d]];
            wgt *= T[d].wq[g[d]];
        }
        double K[9];
        orc_coefficient(P, xi, K);
        /* grad B_i */
        double gi[3] = {0, 0, 0};
        for (int k = 0; k < n; ++k) {
            double v = 1.0;
            for (int d = 0; d < n; ++d) v *= tab_get(&T[d], g[d], ii[d], d == k);
            gi[k] = v;
        }
        /* K^T grad B_i, so that grad B_i^T K grad B_j = (K^T gi) . gj */
        double Kgi[3] = {0, 0, 0};
        for (int l = 0; l < n; ++l) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += gi[k] * K[k * 3 + l];
            Kgi[l] = s;
        }
        for (int s = 0; s < S; ++s) {
            int jj[3] = {0, 0, 0}, ok = 1, rs = s;
            for (int d = 0; d < n; ++d) {
                int delta = rs % w - p; rs /= w;
                jj[d] = ii[d] + delta;
                if (jj[d] < 0 || jj[d] >= m[d]) ok = 0;
                /* B_j vanishes on this element unless e_d <= j_d <= e_d + p */
                else if (jj[d] < e[d] || jj[d] > e[d] + p) ok = 0;
            }
            if (!ok) continue;
            double acc = 0.0;
            for (int l = 0; l < n; ++l) {
                double v = 1.0;
                for (int d = 0; d < n; ++d) v *= tab_get(&T[d], g[d], jj[d], d == l);
                acc += Kgi[l] * v;
            }
            out[s] += wgt * acc;
        }
    }
}

/* |det Dphi(xi)|: the weight of the mass form m(u,v) = int_Omega u v dx pulled
   back to the parameter domain (Sec. 8, proof of the mass-matrix corollary). */
static double jac_det_abs(const orc_problem* P, const double* xi)
{
    double x[3], J[9];
    orc_map(P, xi, x, J);
    double det;
    if (P->dim == 2) {
        det = J[0] * J[4] - J[1] * J[3];
    } else {
        det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
              J[2] * (J[3] * J[7] - J[4] * J[6]);
    }
    return fabs(det);
}

/* Mass row i: M_ij = sum_g w_g |det Dphi(g)| B_i(g) B_j(g) over the elements of
   supp(B_i), the same Gauss rule and slot order as exact_row. */
static void mass_row(const orc_problem* P, const tab1d* T, int64_t row, double* out)
{
    int n = P->dim, p = P->p, w = 2 * p + 1;
    int S = orc_num_slots(P);
    int m[3] = {1, 1, 1}, ii[3] = {0, 0, 0};
    for (int d = 0; d < n; ++d) m[d] = P->n_el[d] + p;
    int64_t rem = row;
    for (int d = 0; d < n; ++d) { ii[d] = (int)(rem % m[d]); rem /= m[d]; }
    for (int s = 0; s < S; ++s) out[s] = 0.0;
    int elo[3] = {0, 0, 0}, ehi[3] = {0, 0, 0};
    for (int d = 0; d < n; ++d) {
        elo[d] = ii[d] - p < 0 ? 0 : ii[d] - p;
        ehi[d] = ii[d] > P->n_el[d] - 1 ? P->n_el[d] - 1 : ii[d];
    }
    int e[3] = {0, 0, 0}, r[3] = {0, 0, 0};
    for (e[2] = (n == 3 ? elo[2] : 0); e[2] <= (n == 3 ? ehi[2] : 0); ++e[2])
    for (e[1] = elo[1]; e[1] <= ehi[1]; ++e[1])
    for (e[0] = elo[0]; e[0] <= ehi[0]; ++e[0])
    for (r[2] = 0; r[2] <= (n == 3 ? p : 0); ++r[2])
    for (r[1] = 0; r[1] <= p; ++r[1])
    for (r[0] = 0; r[0] <= p; ++r[0]) {
        int g[3] = {0, 0, 0};
        double xi[3] = {0, 0, 0}, wgt = 1.0;
        for (int d = 0; d < n; ++d) {
            g[d] = e[d] * (p + 1) + r[d];
            xi[d] = T[d].xi[g[d]];
            wgt *= T[d].wq[g[d]];
        }
        wgt *= jac_det_abs(P, xi);
        double bi = 1.0;
        for (int d = 0; d < n; ++d) bi *= tab_get(&T[d], g[d], ii[d], 0);
        for (int s = 0; s < S; ++s) {
            int jj[3] = {0, 0, 0}, ok = 1, rs = s;
            for (int d = 0; d < n; ++d) {
                int delta = rs % w - p; rs /= w;
                jj[d] = ii[d] + delta;
                if (jj[d] < 0 || jj[d] >= m[d]) ok = 0;
                else if (jj[d] < e[d] || jj[d] > e[d] + p) ok = 0;
            }
            if (!ok) continue;
            double bj = 1.0;
            for (int d = 0; d < n; ++d) bj *= tab_get(&T[d], g[d], jj[d], 0);
            out[s] += wgt * bi * bj;
        }
    }
}

static int build_tables(const orc_problem* P, tab1d* T)
{
    for (int d = 0; d < P->dim; ++d)
        if (tab_build(P->p, P->n_el[d], &T[d])) return -2;
    return 0;
}

/* Exact rows for an explicit list of row indices; out is [nrows][S]. */
int orc_exact_rows(const orc_problem* P, int64_t nrows, const int64_t* rows, double* out)
{
    if (!problem_ok(P)) return -1;
    int64_t N = orc_num_dofs(P);
    for (int64_t r = 0; r < nrows; ++r) if (rows[r] < 0 || rows[r] >= N) return -1;
    tab1d T[3];
    memset(T, 0, sizeof(T));
    if (build_tables(P, T)) return -2;
    int S = orc_num_slots(P);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) exact_row(P, T, rows[r], out + r * S);
    for (int d = 0; d < P->dim; ++d) tab_free(&T[d]);
    return 0;
}

/* Mass rows (mass_row) for an explicit list of row indices; out is [nrows][S]. */
int orc_mass_rows(const orc_problem* P, int64_t nrows, const int64_t* rows, double* out)
{
    if (!problem_ok(P)) return -1;
    int64_t N = orc_num_dofs(P);
    for (int64_t r = 0; r < nrows; ++r) if (rows[r] < 0 || rows[r] >= N) return -1;
    tab1d T[3];
    memset(T, 0, sizeof(T));
    if (build_tables(P, T)) return -2;
    int S = orc_num_slots(P);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) mass_row(P, T, rows[r], out + r * S);
    for (int d = 0; d < P->dim; ++d) tab_free(&T[d]);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Element-by-element assembly into a dense N x N matrix (tiny meshes   */
/* only): the textbook loop, used to cross-check the row-wise loop.    */
/* ------------------------------------------------------------------ */
int orc_elementwise_dense(const orc_problem* P, double* A /* N*N, row-major */)
{
    if (!problem_ok(P)) return -1;
    int n = P->dim, p = P->p, nl = p + 1;
    int64_t N = orc_num_dofs(P);
    if (N > 20000) return -1;
    int m[3] = {1, 1, 1};
    for (int d = 0; d < n; ++d) m[d] = P->n_el[d] + p;
    tab1d T[3];
    memset(T, 0, sizeof(T));
    if (build_tables(P, T)) return -2;
    memset(A, 0, sizeof(double) * (size_t)(N * N));
    int nloc = 1;
    for (int d = 0; d < n; ++d) nloc *= nl;
    double* grad = (double*)malloc(sizeof(double) * nloc * 3);
    int64_t* glob = (int64_t*)malloc(sizeof(int64_t) * nloc);
    int e[3] = {0, 0, 0}, r[3] = {0, 0, 0};
    for (e[2] = 0; e[2] < (n == 3 ? P->n_el[2] : 1); ++e[2])
    for (e[1] = 0; e[1] < P->n_el[1]; ++e[1])
    for (e[0] = 0; e[0] < P->n_el[0]; ++e[0]) {
        /* local functions a = (a_0, a_1, a_2), global index e + a */
        for (int la = 0; la < nloc; ++la) {
            int rs = la, gidx[3] = {0, 0, 0};
            for (int d = 0; d < n; ++d) { gidx[d] = e[d] + rs % nl; rs /= nl; }
            glob[la] = gidx[0] + (int64_t)m[0] * (gidx[1] + (int64_t)m[1] * gidx[2]);
        }
        for (r[2] = 0; r[2] <= (n == 3 ? p : 0); ++r[2])
        for (r[1] = 0; r[1] <= p; ++r[1])
        for (r[0] = 0; r[0] <= p; ++r[0]) {
            int g[3] = {0, 0, 0};
            double xi[3] = {0, 0, 0}, wgt = 1.0;
            for (int d = 0; d < n; ++d) {
                g[d] = e[d] * nl + r[d];
                xi[d] = T[d].xi[g[d]];
                wgt *= T[d].wq[g[d]];
            }
            double K[9];
            orc_coefficient(P, xi, K);
            for (int la = 0; la < nloc; ++la) {
                int rs = la, a[3] = {0, 0, 0};
                for (int d = 0; d < n; ++d) { a[d] = rs % nl; rs /= nl; }
                for (int k = 0; k < n; ++k) {
                    double v = 1.0;
                    for (int d = 0; d < n; ++d)
                        v *= (d == k) ? T[d].der[g[d] * nl + a[d]] : T[d].val[g[d] * nl + a[d]];
                    grad[la * 3 + k] = v;
                }
            }
            for (int la = 0; la < nloc; ++la)
                for (int lb = 0; lb < nloc; ++lb) {
                    double s = 0.0;
                    for (int k = 0; k < n; ++k)
                        for (int l = 0; l < n; ++l)
                            s += grad[la * 3 + k] * K[k * 3 + l] * grad[lb * 3 + l];
                    A[glob[la] * N + glob[lb]] += wgt * s;
                }
        }
    }
    free(grad); free(glob);
    for (int d = 0; d < n; ++d) tab_free(&T[d]);
    return 0;
}

/* Number of threads the OpenMP loops use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Manufactured solution u(x) = prod_d sin(k pi x_d), k = 1 and k = 20  */
/* being the paper's "low-" and "high-frequency" Poisson solutions     */
/* (Sec. 7.3): the load vector                                          */
/*   F_i = a(u, B_i) = int_Omega kappa grad u . grad B_i dx            */
/* and the energy a(u, u), pulled back to the parameter domain with    */
/* the same (p+1)-point Gauss rule as the stiffness matrix:            */
/*   grad B_i = J^{-T} grad_xi B_i,  dx = |det J| dxi  (eq. ChangeOfVars). */
/* ------------------------------------------------------------------ */
static void mms_point(const orc_problem* P, int freq, const double* xi, double* gradu_pull, double* dens)
{
    int n = P->dim;
    double x[3] = {0, 0, 0}, J[9];
    orc_map(P, xi, x, J);
    double gu[3] = {0, 0, 0};
    for (int a = 0; a < n; ++a) {
        double v = freq * ORC_PI * cos(freq * ORC_PI * x[a]);
        for (int b = 0; b < n; ++b) if (b != a) v *= sin(freq * ORC_PI * x[b]);
        gu[a] = v;
    }
    /* inverse of J by cofactors: Jinv[b][a] = cof[a][b] / det */
    double det, Jinv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (n == 2) {
        det = J[0] * J[4] - J[1] * J[3];
        Jinv[0] = J[4] / det; Jinv[1] = -J[1] / det; Jinv[3] = -J[3] / det; Jinv[4] = J[0] / det;
    } else {
        det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
              J[2] * (J[3] * J[7] - J[4] * J[6]);
        Jinv[0] = (J[4] * J[8] - J[5] * J[7]) / det;
        Jinv[1] = (J[2] * J[7] - J[1] * J[8]) / det;
        Jinv[2] = (J[1] * J[5] - J[2] * J[4]) / det;
        Jinv[3] = (J[5] * J[6] - J[3] * J[8]) / det;
        Jinv[4] = (J[0] * J[8] - J[2] * J[6]) / det;
        Jinv[5] = (J[2] * J[3] - J[0] * J[5]) / det;
        Jinv[6] = (J[3] * J[7] - J[4] * J[6]) / det;
        Jinv[7] = (J[1] * J[6] - J[0] * J[7]) / det;
        Jinv[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    }
    double f = orc_kappa(P, x) * fabs(det);
    /* grad u . (J^{-T} grad_xi B) = (J^{-1} grad u) . grad_xi B */
    double g2 = 0.0;
    for (int b = 0; b < n; ++b) {
        double s = 0.0;
        for (int a = 0; a < n; ++a) s += Jinv[b * 3 + a] * gu[a];
        gradu_pull[b] = f * s;
        g2 += gu[b] * gu[b];
    }
    *dens = f * g2;
}

int orc_manufactured_load(const orc_problem* P, int freq, double* F /* N */, double* energy)
{
    if (!problem_ok(P) || freq < 1) return -1;
    tab1d T[3];
    memset(T, 0, sizeof(T));
    if (build_tables(P, T)) return -2;
    int n = P->dim, p = P->p;
    int64_t N = orc_num_dofs(P);
    int m[3] = {1, 1, 1};
    for (int d = 0; d < n; ++d) m[d] = P->n_el[d] + p;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t row = 0; row < N; ++row) {
        int ii[3] = {0, 0, 0};
        int64_t rem = row;
        for (int d = 0; d < n; ++d) { ii[d] = (int)(rem % m[d]); rem /= m[d]; }
        int elo[3] = {0, 0, 0}, ehi[3] = {0, 0, 0};
        for (int d = 0; d < n; ++d) {
            elo[d] = ii[d] - p < 0 ? 0 : ii[d] - p;
            ehi[d] = ii[d] > P->n_el[d] - 1 ? P->n_el[d] - 1 : ii[d];
        }
        double acc = 0.0;
        int e[3] = {0, 0, 0}, r[3] = {0, 0, 0};
        for (e[2] = (n == 3 ? elo[2] : 0); e[2] <= (n == 3 ? ehi[2] : 0); ++e[2])
        for (e[1] = elo[1]; e[1] <= ehi[1]; ++e[1])
        for (e[0] = elo[0]; e[0] <= ehi[0]; ++e[0])
        for (r[2] = 0; r[2] <= (n == 3 ? p : 0); ++r[2])
        for (r[1] = 0; r[1] <= p; ++r[1])
        for (r[0] = 0; r[0] <= p; ++r[0]) {
            int g[3] = {0, 0, 0};
            double xi[3] = {0, 0, 0}, wgt = 1.0;
            for (int d = 0; d < n; ++d) {
                g[d] = e[d] * (p + 1) + r[d];
                xi[d] = T[d].xi[g[d]];
                wgt *= T[d].wq[g[d]];
            }
            double gp[3], dens;
            mms_point(P, freq, xi, gp, &dens);
            for (int k = 0; k < n; ++k) {
                double v = 1.0;
                for (int d = 0; d < n; ++d) v *= tab_get(&T[d], g[d], ii[d], d == k);
                acc += wgt * gp[k] * v;
            }
        }
        F[row] = acc;
    }
    /* energy: every Gauss point of the patch once */
    double en = 0.0;
    int G[3] = {1, 1, 1};
    for (int d = 0; d < n; ++d) G[d] = T[d].G;
    for (int g2 = 0; g2 < G[2]; ++g2)
    for (int g1 = 0; g1 < G[1]; ++g1)
    for (int g0 = 0; g0 < G[0]; ++g0) {
        int gg[3] = {g0, g1, g2};
        double xi[3] = {0, 0, 0}, wgt = 1.0;
        for (int d = 0; d < n; ++d) { xi[d] = T[d].xi[gg[d]]; wgt *= T[d].wq[gg[d]]; }
        double gp[3], dens;
        mms_point(P, freq, xi, gp, &dens);
        en += wgt * dens;
    }
    *energy = en;
    for (int d = 0; d < P->dim; ++d) tab_free(&T[d]);
    return 0;
}
