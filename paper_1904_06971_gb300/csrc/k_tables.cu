// K1: Gauss rule, B-spline values/derivatives at the Gauss points and the 1-D
//     pair-weight tables of the sum-factorised quadrature.
// K2: the coefficient tensor K = kappa(phi) |det Dphi| Dphi^{-1} Dphi^{-T}
//     (eq. BilinearFormPoissonTensor) at the Gauss points of each box.
#include <math_constants.h>

#include "arith.cuh"
#include "dfmath.cuh"
#include "bspline3.cuh"
#include "iga_internal.cuh"

namespace iga {

// ---------------------------------------------------------------------------
// (p+1)-point Gauss-Legendre rule on [0,1]: Newton's method on the Legendre
// polynomial P_n evaluated by its three-term recurrence; node k of n on
// [-1,1] starts from cos(pi (k + 3/4) / (n + 1/2)).
// ---------------------------------------------------------------------------
__device__ void legendre_eval(int n, double z, double& pn, double& dpn)
{
    double a = 1.0, b = z;                   // P_0, P_1
    for (int j = 2; j <= n; ++j) {
        double c = ((2 * j - 1) * z * b - (j - 1) * a) / j;
        a = b;
        b = c;
    }
    pn = (n == 0) ? 1.0 : b;
    dpn = n * (z * b - a) / (z * z - 1.0);
}

__device__ void gauss_node(int n, int k, double& x01, double& w01)
{
    double z = cospi((k + 0.75) / (n + 0.5));
    double pn, dpn;
    for (int it = 0; it < 64; ++it) {
        legendre_eval(n, z, pn, dpn);
        double dz = pn / dpn;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    legendre_eval(n, z, pn, dpn);
    // ascending order on [0,1]: root k (descending in z) goes to slot n-1-k
    x01 = 0.5 * (1.0 + z);
    w01 = 1.0 / ((1.0 - z * z) * dpn * dpn);
}

// open uniform knot t_k of degree p with n_el elements (m = n_el + p functions)
__device__ __forceinline__ double knot(int k, int p, int n_el)
{
    if (k <= p) return 0.0;
    if (k >= n_el + p) return 1.0;
    return (double)(k - p) / (double)n_el;
}

// Values N[a] and derivatives D[a], a = 0..p, of the p+1 B-splines e..e+p that
// are nonzero on element e at xi, by the local triangular Cox-de Boor scheme
// (span mu = e + p); derivatives from the degree p-1 values.
__device__ void basis_on_element(int p, int n_el, int e, double xi, double* N, double* D)
{
    const int mu = e + p;
    double left[kMaxP + 1], right[kMaxP + 1], prev[kMaxP + 1];
    N[0] = 1.0;
    prev[0] = 1.0;
    for (int k = 1; k <= p; ++k) {
        left[k] = xi - knot(mu + 1 - k, p, n_el);
        right[k] = knot(mu + k, p, n_el) - xi;
        double saved = 0.0;
        for (int r = 0; r < k; ++r) {
            double tmp = N[r] / (right[r + 1] + left[k - r]);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[k - r] * tmp;
        }
        N[k] = saved;
        if (k == p - 1)
            for (int r = 0; r <= k; ++r) prev[r] = N[r];
    }
    // N'_{i,p} = p ( N_{i,p-1} / (t_{i+p} - t_i) - N_{i+1,p-1} / (t_{i+p+1} - t_{i+1}) ), i = e + a
    for (int a = 0; a <= p; ++a) {
        int i = e + a;
        double d = 0.0;
        if (a >= 1) d += prev[a - 1] / (knot(i + p, p, n_el) - knot(i, p, n_el));
        if (a <= p - 1) d -= prev[a] / (knot(i + p + 1, p, n_el) - knot(i + 1, p, n_el));
        D[a] = p * d;
    }
}

struct BasisArgs {
    float2* tdf[3];
    double* gx[3];
    double* sx[3];
    double* cx[3];
    double* bv[3];
    double* bd[3];
    double* wq[3];
};

__global__ void __launch_bounds__(kBlock) k_basis(Geo g, BasisArgs A)
{
    __shared__ double sgx[kMaxP + 1], sgw[kMaxP + 1];
    const int d = blockIdx.y;
    const int p = g.p, Q = p + 1;
    if (threadIdx.x < Q) {
        double x, w;
        gauss_node(Q, threadIdx.x, x, w);
        sgx[Q - 1 - threadIdx.x] = x;
        sgw[Q - 1 - threadIdx.x] = w;
    }
    __syncthreads();
    const int n_el = g.n_el[d];
    const int G = n_el * Q;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= G) return;
    const int e = gi / Q, r = gi % Q;
    const double h = 1.0 / n_el;
    const double xi = (e + sgx[r]) * h;
    A.gx[d][gi] = xi;
    double s, c;
    sincospi(xi, &s, &c);
    A.sx[d][gi] = s;
    A.cx[d][gi] = c;
    A.tdf[d][4 * gi + 0] = PolDF::from_double(s);
    A.tdf[d][4 * gi + 1] = PolDF::from_double(CUDART_PI * c);
    sincospi(2.0 * xi, &s, &c);
    A.sx[d][G + gi] = s;          // sin(2 pi xi), cos(2 pi xi) after the first G entries
    A.cx[d][G + gi] = c;
    A.tdf[d][4 * gi + 2] = PolDF::from_double(s);
    A.tdf[d][4 * gi + 3] = PolDF::from_double(c);
    A.wq[d][gi] = sgw[r] * h;
    double N[kMaxP + 1], D[kMaxP + 1];
    basis_on_element(p, n_el, e, xi, N, D);
    for (int a = 0; a <= p; ++a) {
        A.bv[d][gi * Q + a] = N[a];
        A.bd[d][gi * Q + a] = D[a];
    }
}

cudaError_t launch_basis(const Geo& g, double* gx[3], double* sx[3], double* cx[3],
                         double* bv[3], double* bd[3], double* wq[3], float2* tdf[3], cudaStream_t s)
{
    BasisArgs A;
    int Gmax = 0;
    for (int d = 0; d < 3; ++d) {
        A.tdf[d] = tdf[d];
        A.gx[d] = gx[d]; A.sx[d] = sx[d]; A.cx[d] = cx[d];
        A.bv[d] = bv[d]; A.bd[d] = bd[d]; A.wq[d] = wq[d];
        if (d < g.dim && g.n_el[d] * (g.p + 1) > Gmax) Gmax = g.n_el[d] * (g.p + 1);
    }
    dim3 grid((Gmax + kBlock - 1) / kBlock, g.dim);
    launch_begin(K_BASIS, s);
    k_basis<<<grid, kBlock, 0, s>>>(g, A);
    launch_end(K_BASIS, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pair weights.  For direction d, row function i, offset delta (column
// j = i + delta) and local point t = a (p+1) + r of supp(B_i) (element
// e = i - p + a, Gauss point r), pattern pat = 2 alpha + beta:
//   X[i][delta + p][t][pat] = w_r h  b_i^(alpha)(x_g)  b_j^(beta)(x_g),
// zero when e is outside the mesh, j outside [0, m) or b_j vanishes on e.
// The product over directions of these factors, summed over the Gauss
// points, is the quadrature of d^alpha B_i d^beta B_j (Sec. 3.2, eq. ChangeOfVars).
// ---------------------------------------------------------------------------
struct PairArgs {
    const double* bv[3];
    const double* bd[3];
    const double* wq[3];
    double* X[3];
    void* Xs[3];
};

template <class Pol>
__global__ void __launch_bounds__(kBlock) k_pairs(Geo g, PairArgs A)
{
    const int d = blockIdx.y;
    const int p = g.p, Q = p + 1, W = 2 * p + 1, TT = Q * Q;
    const int m = g.m[d], n_el = g.n_el[d];
    const int64_t total = (int64_t)4 * m * W * TT;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int pat = (int)(idx % 4);
    int64_t rest = idx / 4;
    const int t = (int)(rest % TT);
    rest /= TT;
    const int dd = (int)(rest % W);
    const int i = (int)(rest / W);
    const int alpha = pat >> 1, beta = pat & 1;
    const int e = i - p + t / Q, r = t % Q;
    const int j = i + dd - p;
    double v = 0.0;
    if (e >= 0 && e < n_el && j >= 0 && j < m && j - e >= 0 && j - e <= p) {
        const int gi = e * Q + r;
        const double bi = alpha ? A.bd[d][gi * Q + (i - e)] : A.bv[d][gi * Q + (i - e)];
        const double bj = beta ? A.bd[d][gi * Q + (j - e)] : A.bv[d][gi * Q + (j - e)];
        v = A.wq[d][gi] * bi * bj;
    }
    A.X[d][idx] = v;
    if (Pol::kind != kArithF64) reinterpret_cast<typename Pol::store*>(A.Xs[d])[idx] = Pol::from_double(v);
}

cudaError_t launch_pairs(const Geo& g, double* const bv[3], double* const bd[3],
                         double* const wq[3], double* X[3], void* Xs[3], int arith, cudaStream_t s)
{
    PairArgs A;
    int64_t maxn = 0;
    const int p = g.p;
    for (int d = 0; d < 3; ++d) {
        A.bv[d] = bv[d]; A.bd[d] = bd[d]; A.wq[d] = wq[d]; A.X[d] = X[d]; A.Xs[d] = Xs[d];
        if (d < g.dim) {
            int64_t n = (int64_t)4 * g.m[d] * (2 * p + 1) * (p + 1) * (p + 1);
            if (n > maxn) maxn = n;
        }
    }
    dim3 grid((unsigned)((maxn + kBlock - 1) / kBlock), g.dim);
    launch_begin(K_PAIRS, s);
    if (arith == kArithDF) k_pairs<PolDF><<<grid, kBlock, 0, s>>>(g, A);
    else if (arith == kArithF32) k_pairs<PolF32><<<grid, kBlock, 0, s>>>(g, A);
    else k_pairs<PolF64><<<grid, kBlock, 0, s>>>(g, A);
    launch_end(K_PAIRS, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K2: coefficient fields of a box, SoA over the box's Gauss points
// ([field][g2][g1][g0], g0 fastest).  Fields: 3-D C00 C01 C02 C11 C12 C22,
// 2-D C00 C01 C11.
// ---------------------------------------------------------------------------
__device__ double kappa_at(const Geo& g, const double* x)
{
    switch (g.kappa_kind) {
    case IGA_KAPPA_CONST:
        return g.ka;
    case IGA_KAPPA_SIN2D:
        return g.ka + g.kb * sinpi(2.0 * x[0]) * sinpi(2.0 * x[1]);
    case IGA_KAPPA_EXPSIN3D:
        return exp(g.kb * sinpi(2.0 * x[0]) * cospi(2.0 * x[1]) * sinpi(2.0 * x[2]));
    case IGA_KAPPA_POLY: {
        const int D = g.kappa_deg + 1;
        double v = 0.0;
        const int cmax = (g.dim == 3) ? D : 1;
        for (int c = cmax - 1; c >= 0; --c) {
            double vb = 0.0;
            for (int b = D - 1; b >= 0; --b) {
                double va = 0.0;
                for (int a = D - 1; a >= 0; --a) va = va * x[0] + g.poly[a + D * (b + D * c)];
                vb = vb * x[1] + va;
            }
            v = (g.dim == 3) ? v * x[2] + vb : vb;
        }
        return v;
    }
    case IGA_KAPPA_BSPLINE3: {
        int f[3] = {0, 0, 0};
        double N[3][4] = {{1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}};
        for (int d = 0; d < g.dim; ++d) {
            const double xd = fmin(fmax(x[d], 0.0), 1.0);
            cubic_open_basis(g.knc[d] - 3, xd, f[d], N[d]);
        }
        const int n0 = g.knc[0], n1 = g.knc[1];
        const int nc2 = (g.dim == 3) ? 4 : 1;
        double v = 0.0;
        for (int c = 0; c < nc2; ++c)
            for (int b = 0; b < 4; ++b) {
                const double* row = g.kctrl + f[0] + (int64_t)n0 * ((f[1] + b) + (int64_t)n1 * (f[2] + c));
                const double w = N[1][b] * N[2][c];
                v += w * (((row[0] * N[0][0] + row[1] * N[0][1]) + row[2] * N[0][2]) + row[3] * N[0][3]);
            }
        return v;
    }
    default:
        return 0.0;
    }
}

// kappa at the physical point x (double-float) for IGA_KAPPA_BSPLINE3: the cubic
// basis per direction in double-float and the 4^n control values from their
// double-float copy.
__device__ df2 kappa_bspline_df(const Geo& g, const df2* x)
{
    int f[3] = {0, 0, 0};
    df2 N[3][4];
    for (int d = 0; d < 3; ++d) {
        N[d][0] = df2{1.f, 0.f};
        N[d][1] = N[d][2] = N[d][3] = df2{0.f, 0.f};
    }
    for (int d = 0; d < g.dim; ++d) {
        const int ne = g.knc[d] - 3;
        df2 xc = x[d];
        if (xc.h <= 0.f) xc = df2{0.f, 0.f};
        else if (xc.h >= 1.f) xc = df2{1.f, 0.f};
        int e = (int)(xc.h * (float)ne);
        e = e < 0 ? 0 : (e > ne - 1 ? ne - 1 : e);
        cubic_open_basis_df_span(ne, e, xc, N[d]);
        f[d] = e;
    }
    const int n0 = g.knc[0], n1 = g.knc[1];
    const int nc2 = (g.dim == 3) ? 4 : 1;
    df2 v = {0.f, 0.f};
    for (int c = 0; c < nc2; ++c)
        for (int b = 0; b < 4; ++b) {
            const float2* row = g.kctrl_df + f[0] + (int64_t)n0 * ((f[1] + b) + (int64_t)n1 * (f[2] + c));
            df2 r = df_mul(df2{row[0].x, row[0].y}, N[0][0]);
#pragma unroll
            for (int a = 1; a < 4; ++a) r = df_fma(df2{row[a].x, row[a].y}, N[0][a], r);
            v = df_fma(df_mul(N[1][b], N[2][c]), r, v);
        }
    return v;
}

__global__ void k_split_ctrl(const double* ctrl, int64_t n, float2* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = d2df_split(ctrl[i]);
}

cudaError_t launch_split_ctrl(const double* ctrl, int64_t n, float2* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    launch_begin(K_COEF, s);
    k_split_ctrl<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(ctrl, n, out);
    launch_end(K_COEF, s);
    return cudaGetLastError();
}

template <int DIM, class Pol>
__global__ void __launch_bounds__(kBlock) k_coef(Geo g, Tables T, BoxSet bs, double* scratch)
{
    Box b;
    get_box(bs, DIM, g.p, 0, blockIdx.x, b);
    const int Q = g.p + 1;
    const int64_t G0 = (int64_t)b.E[0] * Q, G1 = (int64_t)b.E[1] * Q, G2 = (DIM == 3) ? (int64_t)b.E[2] * Q : 1;
    const int64_t npts = G0 * G1 * G2;
    const int64_t item = (int64_t)(blockIdx.x - b.blk[0]) * kBlock + threadIdx.x;
    if (item >= npts) return;
    int gl[3];
    gl[0] = (int)(item % G0);
    gl[1] = (int)((item / G0) % G1);
    gl[2] = (int)(item / (G0 * G1));
    double xi[3] = {0, 0, 0}, x[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    int gg[3];
    for (int d = 0; d < DIM; ++d) {
        gg[d] = b.elo[d] * Q + gl[d];
        xi[d] = T.gx[d][gg[d]];
    }
    typename Pol::store* out = reinterpret_cast<typename Pol::store*>(scratch + b.c_off);
    if (g.form == kFormMass) {
        // the mass form's only field: |det Dphi| (Sec. 8), det = 1 + amp sum_b gr_b
        // for the sine-product map.  FP32 contractions take it in FP32, double-float
        // ones in double-float arithmetic (FP32 pipe), FP64 ones in FP64.
        if (Pol::kind != kArithF64 && g.coef_df && g.map_kind == IGA_MAP_SINPROD) {
            df2 sv[3], pcv[3];
            for (int d = 0; d < DIM; ++d) {
                const float2* t4 = T.tdf[d] + 4 * gg[d];
                sv[d] = df2{t4[0].x, t4[0].y};
                pcv[d] = df2{t4[1].x, t4[1].y};
            }
            if (Pol::kind == kArithF32) {
                float gsum = (DIM == 3) ? pcv[0].h * (sv[1].h * sv[2].h) + pcv[1].h * (sv[0].h * sv[2].h) +
                                              pcv[2].h * (sv[0].h * sv[1].h)
                                        : pcv[0].h * sv[1].h + pcv[1].h * sv[0].h;
                reinterpret_cast<float*>(out)[item] = fabsf(fmaf(g.amp_df[0], gsum, 1.f));
                return;
            }
            df2 gsum;
            if (DIM == 3) {
                gsum = df_add(df_add(df_mul(pcv[0], df_mul(sv[1], sv[2])), df_mul(pcv[1], df_mul(sv[0], sv[2]))),
                              df_mul(pcv[2], df_mul(sv[0], sv[1])));
            } else {
                gsum = df_add(df_mul(pcv[0], sv[1]), df_mul(pcv[1], sv[0]));
            }
            const df2 det = df_abs(df_fma(df2{g.amp_df[0], g.amp_df[1]}, gsum, df2{1.f, 0.f}));
            reinterpret_cast<float2*>(out)[item] = make_float2(det.h, det.l);
            return;
        }
        double det = 1.0;
        if (g.map_kind == IGA_MAP_SINPROD) {
            // Dphi = I + amp 1 gr^T, gr_b = dP/dxi_b: det = 1 + amp sum_b gr_b
            double sv[3], cv[3], gsum = 0.0;
            for (int d = 0; d < DIM; ++d) { sv[d] = T.sx[d][gg[d]]; cv[d] = T.cx[d][gg[d]]; }
            for (int bdir = 0; bdir < DIM; ++bdir) {
                double dP = CUDART_PI * cv[bdir];
                for (int j = 0; j < DIM; ++j) if (j != bdir) dP *= sv[j];
                gsum += dP;
            }
            det = 1.0 + g.amp * gsum;
        } else if (g.map_kind == IGA_MAP_AFFINE) {
            const double* A = g.aff;
            det = (DIM == 2) ? A[0] * A[4] - A[1] * A[3]
                             : A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                                   A[2] * (A[3] * A[7] - A[4] * A[6]);
        }
        out[item] = Pol::from_double(fabs(det));
        return;
    }
    if (Pol::kind == kArithF32 && g.coef_df) {
        // FP32 contractions: the same formulas in FP32 (the hi parts of the
        // double-float tables), whose rounding is of the order of the FP32
        // contractions' own.
        float sv[3], pcv[3], S2[3], C2[3];
        for (int d = 0; d < DIM; ++d) {
            const float2* t4 = T.tdf[d] + 4 * gg[d];
            sv[d] = t4[0].x; pcv[d] = t4[1].x; S2[d] = t4[2].x; C2[d] = t4[3].x;
        }
        float gr[3], P;
        if (DIM == 3) {
            gr[0] = pcv[0] * (sv[1] * sv[2]);
            gr[1] = pcv[1] * (sv[0] * sv[2]);
            gr[2] = pcv[2] * (sv[0] * sv[1]);
            P = sv[0] * (sv[1] * sv[2]);
        } else {
            gr[0] = pcv[0] * sv[1];
            gr[1] = pcv[1] * sv[0];
            gr[2] = 0.f;
            P = sv[0] * sv[1];
        }
        float gsum = 0.f, gg2 = 0.f;
        for (int d = 0; d < DIM; ++d) { gsum += gr[d]; gg2 = fmaf(gr[d], gr[d], gg2); }
        const float amp = g.amp_df[0];
        const float det = fmaf(amp, gsum, 1.f);
        const float cc = amp / det;
        const float c2g = cc * cc * gg2;
        float kap = g.ka_df[0];
        if (g.kappa_kind == IGA_KAPPA_SIN2D || g.kappa_kind == IGA_KAPPA_EXPSIN3D) {
            float st, ct;
            sincospif(2.f * amp * P, &st, &ct);
            const float kb = g.kb_df[0];
            const float sin0 = fmaf(S2[0], ct, C2[0] * st);
            if (g.kappa_kind == IGA_KAPPA_SIN2D) {
                kap = fmaf(kb, sin0 * fmaf(S2[1], ct, C2[1] * st), kap);
            } else {
                const float cos1 = C2[1] * ct - S2[1] * st;
                const float sin2 = fmaf(S2[2], ct, C2[2] * st);
                kap = expf(kb * sin0 * cos1 * sin2);
            }
        }
        const float f = kap * fabsf(det);
        int k = 0;
        for (int a = 0; a < DIM; ++a)
            for (int bdir = a; bdir < DIM; ++bdir, ++k) {
                float m = c2g - cc * (gr[a] + gr[bdir]);
                if (a == bdir) m += 1.f;
                reinterpret_cast<float*>(out)[k * npts + item] = f * m;
            }
        return;
    }
    if (Pol::kind != kArithF64 && g.coef_df) {
        // Same formulas as the FP64 branch below, in double-float arithmetic on
        // the FP32 pipe (dfmath.cuh): the result is stored in double-float (or
        // float) anyway, and GB300's FP64 pipe is 64x slower than its FP32 pipe.
        df2 sv[3], pcv[3], S2[3], C2[3];
        for (int d = 0; d < DIM; ++d) {
            const float2* t4 = T.tdf[d] + 4 * gg[d];
            sv[d] = df2{t4[0].x, t4[0].y};
            pcv[d] = df2{t4[1].x, t4[1].y};
            S2[d] = df2{t4[2].x, t4[2].y};
            C2[d] = df2{t4[3].x, t4[3].y};
        }
        df2 gr[3], P;
        if (DIM == 3) {
            const df2 q12 = df_mul(sv[1], sv[2]), q02 = df_mul(sv[0], sv[2]), q01 = df_mul(sv[0], sv[1]);
            gr[0] = df_mul(pcv[0], q12);
            gr[1] = df_mul(pcv[1], q02);
            gr[2] = df_mul(pcv[2], q01);
            P = df_mul(sv[0], q12);
        } else {
            gr[0] = df_mul(pcv[0], sv[1]);
            gr[1] = df_mul(pcv[1], sv[0]);
            gr[2] = df2{0.f, 0.f};
            P = df_mul(sv[0], sv[1]);
        }
        df2 gsum = gr[0], gg2 = df_mul(gr[0], gr[0]);
        for (int d = 1; d < DIM; ++d) {
            gsum = df_add(gsum, gr[d]);
            gg2 = df_fma(gr[d], gr[d], gg2);
        }
        const df2 amp = df2{g.amp_df[0], g.amp_df[1]};
        const df2 det = df_fma(amp, gsum, df2{1.f, 0.f});
        const df2 cc = df_div(amp, det);
        const df2 c2g = df_mul(df_mul(cc, cc), gg2);
        df2 kap = df2{g.ka_df[0], g.ka_df[1]};
        if (g.kappa_kind == IGA_KAPPA_BSPLINE3) {
            // the physical point x_a = xi_a + amp P, then the spline
            df2 x[3];
            for (int a = 0; a < DIM; ++a) {
                const float2 xs = d2df_split(xi[a]);
                x[a] = df_fma(amp, P, df2{xs.x, xs.y});
            }
            kap = kappa_bspline_df(g, x);
        } else if (g.kappa_kind == IGA_KAPPA_SIN2D || g.kappa_kind == IGA_KAPPA_EXPSIN3D) {
            const df2 th = df_add(amp, amp);
            df2 st, ct;
            df_sincospi_small(df_mul(th, P), st, ct);
            const df2 kb = df2{g.kb_df[0], g.kb_df[1]};
            const df2 sin0 = df_fma(S2[0], ct, df_mul(C2[0], st));
            if (g.kappa_kind == IGA_KAPPA_SIN2D) {
                const df2 sin1 = df_fma(S2[1], ct, df_mul(C2[1], st));
                kap = df_fma(kb, df_mul(sin0, sin1), kap);
            } else {
                const df2 cos1 = df_sub(df_mul(C2[1], ct), df_mul(S2[1], st));
                const df2 sin2 = df_fma(S2[2], ct, df_mul(C2[2], st));
                kap = df_exp_small(df_mul(kb, df_mul(sin0, df_mul(cos1, sin2))));
            }
        }
        const df2 f = df_mul(kap, df_abs(det));
        int k = 0;
        for (int a = 0; a < DIM; ++a)
            for (int bdir = a; bdir < DIM; ++bdir, ++k) {
                df2 m = df_add(df_neg(df_mul(cc, df_add(gr[a], gr[bdir]))), c2g);
                if (a == bdir) m = df_add(m, df2{1.f, 0.f});
                const df2 v = df_mul(f, m);
                if (Pol::kind == kArithDF) reinterpret_cast<float2*>(out)[k * npts + item] = make_float2(v.h, v.l);
                else reinterpret_cast<float*>(out)[k * npts + item] = __fadd_rn(v.h, v.l);
            }
        return;
    }
    if (g.map_kind == IGA_MAP_SINPROD) {
        // x = xi + amp P 1 with P = prod_j sin(pi xi_j): Dphi = I + amp 1 gr^T,
        // gr_b = dP / dxi_b.  A rank-one update of I, so (Sherman-Morrison)
        //   det = 1 + amp sum_b gr_b,  Dphi^{-1} = I - c 1 gr^T,  c = amp / det,
        //   Dphi^{-1} Dphi^{-T} = I - c (1 gr^T + gr 1^T) + c^2 |gr|^2 1 1^T.
        double s[3], c[3], P = 1.0;
        for (int d = 0; d < DIM; ++d) { s[d] = T.sx[d][gg[d]]; c[d] = T.cx[d][gg[d]]; P *= s[d]; }
        double gr[3], gsum = 0.0, gg2 = 0.0;
        for (int bdir = 0; bdir < DIM; ++bdir) {
            double dP = CUDART_PI * c[bdir];
            for (int j = 0; j < DIM; ++j) if (j != bdir) dP *= s[j];
            gr[bdir] = dP;
            gsum += dP;
            gg2 += dP * dP;
        }
        const double det = 1.0 + g.amp * gsum;
        const double cc = g.amp / det;
        // kappa at x_a = xi_a + amp P: sin / cos of 2 pi x_a by angle addition from the
        // tabulated sin / cos of 2 pi xi_a and one sincos of 2 pi amp P
        double kap;
        if (g.kappa_kind == IGA_KAPPA_SIN2D || g.kappa_kind == IGA_KAPPA_EXPSIN3D) {
            double st, ct;
            sincospi(2.0 * g.amp * P, &st, &ct);
            const int64_t G0 = (int64_t)g.n_el[0] * Q, G1 = (int64_t)g.n_el[1] * Q;
            const double S0 = T.sx[0][G0 + gg[0]], C0 = T.cx[0][G0 + gg[0]];
            const double S1 = T.sx[1][G1 + gg[1]], C1 = T.cx[1][G1 + gg[1]];
            const double sin0 = S0 * ct + C0 * st;
            if (g.kappa_kind == IGA_KAPPA_SIN2D) {
                kap = g.ka + g.kb * sin0 * (S1 * ct + C1 * st);
            } else {
                const int64_t G2 = (int64_t)g.n_el[2] * Q;
                const double S2 = T.sx[2][G2 + gg[2]], C2 = T.cx[2][G2 + gg[2]];
                kap = exp(g.kb * sin0 * (C1 * ct - S1 * st) * (S2 * ct + C2 * st));
            }
        } else {
            for (int a = 0; a < DIM; ++a) x[a] = xi[a] + g.amp * P;
            kap = kappa_at(g, x);
        }
        const double f = kap * fabs(det), c2g = cc * cc * gg2;
        int k = 0;
        for (int a = 0; a < DIM; ++a)
            for (int bdir = a; bdir < DIM; ++bdir, ++k)
                out[k * npts + item] = Pol::from_double(f * ((a == bdir ? 1.0 : 0.0) - cc * (gr[a] + gr[bdir]) + c2g));
        return;
    } else if (g.map_kind == IGA_MAP_AFFINE) {
        for (int a = 0; a < DIM; ++a) {
            x[a] = g.aff[9 + a];
            for (int bdir = 0; bdir < DIM; ++bdir) {
                J[a][bdir] = g.aff[a * 3 + bdir];
                x[a] += J[a][bdir] * xi[bdir];
            }
        }
    } else {
        for (int a = 0; a < DIM; ++a) { x[a] = xi[a]; J[a][a] = 1.0; }
    }
    const double kap = kappa_at(g, x);
    // K = kappa |det J| J^{-1} J^{-T} = kappa / |det J| adj(J) adj(J)^T
    if (DIM == 2) {
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double a00 = J[1][1], a01 = -J[0][1], a10 = -J[1][0], a11 = J[0][0];
        const double f = kap / fabs(det);
        out[0 * npts + item] = Pol::from_double(f * (a00 * a00 + a01 * a01));
        out[1 * npts + item] = Pol::from_double(f * (a00 * a10 + a01 * a11));
        out[2 * npts + item] = Pol::from_double(f * (a10 * a10 + a11 * a11));
    } else {
        double adj[3][3];
        adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
        const double f = kap / fabs(det);
        auto row = [&](int a, int c) { return adj[a][0] * adj[c][0] + adj[a][1] * adj[c][1] + adj[a][2] * adj[c][2]; };
        out[0 * npts + item] = Pol::from_double(f * row(0, 0));
        out[1 * npts + item] = Pol::from_double(f * row(0, 1));
        out[2 * npts + item] = Pol::from_double(f * row(0, 2));
        out[3 * npts + item] = Pol::from_double(f * row(1, 1));
        out[4 * npts + item] = Pol::from_double(f * row(1, 2));
        out[5 * npts + item] = Pol::from_double(f * row(2, 2));
    }
}

void prepare_coef_df(Geo& g, int arith)
{
    auto split = [](double v, float* out) {
        out[0] = (float)v;
        out[1] = (float)(v - (double)out[0]);
    };
    split(g.amp, g.amp_df);
    split(g.ka, g.ka_df);
    split(g.kb, g.kb_df);
    const bool kappa_ok = g.kappa_kind == IGA_KAPPA_CONST || g.kappa_kind == IGA_KAPPA_SIN2D ||
                          (g.kappa_kind == IGA_KAPPA_EXPSIN3D && fabs(g.kb) <= 1.0) ||
                          (g.kappa_kind == IGA_KAPPA_BSPLINE3 && g.kctrl_split);
    g.coef_df = (arith != kArithF64 && g.map_kind == IGA_MAP_SINPROD && fabs(g.amp) <= 0.07 && kappa_ok) ? 1 : 0;
}

cudaError_t launch_coef(const Geo& g, const Tables& T, const BoxSet& bs, int64_t nblocks,
                        double* scratch, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    launch_begin(K_COEF, s);
    const unsigned grid = (unsigned)nblocks;
    if (g.dim == 3) {
        if (T.arith == kArithDF) k_coef<3, PolDF><<<grid, kBlock, 0, s>>>(g, T, bs, scratch);
        else if (T.arith == kArithF32) k_coef<3, PolF32><<<grid, kBlock, 0, s>>>(g, T, bs, scratch);
        else k_coef<3, PolF64><<<grid, kBlock, 0, s>>>(g, T, bs, scratch);
    } else {
        if (T.arith == kArithDF) k_coef<2, PolDF><<<grid, kBlock, 0, s>>>(g, T, bs, scratch);
        else if (T.arith == kArithF32) k_coef<2, PolF32><<<grid, kBlock, 0, s>>>(g, T, bs, scratch);
        else k_coef<2, PolF64><<<grid, kBlock, 0, s>>>(g, T, bs, scratch);
    }
    launch_end(K_COEF, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Manufactured solution u(x) = prod_d sin(k pi x_d) of the paper's Poisson
// experiments (Sec. 7.3; k = 1 and k = 20 there): load F_i = a(u, B_i) = int kappa grad u . grad B_i dx
// and energy a(u, u), pulled back with the assembly's Gauss rule
// (grad B_i = J^{-T} grad_xi B_i, dx = |det J| dxi, eq. ChangeOfVars), in FP64.
// Pass 1 (every Gauss point of the patch): v = w kappa |det J| J^{-1} grad u
// and e = w kappa |det J| |grad u|^2.  Pass 2 (one thread per basis function):
// F_i = sum over the Gauss points of supp(B_i) of v . grad_xi B_i.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_mms_points(Geo g, MmsArgs A)
{
    const int Q = g.p + 1;
    const int64_t G0 = (int64_t)g.n_el[0] * Q, G1 = (int64_t)g.n_el[1] * Q;
    const int64_t G2 = (DIM == 3) ? (int64_t)g.n_el[2] * Q : 1;
    const int64_t npts = G0 * G1 * G2;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= npts) return;
    const int gg[3] = {(int)(item % G0), (int)((item / G0) % G1), (int)(item / (G0 * G1))};
    double xi[3] = {0, 0, 0}, x[3] = {0, 0, 0}, w = 1.0;
    for (int d = 0; d < DIM; ++d) { xi[d] = A.gx[d][gg[d]]; w *= A.wq[d][gg[d]]; }
    double Ji[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, det = 1.0;
    if (g.map_kind == IGA_MAP_SINPROD) {
        // J = I + amp 1 gr^T: det = 1 + amp sum gr, J^{-1} = I - c 1 gr^T, c = amp / det
        double sv[3], cv[3], P = 1.0, gr[3] = {0, 0, 0}, gsum = 0.0;
        for (int d = 0; d < DIM; ++d) { sincospi(xi[d], &sv[d], &cv[d]); P *= sv[d]; }
        for (int b = 0; b < DIM; ++b) {
            double v = CUDART_PI * cv[b];
            for (int j = 0; j < DIM; ++j) if (j != b) v *= sv[j];
            gr[b] = v;
            gsum += v;
        }
        det = 1.0 + g.amp * gsum;
        const double c = g.amp / det;
        for (int a = 0; a < DIM; ++a) {
            x[a] = xi[a] + g.amp * P;
            for (int b = 0; b < DIM; ++b) Ji[a][b] = (a == b ? 1.0 : 0.0) - c * gr[b];
        }
    } else if (g.map_kind == IGA_MAP_AFFINE) {
        double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int a = 0; a < DIM; ++a) {
            x[a] = g.aff[9 + a];
            for (int b = 0; b < DIM; ++b) { J[a][b] = g.aff[a * 3 + b]; x[a] += J[a][b] * xi[b]; }
        }
        if (DIM == 2) {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det; Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
        } else {
            det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                  J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    // cofactor of J[b][a] over det
                    const int r0 = (b + 1) % 3, r1 = (b + 2) % 3, c0 = (a + 1) % 3, c1 = (a + 2) % 3;
                    Ji[a][b] = (J[r0][c0] * J[r1][c1] - J[r0][c1] * J[r1][c0]) / det;
                }
        }
    } else {
        for (int a = 0; a < DIM; ++a) x[a] = xi[a];
    }
    double su[3], cu[3];
    for (int d = 0; d < DIM; ++d) sincospi((double)A.freq * x[d], &su[d], &cu[d]);
    double gu[3] = {0, 0, 0}, g2 = 0.0;
    for (int a = 0; a < DIM; ++a) {
        double v = A.freq * CUDART_PI * cu[a];
        for (int b = 0; b < DIM; ++b) if (b != a) v *= su[b];
        gu[a] = v;
        g2 += v * v;
    }
    const double f = w * kappa_at(g, x) * fabs(det);
    for (int a = 0; a < DIM; ++a) {
        double v = 0.0;
        for (int b = 0; b < DIM; ++b) v += Ji[a][b] * gu[b];
        A.V[a * npts + item] = f * v;
    }
    A.E[item] = f * g2;
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) k_mms_rows(Geo g, MmsArgs A, double* F)
{
    const int p = g.p, Q = p + 1;
    const int64_t N = (int64_t)g.m[0] * g.m[1] * (DIM == 3 ? g.m[2] : 1);
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    const int64_t G0 = (int64_t)g.n_el[0] * Q, G1 = (int64_t)g.n_el[1] * Q;
    const int64_t G2 = (DIM == 3) ? (int64_t)g.n_el[2] * Q : 1;
    const int64_t npts = G0 * G1 * G2;
    const int ii[3] = {(int)(row % g.m[0]), (int)((row / g.m[0]) % g.m[1]), (int)(row / ((int64_t)g.m[0] * g.m[1]))};
    int elo[3] = {0, 0, 0}, ehi[3] = {0, 0, 0};
    for (int d = 0; d < DIM; ++d) { elo[d] = max(0, ii[d] - p); ehi[d] = min(g.n_el[d] - 1, ii[d]); }
    double acc = 0.0;
    for (int e2 = elo[2]; e2 <= ehi[2]; ++e2)
    for (int r2 = 0; r2 < (DIM == 3 ? Q : 1); ++r2) {
        const int g2i = e2 * Q + r2;
        const double v2 = (DIM == 3) ? A.bv[2][g2i * Q + (ii[2] - e2)] : 1.0;
        const double d2 = (DIM == 3) ? A.bd[2][g2i * Q + (ii[2] - e2)] : 0.0;
        for (int e1 = elo[1]; e1 <= ehi[1]; ++e1)
        for (int r1 = 0; r1 < Q; ++r1) {
            const int g1i = e1 * Q + r1;
            const double v1 = A.bv[1][g1i * Q + (ii[1] - e1)], d1 = A.bd[1][g1i * Q + (ii[1] - e1)];
            for (int e0 = elo[0]; e0 <= ehi[0]; ++e0)
            for (int r0 = 0; r0 < Q; ++r0) {
                const int g0i = e0 * Q + r0;
                const double v0 = A.bv[0][g0i * Q + (ii[0] - e0)], d0 = A.bd[0][g0i * Q + (ii[0] - e0)];
                const int64_t pt = g0i + G0 * (g1i + G1 * (int64_t)(DIM == 3 ? g2i : 0));
                double t = A.V[pt] * d0 * v1 + A.V[npts + pt] * v0 * d1;
                if (DIM == 3) t = t * v2 + A.V[2 * npts + pt] * v0 * v1 * d2;
                acc += t;
            }
        }
    }
    F[row] = acc;
}

// deterministic sum: per-block tree sums in a fixed order, then one block over the partial sums
__global__ void __launch_bounds__(kBlock) k_sum_partial(int64_t n, const double* a, double* partial)
{
    __shared__ double sh[kBlock];
    double s = 0.0;
    const int64_t per = (int64_t)kBlock * 8;
    const int64_t base = (int64_t)blockIdx.x * per;
    for (int k = 0; k < 8; ++k) {
        const int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
        if (i < n) s += a[i];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

cudaError_t launch_manufactured(const Geo& g, const MmsArgs& A, double* F, double* energy, double* partial,
                                int64_t npart, cudaStream_t s)
{
    const int Q = g.p + 1;
    int64_t npts = 1, N = 1;
    for (int d = 0; d < g.dim; ++d) { npts *= (int64_t)g.n_el[d] * Q; N *= g.m[d]; }
    const unsigned gp = (unsigned)((npts + kBlock - 1) / kBlock), gr = (unsigned)((N + kBlock - 1) / kBlock);
    launch_begin(K_MMS, s);
    if (g.dim == 3) k_mms_points<3><<<gp, kBlock, 0, s>>>(g, A);
    else k_mms_points<2><<<gp, kBlock, 0, s>>>(g, A);
    launch_end(K_MMS, s);
    launch_begin(K_MMS, s);
    if (g.dim == 3) k_mms_rows<3><<<gr, kBlock, 0, s>>>(g, A, F);
    else k_mms_rows<2><<<gr, kBlock, 0, s>>>(g, A, F);
    launch_end(K_MMS, s);
    // energy: sum of E over the points, then of the partial sums (both deterministic)
    int64_t n = npts;
    const double* src = A.E;
    double* bufs[2] = {partial, partial + npart};
    int k = 0;
    while (true) {
        const int64_t nb = (n + (int64_t)kBlock * 8 - 1) / ((int64_t)kBlock * 8);
        double* dst = (nb == 1) ? energy : bufs[k];
        launch_begin(K_MMS, s);
        k_sum_partial<<<(unsigned)nb, kBlock, 0, s>>>(n, src, dst);
        launch_end(K_MMS, s);
        if (nb == 1) break;
        src = dst;
        n = nb;
        k ^= 1;
    }
    return cudaGetLastError();
}

}  // namespace iga
