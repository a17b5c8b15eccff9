// Adjoint of L = ybar^T A~(kappa) x with respect to the control values c of a
// B-spline diffusion coefficient kappa (IGA_KAPPA_BSPLINE3).
//
// Every step of the surrogate is linear in kappa, and A_ij = sum_g w_g kappa(phi(g))
// grad B_i^T G(g) grad B_j with G = |det Dphi| Dphi^{-1} Dphi^{-T} (Sec. 3.2), so
// every contribution to dL/dc_k has the form sum_g N_k(phi(g)) s(g) for a field s
// on the Gauss points:
//
//   L = sum_{i != j} ybar_i (x_j - x_i) A~_ij              (kernel-preserving diagonal, Sec. 5.3)
//     = ybar^T A x - (R ybar)^T A (R x) + (R(ybar.x))^T A (R 1)    [entries with an exact value]
//       + sum_delta sum_s Phibar_delta(s) A_{s, s+delta}             [interpolated entries]
//
// with R the restriction to Omega~ (A 1 = 0 for every kappa removes the diagonal
// term of the first line).  The first line is a sum of bilinear forms a^T A b,
// whose kappa-derivative field is w_g grad u_a^T G grad u_b (u_v = sum_i v_i B_i),
// evaluated by sum factorisation.  Phibar is the transposed interpolation of the
// weights Z_delta(i) = (ybar_i - ybar_{i+delta})(x_{i+delta} - x_i) of the
// interpolated entries (Sec. 4.1, transposed), and each sample row s adds the
// field w_g grad B_s^T G grad u_{w_s} with w_s = sum_delta Phibar_delta(s) e_{s+delta}
// on the support of B_s.  Finally dL/dc_k = sum_g N_k(phi(g)) s(g).
//
// The basis tables are recomputed by every call.  The sum-factorised fields and
// the geometry are FP64; the point field's gradients and quadratic forms and
// the scatter to the control values (cubic basis and window sums) run in
// double-float arithmetic on the FP32 pipe (GB300's FP64 pipe bounded them).
#include <math_constants.h>

#include "arith.cuh"
#include "bspline3.cuh"
#include "iga_internal.cuh"

namespace iga {

// ---------------------------------------------------------------------------
// geometry at a Gauss point: physical point x and G = |det J| J^{-1} J^{-T}
// ---------------------------------------------------------------------------
__device__ void adj_geometry(const Geo& g, const double* xi, const double* s1, const double* c1, double* x,
                             double G[3][3])
{
    const int n = g.dim;
    double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (g.map_kind == IGA_MAP_SINPROD) {
        // x_a = xi_a + amp prod_j sin(pi xi_j): J = I + amp 1 grad(P)^T
        double P = 1.0;
        for (int d = 0; d < n; ++d) P *= s1[d];
        for (int a = 0; a < n; ++a) x[a] = xi[a] + g.amp * P;
        for (int b = 0; b < n; ++b) {
            double dP = CUDART_PI * c1[b];
            for (int d = 0; d < n; ++d)
                if (d != b) dP *= s1[d];
            for (int a = 0; a < n; ++a) J[a][b] += g.amp * dP;
        }
    } else if (g.map_kind == IGA_MAP_AFFINE) {
        for (int a = 0; a < n; ++a) {
            x[a] = g.aff[9 + a];
            for (int b = 0; b < n; ++b) {
                J[a][b] = g.aff[a * 3 + b];
                x[a] += J[a][b] * xi[b];
            }
        }
    } else {
        for (int a = 0; a < n; ++a) x[a] = xi[a];
    }
    // adjugate: J^{-1} = adj(J) / det, so G = |det| adj adj^T / det^2 = adj adj^T / |det|
    double adj[3][3], det;
    if (n == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        adj[0][0] = J[1][1]; adj[0][1] = -J[0][1];
        adj[1][0] = -J[1][0]; adj[1][1] = J[0][0];
    } else {
        adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
        adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    }
    const double rd = 1.0 / fabs(det);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += adj[a][k] * adj[b][k];
            G[a][b] = rd * v;
        }
}

// physical point alone (no Jacobian)
__device__ __forceinline__ void adj_point(const Geo& g, const double* xi, const double* s1, double* x)
{
    const int n = g.dim;
    if (g.map_kind == IGA_MAP_SINPROD) {
        double P = 1.0;
        for (int d = 0; d < n; ++d) P *= s1[d];
        for (int a = 0; a < n; ++a) x[a] = xi[a] + g.amp * P;
    } else if (g.map_kind == IGA_MAP_AFFINE) {
        for (int a = 0; a < n; ++a) {
            x[a] = g.aff[9 + a];
            for (int b = 0; b < n; ++b) x[a] += g.aff[a * 3 + b] * xi[b];
        }
    } else {
        for (int a = 0; a < n; ++a) x[a] = xi[a];
    }
}

__device__ __forceinline__ double quad_form(int n, const double G[3][3], const double* u, const double* v)
{
    double s = 0.0;
    for (int a = 0; a < n; ++a) {
        double t = 0.0;
        for (int b = 0; b < n; ++b) t += G[a][b] * v[b];
        s += u[a] * t;
    }
    return s;
}

// ---------------------------------------------------------------------------
// Gradient of u_v at every Gauss point, sum-factorised:
//   pass 0 (direction 0): W0[k][i2][i1][g0] = sum_a B0^(k)(g0) v[e0+a, i1, i2], k = value / derivative
//   pass 1 (direction 1): W1[0] = sum_b B1 W0[0], W1[1] = sum_b B1 W0[1], W1[2] = sum_b B1' W0[0]
//   (3-D) the point kernel finishes direction 2.  In 2-D, W1[1], W1[2] are the gradient.
// ---------------------------------------------------------------------------
__global__ void k_adj_pass0(Geo g, AdjTables T, const double* v, double* W0)
{
    const int Q = g.p + 1;
    const int G0 = g.n_el[0] * Q, m0 = g.m[0], m1 = g.m[1], m2 = (g.dim == 3) ? g.m[2] : 1;
    const int64_t tot = (int64_t)m2 * m1 * G0;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int g0 = (int)(idx % G0);
    const int64_t l = idx / G0;                  // i1 + m1 i2
    const int e0 = g0 / Q;
    const double* vl = v + l * m0 + e0;
    double a0 = 0.0, a1 = 0.0;
    for (int a = 0; a < Q; ++a) {
        a0 += T.bv[0][g0 * Q + a] * vl[a];
        a1 += T.bd[0][g0 * Q + a] * vl[a];
    }
    W0[idx] = a0;
    W0[tot + idx] = a1;
}

__global__ void k_adj_pass1(Geo g, AdjTables T, const double* W0, double* W1)
{
    const int Q = g.p + 1;
    const int G0 = g.n_el[0] * Q, G1 = g.n_el[1] * Q, m1 = g.m[1], m2 = (g.dim == 3) ? g.m[2] : 1;
    const int64_t tot = (int64_t)m2 * G1 * G0, tot0 = (int64_t)m2 * m1 * G0;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int g0 = (int)(idx % G0);
    const int g1 = (int)((idx / G0) % G1);
    const int i2 = (int)(idx / ((int64_t)G0 * G1));
    const int e1 = g1 / Q;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int b = 0; b < Q; ++b) {
        const int64_t o = ((int64_t)i2 * m1 + e1 + b) * G0 + g0;
        const double bv = T.bv[1][g1 * Q + b], bd = T.bd[1][g1 * Q + b];
        a0 += bv * W0[o];
        a1 += bv * W0[tot0 + o];
        a2 += bd * W0[o];
    }
    // stored as double-float pairs (same 8 bytes) for the point field, which works in double-float
    float2* W1f = reinterpret_cast<float2*>(W1);
    W1f[idx] = d2df_split(a0);
    W1f[tot + idx] = d2df_split(a1);
    W1f[2 * tot + idx] = d2df_split(a2);
}

// gradient of u at point (g0, g1, g2) from its W1 array (3-D) or directly (2-D), in
// double-float; bv2 / bd2 are the direction-2 basis values and derivatives at g2
__device__ __forceinline__ void adj_grad_df(const Geo& g, const df2* bv2, const df2* bd2, const float2* W1,
                                            int64_t tot1, int g0, int g1, int g2, df2* du)
{
    const int Q = g.p + 1;
    const int G0 = g.n_el[0] * Q, G1 = g.n_el[1] * Q;
    auto ld = [](float2 v) { return df2{v.x, v.y}; };
    if (g.dim == 2) {
        const int64_t o = (int64_t)g1 * G0 + g0;
        du[0] = ld(W1[tot1 + o]);
        du[1] = ld(W1[2 * tot1 + o]);
        return;
    }
    const int e2 = g2 / Q;
    df2 d0 = {0.f, 0.f}, d1 = {0.f, 0.f}, d2 = {0.f, 0.f};
    for (int c = 0; c < Q; ++c) {
        const int64_t o = ((int64_t)(e2 + c) * G1 + g1) * G0 + g0;
        d0 = df_add(d0, df_mul(bv2[c], ld(W1[tot1 + o])));
        d1 = df_add(d1, df_mul(bv2[c], ld(W1[2 * tot1 + o])));
        d2 = df_add(d2, df_mul(bd2[c], ld(W1[o])));
    }
    du[0] = d0; du[1] = d1; du[2] = d2;
}

__device__ __forceinline__ df2 quad_form_df(int n, const df2 G[3][3], const df2* u, const df2* v)
{
    df2 s = {0.f, 0.f};
    for (int a = 0; a < n; ++a) {
        df2 t = {0.f, 0.f};
        for (int b = 0; b < n; ++b) t = df_add(t, df_mul(G[a][b], v[b]));
        s = df_add(s, df_mul(u[a], t));
    }
    return s;
}

// s(g) = w_g sum_t sign_t grad u_{a_t}^T G grad u_{b_t} at every Gauss point: the geometry in
// FP64, the gradients and quadratic forms in double-float on the FP32 pipe
__global__ void k_adj_points(Geo g, AdjTables T, AdjTerms terms, double* spt)
{
    const int Q = g.p + 1;
    const int G0 = g.n_el[0] * Q, G1 = g.n_el[1] * Q, G2 = (g.dim == 3) ? g.n_el[2] * Q : 1;
    const int64_t tot = (int64_t)G0 * G1 * G2;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int g0 = (int)(idx % G0);
    const int g1 = (int)((idx / G0) % G1);
    const int g2 = (int)(idx / ((int64_t)G0 * G1));
    const int gg[3] = {g0, g1, g2};
    double xi[3] = {0, 0, 0}, s1[3] = {0, 0, 0}, c1[3] = {0, 0, 0}, x[3], G[3][3];
    double w = 1.0;
    for (int d = 0; d < g.dim; ++d) {
        xi[d] = T.gx[d][gg[d]];
        s1[d] = T.sx[d][gg[d]];
        c1[d] = T.cx[d][gg[d]];
        w *= T.wq[d][gg[d]];
    }
    adj_geometry(g, xi, s1, c1, x, G);
    df2 Gd[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const float2 v = (a < g.dim && b < g.dim) ? d2df_split(G[a][b]) : make_float2(0.f, 0.f);
            Gd[a][b] = df2{v.x, v.y};
        }
    df2 bv2[kMaxP + 1], bd2[kMaxP + 1];
    if (g.dim == 3)
        for (int c = 0; c < Q; ++c) {
            const float2 v = d2df_split(T.bv[2][g2 * Q + c]), dd = d2df_split(T.bd[2][g2 * Q + c]);
            bv2[c] = df2{v.x, v.y};
            bd2[c] = df2{dd.x, dd.y};
        }
    df2 sacc = {0.f, 0.f};
    for (int t = 0; t < terms.n; ++t) {
        df2 du[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, dv[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        adj_grad_df(g, bv2, bd2, reinterpret_cast<const float2*>(terms.Wa[t]), terms.tot1, g0, g1, g2, du);
        adj_grad_df(g, bv2, bd2, reinterpret_cast<const float2*>(terms.Wb[t]), terms.tot1, g0, g1, g2, dv);
        const df2 q = quad_form_df(g.dim, Gd, du, dv);
        sacc = df_add(sacc, terms.sign[t] < 0.0 ? df_neg(q) : q);
    }
    const float2 ws = d2df_split(w);
    const df2 r = df_mul(df2{ws.x, ws.y}, sacc);
    spt[idx] = df2d_exact(r.h, r.l);
}

// ---------------------------------------------------------------------------
// Transposed interpolation (common domain Omega~ = [k0, k1]^n).
//   Z_u(j) = (ybar_i - ybar_{i+delta})(x_{i+delta} - x_i), i = k0 + j, for i, i + delta in Omega~
//   C0[u][j2][j1][a0] = sum_{j0} Z_u(j) E0[j0][a0]        (2-D: [u][j1][a0])
//   C1[u][j2][a1][a0] = sum_{j1} C0 E1[j1][a1]            (2-D: the sample table)
//   table[u][a2][a1][a0] = sum_{j2} C1 E2[j2][a2]           (3-D)
// then the transposed collocation solves B^T y = r per direction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double eval_at(const SplineBufs& sb, int d, int v, int qe, int j, int a)
{
    const int o = a - sb.espan[d][v][j];
    return (o >= 0 && o <= qe) ? sb.eval[d][v][(int64_t)j * (qe + 1) + o] : 0.0;
}

__global__ void k_adj_interp0(Geo g, SplinePlan sp, SplineBufs sb, const double* ybar, const double* x, double* C0)
{
    const int W = sp.nv, P = (W - 1) / 2;
    const int L0 = sp.L[0][P], L1 = sp.L[1][P], L2 = (sp.dim == 3) ? sp.L[2][P] : 1;
    const int ns0 = sp.nu[0];
    const int64_t S_up = sp.S - 1 - sp.c;
    const int64_t tot = S_up * L2 * L1 * ns0;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int a0 = (int)(idx % ns0);
    const int j1 = (int)((idx / ns0) % L1);
    const int j2 = (int)((idx / ((int64_t)ns0 * L1)) % L2);
    const int64_t u = idx / ((int64_t)ns0 * L1 * L2);
    int s = sp.c + 1 + (int)u;
    int dl[3] = {0, 0, 0};
    for (int d = 0; d < sp.dim; ++d) { dl[d] = s % W - P; s /= W; }
    const int v0 = dl[0] + P, qe0 = sp.qe[0][v0];
    const int k0 = sp.r0[0], k1[3] = {sp.r1[0], sp.r1[1], sp.r1[2]};
    const int i1 = sp.r0[1] + j1, i2 = (sp.dim == 3) ? sp.r0[2] + j2 : 0;
    const int n1 = i1 + dl[1], n2 = i2 + dl[2];
    double acc = 0.0;
    if (n1 >= sp.r0[1] && n1 <= k1[1] && (sp.dim == 2 || (n2 >= sp.r0[2] && n2 <= k1[2]))) {
        const int m0 = g.m[0], m1 = g.m[1];
        for (int j0 = 0; j0 < L0; ++j0) {
            const double e = eval_at(sb, 0, v0, qe0, j0, a0);
            if (e == 0.0) continue;
            const int i0 = k0 + j0, n0 = i0 + dl[0];
            if (n0 < k0 || n0 > k1[0]) continue;
            const int64_t ii = i0 + (int64_t)m0 * (i1 + (int64_t)m1 * i2);
            const int64_t jj = n0 + (int64_t)m0 * (n1 + (int64_t)m1 * n2);
            acc += e * (ybar[ii] - ybar[jj]) * (x[jj] - x[ii]);
        }
    }
    C0[idx] = acc;
}

// contract direction d (1 or 2) of an array [u][outer][L_d][inner] into [u][outer][ns_d][inner]
__global__ void k_adj_interp_dir(SplinePlan sp, SplineBufs sb, int d, int64_t outer, int64_t inner,
                                 const double* in, double* out)
{
    const int W = sp.nv, P = (W - 1) / 2;
    const int Ld = sp.L[d][P], nsd = sp.nu[d];
    const int64_t S_up = sp.S - 1 - sp.c;
    const int64_t tot = S_up * outer * nsd * inner;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int64_t in_i = idx % inner;
    const int a = (int)((idx / inner) % nsd);
    const int64_t ou = idx / (inner * nsd);           // u * outer + o
    int s = sp.c + 1 + (int)(ou / outer);
    int v = 0;
    for (int e = 0; e <= d; ++e) { v = s % W; s /= W; }
    const int qe = sp.qe[d][v];
    const double* src = in + ou * Ld * inner + in_i;
    double acc = 0.0;
    for (int j = 0; j < Ld; ++j) {
        const double e = eval_at(sb, d, v, qe, j, a);
        if (e != 0.0) acc += e * src[(int64_t)j * inner];
    }
    out[idx] = acc;
}

// transposed collocation solve B^T y = r (B = L U, unit lower L) along direction d, in place
__global__ void k_adj_solve_t(SplinePlan sp, SplineBufs sb, int d, double* table)
{
    const int W = sp.nv, P = (W - 1) / 2;
    const int64_t lines = sp.n_samples / sp.nu[d];
    const int64_t S_up = sp.S - 1 - sp.c;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= S_up * lines) return;
    const int64_t u = idx / lines, l = idx % lines;
    int s = sp.c + 1 + (int)u;
    int v = 0;
    for (int e = 0; e <= d; ++e) { v = s % W; s /= W; }
    (void)P;
    int64_t st = 1;
    for (int e = 0; e < d; ++e) st *= sp.nu[e];
    const int ns = sp.ns[d][v];
    double* y = table + u * sp.n_samples + (l % st) + (l / st) * st * ns;
    const double* B = sb.lu[d][v];
    const int bl = sb.band[2 * (d * kMaxV + v)], bu = sb.band[2 * (d * kMaxV + v) + 1];
    // U^T z = r: z_r = (r_r - sum_{c<r} U_cr z_c) / U_rr, U_cr = B[c][r] for r - bu <= c < r
    for (int r = 0; r < ns; ++r) {
        double acc = y[r * st];
        for (int c = max(0, r - bu); c < r; ++c) acc -= B[(int64_t)c * ns + r] * y[c * st];
        y[r * st] = acc / B[(int64_t)r * ns + r];
    }
    // L^T y = z: y_r = z_r - sum_{c>r} L_cr y_c, L_cr = B[c][r] for r < c <= r + bl
    for (int r = ns - 2; r >= 0; --r) {
        double acc = y[r * st];
        for (int c = r + 1; c < min(ns, r + bl + 1); ++c) acc -= B[(int64_t)c * ns + r] * y[c * st];
        y[r * st] = acc;
    }
}

// ---------------------------------------------------------------------------
// Sample rows: s(g) += w_g grad B_s^T G grad u_{w_s} on supp(B_s),
// w_s = sum_{delta upper} Phibar_delta(s) e_{s+delta}.  One block per sample row.
// ---------------------------------------------------------------------------
__global__ void k_adj_samples(Geo g, AdjTables T, SplinePlan sp, const double* phibar, double* spt)
{
    const int p = g.p, Q = p + 1, W = 2 * p + 1, n = g.dim;
    const int C = sp.c;
    const int64_t sid = blockIdx.x;
    int srow[3] = {0, 0, 0};
    {
        int64_t rem = sid;
        for (int d = 0; d < n; ++d) {
            srow[d] = axis_sample(sp.ax[d], (int)(rem % sp.nu[d]));
            rem /= sp.nu[d];
        }
    }
    const int G0 = g.n_el[0] * Q, G1 = g.n_el[1] * Q;
    int npts = 1;
    for (int d = 0; d < n; ++d) npts *= Q * Q;
    for (int t = threadIdx.x; t < npts; t += blockDim.x) {
        int gg[3] = {0, 0, 0}, e[3] = {0, 0, 0};
        int rem = t;
        for (int d = 0; d < n; ++d) {
            const int loc = rem % (Q * Q);
            rem /= Q * Q;
            e[d] = srow[d] - p + loc / Q;
            gg[d] = e[d] * Q + loc % Q;
        }
        double xi[3] = {0, 0, 0}, s1[3] = {0, 0, 0}, c1[3] = {0, 0, 0}, x[3], G[3][3];
        double w = 1.0;
        for (int d = 0; d < n; ++d) {
            xi[d] = T.gx[d][gg[d]];
            s1[d] = T.sx[d][gg[d]];
            c1[d] = T.cx[d][gg[d]];
            w *= T.wq[d][gg[d]];
        }
        adj_geometry(g, xi, s1, c1, x, G);
        // 1-D values / derivatives of the active functions e_d + b, b = 0..p
        double bv[3][kMaxP + 1], bd[3][kMaxP + 1];
        for (int d = 0; d < 3; ++d)
            for (int b = 0; b <= p; ++b) {
                bv[d][b] = (d < n) ? T.bv[d][gg[d] * Q + b] : 1.0;
                bd[d][b] = (d < n) ? T.bd[d][gg[d] * Q + b] : 0.0;
            }
        const int as0 = srow[0] - e[0], as1 = srow[1] - e[1], as2 = (n == 3) ? srow[2] - e[2] : 0;
        double dB[3] = {bd[0][as0] * bv[1][as1] * bv[2][as2], bv[0][as0] * bd[1][as1] * bv[2][as2],
                        bv[0][as0] * bv[1][as1] * bd[2][as2]};
        double du[3] = {0, 0, 0};
        const int c2max = (n == 3) ? p : 0;
        for (int c2 = 0; c2 <= c2max; ++c2)
            for (int c1b = 0; c1b <= p; ++c1b)
                for (int c0 = 0; c0 <= p; ++c0) {
                    const int dl0 = e[0] + c0 - srow[0], dl1 = e[1] + c1b - srow[1];
                    const int dl2 = (n == 3) ? e[2] + c2 - srow[2] : 0;
                    const int slot = (dl0 + p) + W * ((dl1 + p) + W * (n == 3 ? dl2 + p : 0));
                    if (slot <= C) continue;
                    const double f = phibar[(int64_t)(slot - C - 1) * sp.n_samples + sid];
                    du[0] += f * bd[0][c0] * bv[1][c1b] * bv[2][c2];
                    du[1] += f * bv[0][c0] * bd[1][c1b] * bv[2][c2];
                    du[2] += f * bv[0][c0] * bv[1][c1b] * bd[2][c2];
                }
        const double val = w * quad_form(n, G, dB, du);
        const int64_t pi = gg[0] + (int64_t)G0 * (gg[1] + (int64_t)G1 * gg[2]);
        atomicAdd(spt + pi, val);
    }
}

// ---------------------------------------------------------------------------
// dL/dc_k = sum_g N_k(phi(g)) s(g).  One warp per element.  An element maps into
// at most two spans of the kappa spline per direction when its physical size is
// below the spline's, so its contributions fall into a window of 5^n control
// values starting at the smallest span its points touch.  The points' data
// (s(g), the 4 basis values per direction, the span offsets) are staged in
// shared memory 64 at a time; lane (kb, kc) then owns the window line
// (0..4, kb, kc) and sums the contributions of all points into 5 registers, so
// the element needs no atomics until one global atomic per window entry.
// Points whose span falls outside the window add their contributions directly.
// ---------------------------------------------------------------------------
constexpr int kScatterWarps = 4;
constexpr int kStage = 64;

__global__ void __launch_bounds__(32 * kScatterWarps) k_adj_scatter(Geo g, AdjTables T, const double* spt,
                                                                    double* grad)
{
    // s(g) then N0[4], N1[4], N2[4], as double-float pairs
    __shared__ df2 sN[kScatterWarps][kStage][13];
    __shared__ int sO[kScatterWarps][kStage];          // window offsets o0 + 4 o1 + 16 o2, or -1
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int p = g.p, Q = p + 1, n = g.dim;
    const int G0 = g.n_el[0] * Q, G1 = g.n_el[1] * Q;
    const int64_t nel = (int64_t)g.n_el[0] * g.n_el[1] * (n == 3 ? g.n_el[2] : 1);
    int npt = 1;
    for (int d = 0; d < n; ++d) npt *= Q;
    const int n0 = g.knc[0], n1 = g.knc[1];
    // the window line of this lane
    const bool owner = (n == 3) ? lane < 25 : lane < 5;
    const int kb = lane % 5, kc = (n == 3) ? lane / 5 : 0;
    for (int64_t el = (int64_t)blockIdx.x * kScatterWarps + wid; el < nel; el += (int64_t)gridDim.x * kScatterWarps) {
        const int e[3] = {(int)(el % g.n_el[0]), (int)((el / g.n_el[0]) % g.n_el[1]),
                          (int)(el / ((int64_t)g.n_el[0] * g.n_el[1]))};
        // smallest span per direction over the element's points
        int flo[3] = {1 << 30, 1 << 30, 1 << 30};
        for (int t = lane; t < npt; t += 32) {
            int rem = t;
            double xi[3] = {0, 0, 0}, s1[3] = {0, 0, 0}, x[3];
            for (int d = 0; d < n; ++d) {
                const int gd = e[d] * Q + rem % Q;
                rem /= Q;
                xi[d] = T.gx[d][gd];
                s1[d] = T.sx[d][gd];
            }
            adj_point(g, xi, s1, x);
            for (int d = 0; d < n; ++d) {
                const int ne = g.knc[d] - 3;
                int f = (int)(fmin(fmax(x[d], 0.0), 1.0) * ne);
                f = f > ne - 1 ? ne - 1 : f;
                flo[d] = min(flo[d], f);
            }
        }
        for (int d = 0; d < n; ++d) flo[d] = __reduce_min_sync(0xffffffffu, flo[d]);
        df2 acc[5];
#pragma unroll
        for (int ka = 0; ka < 5; ++ka) acc[ka] = df2{0.f, 0.f};
        for (int base = 0; base < npt; base += kStage) {
            __syncwarp();
            for (int tl = lane; tl < kStage; tl += 32) {
                const int t = base + tl;
                int o = -1;
                if (t < npt) {
                    int rem = t;
                    int gd[3] = {0, 0, 0};
                    double xi[3] = {0, 0, 0}, s1[3] = {0, 0, 0}, x[3];
                    for (int d = 0; d < n; ++d) {
                        gd[d] = e[d] * Q + rem % Q;
                        rem /= Q;
                        xi[d] = T.gx[d][gd[d]];
                        s1[d] = T.sx[d][gd[d]];
                    }
                    adj_point(g, xi, s1, x);
                    const double sv = spt[gd[0] + (int64_t)G0 * (gd[1] + (int64_t)G1 * gd[2])];
                    int f[3] = {0, 0, 0};
                    df2 N[3][4];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        N[d][0] = df2{1.f, 0.f};
                        N[d][1] = N[d][2] = N[d][3] = df2{0.f, 0.f};
                    }
                    bool inwin = true;
                    for (int d = 0; d < n; ++d) {
                        const double xc = fmin(fmax(x[d], 0.0), 1.0);
                        const float2 xs = d2df_split(xc);
                        cubic_open_basis_df(g.knc[d] - 3, xc, df2{xs.x, xs.y}, f[d], N[d]);
                        inwin = inwin && (f[d] - flo[d] <= 1);
                    }
                    if (inwin) {
                        o = (f[0] - flo[0]) + 4 * (f[1] - flo[1]) + 16 * (n == 3 ? f[2] - flo[2] : 0);
                        const float2 svs = d2df_split(sv);
                        sN[wid][tl][0] = df2{svs.x, svs.y};
                        for (int d = 0; d < 3; ++d)
                            for (int a = 0; a < 4; ++a) sN[wid][tl][1 + 4 * d + a] = N[d][a];
                    } else {
                        // a point outside the element's window: its 4^n contributions directly (rare)
                        const int cmax = (n == 3) ? 4 : 1;
                        for (int c = 0; c < cmax; ++c)
                            for (int b = 0; b < 4; ++b)
                                for (int a = 0; a < 4; ++a) {
                                    const df2 w = df_mul(df_mul(N[0][a], N[1][b]), N[2][c]);
                                    atomicAdd(grad + (f[0] + a) + (int64_t)n0 * ((f[1] + b) + (int64_t)n1 * (f[2] + c)),
                                              sv * df2d_exact(w.h, w.l));
                                }
                    }
                }
                sO[wid][tl] = o;
            }
            __syncwarp();
            if (owner) {
                const int cnt = min(kStage, npt - base);
                for (int tl = 0; tl < cnt; ++tl) {
                    const int o = sO[wid][tl];
                    if (o < 0) continue;
                    const int b = kb - ((o >> 2) & 3), c = kc - (o >> 4), o0 = o & 3;
                    if (b < 0 || b > 3 || c < 0 || c > 3) continue;
                    const df2* D = sN[wid][tl];
                    const df2 w = df_mul(df_mul(D[0], D[5 + b]), D[9 + c]);
#pragma unroll
                    for (int ka = 0; ka < 5; ++ka) {
                        const int a = ka - o0;
                        if (a >= 0 && a <= 3) acc[ka] = df_add(acc[ka], df_mul(w, D[1 + a]));
                    }
                }
            }
        }
        if (owner) {
            const int kbg = flo[1] + kb, kcg = (n == 3) ? flo[2] + kc : 0;
            if (kbg < g.knc[1] && (n == 2 || kcg < g.knc[2]))
                for (int ka = 0; ka < 5; ++ka) {
                    const int kag = flo[0] + ka;
                    if ((acc[ka].h != 0.f || acc[ka].l != 0.f) && kag < g.knc[0])
                        atomicAdd(grad + kag + (int64_t)n0 * (kbg + (int64_t)n1 * kcg), df2d_exact(acc[ka].h, acc[ka].l));
                }
        }
    }
}

// The restricted vectors of the exact-entry terms: out = [R ybar, R x, R(ybar . x), R 1],
// R the restriction to the rows of Omega~ = [r0, r1]^n.
__global__ void k_adj_vectors(Geo g, SplinePlan sp, const double* ybar, const double* x, double* out)
{
    const int64_t N = (int64_t)g.m[0] * g.m[1] * (g.dim == 3 ? g.m[2] : 1);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int i0 = (int)(i % g.m[0]), i1 = (int)((i / g.m[0]) % g.m[1]);
    const int i2 = (g.dim == 3) ? (int)(i / ((int64_t)g.m[0] * g.m[1])) : 0;
    const bool in = i0 >= sp.r0[0] && i0 <= sp.r1[0] && i1 >= sp.r0[1] && i1 <= sp.r1[1] &&
                    (g.dim == 2 || (i2 >= sp.r0[2] && i2 <= sp.r1[2]));
    out[i] = in ? ybar[i] : 0.0;
    out[N + i] = in ? x[i] : 0.0;
    out[2 * N + i] = in ? ybar[i] * x[i] : 0.0;
    out[3 * N + i] = in ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_adj_vectors(const Geo& g, const SplinePlan& sp, const double* ybar, const double* x, double* out,
                               cudaStream_t s)
{
    const int64_t N = (int64_t)g.m[0] * g.m[1] * (g.dim == 3 ? g.m[2] : 1);
    launch_begin(K_ADJ_FIELDS, s);
    k_adj_vectors<<<blocks_for(N, kBlock), kBlock, 0, s>>>(g, sp, ybar, x, out);
    launch_end(K_ADJ_FIELDS, s);
    return cudaGetLastError();
}

cudaError_t launch_adj_grad_field(const Geo& g, const AdjTables& T, const double* v, double* W0, double* W1,
                                  cudaStream_t s)
{
    const int Q = g.p + 1;
    const int64_t m2 = (g.dim == 3) ? g.m[2] : 1;
    const int64_t tot0 = m2 * g.m[1] * (int64_t)g.n_el[0] * Q;
    const int64_t tot1 = m2 * (int64_t)g.n_el[1] * Q * g.n_el[0] * Q;
    launch_begin(K_ADJ_FIELDS, s);
    k_adj_pass0<<<blocks_for(tot0, kBlock), kBlock, 0, s>>>(g, T, v, W0);
    launch_end(K_ADJ_FIELDS, s);
    launch_begin(K_ADJ_FIELDS, s);
    k_adj_pass1<<<blocks_for(tot1, kBlock), kBlock, 0, s>>>(g, T, W0, W1);
    launch_end(K_ADJ_FIELDS, s);
    return cudaGetLastError();
}

cudaError_t launch_adj_points(const Geo& g, const AdjTables& T, const AdjTerms& terms, double* spt, cudaStream_t s)
{
    const int Q = g.p + 1;
    int64_t tot = 1;
    for (int d = 0; d < g.dim; ++d) tot *= (int64_t)g.n_el[d] * Q;
    launch_begin(K_ADJ_POINTS, s);
    k_adj_points<<<blocks_for(tot, kBlock), kBlock, 0, s>>>(g, T, terms, spt);
    launch_end(K_ADJ_POINTS, s);
    return cudaGetLastError();
}

cudaError_t launch_adj_interp(const Geo& g, const SplinePlan& sp, const SplineBufs& sb, const double* ybar,
                              const double* x, double* C0, double* C1, double* table, cudaStream_t s)
{
    const int P = (sp.nv - 1) / 2;
    const int64_t S_up = sp.S - 1 - sp.c;
    const int64_t L1 = sp.L[1][P], L2 = (sp.dim == 3) ? sp.L[2][P] : 1;
    const int64_t nu0 = sp.nu[0], nu1 = sp.nu[1];
    launch_begin(K_ADJ_INTERP, s);
    k_adj_interp0<<<blocks_for(S_up * L2 * L1 * nu0, kBlock), kBlock, 0, s>>>(g, sp, sb, ybar, x, C0);
    launch_end(K_ADJ_INTERP, s);
    // direction 1: [u][L2][L1][nu0] -> [u][L2][nu1][nu0] (the sample table itself in 2-D)
    double* out1 = (sp.dim == 3) ? C1 : table;
    launch_begin(K_ADJ_INTERP, s);
    k_adj_interp_dir<<<blocks_for(S_up * L2 * nu1 * nu0, kBlock), kBlock, 0, s>>>(sp, sb, 1, L2, nu0, C0, out1);
    launch_end(K_ADJ_INTERP, s);
    if (sp.dim == 3) {
        const int64_t nu2 = sp.nu[2];
        launch_begin(K_ADJ_INTERP, s);
        k_adj_interp_dir<<<blocks_for(S_up * nu2 * nu1 * nu0, kBlock), kBlock, 0, s>>>(sp, sb, 2, 1, nu1 * nu0,
                                                                                      C1, table);
        launch_end(K_ADJ_INTERP, s);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    for (int d = 0; d < sp.dim; ++d) {
        const int64_t n = S_up * (sp.n_samples / sp.nu[d]);
        launch_begin(K_ADJ_INTERP, s);
        k_adj_solve_t<<<blocks_for(n, 128), 128, 0, s>>>(sp, sb, d, table);
        launch_end(K_ADJ_INTERP, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_samples(const Geo& g, const AdjTables& T, const SplinePlan& sp, const double* phibar,
                               double* spt, cudaStream_t s)
{
    if (sp.n_samples <= 0) return cudaSuccess;
    launch_begin(K_ADJ_SAMPLES, s);
    k_adj_samples<<<(unsigned)sp.n_samples, 256, 0, s>>>(g, T, sp, phibar, spt);
    launch_end(K_ADJ_SAMPLES, s);
    return cudaGetLastError();
}

cudaError_t launch_adj_scatter(const Geo& g, const AdjTables& T, const double* spt, double* grad, cudaStream_t s)
{
    int64_t nel = 1;
    for (int d = 0; d < g.dim; ++d) nel *= g.n_el[d];
    int64_t blocks = (nel + kScatterWarps - 1) / kScatterWarps;
    if (blocks > 152 * 16) blocks = 152 * 16;
    launch_begin(K_ADJ_SCATTER, s);
    k_adj_scatter<<<(unsigned)blocks, 32 * kScatterWarps, 0, s>>>(g, T, spt, grad);
    launch_end(K_ADJ_SCATTER, s);
    return cudaGetLastError();
}

}  // namespace iga
