// K4: per-offset tensor-product B-spline interpolation of the stencil
//     functions through their samples (Sec. 4.1, Sec. 6).
// K5: surrogate rows of eq. DefinitionOfSurrogateMatrixSymmetricKernel
//     (Sec. 5.3) written into the stencil-ELL values (pass 1, rows with
//     interpolated entries), then the kernel-preserving diagonal of every row
//     (pass 2).
//
// Each offset delta interpolates, per direction d, through the samples of the
// variant v = delta_d + p (SplinePlan, variant_sample): abscissae t_a, a = 0..ns-1.  The knot vector of degree q has (q+1)-fold end knots at t_0 and
// t_{ns-1} and interior knots at t_{(q+1)/2} .. t_{ns-1-(q+1)/2} (odd q) or at the
// midpoints (t_r + t_{r+1})/2, r = q/2 .. ns-2-q/2 (even q) -- the not-a-knot
// interpolating spline.  Spans are half-open [kn_mu, kn_mu+1) except the last.
// The collocation matrix is totally positive and banded, so it is factored
// without pivoting and the factors keep its band.
#include "arith.cuh"
#include "iga_internal.cuh"

namespace iga {

__device__ int find_span(const double* kn, int ns, int q, double x)
{
    if (x >= kn[ns]) return ns - 1;
    int lo = q, hi = ns;                 // kn[lo] <= x < kn[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (x < kn[mid]) hi = mid;
        else lo = mid;
    }
    return lo;
}

// values of the q+1 B-splines mu-q..mu at x (local triangular Cox-de Boor)
__device__ void spline_basis(const double* kn, int mu, int q, double x, double* N)
{
    double left[kMaxQ + 1], right[kMaxQ + 1];
    N[0] = 1.0;
    for (int k = 1; k <= q; ++k) {
        left[k] = x - kn[mu + 1 - k];
        right[k] = kn[mu + k] - x;
        double saved = 0.0;
        for (int r = 0; r < k; ++r) {
            double tmp = N[r] / (right[r + 1] + left[k - r]);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[k - r] * tmp;
        }
        N[k] = saved;
    }
}

// variant (v_0, v_1, v_2) of interpolated slot u: v_d = delta_d + p of slot first + u
__device__ __forceinline__ void slot_variants(const SplinePlan& sp, int64_t u, int v[3])
{
    const int W = sp.nv;
    int s = sp.first + (int)u;
    for (int d = 0; d < 3; ++d) {
        v[d] = (d < sp.dim) ? s % W : 0;
        s /= W;
    }
}

// One block per (variant, direction): sample list, knots, collocation matrix,
// banded LU, evaluation tables.
__global__ void k_spline_setup(SplinePlan sp, SplineBufs sb)
{
    extern __shared__ double smem[];
    __shared__ int sbl, sbu;
    const int v = blockIdx.x, d = blockIdx.y;
    const int ns = sp.ns[d][v], q = sp.qe[d][v], k0 = sp.k0[d][v], L = sp.L[d][v];
    if (L <= 0 || ns <= 0) return;
    const SampleAxis ax = sp.ax[d];
    const int nu = sp.nu[d];
    double* ts = smem;               // [ns] abscissae
    double* kn = smem + ns;          // [ns + q + 1] knots
    const int nk = ns + q + 1;
    if (threadIdx.x == 0) {
        sbl = 0; sbu = 0;
        int r = 0;
        for (int a = 0; a < nu; ++a) {
            const int t = axis_sample(ax, a);
            const bool in = variant_sample(ax, sp.all, t, k0, k0 + L - 1) && r < ns;
            sb.inv[d][v][a] = in ? r : -1;
            if (in) { sb.pos[d][v][r] = a; ts[r] = (double)t; ++r; }
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nk; r += blockDim.x) {
        double x;
        if (r <= q) x = ts[0];
        else if (r >= ns) x = ts[ns - 1];
        else if (q & 1) x = ts[(q + 1) / 2 + (r - q - 1)];
        else {
            const int a = q / 2 + (r - q - 1);
            x = 0.5 * (ts[a] + ts[a + 1]);
        }
        kn[r] = x;
    }
    double* B = sb.lu[d][v];
    for (int64_t k = threadIdx.x; k < (int64_t)ns * ns; k += blockDim.x) B[k] = 0.0;
    __syncthreads();
    // collocation rows: B[r][c] = N_c(t_r)
    for (int r = threadIdx.x; r < ns; r += blockDim.x) {
        const double x = ts[r];
        const int mu = find_span(kn, ns, q, x);
        double N[kMaxQ + 1];
        spline_basis(kn, mu, q, x, N);
        for (int a = 0; a <= q; ++a) B[(int64_t)r * ns + mu - q + a] = N[a];
        atomicMax(&sbl, r - (mu - q));
        atomicMax(&sbu, mu - r);
    }
    __syncthreads();
    const int bl = sbl, bu = sbu;
    // banded LU without pivoting: B = L U, L unit lower (stored below the diagonal)
    for (int k = 0; k < ns - 1; ++k) {
        const double piv = B[(int64_t)k * ns + k];
        const int rhi = min(ns, k + bl + 1), chi = min(ns, k + bu + 1);
        for (int r = k + 1 + threadIdx.x; r < rhi; r += blockDim.x) {
            const double l = B[(int64_t)r * ns + k] / piv;
            B[(int64_t)r * ns + k] = l;
            for (int c = k + 1; c < chi; ++c) B[(int64_t)r * ns + c] -= l * B[(int64_t)k * ns + c];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sb.band[2 * (d * kMaxV + v)] = bl;
        sb.band[2 * (d * kMaxV + v) + 1] = bu;
    }
    // evaluation at every domain index k0 + k
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const double x = (double)(k0 + k);
        const int mu = find_span(kn, ns, q, x);
        double N[kMaxQ + 1];
        spline_basis(kn, mu, q, x, N);
        sb.espan[d][v][k] = mu - q;
        for (int a = 0; a <= q; ++a) {
            sb.eval[d][v][(int64_t)k * (q + 1) + a] = N[a];
            if (d == 0) sb.eval0[v][(int64_t)a * L + k] = PolDF::from_double(N[a]);
        }
    }
}

// Solve the collocation system along direction d for every upper offset and every
// line of its sample grid, in place in the sample table rows c+1 .. S-1.  Thread
// per (offset, line of the full sample grid); lines through positions that are
// not samples of the offset return.
__global__ void k_spline_solve(SplinePlan sp, int d, SplineBufs sb, double* samples)
{
    const int64_t lines = sp.n_samples / sp.nu[d];
    const int64_t S_up = sp.S - sp.first;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= S_up * lines) return;
    const int64_t u = idx / lines;
    int64_t l = idx % lines;
    int v[3];
    slot_variants(sp, u, v);
    int64_t base = 0, st = 1, std_ = 1;
    for (int e = 0; e < sp.dim; ++e) {
        if (e == d) { std_ = st; st *= sp.nu[e]; continue; }
        const int pos = (int)(l % sp.nu[e]);
        l /= sp.nu[e];
        if (sp.ns[e][v[e]] <= 0 || sb.inv[e][v[e]][pos] < 0) return;
        base += pos * st;
        st *= sp.nu[e];
    }
    const int ns = sp.ns[d][v[d]];
    if (ns <= 0) return;
    double* x = samples + (sp.first + u) * sp.n_samples + base;
    const int* ps = sb.pos[d][v[d]];
    const double* B = sb.lu[d][v[d]];
    const int bl = sb.band[2 * (d * kMaxV + v[d])], bu = sb.band[2 * (d * kMaxV + v[d]) + 1];
    for (int r = 1; r < ns; ++r) {
        double acc = x[ps[r] * std_];
        for (int c = max(0, r - bl); c < r; ++c) acc -= B[(int64_t)r * ns + c] * x[ps[c] * std_];
        x[ps[r] * std_] = acc;
    }
    for (int r = ns - 1; r >= 0; --r) {
        double acc = x[ps[r] * std_];
        for (int c = r + 1; c < min(ns, r + bu + 1); ++c) acc -= B[(int64_t)r * ns + c] * x[ps[c] * std_];
        x[ps[r] * std_] = acc / B[(int64_t)r * ns + r];
    }
}

// Partially evaluated coefficients: contract directions 2 (3-D) and 1 at every
// domain index, keeping the coefficient index a0 of direction 0 (all indices
// relative to the offset's own samples and domain):
//   3-D: partial[u][j2][j1][a0] = sum_{b,c} coef[u][a0, s1(j1)+b, s2(j2)+c] E1[j1][b] E2[j2][c]
//   2-D: partial[u][j1][a0]     = sum_b     coef[u][a0, s1(j1)+b]          E1[j1][b]
// Sum-factorised: first direction 2 into mid[u][j2][b'][a0] (3-D only), then direction 1.
__global__ void k_spline_mid(SplinePlan sp, SplineBufs sb, const double* samples, double* mid)
{
    const int nu0 = sp.nu[0], nu1 = sp.nu[1], L2 = sp.Lmax[2];
    const int64_t S_up = sp.S - sp.first;
    const int64_t total = S_up * L2 * nu1 * nu0;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int a0 = (int)(idx % nu0);
    const int b1 = (int)((idx / nu0) % nu1);
    const int j2 = (int)((idx / ((int64_t)nu0 * nu1)) % L2);
    const int64_t u = idx / ((int64_t)nu0 * nu1 * L2);
    int v[3];
    slot_variants(sp, u, v);
    if (a0 >= sp.ns[0][v[0]] || b1 >= sp.ns[1][v[1]] || j2 >= sp.L[2][v[2]]) return;
    const double* coef = samples + (sp.first + u) * sp.n_samples;
    const int q2 = sp.qe[2][v[2]];
    const int s2 = sb.espan[2][v[2]][j2];
    const int* p2 = sb.pos[2][v[2]];
    const double* E2 = sb.eval[2][v[2]] + (int64_t)j2 * (q2 + 1);
    const int64_t o01 = sb.pos[0][v[0]][a0] + (int64_t)nu0 * sb.pos[1][v[1]][b1];
    const int64_t plane = (int64_t)nu0 * nu1;
    double acc = 0.0;
    for (int c = 0; c <= q2; ++c) acc += coef[o01 + plane * p2[s2 + c]] * E2[c];
    mid[idx] = acc;
}

__global__ void k_spline_partial(SplinePlan sp, SplineBufs sb, const double* samples, const double* mid)
{
    const int nu0 = sp.nu[0], nu1 = sp.nu[1];
    const int L1 = sp.Lmax[1], L2 = (sp.dim == 3) ? sp.Lmax[2] : 1;
    const int64_t S_up = sp.S - sp.first;
    const int64_t total = S_up * L2 * L1 * nu0;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int a0 = (int)(idx % nu0);
    const int j1 = (int)((idx / nu0) % L1);
    const int j2 = (int)((idx / ((int64_t)nu0 * L1)) % L2);
    const int64_t u = idx / ((int64_t)nu0 * L1 * L2);
    int v[3];
    slot_variants(sp, u, v);
    if (a0 >= sp.ns[0][v[0]] || j1 >= sp.L[1][v[1]] || (sp.dim == 3 && j2 >= sp.L[2][v[2]])) return;
    const int q1 = sp.qe[1][v[1]];
    const int s1 = sb.espan[1][v[1]][j1];
    const double* E1 = sb.eval[1][v[1]] + (int64_t)j1 * (q1 + 1);
    double acc = 0.0;
    if (sp.dim == 3) {
        // mid[u][j2][b'][a0], b' relative to the offset's first sample of direction 1
        const double* src = mid + ((u * L2 + j2) * (int64_t)nu1) * nu0 + a0;
        for (int b = 0; b <= q1; ++b) acc += src[(int64_t)nu0 * (s1 + b)] * E1[b];
    } else {
        const double* src = samples + (sp.first + u) * sp.n_samples + sb.pos[0][v[0]][a0];
        const int* p1 = sb.pos[1][v[1]];
        for (int b = 0; b <= q1; ++b) acc += src[(int64_t)nu0 * p1[s1 + b]] * E1[b];
    }
    sb.partial[idx] = PolDF::from_double(acc);
}

cudaError_t launch_spline_setup(const SplinePlan& sp, const SplineBufs& sb, cudaStream_t s)
{
    int nkmax = 0;
    for (int d = 0; d < sp.dim; ++d)
        for (int v = 0; v < sp.nv; ++v) nkmax = max(nkmax, 2 * sp.ns[d][v] + sp.qe[d][v] + 1);
    launch_begin(K_SPLINE_SETUP, s);
    k_spline_setup<<<dim3(sp.nv, sp.dim), 256, (size_t)nkmax * sizeof(double), s>>>(sp, sb);
    launch_end(K_SPLINE_SETUP, s);
    return cudaGetLastError();
}

cudaError_t launch_spline(const Geo& g, const SplinePlan& sp, double* samples,
                          const SplineBufs& sb, cudaStream_t s)
{
    (void)g;
    cudaError_t err = launch_spline_setup(sp, sb, s);
    if (err != cudaSuccess) return err;
    const int64_t S_up = sp.S - sp.first;
    for (int d = 0; d < sp.dim; ++d) {
        const int64_t n = S_up * (sp.n_samples / sp.nu[d]);
        launch_begin(K_SPLINE_SOLVE, s);
        k_spline_solve<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(sp, d, sb, samples);
        launch_end(K_SPLINE_SOLVE, s);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (sp.dim == 3) {
        const int64_t nmid = S_up * sp.Lmax[2] * (int64_t)sp.nu[1] * sp.nu[0];
        launch_begin(K_SPLINE_PARTIAL, s);
        k_spline_mid<<<(unsigned)((nmid + kBlock - 1) / kBlock), kBlock, 0, s>>>(sp, sb, samples, sb.mid);
        launch_end(K_SPLINE_PARTIAL, s);
    }
    const int64_t total = S_up * (sp.dim == 3 ? sp.Lmax[2] : 1) * (int64_t)sp.Lmax[1] * sp.nu[0];
    launch_begin(K_SPLINE_PARTIAL, s);
    k_spline_partial<<<(unsigned)((total + kBlock - 1) / kBlock), kBlock, 0, s>>>(sp, sb, samples, sb.mid);
    launch_end(K_SPLINE_PARTIAL, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K5, rows of the region R = [r0, r1]^n of rows with interpolated entries (the
// box Omega~, or the cardinal box with per-offset domains): for each slot with
// column j = i + delta,
//      j in R, j > i : Phi~_delta(x~_i)                      (interpolated)
//      j in R, j < i : Phi~_{-delta}(x~_j)  (= A~_ji, the copied entry)
//      j outside R   : A_ji from the exact frame row j (= A_ij)
// then, for every row, diagonal := -(off-diagonal sum).
// The interpolant is evaluated in double-float arithmetic on the FP32 pipe
// (about 48 significand bits); the diagonal sums are FP64.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T from_df(const DFAcc& a) { return df2d_exact(a.h, a.l); }
template <>
__device__ __forceinline__ float from_df<float>(const DFAcc& a) { return __fadd_rn(a.h, a.l); }

// Pass 1 (rows of R only): one thread per (row, delta_1, delta_2) writes the
// 2p+1 slots delta_0 = -p..p of that row.
template <int P, int DIM, typename T>
__global__ void __launch_bounds__(kBlock) k_fill(Geo g, SplinePlan sp, SplineBufs sb, T* vals)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    constexpr int C = (S - 1) / 2;
    constexpr int NPAIR = (DIM == 3) ? W * W : W;
    const int R0 = sp.r1[0] - sp.r0[0] + 1, R1 = sp.r1[1] - sp.r0[1] + 1;
    const int R2 = (DIM == 3) ? sp.r1[2] - sp.r0[2] + 1 : 1;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)R0 * R1 * R2 * NPAIR;
    if (item >= total) return;
    const int e0i = (int)(item % R0);
    int64_t rest = item / R0;
    const int pr = (int)(rest % NPAIR);
    rest /= NPAIR;
    const int e1i = (int)(rest % R1);
    const int e2i = (int)(rest / R1);
    const int d1 = pr % W, d2 = (DIM == 3) ? pr / W : P;
    const int m0 = g.m[0], m1 = g.m[1];
    const int64_t N = (int64_t)m0 * m1 * ((DIM == 3) ? g.m[2] : 1);
    const int i0 = sp.r0[0] + e0i, i1 = sp.r0[1] + e1i, i2 = (DIM == 3) ? sp.r0[2] + e2i : 0;
    const int64_t i = i0 + (int64_t)m0 * (i1 + (int64_t)m1 * i2);
    const int dl1 = d1 - P, dl2 = (DIM == 3) ? d2 - P : 0;
    const int j1 = i1 + dl1, j2 = i2 + dl2;
    const bool in12 = (j1 >= sp.r0[1] && j1 <= sp.r1[1]) && (DIM == 2 || (j2 >= sp.r0[2] && j2 <= sp.r1[2]));
    const int L2x = (DIM == 3) ? sp.Lmax[2] : 1, L1x = sp.Lmax[1], nu0 = sp.nu[0];
    // domain indices in directions 1, 2 of the upper evaluation (at i, variants d1, d2)
    // and of the lower one (at j, variants 2P - d1, 2P - d2)
    const int up1 = i1 - sp.k0[1][d1], up2 = (DIM == 3) ? i2 - sp.k0[2][d2] : 0;
    const int lo1 = j1 - sp.k0[1][2 * P - d1], lo2 = (DIM == 3) ? j2 - sp.k0[2][2 * P - d2] : 0;
    const int sbase = W * (d1 + W * ((DIM == 3) ? d2 : 0));
#pragma unroll
    for (int d0 = 0; d0 < W; ++d0) {
        const int s = sbase + d0;
        if (s == C && sp.first > C) continue;     // kernel-preserving: the diagonal comes from pass 2
        const int j0 = i0 + d0 - P;
        T out;
        if (in12 && j0 >= sp.r0[0] && j0 <= sp.r1[0]) {
            // upper (diagonal included for the symmetric surrogate): Phi~_delta at i;
            // lower: Phi~_{-delta} at j
            const bool upper = s >= sp.first;
            const int u = upper ? s - sp.first : (S - 1 - s) - sp.first;
            const int v0 = upper ? d0 : 2 * P - d0;
            const int x0 = (upper ? i0 : j0) - sp.k0[0][v0];
            const int x1 = upper ? up1 : lo1, x2 = upper ? up2 : lo2;
            const float2* Pp = sb.partial + (((int64_t)u * L2x + x2) * L1x + x1) * nu0 + sb.espan[0][v0][x0];
            const float2* E = sb.eval0[v0] + x0;
            const int L0v = sp.L[0][v0];
            if constexpr (sizeof(T) == 4) {
                // FP32 values: the hi parts in FP32 (the B-spline weights are a partition of
                // unity, so the sum has no cancellation beyond the FP32 rounding of the value)
                float acc = 0.f;
                for (int k = 0; k <= sp.qe[0][v0]; ++k) acc = __fmaf_rn(E[(int64_t)k * L0v].x, Pp[k].x, acc);
                out = acc;
            } else {
                DFAcc acc = PolDF::zero();
                for (int k = 0; k <= sp.qe[0][v0]; ++k) PolDF::mac(acc, E[(int64_t)k * L0v], Pp[k]);
                out = from_df<T>(acc);
            }
        } else {
            const int64_t jrow = j0 + (int64_t)m0 * (j1 + (int64_t)m1 * j2);
            out = vals[(int64_t)(S - 1 - s) * N + jrow];
        }
        vals[(int64_t)s * N + i] = out;
    }
}

// Pass 1 for the common domain Omega~, where every variant shares the tables of
// variant P: the same mapping as k_fill with those tables held in registers, the
// direction-0 evaluation row of the upper slots loaded once per thread, and the
// Q1 = q_eff + 1 <= 4 terms of the evaluation unrolled.
template <int P, int DIM, typename T, int Q1>
__global__ void __launch_bounds__(kBlock) k_fill_common(Geo g, SplinePlan sp, SplineBufs sb, T* vals)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    constexpr int C = (S - 1) / 2;
    constexpr int NPAIR = (DIM == 3) ? W * W : W;
    const int R0 = sp.r1[0] - sp.r0[0] + 1, R1 = sp.r1[1] - sp.r0[1] + 1;
    const int R2 = (DIM == 3) ? sp.r1[2] - sp.r0[2] + 1 : 1;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)R0 * R1 * R2 * NPAIR) return;
    const int x0 = (int)(item % R0);
    int64_t rest = item / R0;
    const int pr = (int)(rest % NPAIR);
    rest /= NPAIR;
    const int x1 = (int)(rest % R1);
    const int x2 = (int)(rest / R1);
    const int d1 = pr % W, d2 = (DIM == 3) ? pr / W : P;
    const int m0 = g.m[0], m1 = g.m[1];
    const int64_t N = (int64_t)m0 * m1 * ((DIM == 3) ? g.m[2] : 1);
    const int i0 = sp.r0[0] + x0, i1 = sp.r0[1] + x1, i2 = (DIM == 3) ? sp.r0[2] + x2 : 0;
    const int64_t i = i0 + (int64_t)m0 * (i1 + (int64_t)m1 * i2);
    const int y1 = x1 + d1 - P, y2 = (DIM == 3) ? x2 + d2 - P : 0;        // box indices of j in directions 1, 2
    const bool in12 = (y1 >= 0 && y1 < R1) && (y2 >= 0 && y2 < R2);
    const int L0 = sp.L[0][P], L1x = sp.Lmax[1], L2x = (DIM == 3) ? sp.Lmax[2] : 1, nu0 = sp.nu[0];
    const int* esp0 = sb.espan[0][P];
    const float2* ev0 = sb.eval0[P];
    float2 Eu[Q1];
#pragma unroll
    for (int k = 0; k < Q1; ++k) Eu[k] = ev0[(int64_t)k * L0 + x0];
    const int su = esp0[x0];
    const int sbase = W * (d1 + W * ((DIM == 3) ? d2 : 0));
    const int64_t up_row = ((int64_t)x2 * L1x + x1) * nu0 + su;      // within one slot's partial field
    const int64_t lo_row = ((int64_t)y2 * L1x + y1) * nu0;
    const int64_t slot_stride = (int64_t)L2x * L1x * nu0;
#pragma unroll
    for (int d0 = 0; d0 < W; ++d0) {
        const int s = sbase + d0;
        if (s == C && sp.first > C) continue;     // kernel-preserving: the diagonal comes from pass 2
        const int y0 = x0 + d0 - P;
        T out;
        if (in12 && y0 >= 0 && y0 < R0) {
            const float2* Pp;
            float2 E[Q1];
            if (s >= sp.first) {    // Phi~_delta at x~_i (the diagonal too for the symmetric surrogate)
                Pp = sb.partial + (int64_t)(s - sp.first) * slot_stride + up_row;
#pragma unroll
                for (int k = 0; k < Q1; ++k) E[k] = Eu[k];
            } else {                // Phi~_{-delta} at x~_j
                Pp = sb.partial + (int64_t)(S - 1 - s - sp.first) * slot_stride + lo_row + esp0[y0];
#pragma unroll
                for (int k = 0; k < Q1; ++k) E[k] = ev0[(int64_t)k * L0 + y0];
            }
            if constexpr (sizeof(T) == 4) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < Q1; ++k) acc = __fmaf_rn(E[k].x, Pp[k].x, acc);
                out = acc;
            } else {
                DFAcc acc = PolDF::zero();
#pragma unroll
                for (int k = 0; k < Q1; ++k) PolDF::mac(acc, E[k], Pp[k]);
                out = from_df<T>(acc);
            }
        } else {
            const int64_t jrow = (i0 + d0 - P) + (int64_t)m0 * ((i1 + d1 - P) + (int64_t)m1 * (i2 + d2 - P));
            out = vals[(int64_t)(S - 1 - s) * N + jrow];
        }
        vals[(int64_t)s * N + i] = out;
    }
}

// Pass 1 and the kernel-preserving diagonal together for the common domain
// Omega~: one block per line (x1, x2) of Omega~ rows along direction 0.  The
// block stages in shared memory the partially evaluated field of every
// interpolated slot at its own line (upper entries, Phi~_delta at x~_i) and at
// the neighbouring line of each lower slot (Phi~_{-delta} at x~_j), plus the
// direction-0 evaluation table.  The line's rows are cut into chunks of 32 and
// each warp owns one chunk (lane = row) and a share of the offset pairs
// (delta_1, delta_2): everything that depends on the pair or on the slot --
// frame or interpolated column block, upper or lower slot, partial row -- is
// the same for all lanes, so the warp never diverges except at the two ends
// of the line.  For each pair it writes the 2p+1 slots delta_0 = -p..p
// (consecutive rows of one slot are contiguous: coalesced), gathering the frame
// columns, and adds the row sum for the diagonal.  FP64 values: the interpolant
// in double-float (the first product starts the sum exactly), converted with
// one FP64 add of the two exactly converted halves (measured faster than the
// integer-only df2d_exact here, although the adds keep GB300's FP64 pipe ~60 %
// busy); the row sum in renormalised
// double-float (interpolated entries) and FP64 (frame entries, a minority); the
// warps' partial sums of a row added in FP64 in a fixed order.  FP32 values:
// FP32 evaluation and a compensated FP32 row sum.
constexpr int kFillLineThreads = 512;
constexpr int kFillLineWarps = kFillLineThreads / 32;

struct FillLineSmem {
    int U, nu0, R0, nch, wpc;
    size_t bytes;
};
__host__ __device__ inline FillLineSmem fill_line_smem(int S, int first, int nu0, int R0, int Q1)
{
    FillLineSmem f;
    f.U = S - first;
    f.nu0 = nu0;
    f.R0 = R0;
    f.nch = (R0 + 31) / 32;                                   // chunks of 32 rows
    f.wpc = f.nch > 0 ? kFillLineWarps / f.nch : 0;           // warps per chunk (0: too long a line)
    // partial rows (upper, lower), evaluation table [R0][Q1], spans (padded to 16 bytes), two doubles per thread
    f.bytes = ((size_t)2 * f.U * nu0 + (size_t)Q1 * R0) * sizeof(float2) + (size_t)((R0 + 3) / 4) * 16 +
              (size_t)kFillLineThreads * 2 * sizeof(double);
    return f;
}

// renormalised double-float accumulation a += (bh, bl)
__device__ __forceinline__ void df_add2(float& ah, float& al, float bh, float bl)
{
    const float s = __fadd_rn(ah, bh);
    const float z = __fsub_rn(s, ah);
    float t = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, z)), __fsub_rn(bh, z));
    t = __fadd_rn(t, __fadd_rn(al, bl));
    ah = __fadd_rn(s, t);
    al = __fsub_rn(t, __fsub_rn(ah, s));
}

// sum_k E[k] row[k] in double-float: the first product exactly, then PolDF::mac
template <int Q1>
__device__ __forceinline__ DFAcc fill_eval_df(const float2* E, const float2* row)
{
    DFAcc acc;
    acc.h = __fmul_rn(E[0].x, row[0].x);
    float pe = __fmaf_rn(E[0].x, row[0].x, -acc.h);
    pe = __fmaf_rn(E[0].x, row[0].y, pe);
    acc.l = __fmaf_rn(E[0].y, row[0].x, pe);
#pragma unroll
    for (int k = 1; k < Q1; ++k) PolDF::mac(acc, E[k], row[k]);
    return acc;
}

template <int P, int DIM, typename T, int Q1>
__global__ void __launch_bounds__(kFillLineThreads) k_fill_line(Geo g, SplinePlan sp, SplineBufs sb, T* vals)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    constexpr int C = (S - 1) / 2;
    constexpr int NPAIR = (DIM == 3) ? W * W : W;
    extern __shared__ __align__(16) unsigned char fl_smem[];
    const int R0 = sp.r1[0] - sp.r0[0] + 1, R1 = sp.r1[1] - sp.r0[1] + 1;
    const int R2 = (DIM == 3) ? sp.r1[2] - sp.r0[2] + 1 : 1;
    const int first = sp.first;
    const bool kp = first > C;                     // kernel-preserving: the diagonal is minus the row sum
    const FillLineSmem f = fill_line_smem(S, first, sp.nu[0], R0, Q1);
    const int nu0 = f.nu0, U = f.U;
    float2* sPu = reinterpret_cast<float2*>(fl_smem);
    float2* sPl = sPu + (size_t)U * nu0;
    float2* sE = sPl + (size_t)U * nu0;            // [x0][k]
    int* sSp = reinterpret_cast<int*>(sE + (size_t)Q1 * R0);
    double* sD = reinterpret_cast<double*>(fl_smem + (f.bytes - (size_t)kFillLineThreads * 2 * sizeof(double)));
    const int x1 = (int)(blockIdx.x % (unsigned)R1), x2 = (int)(blockIdx.x / (unsigned)R1);
    const int tid = threadIdx.x;
    const int L0 = sp.L[0][P], L1x = sp.Lmax[1], L2x = (DIM == 3) ? sp.Lmax[2] : 1;
    const int64_t slot_stride = (int64_t)L2x * L1x * nu0;
    // stage the partial-field rows, the evaluation table and the spans
    for (int idx = tid; idx < U * nu0; idx += kFillLineThreads) {
        const int u = idx / nu0, a = idx - u * nu0;
        sPu[idx] = sb.partial[(int64_t)u * slot_stride + ((int64_t)x2 * L1x + x1) * nu0 + a];
        const int sl = S - 1 - first - u;          // lower slot whose mirror is u
        const int d1 = (sl / W) % W, d2 = (DIM == 3) ? sl / (W * W) : P;
        const int y1 = x1 + d1 - P, y2 = (DIM == 3) ? x2 + d2 - P : 0;
        if (y1 >= 0 && y1 < R1 && y2 >= 0 && y2 < R2)
            sPl[idx] = sb.partial[(int64_t)u * slot_stride + ((int64_t)y2 * L1x + y1) * nu0 + a];
    }
    for (int idx = tid; idx < Q1 * R0; idx += kFillLineThreads) {
        const int x0 = idx / Q1, k = idx - x0 * Q1;
        sE[idx] = sb.eval0[P][(int64_t)k * L0 + x0];
    }
    for (int x0 = tid; x0 < R0; x0 += kFillLineThreads) sSp[x0] = sb.espan[0][P][x0];
    __syncthreads();

    const int m0 = g.m[0], m1 = g.m[1];
    const int64_t N = (int64_t)m0 * m1 * ((DIM == 3) ? g.m[2] : 1);
    const int i1 = sp.r0[1] + x1, i2 = (DIM == 3) ? sp.r0[2] + x2 : 0;
    const int warp = tid >> 5, lane = tid & 31;
    const int wpc = f.wpc, ch = warp / wpc, wi = warp - ch * wpc;
    const bool wact = ch < f.nch;                  // warps past nch * wpc idle
    const int x0 = ch * 32 + lane;
    const bool act = wact && x0 < R0;
    const int x0c = act ? x0 : 0;
    const int64_t i = sp.r0[0] + x0 + (int64_t)m0 * (i1 + (int64_t)m1 * i2);
    float dh = 0.f, dl = 0.f;                      // double-float / compensated FP32 row sum
    double dframe = 0.0;                           // FP64 sum of gathered frame entries (FP64 values)
    if (wact) {
        const int sp0 = sSp[x0c];
        float2 Eu[Q1];                             // direction-0 evaluation row of the upper entries (at x~_i)
#pragma unroll
        for (int k = 0; k < Q1; ++k) Eu[k] = sE[x0c * Q1 + k];
        for (int pr = wi; pr < NPAIR; pr += wpc) {
            const int d1 = pr % W, d2 = (DIM == 3) ? pr / W : P;
            const int y1 = x1 + d1 - P, y2 = (DIM == 3) ? x2 + d2 - P : 0;
            const bool in12 = y1 >= 0 && y1 < R1 && y2 >= 0 && y2 < R2;
            const int sbase = W * (d1 + W * ((DIM == 3) ? d2 : 0));
            // frame columns of the pair (the exact A_ji of frame row j), all loads issued before the
            // pair's stores: they read frame rows, which this kernel never writes
            const int64_t jb = i - P + (int64_t)m0 * ((d1 - P) + (int64_t)m1 * (d2 - P));
            T gv[W];
#pragma unroll
            for (int d0 = 0; d0 < W; ++d0) {
                const int y0 = x0 + d0 - P;
                const bool gat = act && !(in12 && y0 >= 0 && y0 < R0) && !(kp && sbase + d0 == C);
                gv[d0] = gat ? vals[(int64_t)(S - 1 - sbase - d0) * N + jb + d0] : (T)0;
            }
#pragma unroll
            for (int d0 = 0; d0 < W; ++d0) {
                const int s = sbase + d0;
                if (kp && s == C) continue;
                const int y0 = x0 + d0 - P;
                T out;
                if (in12 && y0 >= 0 && y0 < R0) {
                    // upper slot: this line's partial row at x~_i; lower slot: the mirror's at x~_j
                    const bool upper = s >= first;
                    const int y0c = act ? y0 : 0;
                    const float2* row = upper ? sPu + (size_t)(s - first) * nu0 + sp0
                                              : sPl + (size_t)(S - 1 - s - first) * nu0 + sSp[y0c];
                    float2 E[Q1];
#pragma unroll
                    for (int k = 0; k < Q1; ++k) E[k] = upper ? Eu[k] : sE[y0c * Q1 + k];
                    if constexpr (sizeof(T) == 4) {
                        float acc = 0.f;
#pragma unroll
                        for (int k = 0; k < Q1; ++k) acc = __fmaf_rn(E[k].x, row[k].x, acc);
                        out = acc;
                        const float t = __fadd_rn(dh, acc);
                        const float z = __fsub_rn(t, dh);
                        dl = __fadd_rn(dl, __fadd_rn(__fsub_rn(dh, __fsub_rn(t, z)), __fsub_rn(acc, z)));
                        dh = t;
                    } else {
                        const DFAcc acc = fill_eval_df<Q1>(E, row);
                        out = f2d_exact(acc.h) + f2d_exact(acc.l);
                        if (kp) df_add2(dh, dl, acc.h, acc.l);
                    }
                } else {
                    out = gv[d0];
                    if constexpr (sizeof(T) == 4) {
                        const float v = (float)out;
                        const float t = __fadd_rn(dh, v);
                        const float z = __fsub_rn(t, dh);
                        dl = __fadd_rn(dl, __fadd_rn(__fsub_rn(dh, __fsub_rn(t, z)), __fsub_rn(v, z)));
                        dh = t;
                    } else {
                        dframe += (double)out;
                    }
                }
                if (act) vals[(int64_t)s * N + i] = out;
            }
        }
    }
    if (kp) {
        // the partial sums of a row (one per warp of its chunk), added in a fixed order by the chunk's first warp
        if (sizeof(T) == 4) { sD[2 * tid] = (double)dh; sD[2 * tid + 1] = (double)dl; }
        else { sD[2 * tid] = df2d_exact(dh, dl); sD[2 * tid + 1] = dframe; }
        __syncthreads();
        if (act && wi == 0) {
            double sum = 0.0, lo = 0.0;
            for (int w = 0; w < wpc; ++w) {
                const int t = (ch * wpc + w) * 32 + lane;
                sum += sD[2 * t];
                lo += sD[2 * t + 1];
            }
            vals[(int64_t)C * N + i] = (T)(-(sum + lo));
        }
    }
}

// FP32 values: the same pass with thread (ty, x0) taking row x0 of the line and
// the offset pairs ty, ty + Y, ... (evaluation table [k][x0]).  For FP32 values
// it is faster than the warp-per-chunk kernel above (1.10 against 1.42 ms at
// 96^3 p = 4); for FP64 values slower (2.73 against 2.50 ms).
template <int P, int DIM, typename T, int Q1>
__global__ void __launch_bounds__(kFillLineThreads) k_fill_line_rows(Geo g, SplinePlan sp, SplineBufs sb, T* vals)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    constexpr int C = (S - 1) / 2;
    extern __shared__ __align__(16) unsigned char fl_smem[];
    const int R0 = sp.r1[0] - sp.r0[0] + 1, R1 = sp.r1[1] - sp.r0[1] + 1;
    const int R2 = (DIM == 3) ? sp.r1[2] - sp.r0[2] + 1 : 1;
    const int first = sp.first;
    const bool kp = first > C;                     // kernel-preserving: the diagonal is minus the row sum
    const FillLineSmem f = fill_line_smem(S, first, sp.nu[0], R0, Q1);
    const int nu0 = f.nu0, U = f.U;
    const int XR = R0 < kFillLineThreads ? R0 : kFillLineThreads, Y = kFillLineThreads / XR;
    float2* sPu = reinterpret_cast<float2*>(fl_smem);
    float2* sPl = sPu + (size_t)U * nu0;
    float2* sE = sPl + (size_t)U * nu0;
    int* sSp = reinterpret_cast<int*>(sE + (size_t)Q1 * R0);
    double* sD = reinterpret_cast<double*>(fl_smem + (f.bytes - (size_t)kFillLineThreads * 2 * sizeof(double)));
    const int x1 = (int)(blockIdx.x % (unsigned)R1), x2 = (int)(blockIdx.x / (unsigned)R1);
    const int tid = threadIdx.x;
    const int L0 = sp.L[0][P], L1x = sp.Lmax[1], L2x = (DIM == 3) ? sp.Lmax[2] : 1;
    const int64_t slot_stride = (int64_t)L2x * L1x * nu0;
    // stage the partial-field rows, the evaluation table and the spans
    for (int idx = tid; idx < U * nu0; idx += kFillLineThreads) {
        const int u = idx / nu0, a = idx - u * nu0;
        sPu[idx] = sb.partial[(int64_t)u * slot_stride + ((int64_t)x2 * L1x + x1) * nu0 + a];
        const int sl = S - 1 - first - u;          // lower slot whose mirror is u
        const int d1 = (sl / W) % W, d2 = (DIM == 3) ? sl / (W * W) : P;
        const int y1 = x1 + d1 - P, y2 = (DIM == 3) ? x2 + d2 - P : 0;
        if (y1 >= 0 && y1 < R1 && y2 >= 0 && y2 < R2)
            sPl[idx] = sb.partial[(int64_t)u * slot_stride + ((int64_t)y2 * L1x + y1) * nu0 + a];
    }
    for (int idx = tid; idx < Q1 * R0; idx += kFillLineThreads) {
        const int k = idx / R0, x0 = idx - k * R0;
        sE[idx] = sb.eval0[P][(int64_t)k * L0 + x0];
    }
    for (int x0 = tid; x0 < R0; x0 += kFillLineThreads) sSp[x0] = sb.espan[0][P][x0];
    __syncthreads();

    const int m0 = g.m[0], m1 = g.m[1];
    const int64_t N = (int64_t)m0 * m1 * ((DIM == 3) ? g.m[2] : 1);
    const int i1 = sp.r0[1] + x1, i2 = (DIM == 3) ? sp.r0[2] + x2 : 0;
    const int ty = tid / XR, tx = tid - ty * XR;
    for (int xb = 0; xb < R0; xb += XR) {
        const int x0 = xb + tx;
        const bool active = ty < Y && x0 < R0;
        const int i0 = sp.r0[0] + x0;
        const int64_t i = i0 + (int64_t)m0 * (i1 + (int64_t)m1 * i2);
        float dh = 0.f, dl = 0.f;             // double-float / compensated FP32 row sum
        double dframe = 0.0;                  // FP64 sum of gathered frame entries (FP64 values)
        if (active) {
            const int sp0 = sSp[x0];
            float2 Eu[Q1];                    // direction-0 evaluation row of the upper entries (at x~_i)
#pragma unroll
            for (int k = 0; k < Q1; ++k) Eu[k] = sE[k * R0 + x0];
            constexpr int NPAIR = (DIM == 3) ? W * W : W;
            for (int pr = ty; pr < NPAIR; pr += Y) {
                const int d1 = pr % W, d2 = (DIM == 3) ? pr / W : P;
                const int y1 = x1 + d1 - P, y2 = (DIM == 3) ? x2 + d2 - P : 0;
                const bool in12 = y1 >= 0 && y1 < R1 && y2 >= 0 && y2 < R2;
                const int sbase = W * (d1 + W * ((DIM == 3) ? d2 : 0));
                // frame columns of the pair (the exact A_ji of frame row j), all loads issued before the
                // pair's stores: they read frame rows, which this kernel never writes
                const int64_t jb = i - P + (int64_t)m0 * ((d1 - P) + (int64_t)m1 * (d2 - P));
                T gv[W];
#pragma unroll
                for (int d0 = 0; d0 < W; ++d0) {
                    const int y0 = x0 + d0 - P;
                    const bool gat = !(in12 && y0 >= 0 && y0 < R0) && !(kp && sbase + d0 == C);
                    gv[d0] = gat ? vals[(int64_t)(S - 1 - sbase - d0) * N + jb + d0] : (T)0;
                }
#pragma unroll
                for (int d0 = 0; d0 < W; ++d0) {
                    const int s = sbase + d0;
                    if (kp && s == C) continue;
                    const int y0 = x0 + d0 - P;
                    T out;
                    if (in12 && y0 >= 0 && y0 < R0) {
                        const bool upper = s >= first;
                        const float2* row = upper ? sPu + (size_t)(s - first) * nu0 + sp0
                                                  : sPl + (size_t)(S - 1 - s - first) * nu0 + sSp[y0];
                        if constexpr (sizeof(T) == 4) {
                            float acc = 0.f;
#pragma unroll
                            for (int k = 0; k < Q1; ++k)
                                acc = __fmaf_rn(upper ? Eu[k].x : sE[k * R0 + y0].x, row[k].x, acc);
                            out = acc;
                            const float t = __fadd_rn(dh, acc);
                            const float z = __fsub_rn(t, dh);
                            dl = __fadd_rn(dl, __fadd_rn(__fsub_rn(dh, __fsub_rn(t, z)), __fsub_rn(acc, z)));
                            dh = t;
                        } else {
                            DFAcc acc = PolDF::zero();
#pragma unroll
                            for (int k = 0; k < Q1; ++k) PolDF::mac(acc, upper ? Eu[k] : sE[k * R0 + y0], row[k]);
                            out = df2d_exact(acc.h, acc.l);
                            if (kp) df_add2(dh, dl, acc.h, acc.l);
                        }
                    } else {
                        out = gv[d0];
                        if constexpr (sizeof(T) == 4) {
                            const float v = (float)out;
                            const float t = __fadd_rn(dh, v);
                            const float z = __fsub_rn(t, dh);
                            dl = __fadd_rn(dl, __fadd_rn(__fsub_rn(dh, __fsub_rn(t, z)), __fsub_rn(v, z)));
                            dh = t;
                        } else {
                            dframe += (double)out;
                        }
                    }
                    vals[(int64_t)s * N + i] = out;
                }
            }
        }
        if (kp) {
            // the Y partial sums of each row, added in a fixed order by thread ty = 0
            if (sizeof(T) == 4) { sD[2 * tid] = (double)dh; sD[2 * tid + 1] = (double)dl; }
            else { sD[2 * tid] = df2d_exact(dh, dl); sD[2 * tid + 1] = dframe; }
            __syncthreads();
            if (active && ty == 0) {
                double sum = 0.0, lo = 0.0;
                for (int y = 0; y < Y; ++y) {
                    sum += sD[2 * (y * XR + tx)];
                    lo += sD[2 * (y * XR + tx) + 1];
                }
                vals[(int64_t)C * N + i] = (T)(-(sum + lo));
            }
            __syncthreads();
        }
    }
}

template <int P, int DIM, typename T, int Q1>
static bool fill_line_launch(const Geo& g, const SplinePlan& sp, const SplineBufs& sb, T* vals, cudaStream_t s)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    const int R0 = sp.r1[0] - sp.r0[0] + 1, R1 = sp.r1[1] - sp.r0[1] + 1;
    const int R2 = (DIM == 3) ? sp.r1[2] - sp.r0[2] + 1 : 1;
    const FillLineSmem f = fill_line_smem(S, sp.first, sp.nu[0], R0, Q1);
    constexpr bool rows = sizeof(T) == 4;
    if (f.bytes > (size_t)160 * 1024 || (!rows && f.wpc < 1)) return false;
    static bool attr_set = false;          // the attribute is idempotent; setting it twice is harmless
    if (!attr_set) {
        // set once outside any stream capture (a capture then uses the fallback kernels until then)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
        const void* fn = nullptr;
        if constexpr (rows) fn = (const void*)k_fill_line_rows<P, DIM, T, Q1>;
        else fn = (const void*)k_fill_line<P, DIM, T, Q1>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) != cudaSuccess)
            return false;
        attr_set = true;
    }
    const unsigned grid = (unsigned)((int64_t)R1 * R2);
    if constexpr (rows) k_fill_line_rows<P, DIM, T, Q1><<<grid, kFillLineThreads, f.bytes, s>>>(g, sp, sb, vals);
    else k_fill_line<P, DIM, T, Q1><<<grid, kFillLineThreads, f.bytes, s>>>(g, sp, sb, vals);
    return true;
}

template <int P, int DIM, typename T>
static bool fill_line_q(const Geo& g, const SplinePlan& sp, const SplineBufs& sb, T* vals, cudaStream_t s)
{
    switch (sp.qe[0][P] + 1) {
    case 1: return fill_line_launch<P, DIM, T, 1>(g, sp, sb, vals, s);
    case 2: return fill_line_launch<P, DIM, T, 2>(g, sp, sb, vals, s);
    case 3: return fill_line_launch<P, DIM, T, 3>(g, sp, sb, vals, s);
    case 4: return fill_line_launch<P, DIM, T, 4>(g, sp, sb, vals, s);
    default: return false;      // q > 3: the general kernels
    }
}

// The kernel-preserving diagonal of the frame rows only (rows with an index
// outside [r0, r1] in some direction), after k_fill_line wrote those of Omega~.
// Thread t takes the t-th frame row: first the planes i2 outside [r0_2, r1_2],
// then the lines i1 outside [r0_1, r1_1] of the other planes, then the rows i0
// outside [r0_0, r1_0] of the remaining lines (consecutive threads take
// consecutive rows of one line: coalesced), so that every thread of the grid has
// a row (0.65 against 0.98 ms for a grid over all rows at 96^3 p = 4).  FP64
// sums (splitting the values into double-float pairs by integer operations took
// twice as long).
struct FrameRows {
    int m0, m1, m2;
    int r0[3], r1[3];
    int64_t nA, nB, nC;       // frame rows in the outer planes, outer lines, outer row runs
};

__device__ __forceinline__ int frame_index(int k, int lo, int hi)   // k-th index outside [lo, hi]
{
    return k < lo ? k : hi + 1 + (k - lo);
}

template <int P, int DIM, typename T>
__global__ void __launch_bounds__(kBlock) k_diag_frame(FrameRows fr, T* vals)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    constexpr int C = (S - 1) / 2;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= fr.nA + fr.nB + fr.nC) return;
    const int64_t plane = (int64_t)fr.m0 * fr.m1;
    int i0, i1, i2;
    if (t < fr.nA) {
        i2 = frame_index((int)(t / plane), fr.r0[2], fr.r1[2]);
        const int64_t r = t % plane;
        i1 = (int)(r / fr.m0);
        i0 = (int)(r % fr.m0);
    } else if ((t -= fr.nA) < fr.nB) {
        const int nb1 = fr.r0[1] + fr.m1 - 1 - fr.r1[1];
        const int64_t per = (int64_t)nb1 * fr.m0;
        i2 = fr.r0[2] + (int)(t / per);
        const int64_t r = t % per;
        i1 = frame_index((int)(r / fr.m0), fr.r0[1], fr.r1[1]);
        i0 = (int)(r % fr.m0);
    } else {
        t -= fr.nB;
        const int nc0 = fr.r0[0] + fr.m0 - 1 - fr.r1[0];
        const int R1 = fr.r1[1] - fr.r0[1] + 1;
        const int64_t line = t / nc0;
        i2 = fr.r0[2] + (int)(line / R1);
        i1 = fr.r0[1] + (int)(line % R1);
        i0 = frame_index((int)(t % nc0), fr.r0[0], fr.r1[0]);
    }
    const int64_t N = plane * fr.m2;
    const int64_t i = i0 + (int64_t)fr.m0 * (i1 + (int64_t)fr.m1 * i2);
    // four interleaved partial sums keep more loads in flight; combined in a fixed order
    double part[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int s = 0; s < S; ++s)
        if (s != C) part[s & 3] += (double)vals[(int64_t)s * N + i];
    vals[(int64_t)C * N + i] = (T)(-((part[0] + part[1]) + (part[2] + part[3])));
}

// FP32 values: one thread per row of the whole patch, the rows of Omega~ leaving
// at once (measured faster for FP32 values than the frame-row enumeration above,
// 0.38 against 0.69 ms at 96^3 p = 4; for FP64 values the enumeration wins).
template <int P, int DIM>
__global__ void __launch_bounds__(kBlock) k_diag_frame_f32(FrameRows fr, float* vals)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    constexpr int C = (S - 1) / 2;
    const int64_t N = (int64_t)fr.m0 * fr.m1 * fr.m2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int i0 = (int)(i % fr.m0), i1 = (int)((i / fr.m0) % fr.m1), i2 = (int)(i / ((int64_t)fr.m0 * fr.m1));
    if (i0 >= fr.r0[0] && i0 <= fr.r1[0] && i1 >= fr.r0[1] && i1 <= fr.r1[1] && i2 >= fr.r0[2] && i2 <= fr.r1[2]) return;
    float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
#pragma unroll 4
    for (int s = 0; s < S; ++s) {
        if (s == C) continue;
        const float v = vals[(int64_t)s * N + i];
        const int k = s & 1;
        const float t = __fadd_rn(hi[k], v);
        const float z = __fsub_rn(t, hi[k]);
        lo[k] = __fadd_rn(lo[k], __fadd_rn(__fsub_rn(hi[k], __fsub_rn(t, z)), __fsub_rn(v, z)));
        hi[k] = t;
    }
    vals[(int64_t)C * N + i] = (float)(-((double)hi[0] + (double)hi[1] + ((double)lo[0] + (double)lo[1])));
}

template <int P, int DIM, typename T>
static bool fill_common_q(const Geo& g, const SplinePlan& sp, const SplineBufs& sb, T* vals, unsigned grid,
                          cudaStream_t s)
{
    switch (sp.qe[0][P] + 1) {
    case 1: k_fill_common<P, DIM, T, 1><<<grid, kBlock, 0, s>>>(g, sp, sb, vals); return true;
    case 2: k_fill_common<P, DIM, T, 2><<<grid, kBlock, 0, s>>>(g, sp, sb, vals); return true;
    case 3: k_fill_common<P, DIM, T, 3><<<grid, kBlock, 0, s>>>(g, sp, sb, vals); return true;
    case 4: k_fill_common<P, DIM, T, 4><<<grid, kBlock, 0, s>>>(g, sp, sb, vals); return true;
    default: return false;      // q > 3: the general kernel
    }
}

// Pass 2 (every row): the kernel-preserving diagonal, minus the sum of the
// row's stored off-diagonal values.  For FP64 values the sum is FP64, whose
// rounding stays ~1e-15 of the row's mass even for 1330 terms (a double-float sum
// with the contractions' cheap accumulation lost ~1e-12); for FP32 values a
// compensated FP32 sum is far more accurate than the FP32 result.
template <int P, int DIM, typename T>
__global__ void __launch_bounds__(kBlock) k_diag(int64_t N, T* vals)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    constexpr int C = (S - 1) / 2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if constexpr (sizeof(T) == 4) {
        // FP32 values: two compensated FP32 sums (Knuth two-sum per term; the error
        // terms collected in a second float) on the FP32 pipe; far below the rounding
        // of the FP32 result
        float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
#pragma unroll 4
        for (int s = 0; s < S; ++s) {
            if (s == C) continue;
            const float v = (float)vals[(int64_t)s * N + i];
            const int k = s & 1;
            const float t = __fadd_rn(hi[k], v);
            const float z = __fsub_rn(t, hi[k]);
            lo[k] = __fadd_rn(lo[k], __fadd_rn(__fsub_rn(hi[k], __fsub_rn(t, z)), __fsub_rn(v, z)));
            hi[k] = t;
        }
        vals[(int64_t)C * N + i] = (T)(-((double)hi[0] + (double)hi[1] + ((double)lo[0] + (double)lo[1])));
    } else {
        // four interleaved partial sums keep more loads in flight; combined in a fixed order
        double part[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
        for (int s = 0; s < S; ++s)
            if (s != C) part[s & 3] += (double)vals[(int64_t)s * N + i];
        vals[(int64_t)C * N + i] = (T)(-((part[0] + part[1]) + (part[2] + part[3])));
    }
}

template <int P>
static void fill_p(const Geo& g, const SplinePlan& sp, int empty_box, const SplineBufs& sb, void* ell,
                   int f32, cudaStream_t s)
{
    const int W = 2 * P + 1;
    const int64_t N = (int64_t)g.m[0] * g.m[1] * (g.dim == 3 ? g.m[2] : 1);
    const unsigned gdiag = (unsigned)((N + kBlock - 1) / kBlock);
    bool line = false;          // k_fill_line wrote the Omega~ rows' diagonals
    if (!empty_box) {
        const int64_t R0 = sp.r1[0] - sp.r0[0] + 1, R1 = sp.r1[1] - sp.r0[1] + 1;
        const int64_t total = R0 * R1 * (g.dim == 3 ? (int64_t)(sp.r1[2] - sp.r0[2] + 1) * W * W : W);
        const unsigned gfill = (unsigned)((total + kBlock - 1) / kBlock);
        launch_begin(K_FILL, s);
        bool done = false;
        if (sp.all) {
            if (g.dim == 3) line = f32 ? fill_line_q<P, 3, float>(g, sp, sb, (float*)ell, s)
                                       : fill_line_q<P, 3, double>(g, sp, sb, (double*)ell, s);
            else line = f32 ? fill_line_q<P, 2, float>(g, sp, sb, (float*)ell, s)
                            : fill_line_q<P, 2, double>(g, sp, sb, (double*)ell, s);
            done = line;
            if (!done) {
                if (g.dim == 3) done = f32 ? fill_common_q<P, 3, float>(g, sp, sb, (float*)ell, gfill, s)
                                           : fill_common_q<P, 3, double>(g, sp, sb, (double*)ell, gfill, s);
                else done = f32 ? fill_common_q<P, 2, float>(g, sp, sb, (float*)ell, gfill, s)
                                : fill_common_q<P, 2, double>(g, sp, sb, (double*)ell, gfill, s);
            }
        }
        if (!done) {
            if (g.dim == 3) {
                if (f32) k_fill<P, 3, float><<<gfill, kBlock, 0, s>>>(g, sp, sb, (float*)ell);
                else k_fill<P, 3, double><<<gfill, kBlock, 0, s>>>(g, sp, sb, (double*)ell);
            } else {
                if (f32) k_fill<P, 2, float><<<gfill, kBlock, 0, s>>>(g, sp, sb, (float*)ell);
                else k_fill<P, 2, double><<<gfill, kBlock, 0, s>>>(g, sp, sb, (double*)ell);
            }
        }
        launch_end(K_FILL, s);
    }
    if (sp.first <= sp.c && !empty_box) return;      // symmetric surrogate: no kernel-preserving diagonal
    if (g.form == kFormMass) return;                  // mass matrix with an empty Omega~: all rows exact
    launch_begin(K_DIAG, s);
    if (line) {
        FrameRows fr;
        fr.m0 = g.m[0]; fr.m1 = g.m[1]; fr.m2 = g.dim == 3 ? g.m[2] : 1;
        for (int d = 0; d < 3; ++d) {
            fr.r0[d] = d < g.dim ? sp.r0[d] : 0;
            fr.r1[d] = d < g.dim ? sp.r1[d] : 0;
        }
        const int64_t R[3] = {fr.r1[0] - fr.r0[0] + 1, fr.r1[1] - fr.r0[1] + 1, fr.r1[2] - fr.r0[2] + 1};
        fr.nA = (int64_t)(fr.m2 - R[2]) * fr.m0 * fr.m1;
        fr.nB = R[2] * (fr.m1 - R[1]) * fr.m0;
        fr.nC = R[2] * R[1] * (fr.m0 - R[0]);
        const unsigned gframe = (unsigned)((fr.nA + fr.nB + fr.nC + kBlock - 1) / kBlock);
        if (f32) {
            if (g.dim == 3) k_diag_frame_f32<P, 3><<<gdiag, kBlock, 0, s>>>(fr, (float*)ell);
            else k_diag_frame_f32<P, 2><<<gdiag, kBlock, 0, s>>>(fr, (float*)ell);
        } else if (gframe > 0) {
            if (g.dim == 3) k_diag_frame<P, 3, double><<<gframe, kBlock, 0, s>>>(fr, (double*)ell);
            else k_diag_frame<P, 2, double><<<gframe, kBlock, 0, s>>>(fr, (double*)ell);
        }
    } else if (g.dim == 3) {
        if (f32) k_diag<P, 3, float><<<gdiag, kBlock, 0, s>>>(N, (float*)ell);
        else k_diag<P, 3, double><<<gdiag, kBlock, 0, s>>>(N, (double*)ell);
    } else {
        if (f32) k_diag<P, 2, float><<<gdiag, kBlock, 0, s>>>(N, (float*)ell);
        else k_diag<P, 2, double><<<gdiag, kBlock, 0, s>>>(N, (double*)ell);
    }
    launch_end(K_DIAG, s);
}

cudaError_t launch_fill(const Geo& g, const SplinePlan& sp, int empty_box, const SplineBufs& sb,
                        void* ell, int ell_f32, cudaStream_t s)
{
    switch (g.p) {
    case 1: fill_p<1>(g, sp, empty_box, sb, ell, ell_f32, s); break;
    case 2: fill_p<2>(g, sp, empty_box, sb, ell, ell_f32, s); break;
    case 3: fill_p<3>(g, sp, empty_box, sb, ell, ell_f32, s); break;
    case 4: fill_p<4>(g, sp, empty_box, sb, ell, ell_f32, s); break;
    case 5: fill_p<5>(g, sp, empty_box, sb, ell, ell_f32, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace iga
