// K3 for the mass form (Sec. 8): M_ij = sum_g w_g |det Dphi(g)| B_i(g) B_j(g),
// sum-factorised over the same boxes of rows, with the same thread mapping
// and launch sizes as the stiffness stages (k_quad.cu), but one scalar field
// (|det Dphi| at the Gauss points, from k_coef) and only the value-value pair
// weights X_d[i][delta][t][00]:
//
//   stage Z (3-D): field [g2][g1][g0]            -> T1 [(i2,d2)][g1][g0]
//   stage Y      : T1 (3-D) or the field (2-D)   -> T2 [(i2,d2)][(i1,d1)][g0]
//   stage X      : T2                            -> rows [slot][row]
#include "arith.cuh"
#include "iga_internal.cuh"

namespace iga {

// Q consecutive values from an offset that is a multiple of Q (the T2 lines of
// a box start on 16-byte boundaries): 16-byte loads when Q values fill whole
// 16-byte words, else scalar loads.
template <class S, int Q>
__device__ __forceinline__ void load_run_m(const S* p, S* v)
{
    if constexpr ((Q * sizeof(S)) % 16 == 0) {
        const float4* p4 = reinterpret_cast<const float4*>(p);
        float4* v4 = reinterpret_cast<float4*>(v);
#pragma unroll
        for (int k = 0; k < (int)(Q * sizeof(S) / 16); ++k) v4[k] = p4[k];
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = p[k];
    }
}

template <class Pol, int P>
__global__ void __launch_bounds__(kBlock) k_mass_z(Geo g, Tables T, BoxSet bs, double* scratch)
{
    using S = typename Pol::store;
    using A = typename Pol::acc;
    constexpr int Q = P + 1, W = 2 * P + 1, TT = Q * Q;
    Box b;
    get_box(bs, 3, P, 1, blockIdx.x, b);
    const int64_t G0 = (int64_t)b.E[0] * Q, G1 = (int64_t)b.E[1] * Q;
    const int64_t plane = G0 * G1;
    const int64_t item = (int64_t)(blockIdx.x - b.blk[1]) * kBlock + threadIdx.x;
    if (item >= (int64_t)b.R[2] * plane) return;
    const int i3l = (int)(item / plane);
    const int64_t pp = item % plane;
    const int i3 = b.rlo[2] + i3l;
    const S* C = reinterpret_cast<const S*>(scratch + b.c_off);
    const S* Xi = reinterpret_cast<const S*>(T.Xs[2]) + (int64_t)i3 * W * TT * 4;
    A acc[W];
#pragma unroll
    for (int dd = 0; dd < W; ++dd) acc[dd] = Pol::zero();
#pragma unroll
    for (int a = 0; a <= P; ++a) {
        const int e3 = i3 - P + a;
        if (e3 < b.elo[2] || e3 >= b.elo[2] + b.E[2]) continue;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            const int t = a * Q + r;
            const S c0 = C[(int64_t)((e3 - b.elo[2]) * Q + r) * plane + pp];
#pragma unroll
            for (int dd = a; dd <= a + P; ++dd) Pol::mac(acc[dd], Xi[(dd * TT + t) * 4], c0);
        }
    }
    S* T1 = reinterpret_cast<S*>(scratch + b.t1_off);
#pragma unroll
    for (int dd = 0; dd < W; ++dd) T1[((int64_t)i3l * W + dd) * plane + pp] = Pol::to_store(acc[dd]);
}

template <class Pol, int P, int DIM>
__global__ void __launch_bounds__(kBlock) k_mass_y(Geo g, Tables T, BoxSet bs, double* scratch)
{
    using S = typename Pol::store;
    using A = typename Pol::acc;
    constexpr int Q = P + 1, W = 2 * P + 1, TT = Q * Q;
    Box b;
    get_box(bs, DIM, P, 2, blockIdx.x, b);
    const int64_t G0 = (int64_t)b.E[0] * Q, G1 = (int64_t)b.E[1] * Q;
    const int64_t P3 = (DIM == 3) ? (int64_t)b.R[2] * W : 1;
    const int R2 = b.R[1];
    const int64_t item = (int64_t)(blockIdx.x - b.blk[2]) * kBlock + threadIdx.x;
    if (item >= P3 * R2 * G0) return;
    const int64_t g0 = item % G0;
    const int i2l = (int)((item / G0) % R2);
    const int64_t pair3 = item / (G0 * R2);
    const int i2 = b.rlo[1] + i2l;
    const S* Xi = reinterpret_cast<const S*>(T.Xs[1]) + (int64_t)i2 * W * TT * 4;
    const S* in = (DIM == 3) ? reinterpret_cast<const S*>(scratch + b.t1_off) + pair3 * G1 * G0 + g0
                             : reinterpret_cast<const S*>(scratch + b.c_off) + g0;
    A acc[W];
#pragma unroll
    for (int dd = 0; dd < W; ++dd) acc[dd] = Pol::zero();
#pragma unroll
    for (int a = 0; a <= P; ++a) {
        const int e2 = i2 - P + a;
        if (e2 < b.elo[1] || e2 >= b.elo[1] + b.E[1]) continue;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            const int t = a * Q + r;
            const S v = in[(int64_t)((e2 - b.elo[1]) * Q + r) * G0];
#pragma unroll
            for (int dd = a; dd <= a + P; ++dd) Pol::mac(acc[dd], Xi[(dd * TT + t) * 4], v);
        }
    }
    S* T2 = reinterpret_cast<S*>(scratch + b.t2_off);
    const int64_t P2 = (int64_t)R2 * W;
#pragma unroll
    for (int dd = 0; dd < W; ++dd) T2[(pair3 * P2 + (int64_t)i2l * W + dd) * G0 + g0] = Pol::to_store(acc[dd]);
}

// Stage X: same item mapping as k_stage_x (kLinesX lines of one row per thread).
// Rows whose stencil stays among cardinal B-splines share one pair-weight table
// (translation invariance, Sec. 2.2), staged in shared memory: the loads of a
// warp become broadcasts instead of one cache line per thread.
template <class Pol, int P, int DIM>
__global__ void __launch_bounds__(kBlock) k_mass_x(Geo g, Tables T, BoxSet bs, double* scratch, void* ell,
                                                   int ell_f32, int64_t N, double* samples)
{
    using S = typename Pol::store;
    using A = typename Pol::acc;
    constexpr int Q = P + 1, W = 2 * P + 1, TT = Q * Q, LINES = kLinesX;
    __shared__ S sX[W * TT];
    const bool has_card = g.m[0] >= 4 * P + 1;
    const S* X0 = reinterpret_cast<const S*>(T.Xs[0]);
    if (has_card)
        for (int k = threadIdx.x; k < W * TT; k += blockDim.x) sX[k] = X0[((int64_t)(2 * P) * W * TT + k) * 4];
    __syncthreads();
    Box b;
    get_box(bs, DIM, P, 3, blockIdx.x, b);
    const int64_t G0 = (int64_t)b.E[0] * Q;
    const int64_t P3 = (DIM == 3) ? (int64_t)b.R[2] * W : 1;
    const int64_t P2 = (int64_t)b.R[1] * W;
    const int64_t NL = (P2 + LINES - 1) / LINES;
    const int R1 = b.R[0];
    const int64_t item = (int64_t)(blockIdx.x - b.blk[3]) * kBlock + threadIdx.x;
    if (item >= P3 * NL * R1) return;
    const int i1l = (int)(item % R1);
    const int64_t lg = (item / R1) % NL;
    const int64_t pair3 = item / (R1 * NL);
    const int i1 = b.rlo[0] + i1l;
    const int i3 = (DIM == 3) ? b.rlo[2] + (int)(pair3 / W) : 0;
    const int d3 = (DIM == 3) ? (int)(pair3 % W) : 0;
    const bool card = has_card && i1 >= 2 * P && i1 <= g.m[0] - 2 * P - 1;
    // pattern-00 weight of (delta, t): sX[dd * TT + t], or every fourth entry of the global table
    const S* Xi = card ? sX : X0 + (int64_t)i1 * W * TT * 4;
    const int xs = card ? 1 : 4;
    int nl = (int)(P2 - lg * LINES);
    if (nl > LINES) nl = LINES;
    const S* T2[LINES];
#pragma unroll
    for (int l = 0; l < LINES; ++l)
        T2[l] = reinterpret_cast<const S*>(scratch + b.t2_off) + (pair3 * P2 + lg * LINES + (l < nl ? l : 0)) * G0;
    A acc[LINES][W];
#pragma unroll
    for (int l = 0; l < LINES; ++l)
#pragma unroll
        for (int dd = 0; dd < W; ++dd) acc[l][dd] = Pol::zero();
#pragma unroll
    for (int a = 0; a <= P; ++a) {
        const int e1 = i1 - P + a;
        if (e1 < b.elo[0] || e1 >= b.elo[0] + b.E[0]) continue;
        const int64_t o = (int64_t)(e1 - b.elo[0]) * Q;
        __align__(16) S v[LINES][Q];
#pragma unroll
        for (int l = 0; l < LINES; ++l) load_run_m<S, Q>(T2[l] + o, v[l]);
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            const int t = a * Q + r;
#pragma unroll
            for (int dd = a; dd <= a + P; ++dd) {
                const S x = Xi[(dd * TT + t) * xs];
#pragma unroll
                for (int l = 0; l < LINES; ++l) Pol::mac(acc[l][dd], x, v[l][r]);
            }
        }
    }
#pragma unroll
    for (int l = 0; l < LINES; ++l) {
        if (l >= nl) break;
        const int64_t pair2 = lg * LINES + l;
        const int i2 = b.rlo[1] + (int)(pair2 / W);
        const int d2 = (int)(pair2 % W);
        const int slot0 = W * (d2 + W * d3);
        if (b.out_kind == 0) {
            const int64_t row = i1 + (int64_t)g.m[0] * (i2 + (int64_t)g.m[1] * i3);
#pragma unroll
            for (int dd = 0; dd < W; ++dd) {
                if (ell_f32) ((float*)ell)[(int64_t)(slot0 + dd) * N + row] = Pol::to_float(acc[l][dd]);
                else ((double*)ell)[(int64_t)(slot0 + dd) * N + row] = Pol::to_double(acc[l][dd]);
            }
        } else {
#pragma unroll
            for (int dd = 0; dd < W; ++dd)
                samples[(int64_t)(slot0 + dd) * bs.n_samples + b.sample_id] = Pol::to_double(acc[l][dd]);
        }
    }
}

template <class Pol, int P>
static cudaError_t mass_p(const Geo& g, const Tables& T, const BoxSet& bs, const int64_t nb[4], double* scratch,
                          void* ell, int ell_f32, double* samples, cudaStream_t s)
{
    const int64_t N = (int64_t)g.m[0] * g.m[1] * (g.dim == 3 ? g.m[2] : 1);
    if (g.dim == 3) {
        if (nb[1] > 0) {
            launch_begin(K_STAGE_Z, s);
            k_mass_z<Pol, P><<<(unsigned)nb[1], kBlock, 0, s>>>(g, T, bs, scratch);
            launch_end(K_STAGE_Z, s);
        }
        if (nb[2] > 0) {
            launch_begin(K_STAGE_Y, s);
            k_mass_y<Pol, P, 3><<<(unsigned)nb[2], kBlock, 0, s>>>(g, T, bs, scratch);
            launch_end(K_STAGE_Y, s);
        }
        if (nb[3] > 0) {
            launch_begin(K_STAGE_X, s);
            k_mass_x<Pol, P, 3><<<(unsigned)nb[3], kBlock, 0, s>>>(g, T, bs, scratch, ell, ell_f32, N, samples);
            launch_end(K_STAGE_X, s);
        }
    } else {
        if (nb[2] > 0) {
            launch_begin(K_STAGE_Y, s);
            k_mass_y<Pol, P, 2><<<(unsigned)nb[2], kBlock, 0, s>>>(g, T, bs, scratch);
            launch_end(K_STAGE_Y, s);
        }
        if (nb[3] > 0) {
            launch_begin(K_STAGE_X, s);
            k_mass_x<Pol, P, 2><<<(unsigned)nb[3], kBlock, 0, s>>>(g, T, bs, scratch, ell, ell_f32, N, samples);
            launch_end(K_STAGE_X, s);
        }
    }
    return cudaGetLastError();
}

template <class Pol>
static cudaError_t mass_pol(const Geo& g, const Tables& T, const BoxSet& bs, const int64_t nb[4], double* scratch,
                            void* ell, int ell_f32, double* samples, cudaStream_t s)
{
    switch (g.p) {
    case 1: return mass_p<Pol, 1>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    case 2: return mass_p<Pol, 2>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    case 3: return mass_p<Pol, 3>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    case 4: return mass_p<Pol, 4>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    case 5: return mass_p<Pol, 5>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mass_stages(const Geo& g, const Tables& T, const BoxSet& bs, const int64_t nblocks[4],
                               double* scratch, void* ell, int ell_f32, double* samples, cudaStream_t s)
{
    switch (T.arith) {
    case kArithF64: return mass_pol<PolF64>(g, T, bs, nblocks, scratch, ell, ell_f32, samples, s);
    case kArithDF: return mass_pol<PolDF>(g, T, bs, nblocks, scratch, ell, ell_f32, samples, s);
    case kArithF32: return mass_pol<PolF32>(g, T, bs, nblocks, scratch, ell, ell_f32, samples, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace iga
