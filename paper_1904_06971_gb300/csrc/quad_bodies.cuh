// K3: sum-factorised Gauss quadrature of full stencil rows over boxes of rows.
//
// A_ij = sum_{k,l} sum_g K_kl(g) d_k B_i(g) d_l B_j(g) (Sec. 3.2, eq. ChangeOfVars)
// factorises per direction: the Gauss points, the row index i_d and the
// column offset delta_d = j_d - i_d of direction d meet only in the 1-D pair
// weights X_d[i_d][delta_d][t][pat] (k_tables.cu).  The 3-D sum is
// contracted one direction at a time, slowest first, so every stage reads and
// writes arrays whose fastest index is contiguous:
//
//   stage Z (3-D): K fields [6][g2][g1][g0]            -> T1 [8][(i2,d2)][g1][g0]  (two launches of 4 combos)
//   stage Y      : T1 (3-D) or K fields (2-D)          -> T2 [4][(i2,d2)][(i1,d1)][g0]
//   stage X      : T2                                  -> rows [slot][row]
//
// T1 combos (field, pattern in direction 2): (K00,00) (K01,00) (K11,00)
// (K02,01) (K02,10) (K12,01) (K12,10) (K22,11).  T2 groups are indexed by the
// pattern still to be applied in direction 0: 11, 10, 01, 00.  A pattern
// (alpha, beta) puts a derivative on the row function (alpha) and/or the
// column function (beta); the nine (k, l) terms are routed so that each
// reaches its pattern (d_k on B_i, d_l on B_j) in every direction.
//
// The kernels are templated on the arithmetic policy (arith.cuh): FP64,
// double-float on the FP32 pipe, or FP32.
#pragma once

#include "arith.cuh"
#include "iga_internal.cuh"

namespace iga {

// The four pattern weights (00, 01, 10, 11) of one (delta, t) are contiguous:
// two 16-byte loads for double / float2 values, one for float.
template <class S>
__device__ __forceinline__ void load_pats(const S* p, S& x00, S& x01, S& x10, S& x11)
{
    x00 = p[0]; x01 = p[1]; x10 = p[2]; x11 = p[3];
}
template <>
__device__ __forceinline__ void load_pats<float2>(const float2* p, float2& x00, float2& x01, float2& x10, float2& x11)
{
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    x00 = make_float2(a.x, a.y); x01 = make_float2(a.z, a.w);
    x10 = make_float2(b.x, b.y); x11 = make_float2(b.z, b.w);
}
template <>
__device__ __forceinline__ void load_pats<double>(const double* p, double& x00, double& x01, double& x10, double& x11)
{
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    x00 = a.x; x01 = a.y; x10 = b.x; x11 = b.y;
}
template <>
__device__ __forceinline__ void load_pats<float>(const float* p, float& x00, float& x01, float& x10, float& x11)
{
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    x00 = a.x; x01 = a.y; x10 = a.z; x11 = a.w;
}

// Q consecutive values starting at an offset that is a multiple of Q; 16-byte
// vector loads when Q values span whole 16-byte words (then they are aligned).
template <class S, int Q>
__device__ __forceinline__ void load_run(const S* p, S* v)
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

// ---------------------------------------------------------------------------
// stage Z: contract direction 2.  HALF selects combos 0..3 or 4..7 (two launches
// keep the accumulators of one thread small enough for two blocks per SM).
// ---------------------------------------------------------------------------
// SYM is the box's symmetry mode (Box::sym) as a template argument, so that the offsets a
// symmetric box skips leave no branch in the unrolled offset loops; SYM = 2 reads it at run time
// (the FP32 body, whose three copies would spill at its three-blocks-per-SM register budget).
template <int SYM, int P>
__device__ __forceinline__ bool z_skip(int sym, int dd)
{
    if constexpr (SYM == 2) return (sym > 0 && dd < P) || (sym < 0 && dd > P);
    else return (SYM > 0 && dd < P) || (SYM < 0 && dd > P);
}

template <class Pol, int P, int HALF, int SYM>
__device__ __forceinline__ void stage_z_box(const Tables& T, const Box& b, double* scratch, int64_t blk)
{
    using S = typename Pol::store;
    using A = typename Pol::acc;
    constexpr int Q = P + 1, W = 2 * P + 1, TT = Q * Q;
    const int64_t G0 = (int64_t)b.E[0] * Q, G1 = (int64_t)b.E[1] * Q, G2 = (int64_t)b.E[2] * Q;
    const int64_t plane = G0 * G1;
    const int64_t item = (blk - b.blk[1]) * kBlock + threadIdx.x;
    if (item >= (int64_t)b.R[2] * plane) return;
    const int i3l = (int)(item / plane);
    const int64_t pp = item % plane;
    const int i3 = b.rlo[2] + i3l;
    const S* C = reinterpret_cast<const S*>(scratch + b.c_off);
    const int64_t fs = G2 * plane;
    const S* Xi = reinterpret_cast<const S*>(T.Xs[2]) + (int64_t)i3 * W * TT * 4;

    A acc[W][4];
#pragma unroll
    for (int dd = 0; dd < W; ++dd)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[dd][k] = Pol::zero();

    // local element a of supp(B_i) meets supp(B_{i+delta}) exactly for dd = delta + P in [a, a + P]
#pragma unroll
    for (int a = 0; a <= P; ++a) {
        const int e3 = i3 - P + a;
        if (e3 < b.elo[2] || e3 >= b.elo[2] + b.E[2]) continue;
        if constexpr (Pol::kind == kArithF32) {
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            const int t = a * Q + r;
            const int64_t o = (int64_t)((e3 - b.elo[2]) * Q + r) * plane + pp;
            S c0, c1, c2, c3;
            if (HALF == 0) { c0 = C[o]; c1 = C[fs + o]; c2 = C[3 * fs + o]; c3 = C[2 * fs + o]; }
            else { c0 = C[2 * fs + o]; c1 = C[4 * fs + o]; c2 = C[5 * fs + o]; c3 = c0; }
#pragma unroll
            for (int dd = a; dd <= a + P; ++dd) {
                if (z_skip<SYM, P>(b.sym, dd)) continue;   // symmetric: one sign of delta_2
                S x00, x01, x10, x11;
                load_pats(Xi + (dd * TT + t) * 4, x00, x01, x10, x11);
                if (HALF == 0) {
                    Pol::mac(acc[dd][0], x00, c0);   // (K00, 00)
                    Pol::mac(acc[dd][1], x00, c1);   // (K01, 00)
                    Pol::mac(acc[dd][2], x00, c2);   // (K11, 00)
                    Pol::mac(acc[dd][3], x01, c3);   // (K02, 01)
                } else {
                    Pol::mac(acc[dd][0], x10, c0);   // (K02, 10)
                    Pol::mac(acc[dd][1], x01, c1);   // (K12, 01)
                    Pol::mac(acc[dd][2], x10, c1);   // (K12, 10)
                    Pol::mac(acc[dd][3], x11, c2);   // (K22, 11)
                }
            }
        }
        } else {
            // the rolled Gauss-point loop loads the next point's fields before this point's
            // multiply-adds, so that their latency overlaps the arithmetic
            auto load_c = [&](int r, S& c0, S& c1, S& c2, S& c3) {
                const int64_t o = (int64_t)((e3 - b.elo[2]) * Q + r) * plane + pp;
                if (HALF == 0) { c0 = C[o]; c1 = C[fs + o]; c2 = C[3 * fs + o]; c3 = C[2 * fs + o]; }
                else { c0 = C[2 * fs + o]; c1 = C[4 * fs + o]; c2 = C[5 * fs + o]; c3 = c0; }
            };
            S n0, n1, n2, n3;
            load_c(0, n0, n1, n2, n3);
#pragma unroll 1
        for (int r = 0; r < Q; ++r) {
            const int t = a * Q + r;
            const S c0 = n0, c1 = n1, c2 = n2, c3 = n3;
            if (r + 1 < Q) load_c(r + 1, n0, n1, n2, n3);
#pragma unroll
            for (int dd = a; dd <= a + P; ++dd) {
                if (z_skip<SYM, P>(b.sym, dd)) continue;   // symmetric: one sign of delta_2
                S x00, x01, x10, x11;
                load_pats(Xi + (dd * TT + t) * 4, x00, x01, x10, x11);
                if (HALF == 0) {
                    Pol::mac(acc[dd][0], x00, c0);   // (K00, 00)
                    Pol::mac(acc[dd][1], x00, c1);   // (K01, 00)
                    Pol::mac(acc[dd][2], x00, c2);   // (K11, 00)
                    Pol::mac(acc[dd][3], x01, c3);   // (K02, 01)
                } else {
                    Pol::mac(acc[dd][0], x10, c0);   // (K02, 10)
                    Pol::mac(acc[dd][1], x01, c1);   // (K12, 01)
                    Pol::mac(acc[dd][2], x10, c1);   // (K12, 10)
                    Pol::mac(acc[dd][3], x11, c2);   // (K22, 11)
                }
            }
        }
        }
    }
    S* T1 = reinterpret_cast<S*>(scratch + b.t1_off);
    const int64_t P3 = (int64_t)b.R[2] * W;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int dd = 0; dd < W; ++dd)
            if (!z_skip<SYM, P>(b.sym, dd))
                T1[((int64_t)(4 * HALF + k) * P3 + (int64_t)i3l * W + dd) * plane + pp] = Pol::to_store(acc[dd][k]);
}

template <class Pol, int P, int HALF>
__device__ __forceinline__ void stage_z_body(const Geo& g, const Tables& T, const BoxSet& bs, double* scratch,
                                             int64_t blk)
{
    Box b;
    get_box(bs, 3, P, 1, blk, b);
    if constexpr (Pol::kind == kArithF32) stage_z_box<Pol, P, HALF, 2>(T, b, scratch, blk);
    else if (b.sym > 0) stage_z_box<Pol, P, HALF, 1>(T, b, scratch, blk);
    else if (b.sym < 0) stage_z_box<Pol, P, HALF, -1>(T, b, scratch, blk);
    else stage_z_box<Pol, P, HALF, 0>(T, b, scratch, blk);
}

// ---------------------------------------------------------------------------
// stage Y: contract direction 1
// ---------------------------------------------------------------------------
template <class Pol, int P, int DIM>
__device__ __forceinline__ void stage_y_body(const Geo& g, const Tables& T, const BoxSet& bs, double* scratch,
                                             int64_t blk)
{
    using S = typename Pol::store;
    using A = typename Pol::acc;
    constexpr int Q = P + 1, W = 2 * P + 1, TT = Q * Q;
    constexpr int NIN = (DIM == 3) ? 8 : 3;
    Box b;
    get_box(bs, DIM, P, 2, blk, b);
    const int64_t G0 = (int64_t)b.E[0] * Q, G1 = (int64_t)b.E[1] * Q;
    const int64_t P3 = (DIM == 3) ? (int64_t)b.R[2] * W : 1;
    const int R2 = b.R[1];
    const int64_t item = (blk - b.blk[2]) * kBlock + threadIdx.x;
    if (item >= P3 * R2 * G0) return;
    const int64_t g0 = item % G0;
    const int i2l = (int)((item / G0) % R2);
    const int64_t pair3 = item / (G0 * R2);
    // symmetric box: lines of the other sign of delta_2 are not needed; with delta_2 = 0 only one
    // sign of delta_1 (cut_lo: delta_1 >= 0, cut_hi: delta_1 <= 0)
    const int dz = (DIM == 3) ? (int)(pair3 % W) : P;
    if ((b.sym > 0 && dz < P) || (b.sym < 0 && dz > P)) return;
    const bool cut_lo = b.sym > 0 && dz == P, cut_hi = b.sym < 0 && dz == P;
    const int i2 = b.rlo[1] + i2l;
    const S* Xi = reinterpret_cast<const S*>(T.Xs[1]) + (int64_t)i2 * W * TT * 4;

    // input field f at local Gauss point g1 of direction 1
    const S* in;
    int64_t fstride;
    if (DIM == 3) {
        in = reinterpret_cast<const S*>(scratch + b.t1_off) + pair3 * G1 * G0 + g0;
        fstride = P3 * G1 * G0;
    } else {
        in = reinterpret_cast<const S*>(scratch + b.c_off) + g0;
        fstride = G1 * G0;
    }

    A acc[W][4];
#pragma unroll
    for (int dd = 0; dd < W; ++dd)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[dd][k] = Pol::zero();

#pragma unroll
    for (int a = 0; a <= P; ++a) {
        const int e2 = i2 - P + a;
        if (e2 < b.elo[1] || e2 >= b.elo[1] + b.E[1]) continue;
        if constexpr (Pol::kind == kArithF32) {
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            const int t = a * Q + r;
            const int64_t o = (int64_t)((e2 - b.elo[1]) * Q + r) * G0;
            S v[NIN];
#pragma unroll
            for (int f = 0; f < NIN; ++f) v[f] = in[f * fstride + o];
#pragma unroll
            for (int dd = a; dd <= a + P; ++dd) {
                if ((cut_lo && dd < P) || (cut_hi && dd > P)) continue;
                S x00, x01, x10, x11;
                load_pats(Xi + (dd * TT + t) * 4, x00, x01, x10, x11);
                if (DIM == 3) {
                    Pol::mac(acc[dd][0], x00, v[0]);   // A^00 -> group 0 (11 left in direction 0)
                    Pol::mac(acc[dd][1], x01, v[1]);   // A^01 -> group 1 (10)
                    Pol::mac(acc[dd][1], x00, v[3]);   // A^02 -> group 1
                    Pol::mac(acc[dd][2], x10, v[1]);   // A^10 -> group 2 (01)
                    Pol::mac(acc[dd][2], x00, v[4]);   // A^20 -> group 2
                    Pol::mac(acc[dd][3], x11, v[2]);   // A^11 -> group 3 (00)
                    Pol::mac(acc[dd][3], x10, v[5]);   // A^12 -> group 3
                    Pol::mac(acc[dd][3], x01, v[6]);   // A^21 -> group 3
                    Pol::mac(acc[dd][3], x00, v[7]);   // A^22 -> group 3
                } else {
                    Pol::mac(acc[dd][0], x00, v[0]);   // A^00: K00, 00
                    Pol::mac(acc[dd][1], x01, v[1]);   // A^01: K01, 01
                    Pol::mac(acc[dd][2], x10, v[1]);   // A^10: K01, 10
                    Pol::mac(acc[dd][3], x11, v[2]);   // A^11: K11, 11
                }
            }
        }
        } else {
            // the next Gauss point's inputs are loaded before this point's multiply-adds
            S nv[NIN];
            {
                const int64_t o = (int64_t)((e2 - b.elo[1]) * Q) * G0;
#pragma unroll
                for (int f = 0; f < NIN; ++f) nv[f] = in[f * fstride + o];
            }
#pragma unroll 1
        for (int r = 0; r < Q; ++r) {
            const int t = a * Q + r;
            S v[NIN];
#pragma unroll
            for (int f = 0; f < NIN; ++f) v[f] = nv[f];
            if (r + 1 < Q) {
                const int64_t o = (int64_t)((e2 - b.elo[1]) * Q + r + 1) * G0;
#pragma unroll
                for (int f = 0; f < NIN; ++f) nv[f] = in[f * fstride + o];
            }
#pragma unroll
            for (int dd = a; dd <= a + P; ++dd) {
                if ((cut_lo && dd < P) || (cut_hi && dd > P)) continue;
                S x00, x01, x10, x11;
                load_pats(Xi + (dd * TT + t) * 4, x00, x01, x10, x11);
                if (DIM == 3) {
                    Pol::mac(acc[dd][0], x00, v[0]);   // A^00 -> group 0 (11 left in direction 0)
                    Pol::mac(acc[dd][1], x01, v[1]);   // A^01 -> group 1 (10)
                    Pol::mac(acc[dd][1], x00, v[3]);   // A^02 -> group 1
                    Pol::mac(acc[dd][2], x10, v[1]);   // A^10 -> group 2 (01)
                    Pol::mac(acc[dd][2], x00, v[4]);   // A^20 -> group 2
                    Pol::mac(acc[dd][3], x11, v[2]);   // A^11 -> group 3 (00)
                    Pol::mac(acc[dd][3], x10, v[5]);   // A^12 -> group 3
                    Pol::mac(acc[dd][3], x01, v[6]);   // A^21 -> group 3
                    Pol::mac(acc[dd][3], x00, v[7]);   // A^22 -> group 3
                } else {
                    Pol::mac(acc[dd][0], x00, v[0]);   // A^00: K00, 00
                    Pol::mac(acc[dd][1], x01, v[1]);   // A^01: K01, 01
                    Pol::mac(acc[dd][2], x10, v[1]);   // A^10: K01, 10
                    Pol::mac(acc[dd][3], x11, v[2]);   // A^11: K11, 11
                }
            }
        }
        }
    }
    S* T2 = reinterpret_cast<S*>(scratch + b.t2_off);
    const int64_t P2 = (int64_t)R2 * W;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int dd = 0; dd < W; ++dd)
            if (!((cut_lo && dd < P) || (cut_hi && dd > P)))
                T2[(((int64_t)k * P3 + pair3) * P2 + (int64_t)i2l * W + dd) * G0 + g0] = Pol::to_store(acc[dd][k]);
    if constexpr (Pol::kind == kArithDF) {
        if (T.tc64 && b.out_kind == 0 && b.ex_off >= 0) {
            // largest exponent of each T2 line (pair3, i2l W + dd), the groups shifted by sigma_g, for the
            // exact-digit tensor-core stage X: max over this warp's lanes of the same line, one atomic each
            int* ex = reinterpret_cast<int*>(scratch + b.ex_off);
            const unsigned key = (unsigned)(item / G0);
            const unsigned peers = __match_any_sync(__activemask(), key);
            const bool leader = (__ffs(peers) - 1) == (int)(threadIdx.x & 31);
            int sh[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) sh[k] = T.gshift[k];
#pragma unroll
            for (int dd = 0; dd < W; ++dd) {
                int m = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = (int)((__float_as_uint(Pol::to_store(acc[dd][k]).x) >> 23) & 0xffu);
                    if (e > 0) m = max(m, e + sh[k] + kTcExpOffset);
                }
                m = (int)__reduce_max_sync(peers, (unsigned)m);
                if (leader && m > 0) atomicMax(ex + pair3 * P2 + (int64_t)i2l * W + dd, m);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// stage X: contract direction 0 and write the stencil rows.  A thread takes
// LINES consecutive (i1, delta_1) lines of one row i0, so every pair weight it
// loads serves LINES rows of output.
// ---------------------------------------------------------------------------
template <class Pol, int P, int DIM, int LINES>
__device__ __forceinline__ void stage_x_body(const Geo& g, const Tables& T, const BoxSet& bs, double* scratch,
                                             void* ell, int ell_f32, int64_t N, double* samples, int skip_card,
                                             int64_t blk)
{
    using S = typename Pol::store;
    using A = typename Pol::acc;
    constexpr int Q = P + 1, W = 2 * P + 1, TT = Q * Q;
    // Rows whose stencil stays among cardinal B-splines (2p <= i1 <= m0-2p-1)
    // all have the same pair weights (translation invariance, Sec. 2.2): they
    // read one copy from shared memory, so a warp's loads are broadcasts.
    // Loaded before any thread of the block can leave.
    __shared__ __align__(16) S sX[W * TT * 4];
    const bool has_card = g.m[0] >= 4 * P + 1;
    const S* X0 = reinterpret_cast<const S*>(T.Xs[0]);
    if (has_card)
        for (int k = threadIdx.x; k < W * TT * 4; k += blockDim.x) sX[k] = X0[(int64_t)(2 * P) * W * TT * 4 + k];
    __syncthreads();
    Box b;
    get_box(bs, DIM, P, 3, blk, b);
    const int64_t G0 = (int64_t)b.E[0] * Q;
    const int64_t P3 = (DIM == 3) ? (int64_t)b.R[2] * W : 1;
    const int64_t P2 = (int64_t)b.R[1] * W;
    const int64_t NL = (P2 + LINES - 1) / LINES;       // line groups
    const int m0 = g.m[0];
    // With the tensor-core stage X the cardinal rows of the explicit boxes are written there: the
    // threads then run over the box's other rows only, nlo below the cardinal range and the rest
    // above it, so that whole warps carry work (the grid keeps its size; the tail exits).
    int R1 = b.R[0], nlo = R1, hi0 = 0;
    if (skip_card && has_card && b.out_kind == 0) {
        const int lo = b.rlo[0], end = b.rlo[0] + b.R[0];
        nlo = max(0, min(end, 2 * P) - lo);
        hi0 = max(lo, m0 - 2 * P);
        R1 = nlo + max(0, end - hi0);
        if (R1 == 0) return;
    }
    const int64_t item = (blk - b.blk[3]) * kBlock + threadIdx.x;
    if (item >= P3 * NL * R1) return;
    const int i1l = (int)(item % R1);
    const int64_t lg = (item / R1) % NL;
    const int64_t pair3 = item / (R1 * NL);
    const int i1 = (i1l < nlo) ? b.rlo[0] + i1l : hi0 + (i1l - nlo);
    const int i3 = (DIM == 3) ? b.rlo[2] + (int)(pair3 / W) : 0;
    const int d3 = (DIM == 3) ? (int)(pair3 % W) : 0;
    // symmetric box: only the upper (sym = +1) or lower (-1) offsets
    const int dz = (DIM == 3) ? d3 : P;
    if ((b.sym > 0 && dz < P) || (b.sym < 0 && dz > P)) return;
    const bool card = has_card && i1 >= 2 * P && i1 <= m0 - 2 * P - 1;
    const S* Xi = card ? sX : X0 + (int64_t)i1 * W * TT * 4;
    const int64_t gs = P3 * P2 * G0;        // group stride
    int nl = (int)(P2 - lg * LINES);
    if (nl > LINES) nl = LINES;
    if (b.sym != 0 && dz == P) {
        // lines of the other sign of delta_1 are mirrored: nothing to do when all of this thread's are
        bool any = false;
        for (int l = 0; l < nl; ++l) {
            const int d = (int)((lg * LINES + l) % W);
            any = any || (b.sym > 0 ? d >= P : d <= P);
        }
        if (!any) return;
    }
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
        if constexpr (Pol::kind == kArithF32) {
            __align__(16) S v[LINES][4][Q];
#pragma unroll
            for (int l = 0; l < LINES; ++l)
#pragma unroll
                for (int gr = 0; gr < 4; ++gr) load_run<S, Q>(T2[l] + gr * gs + o, v[l][gr]);
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                const int t = a * Q + r;
#pragma unroll
                for (int dd = a; dd <= a + P; ++dd) {
                    S x00, x01, x10, x11;
                    load_pats(Xi + (dd * TT + t) * 4, x00, x01, x10, x11);
#pragma unroll
                    for (int l = 0; l < LINES; ++l) {
                        Pol::mac(acc[l][dd], x11, v[l][0][r]);   // group 0: pattern 11
                        Pol::mac(acc[l][dd], x10, v[l][1][r]);   // group 1: pattern 10
                        Pol::mac(acc[l][dd], x01, v[l][2][r]);   // group 2: pattern 01
                        Pol::mac(acc[l][dd], x00, v[l][3][r]);   // group 3: pattern 00
                    }
                }
            }
        } else {
            // double-float and FP64 bodies are ~12x longer per multiply-add: with the Gauss-point
            // loop unrolled too the kernel outgrew the instruction cache (ncu: "no instruction" the
            // largest stall), so it stays rolled and the T2 values are loaded per point
#pragma unroll 1
            for (int r = 0; r < Q; ++r) {
                const int t = a * Q + r;
                S v[LINES][4];
#pragma unroll
                for (int l = 0; l < LINES; ++l)
#pragma unroll
                    for (int gr = 0; gr < 4; ++gr) v[l][gr] = T2[l][gr * gs + o + r];
#pragma unroll
                for (int dd = a; dd <= a + P; ++dd) {
                    S x00, x01, x10, x11;
                    load_pats(Xi + (dd * TT + t) * 4, x00, x01, x10, x11);
#pragma unroll
                    for (int l = 0; l < LINES; ++l) {
                        Pol::mac(acc[l][dd], x11, v[l][0]);   // group 0: pattern 11
                        Pol::mac(acc[l][dd], x10, v[l][1]);   // group 1: pattern 10
                        Pol::mac(acc[l][dd], x01, v[l][2]);   // group 2: pattern 01
                        Pol::mac(acc[l][dd], x00, v[l][3]);   // group 3: pattern 00
                    }
                }
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
        if (b.sym != 0 && dz == P && (b.sym > 0 ? d2 < P : d2 > P)) continue;   // mirrored line
        // the centre line: one sign of delta_0
        const int dlo = (b.sym > 0 && dz == P && d2 == P) ? P : 0;
        const int dhi = (b.sym < 0 && dz == P && d2 == P) ? P : W - 1;
        if (b.out_kind == 0) {
            const int64_t row = i1 + (int64_t)m0 * (i2 + (int64_t)g.m[1] * i3);
            if (ell_f32) {
                float* out = (float*)ell;
#pragma unroll
                for (int dd = 0; dd < W; ++dd) if (dd >= dlo && dd <= dhi) out[(int64_t)(slot0 + dd) * N + row] = (float)Pol::to_double(acc[l][dd]);
            } else {
                double* out = (double*)ell;
#pragma unroll
                for (int dd = 0; dd < W; ++dd) if (dd >= dlo && dd <= dhi) out[(int64_t)(slot0 + dd) * N + row] = Pol::to_double(acc[l][dd]);
            }
        } else {
#pragma unroll
            for (int dd = 0; dd < W; ++dd)
                samples[(int64_t)(slot0 + dd) * bs.n_samples + b.sample_id] = Pol::to_double(acc[l][dd]);
        }
    }
}

}  // namespace iga
