// K3 kernels: the sum-factorised quadrature stages (bodies in quad_bodies.cuh)
// as one launch per stage, and their launch sequence.
#include "quad_bodies.cuh"

namespace iga {

// FP32 contractions get their own entry points: the Gauss-point loop unrolled
// (short bodies, several points' loads in flight) and three resident blocks per
// SM; the double-float and FP64 bodies are long and keep the rolled loop and the
// compiler's register choice.
template <class Pol, int P, int HALF>
__global__ void __launch_bounds__(kBlock) k_stage_z(Geo g, Tables T, BoxSet bs, double* scratch)
{
    stage_z_body<Pol, P, HALF>(g, T, bs, scratch, blockIdx.x);
}
template <int P, int HALF>
__global__ void __launch_bounds__(kBlock, 3) k_stage_z_f32(Geo g, Tables T, BoxSet bs, double* scratch)
{
    stage_z_body<PolF32, P, HALF>(g, T, bs, scratch, blockIdx.x);
}

template <class Pol, int P, int DIM>
__global__ void __launch_bounds__(kBlock, DIM == 3 ? 2 : 1) k_stage_y(Geo g, Tables T, BoxSet bs, double* scratch)
{
    stage_y_body<Pol, P, DIM>(g, T, bs, scratch, blockIdx.x);
}
template <int P, int DIM>
__global__ void __launch_bounds__(kBlock, 3) k_stage_y_f32(Geo g, Tables T, BoxSet bs, double* scratch)
{
    stage_y_body<PolF32, P, DIM>(g, T, bs, scratch, blockIdx.x);
}

template <class Pol, int P, int DIM, int LINES>
__global__ void __launch_bounds__(kBlock) k_stage_x(Geo g, Tables T, BoxSet bs, double* scratch,
                                                    void* ell, int ell_f32, int64_t N, double* samples, int skip_card)
{
    stage_x_body<Pol, P, DIM, LINES>(g, T, bs, scratch, ell, ell_f32, N, samples, skip_card, blockIdx.x);
}

// ---------------------------------------------------------------------------
template <class Pol, int P>
static cudaError_t stages_p(const Geo& g, const Tables& T, const BoxSet& bs, const int64_t nb[4],
                            double* scratch, void* ell, int ell_f32, double* samples, cudaStream_t s)
{
    const int64_t N = (int64_t)g.m[0] * g.m[1] * (g.dim == 3 ? g.m[2] : 1);
    if (g.dim == 3) {
        if (nb[1] > 0) {
            launch_begin(K_STAGE_Z, s);
            if constexpr (Pol::kind == kArithF32) k_stage_z_f32<P, 0><<<(unsigned)nb[1], kBlock, 0, s>>>(g, T, bs, scratch);
            else k_stage_z<Pol, P, 0><<<(unsigned)nb[1], kBlock, 0, s>>>(g, T, bs, scratch);
            launch_end(K_STAGE_Z, s);
            launch_begin(K_STAGE_Z, s);
            if constexpr (Pol::kind == kArithF32) k_stage_z_f32<P, 1><<<(unsigned)nb[1], kBlock, 0, s>>>(g, T, bs, scratch);
            else k_stage_z<Pol, P, 1><<<(unsigned)nb[1], kBlock, 0, s>>>(g, T, bs, scratch);
            launch_end(K_STAGE_Z, s);
        }
        if (nb[2] > 0) {
            launch_begin(K_STAGE_Y, s);
            if constexpr (Pol::kind == kArithF32) k_stage_y_f32<P, 3><<<(unsigned)nb[2], kBlock, 0, s>>>(g, T, bs, scratch);
            else k_stage_y<Pol, P, 3><<<(unsigned)nb[2], kBlock, 0, s>>>(g, T, bs, scratch);
            launch_end(K_STAGE_Y, s);
        }
        if (nb[3] > 0) {
            int skip = 0;
            if constexpr (Pol::kind == kArithF32 || Pol::kind == kArithDF) {
                const bool want = (Pol::kind == kArithF32) ? (T.tc && ell_f32) : (T.tc64 && !ell_f32);
                if (want && P >= 2) {
                    bool used = false;
                    cudaError_t e = launch_stage_x_tc(g, T, bs, scratch, ell, Pol::kind == kArithDF, N, s, &used);
                    if (e != cudaSuccess) return e;
                    skip = used ? 1 : 0;
                }
            }
            launch_begin(K_STAGE_X, s);
            k_stage_x<Pol, P, 3, kLinesX><<<(unsigned)nb[3], kBlock, 0, s>>>(g, T, bs, scratch, ell, ell_f32, N, samples, skip);
            launch_end(K_STAGE_X, s);
        }
    } else {
        if (nb[2] > 0) {
            launch_begin(K_STAGE_Y, s);
            if constexpr (Pol::kind == kArithF32) k_stage_y_f32<P, 2><<<(unsigned)nb[2], kBlock, 0, s>>>(g, T, bs, scratch);
            else k_stage_y<Pol, P, 2><<<(unsigned)nb[2], kBlock, 0, s>>>(g, T, bs, scratch);
            launch_end(K_STAGE_Y, s);
        }
        if (nb[3] > 0) {
            int skip = 0;
            if constexpr (Pol::kind == kArithF32 || Pol::kind == kArithDF) {
                const bool want = (Pol::kind == kArithF32) ? (T.tc && ell_f32) : (T.tc64 && !ell_f32);
                if (want && P >= 2) {
                    bool used = false;
                    cudaError_t e = launch_stage_x_tc(g, T, bs, scratch, ell, Pol::kind == kArithDF, N, s, &used);
                    if (e != cudaSuccess) return e;
                    skip = used ? 1 : 0;
                }
            }
            launch_begin(K_STAGE_X, s);
            k_stage_x<Pol, P, 2, kLinesX><<<(unsigned)nb[3], kBlock, 0, s>>>(g, T, bs, scratch, ell, ell_f32, N, samples, skip);
            launch_end(K_STAGE_X, s);
        }
    }
    return cudaGetLastError();
}

template <class Pol>
static cudaError_t stages_pol(const Geo& g, const Tables& T, const BoxSet& bs, const int64_t nb[4],
                              double* scratch, void* ell, int ell_f32, double* samples, cudaStream_t s)
{
    switch (g.p) {
    case 1: return stages_p<Pol, 1>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    case 2: return stages_p<Pol, 2>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    case 3: return stages_p<Pol, 3>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    case 4: return stages_p<Pol, 4>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    case 5: return stages_p<Pol, 5>(g, T, bs, nb, scratch, ell, ell_f32, samples, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stages(const Geo& g, const Tables& T, const BoxSet& bs, const int64_t nblocks[4],
                          double* scratch, void* ell, int ell_f32, double* samples, cudaStream_t s)
{
    switch (T.arith) {
    case kArithF64: return stages_pol<PolF64>(g, T, bs, nblocks, scratch, ell, ell_f32, samples, s);
    case kArithDF: return stages_pol<PolDF>(g, T, bs, nblocks, scratch, ell, ell_f32, samples, s);
    case kArithF32: return stages_pol<PolF32>(g, T, bs, nblocks, scratch, ell, ell_f32, samples, s);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Mirror of a symmetric matrix (A_ij = A_ji) over a range of rows whose stages
// computed one half of the offsets: dir = +1 fills slot s below the centre of
// row i from the mirrored slot S-1-s of row j = i + delta_s, dir = -1 the slots
// above the centre the same way; 0 when j lies outside the index range.  One
// thread per (row, slot); consecutive threads take consecutive rows.
// ---------------------------------------------------------------------------
template <int P, int DIM, typename T>
__global__ void __launch_bounds__(kBlock) k_mirror(int m0, int m1, int m2, int64_t row_begin, int64_t count, int dir,
                                                   T* __restrict__ vals)
{
    constexpr int W = 2 * P + 1;
    constexpr int S = (DIM == 3) ? W * W * W : W * W;
    constexpr int C = (S - 1) / 2;
    const int64_t N = (int64_t)m0 * m1 * m2;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    const int64_t i = row_begin + r;
    const int s = dir > 0 ? (int)blockIdx.y : C + 1 + (int)blockIdx.y;     // the slot written
    const int o0 = s % W - P, o1 = (s / W) % W - P, o2 = (DIM == 3) ? s / (W * W) - P : 0;
    const int i0 = (int)(i % m0), i1 = (int)((i / m0) % m1), i2 = (int)(i / ((int64_t)m0 * m1));
    const bool in = i0 + o0 >= 0 && i0 + o0 < m0 && i1 + o1 >= 0 && i1 + o1 < m1 && i2 + o2 >= 0 && i2 + o2 < m2;
    const int64_t j = i + o0 + (int64_t)m0 * (o1 + (int64_t)m1 * o2);
    vals[(int64_t)s * N + i] = in ? vals[(int64_t)(S - 1 - s) * N + j] : (T)0;
}

template <int P>
static void mirror_p(int dim, const int m[3], void* values, int f32, int64_t row_begin, int64_t count, int dir,
                     cudaStream_t s)
{
    const int W = 2 * P + 1;
    const int S = (dim == 3) ? W * W * W : W * W;
    const dim3 grid((unsigned)((count + kBlock - 1) / kBlock), (unsigned)((S - 1) / 2));
    const int m2 = (dim == 3) ? m[2] : 1;
    if (dim == 3) {
        if (f32) k_mirror<P, 3, float><<<grid, kBlock, 0, s>>>(m[0], m[1], m2, row_begin, count, dir, (float*)values);
        else k_mirror<P, 3, double><<<grid, kBlock, 0, s>>>(m[0], m[1], m2, row_begin, count, dir, (double*)values);
    } else {
        if (f32) k_mirror<P, 2, float><<<grid, kBlock, 0, s>>>(m[0], m[1], m2, row_begin, count, dir, (float*)values);
        else k_mirror<P, 2, double><<<grid, kBlock, 0, s>>>(m[0], m[1], m2, row_begin, count, dir, (double*)values);
    }
}

cudaError_t launch_mirror(int dim, int p, const int m[3], void* values, int f32, int64_t row_begin,
                          int64_t count, int dir, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    launch_begin(K_MIRROR, s);
    switch (p) {
    case 1: mirror_p<1>(dim, m, values, f32, row_begin, count, dir, s); break;
    case 2: mirror_p<2>(dim, m, values, f32, row_begin, count, dir, s); break;
    case 3: mirror_p<3>(dim, m, values, f32, row_begin, count, dir, s); break;
    case 4: mirror_p<4>(dim, m, values, f32, row_begin, count, dir, s); break;
    case 5: mirror_p<5>(dim, m, values, f32, row_begin, count, dir, s); break;
    default: break;
    }
    launch_end(K_MIRROR, s);
    return cudaGetLastError();
}
}  // namespace iga
