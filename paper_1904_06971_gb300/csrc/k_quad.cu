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

}  // namespace iga
