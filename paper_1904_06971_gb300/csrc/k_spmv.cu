// K6: stencil SpMV y = A x on the index-free stencil-ELL layout
// (eq. DiscreteVariationalProblems).  One thread per row; the value of slot s
// of row i is vals[s * N + i] (coalesced across consecutive rows) and its
// column is i + delta_0 + m_0 (delta_1 + m_1 delta_2).
//
// FP64 values: GB300 runs FP64 FMAs at 1/64 of the FP32 rate, just below what
// the HBM stream of the values needs, so a quarter of the products (the last
// (2p+1)/4 offsets delta_0 of every run) are formed in double-float arithmetic
// on the FP32 pipe -- x split once into (hi, lo) float pairs, each stored value
// split by integer operations as it streams in, a renormalised double-float
// row sum -- and the rest with FP64 FMAs, so that neither pipe limits the
// stream (more double-float work delays the loads behind it); the two partial
// sums are added once per row.
#include "arith.cuh"
#include "iga_internal.cuh"

namespace iga {

// FP32 values: 1024-thread blocks, the values streamed past L1 (each is read
// once) so that L1 keeps the x neighbourhood the rows of a block share.
constexpr int kSpmvF32Block = 1024;

template <int P, int DIM>
__global__ void __launch_bounds__(kSpmvF32Block) k_spmv_f32(int m0, int m1, int m2, const float* __restrict__ vals,
                                                            const float* __restrict__ x, float* __restrict__ y)
{
    constexpr int W = 2 * P + 1;
    const int64_t N = (int64_t)m0 * m1 * m2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int i0 = (int)(i % m0), i1 = (int)((i / m0) % m1), i2 = (int)(i / ((int64_t)m0 * m1));
    const bool inner = i0 >= P && i0 < m0 - P && i1 >= P && i1 < m1 - P &&
                       (DIM == 2 || (i2 >= P && i2 < m2 - P));
    const int64_t s1 = m0, s2 = (int64_t)m0 * m1;
    float acc = 0.f;
    const int n2 = (DIM == 3) ? W : 1;
    for (int d2 = 0; d2 < n2; ++d2) {
        const int o2 = (DIM == 3) ? d2 - P : 0;
        const bool ok2 = inner || (i2 + o2 >= 0 && i2 + o2 < m2);
        for (int d1 = 0; d1 < W; ++d1) {
            const int o1 = d1 - P;
            const bool ok1 = ok2 && (inner || (i1 + o1 >= 0 && i1 + o1 < m1));
            if (!ok1) continue;
            const int sbase = W * (d1 + W * d2);
            const int64_t jbase = i + o1 * s1 + o2 * s2;
            const float* v = vals + (int64_t)sbase * N + i;
#pragma unroll
            for (int d0 = 0; d0 < W; ++d0) {
                const int o0 = d0 - P;
                if (inner || (i0 + o0 >= 0 && i0 + o0 < m0))
                    acc = fmaf(__ldcs(v + (int64_t)d0 * N), __ldg(x + jbase + o0), acc);
            }
        }
    }
    y[i] = acc;
}

__global__ void __launch_bounds__(kBlock) k_split_x(int64_t n, const double* __restrict__ x, float2* __restrict__ xs)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xs[i] = d2df_split(x[i]);
}

// renormalised double-float accumulation a += b
__device__ __forceinline__ void spmv_add2(float& ah, float& al, float bh, float bl)
{
    const float s = __fadd_rn(ah, bh);
    const float z = __fsub_rn(s, ah);
    float t = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, z)), __fsub_rn(bh, z));
    t = __fadd_rn(t, __fadd_rn(al, bl));
    ah = __fadd_rn(s, t);
    al = __fsub_rn(t, __fsub_rn(ah, s));
}

// (ah, al) += v * b in double-float: v split into (hi, lo) floats by integer
// operations, the product of the high parts exact, the cross terms into the
// low part, then a renormalised sum.
__device__ __forceinline__ void spmv_dfmac(float& ah, float& al, double v, float2 b)
{
    const float2 a = d2df_split(v);
    const float ph = __fmul_rn(a.x, b.x);
    float pe = __fmaf_rn(a.x, b.x, -ph);
    pe = __fmaf_rn(a.x, b.y, pe);
    pe = __fmaf_rn(a.y, b.x, pe);
    spmv_add2(ah, al, ph, pe);
}

// One row of the FP64-value product.  The pointers are deliberately not
// __restrict__ here and the double-float product is a separate function of the
// loaded value: in this form the compiler keeps the loads in program order and
// allocates 44 registers at p = 4 (the other forms tried got 32 or 60), which
// streams 10-20 % faster on GB300 at 96^3 (measured).
template <int P, int DIM>
__device__ __forceinline__ double spmv_df_row(int64_t i, int i0, int i1, int i2, int m0, int m1, int m2, int64_t N,
                                              const double* vals, const double* x, const float2* xs)
{
    constexpr int W = 2 * P + 1;
    constexpr int F64 = W - W / 4;              // slots delta_0 + p < F64 use FP64 FMAs, the rest double-float
    const int64_t s1 = m0, s2 = (int64_t)m0 * m1;
    float ah = 0.f, al = 0.f;
    double a64 = 0.0;
    for (int d2 = 0; d2 < (DIM == 3 ? W : 1); ++d2) {
        const int o2 = (DIM == 3) ? d2 - P : 0;
        if (i2 + o2 < 0 || i2 + o2 >= m2) continue;
        for (int d1 = 0; d1 < W; ++d1) {
            const int o1 = d1 - P;
            if (i1 + o1 < 0 || i1 + o1 >= m1) continue;
            const int64_t jb = i + o1 * s1 + o2 * s2;
            const double* v = vals + (int64_t)(W * (d1 + W * d2)) * N + i;
#pragma unroll
            for (int d0 = 0; d0 < W; ++d0) {
                const int o0 = d0 - P;
                if (i0 + o0 < 0 || i0 + o0 >= m0) continue;
                if (d0 < F64) a64 = fma(v[(int64_t)d0 * N], x[jb + o0], a64);
                else spmv_dfmac(ah, al, v[(int64_t)d0 * N], xs[jb + o0]);
            }
        }
    }
    return df2d_exact(ah, al) + a64;
}

template <int P, int DIM>
__global__ void __launch_bounds__(kBlock) k_spmv_df(int m0, int m1, int m2, const double* __restrict__ vals,
                                                    const double* __restrict__ x, const float2* __restrict__ xs,
                                                    double* __restrict__ y)
{
    const int64_t N = (int64_t)m0 * m1 * m2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int i0 = (int)(i % m0), i1 = (int)((i / m0) % m1), i2 = (int)(i / ((int64_t)m0 * m1));
    y[i] = spmv_df_row<P, DIM>(i, i0, i1, i2, m0, m1, m2, N, vals, x, xs);
}

template <int P>
static void spmv_f32_p(int dim, const int m[3], const float* vals, const float* x, float* y, cudaStream_t s)
{
    const int64_t N = (int64_t)m[0] * m[1] * (dim == 3 ? m[2] : 1);
    const unsigned grid = (unsigned)((N + kSpmvF32Block - 1) / kSpmvF32Block);
    if (dim == 3) k_spmv_f32<P, 3><<<grid, kSpmvF32Block, 0, s>>>(m[0], m[1], m[2], vals, x, y);
    else k_spmv_f32<P, 2><<<grid, kSpmvF32Block, 0, s>>>(m[0], m[1], 1, vals, x, y);
}

cudaError_t pool_alloc(size_t bytes, cudaStream_t s, void** out);

template <int P>
static cudaError_t spmv_df_p(int dim, const int m[3], const double* vals, const double* x, double* y,
                             unsigned grid, cudaStream_t s)
{
    const int64_t N = (int64_t)m[0] * m[1] * (dim == 3 ? m[2] : 1);
    float2* xs = nullptr;
    cudaError_t e = pool_alloc((size_t)N * sizeof(float2), s, (void**)&xs);
    if (e != cudaSuccess) return e;
    k_split_x<<<grid, kBlock, 0, s>>>(N, x, xs);
    if (dim == 3) k_spmv_df<P, 3><<<grid, kBlock, 0, s>>>(m[0], m[1], m[2], vals, x, xs, y);
    else k_spmv_df<P, 2><<<grid, kBlock, 0, s>>>(m[0], m[1], 1, vals, x, xs, y);
    e = cudaGetLastError();
    cudaError_t fe = cudaFreeAsync(xs, s);
    return e != cudaSuccess ? e : fe;
}

cudaError_t launch_spmv(int dim, int p, const int m[3], const void* values, int f32,
                        const void* x, void* y, cudaStream_t s)
{
    const int64_t N = (int64_t)m[0] * m[1] * (dim == 3 ? m[2] : 1);
    const unsigned grid = (unsigned)((N + kBlock - 1) / kBlock);
    launch_begin(K_SPMV, s);
    cudaError_t e = cudaSuccess;
    if (!f32) {
        const double* v = (const double*)values;
        const double* xd = (const double*)x;
        double* yd = (double*)y;
        switch (p) {
        case 1: e = spmv_df_p<1>(dim, m, v, xd, yd, grid, s); break;
        case 2: e = spmv_df_p<2>(dim, m, v, xd, yd, grid, s); break;
        case 3: e = spmv_df_p<3>(dim, m, v, xd, yd, grid, s); break;
        case 4: e = spmv_df_p<4>(dim, m, v, xd, yd, grid, s); break;
        case 5: e = spmv_df_p<5>(dim, m, v, xd, yd, grid, s); break;
        default: break;
        }
    } else {
        const float* v = (const float*)values;
        const float* xf = (const float*)x;
        float* yf = (float*)y;
        switch (p) {
        case 1: spmv_f32_p<1>(dim, m, v, xf, yf, s); break;
        case 2: spmv_f32_p<2>(dim, m, v, xf, yf, s); break;
        case 3: spmv_f32_p<3>(dim, m, v, xf, yf, s); break;
        case 4: spmv_f32_p<4>(dim, m, v, xf, yf, s); break;
        case 5: spmv_f32_p<5>(dim, m, v, xf, yf, s); break;
        default: break;
        }
    }
    launch_end(K_SPMV, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace iga
