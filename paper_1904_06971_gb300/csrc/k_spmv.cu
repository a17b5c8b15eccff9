// K6: stencil SpMV y = A x on the index-free stencil-ELL layout
// (eq. DiscreteVariationalProblems).  One thread per row; the value of slot s
// of row i is vals[s * N + i] (coalesced across consecutive rows) and its
// column is i + delta_0 + m_0 (delta_1 + m_1 delta_2).  Rows whose whole
// stencil stays inside the index range skip the bounds tests.
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

template <int P, int DIM, typename T>
__global__ void __launch_bounds__(kBlock) k_spmv(int m0, int m1, int m2, const T* __restrict__ vals,
                                                 const T* __restrict__ x, T* __restrict__ y)
{
    constexpr int W = 2 * P + 1;
    const int64_t N = (int64_t)m0 * m1 * m2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int i0 = (int)(i % m0), i1 = (int)((i / m0) % m1), i2 = (int)(i / ((int64_t)m0 * m1));
    const bool inner = i0 >= P && i0 < m0 - P && i1 >= P && i1 < m1 - P &&
                       (DIM == 2 || (i2 >= P && i2 < m2 - P));
    const int64_t s1 = m0, s2 = (int64_t)m0 * m1;
    T acc = 0;
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
            const T* v = vals + (int64_t)sbase * N + i;
#pragma unroll
            for (int d0 = 0; d0 < W; ++d0) {
                const int o0 = d0 - P;
                if (inner || (i0 + o0 >= 0 && i0 + o0 < m0))
                    acc = fma(v[(int64_t)d0 * N], __ldg(x + jbase + o0), acc);
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

template <int P, int DIM>
__global__ void __launch_bounds__(kBlock) k_spmv_df(int m0, int m1, int m2, const double* __restrict__ vals,
                                                    const double* __restrict__ x, const float2* __restrict__ xs,
                                                    double* __restrict__ y)
{
    constexpr int W = 2 * P + 1;
    constexpr int F64 = W - W / 4;              // slots delta_0 + p < F64 use FP64 FMAs, the rest double-float
    const int64_t N = (int64_t)m0 * m1 * m2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int i0 = (int)(i % m0), i1 = (int)((i / m0) % m1), i2 = (int)(i / ((int64_t)m0 * m1));
    const bool inner = i0 >= P && i0 < m0 - P && i1 >= P && i1 < m1 - P &&
                       (DIM == 2 || (i2 >= P && i2 < m2 - P));
    const int64_t s1 = m0, s2 = (int64_t)m0 * m1;
    float ah = 0.f, al = 0.f;
    double a64 = 0.0;
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
            const double* v = vals + (int64_t)sbase * N + i;
#pragma unroll
            for (int d0 = 0; d0 < W; ++d0) {
                const int o0 = d0 - P;
                if (d0 < F64) {
                    if (inner || (i0 + o0 >= 0 && i0 + o0 < m0)) a64 = fma(v[(int64_t)d0 * N], __ldg(x + jbase + o0), a64);
                } else if (inner || (i0 + o0 >= 0 && i0 + o0 < m0)) {
                    const float2 a = d2df_split(v[(int64_t)d0 * N]);
                    const float2 b = xs[jbase + o0];
                    // a * b: exact product of the high parts, cross terms into the low part
                    const float ph = __fmul_rn(a.x, b.x);
                    float pe = __fmaf_rn(a.x, b.x, -ph);
                    pe = __fmaf_rn(a.x, b.y, pe);
                    pe = __fmaf_rn(a.y, b.x, pe);
                    spmv_add2(ah, al, ph, pe);
                }
            }
        }
    }
    y[i] = df2d_exact(ah, al) + a64;
}

template <int P>
static void spmv_p(int dim, const int m[3], const void* vals, int f32, const void* x, void* y,
                   unsigned grid, cudaStream_t s)
{
    const int m2 = (dim == 3) ? m[2] : 1;
    if (dim == 3) {
        if (f32) k_spmv<P, 3, float><<<grid, kBlock, 0, s>>>(m[0], m[1], m2, (const float*)vals, (const float*)x, (float*)y);
        else k_spmv<P, 3, double><<<grid, kBlock, 0, s>>>(m[0], m[1], m2, (const double*)vals, (const double*)x, (double*)y);
    } else {
        if (f32) k_spmv<P, 2, float><<<grid, kBlock, 0, s>>>(m[0], m[1], m2, (const float*)vals, (const float*)x, (float*)y);
        else k_spmv<P, 2, double><<<grid, kBlock, 0, s>>>(m[0], m[1], m2, (const double*)vals, (const double*)x, (double*)y);
    }
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
        switch (p) {
        case 1: spmv_p<1>(dim, m, values, f32, x, y, grid, s); break;
        case 2: spmv_p<2>(dim, m, values, f32, x, y, grid, s); break;
        case 3: spmv_p<3>(dim, m, values, f32, x, y, grid, s); break;
        case 4: spmv_p<4>(dim, m, values, f32, x, y, grid, s); break;
        case 5: spmv_p<5>(dim, m, values, f32, x, y, grid, s); break;
        default: break;
        }
    }
    launch_end(K_SPMV, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace iga
