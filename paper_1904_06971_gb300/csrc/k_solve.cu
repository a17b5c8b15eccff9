// Conjugate gradients on the Dirichlet-reduced system A_II u_I = f_I (Sec. 6,
// Remark with eq. BlockSystem: homogeneous Dirichlet dofs -- basis functions
// with an index 0 or m-1 in some direction -- are eliminated).  Vectors keep
// all N entries; Dirichlet entries are held at zero and the masked SpMV zeroes
// the Dirichlet rows, so the iteration acts on the interior block only.
//
// Matrices with FP32 values are solved by iterative refinement: the residual
// r = f - A u is computed in FP64 (FP32 values promoted, FP64 u), an FP32 CG
// solves A d = r to a loose tolerance, and u += d in FP64.
//
// Reductions are two-level with a fixed block count and order, so results are
// deterministic run to run.
#include <cmath>
#include <cstring>

#include "iga_internal.cuh"

namespace iga {

constexpr int kRedBlocks = 304;            // 2 x 152 SMs

__device__ __forceinline__ bool dirichlet(int64_t i, int m0, int m1, int m2, int dim)
{
    const int i0 = (int)(i % m0), i1 = (int)((i / m0) % m1);
    if (i0 == 0 || i0 == m0 - 1 || i1 == 0 || i1 == m1 - 1) return true;
    if (dim == 3) {
        const int i2 = (int)(i / ((int64_t)m0 * m1));
        if (i2 == 0 || i2 == m2 - 1) return true;
    }
    return false;
}

// y = A x on interior rows, 0 on Dirichlet rows.  TV: value type, TX: vector
// type, TA: accumulator type.  x is zero on Dirichlet dofs.
template <int P, int DIM, typename TV, typename TX, typename TA>
__global__ void __launch_bounds__(kBlock) k_spmv_masked(int m0, int m1, int m2, const TV* __restrict__ vals,
                                                        const TX* __restrict__ x, TX* __restrict__ y)
{
    constexpr int W = 2 * P + 1;
    const int64_t N = (int64_t)m0 * m1 * m2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (dirichlet(i, m0, m1, m2, DIM)) { y[i] = (TX)0; return; }
    const int i0 = (int)(i % m0), i1 = (int)((i / m0) % m1), i2 = (int)(i / ((int64_t)m0 * m1));
    const bool inner = i0 >= P && i0 < m0 - P && i1 >= P && i1 < m1 - P && (DIM == 2 || (i2 >= P && i2 < m2 - P));
    const int64_t s1 = m0, s2 = (int64_t)m0 * m1;
    TA acc = 0;
    const int n2 = (DIM == 3) ? W : 1;
    for (int d2 = 0; d2 < n2; ++d2) {
        const int o2 = (DIM == 3) ? d2 - P : 0;
        if (!(inner || (i2 + o2 >= 0 && i2 + o2 < m2))) continue;
        for (int d1 = 0; d1 < W; ++d1) {
            const int o1 = d1 - P;
            if (!(inner || (i1 + o1 >= 0 && i1 + o1 < m1))) continue;
            const TV* v = vals + (int64_t)(W * (d1 + W * d2)) * N + i;
            const int64_t jb = i + o1 * s1 + o2 * s2;
#pragma unroll
            for (int d0 = 0; d0 < W; ++d0) {
                const int o0 = d0 - P;
                if (inner || (i0 + o0 >= 0 && i0 + o0 < m0))
                    acc += (TA)v[(int64_t)d0 * N] * (TA)__ldg(x + jb + o0);
            }
        }
    }
    y[i] = (TX)acc;
}

// partial[b] = sum over the block's grid-stride share of a[i] * b[i] (FP64)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_dot_partial(int64_t n, const T* a, const T* b, double* partial)
{
    __shared__ double sh[kBlock];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)b[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(int nb, const double* partial, double* out)
{
    __shared__ double sh[kBlock];
    double s = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s += partial[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// x += alpha p ; r -= alpha q   (alpha = num / den read on the device)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_update(int64_t n, const double* num, const double* den, T* x,
                                                      const T* p, T* r, const T* q)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = *num / *den;
    x[i] = (T)((double)x[i] + alpha * (double)p[i]);
    r[i] = (T)((double)r[i] - alpha * (double)q[i]);
}

// p = r + beta p   (beta = num / den on the device)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_dir(int64_t n, const double* num, const double* den, const T* r, T* p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double beta = *num / *den;
    p[i] = (T)((double)r[i] + beta * (double)p[i]);
}

// dst = src on interior dofs, 0 on Dirichlet dofs (with type conversion and a scale)
template <typename TS, typename TD>
__global__ void __launch_bounds__(kBlock) k_mask_copy(int64_t n, int m0, int m1, int m2, int dim, const TS* src,
                                                      double scale, TD* dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[i] = dirichlet(i, m0, m1, m2, dim) ? (TD)0 : (TD)((double)src[i] * scale);
}

// u += scale * d
__global__ void __launch_bounds__(kBlock) k_add_scaled(int64_t n, const float* d, double scale, double* u)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u[i] += scale * (double)d[i];
}

// r = f - y on interior dofs, 0 elsewhere
template <typename T>
__global__ void __launch_bounds__(kBlock) k_residual(int64_t n, int m0, int m1, int m2, int dim, const T* f,
                                                     const T* y, T* r)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r[i] = dirichlet(i, m0, m1, m2, dim) ? (T)0 : (T)(f[i] - y[i]);
}

// ---------------------------------------------------------------------------
struct SolveCtx {
    int dim, p, m[3];
    int64_t N;
    const void* vals;
    int f32;
    cudaStream_t s;
    double* partial;     // [kRedBlocks]
    double* scal;        // [6] device scalars
    unsigned grid;
};

template <int P, int DIM, typename TV, typename TX, typename TA>
static void spmv_m(const SolveCtx& c, const TX* x, TX* y)
{
    launch_begin(K_SOLVE, c.s);
    k_spmv_masked<P, DIM, TV, TX, TA><<<c.grid, kBlock, 0, c.s>>>(c.m[0], c.m[1], DIM == 3 ? c.m[2] : 1,
                                                                  (const TV*)c.vals, x, y);
    launch_end(K_SOLVE, c.s);
}

// y = A x with the value type of the matrix, vector type TX, accumulator TA
template <typename TX, typename TA>
static void spmv_dispatch(const SolveCtx& c, const TX* x, TX* y)
{
#define IGA_SPMV_CASE(PP)                                                              \
    case PP:                                                                           \
        if (c.dim == 3) {                                                              \
            if (c.f32) spmv_m<PP, 3, float, TX, TA>(c, x, y);                          \
            else spmv_m<PP, 3, double, TX, TA>(c, x, y);                               \
        } else {                                                                       \
            if (c.f32) spmv_m<PP, 2, float, TX, TA>(c, x, y);                          \
            else spmv_m<PP, 2, double, TX, TA>(c, x, y);                               \
        }                                                                              \
        break;
    switch (c.p) {
        IGA_SPMV_CASE(1)
        IGA_SPMV_CASE(2)
        IGA_SPMV_CASE(3)
        IGA_SPMV_CASE(4)
        IGA_SPMV_CASE(5)
    default: break;
    }
#undef IGA_SPMV_CASE
}

template <typename T>
static void dot(const SolveCtx& c, const T* a, const T* b, double* out)
{
    launch_begin(K_SOLVE, c.s);
    k_dot_partial<T><<<kRedBlocks, kBlock, 0, c.s>>>(c.N, a, b, c.partial);
    launch_end(K_SOLVE, c.s);
    launch_begin(K_SOLVE, c.s);
    k_dot_final<<<1, kBlock, 0, c.s>>>(kRedBlocks, c.partial, out);
    launch_end(K_SOLVE, c.s);
}

static cudaError_t read_scalar(const SolveCtx& c, const double* d, double* h)
{
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, c.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
    return e;
}

// Plain CG on interior dofs: x (in: start, out: solution), b right-hand side
// (zero on Dirichlet dofs).  Work vectors r, p, q.  Stops when ||r|| <= tol ||b||.
template <typename T, typename TA>
static cudaError_t cg_core(const SolveCtx& c, const T* b, T* x, T* r, T* p, T* q, double tol, int maxit,
                           int check_every, int* iters, double* relres)
{
    double* d_bb = c.scal + 0;
    double* d_rr = c.scal + 1;
    double* d_rr_new = c.scal + 2;
    double* d_pq = c.scal + 3;
    // r = b - A x
    spmv_dispatch<T, TA>(c, x, q);
    launch_begin(K_SOLVE, c.s);
    k_residual<T><<<c.grid, kBlock, 0, c.s>>>(c.N, c.m[0], c.m[1], c.dim == 3 ? c.m[2] : 1, c.dim, b, q, r);
    launch_end(K_SOLVE, c.s);
    cudaMemcpyAsync(p, r, c.N * sizeof(T), cudaMemcpyDeviceToDevice, c.s);
    dot<T>(c, b, b, d_bb);
    dot<T>(c, r, r, d_rr);
    double bb = 0, rr = 0;
    cudaError_t e = read_scalar(c, d_bb, &bb);
    if (e == cudaSuccess) e = read_scalar(c, d_rr, &rr);
    if (e != cudaSuccess) return e;
    if (bb == 0.0) {
        *iters = 0;
        *relres = 0.0;
        return cudaSuccess;
    }
    int it = 0;
    double rel = std::sqrt(rr / bb);
    while (rel > tol && it < maxit) {
        spmv_dispatch<T, TA>(c, p, q);
        dot<T>(c, p, q, d_pq);
        launch_begin(K_SOLVE, c.s);
        k_cg_update<T><<<c.grid, kBlock, 0, c.s>>>(c.N, d_rr, d_pq, x, p, r, q);
        launch_end(K_SOLVE, c.s);
        dot<T>(c, r, r, d_rr_new);
        launch_begin(K_SOLVE, c.s);
        k_cg_dir<T><<<c.grid, kBlock, 0, c.s>>>(c.N, d_rr_new, d_rr, r, p);
        launch_end(K_SOLVE, c.s);
        cudaMemcpyAsync(d_rr, d_rr_new, sizeof(double), cudaMemcpyDeviceToDevice, c.s);
        ++it;
        if (it % check_every == 0 || it == maxit) {
            if ((e = read_scalar(c, d_rr, &rr)) != cudaSuccess) return e;
            rel = std::sqrt(rr / bb);
        }
    }
    *iters = it;
    *relres = rel;
    return cudaGetLastError();
}

}  // namespace iga

using namespace iga;

// Implemented in iga_api.cu: access to the matrix fields.
namespace iga {
int matrix_fields(iga_matrix_t A, int* dim, int* p, int m[3], int64_t* N, const void** vals, int* f32);
cudaError_t pool_alloc(size_t bytes, cudaStream_t s, void** out);
}

extern "C" int iga_cg(iga_matrix_t A, const double* f, double* u, double tol, int maxit, void* stream,
                      int* iters, double* relres)
{
    iga::report_error(IGA_OK, "");
    if (!A || !f || !u || !iters || !relres) return iga::report_error(IGA_EINVAL, "iga_cg: null argument");
    if (!(tol > 0.0) || maxit < 1) return iga::report_error(IGA_EINVAL, "iga_cg: need tol > 0 and maxit >= 1");
    SolveCtx c;
    memset(&c, 0, sizeof(c));
    if (matrix_fields(A, &c.dim, &c.p, c.m, &c.N, &c.vals, &c.f32) != IGA_OK) return IGA_EINVAL;
    c.s = (cudaStream_t)stream;
    c.grid = (unsigned)((c.N + kBlock - 1) / kBlock);
    const int64_t N = c.N;
    const size_t vec64 = ((size_t)N * 8 + 255) / 256 * 256, vec32 = ((size_t)N * 4 + 255) / 256 * 256;
    const size_t bytes = 4096 + (c.f32 ? 4 * vec64 + 5 * vec32 : 3 * vec64);
    char* buf = nullptr;
    cudaError_t e = pool_alloc(bytes, c.s, (void**)&buf);
    if (e != cudaSuccess) return iga::report_error(IGA_ENOMEM, "iga_cg: scratch allocation failed");
    c.partial = (double*)buf;
    c.scal = (double*)(buf + kRedBlocks * 8);
    char* w = buf + 4096;
    const int m2 = c.dim == 3 ? c.m[2] : 1;
    if (e == cudaSuccess && !c.f32) {
        double *r = (double*)w, *p = (double*)(w + vec64), *q = (double*)(w + 2 * vec64);
        // start from u = 0 on every dof
        cudaMemsetAsync(u, 0, N * sizeof(double), c.s);
        e = cg_core<double, double>(c, f, u, r, p, q, tol, maxit, 10, iters, relres);
    } else if (e == cudaSuccess) {
        // iterative refinement: FP64 residual, FP32 inner CG
        double *rd = (double*)w, *yd = (double*)(w + vec64), *fm = (double*)(w + 2 * vec64);
        float *b32 = (float*)(w + 4 * vec64), *d32 = (float*)(w + 4 * vec64 + vec32);
        float *r32 = (float*)(w + 4 * vec64 + 2 * vec32), *p32 = (float*)(w + 4 * vec64 + 3 * vec32);
        float* q32 = (float*)(w + 4 * vec64 + 4 * vec32);
        cudaMemsetAsync(u, 0, N * sizeof(double), c.s);
        launch_begin(K_SOLVE, c.s);
        k_mask_copy<double, double><<<c.grid, kBlock, 0, c.s>>>(N, c.m[0], c.m[1], m2, c.dim, f, 1.0, fm);
        launch_end(K_SOLVE, c.s);
        double ff = 0.0;
        dot<double>(c, fm, fm, c.scal + 4);
        e = read_scalar(c, c.scal + 4, &ff);
        int total = 0, outer = 0;
        double rel = 1.0;
        while (e == cudaSuccess && ff > 0.0) {
            // r = f - A u in FP64 (FP32 values promoted)
            spmv_dispatch<double, double>(c, u, yd);
            launch_begin(K_SOLVE, c.s);
            k_residual<double><<<c.grid, kBlock, 0, c.s>>>(N, c.m[0], c.m[1], m2, c.dim, fm, yd, rd);
            launch_end(K_SOLVE, c.s);
            double rr = 0.0;
            dot<double>(c, rd, rd, c.scal + 5);
            if ((e = read_scalar(c, c.scal + 5, &rr)) != cudaSuccess) break;
            rel = std::sqrt(rr / ff);
            if (rel <= tol || total >= maxit || outer >= 50) break;
            // solve A d = r in FP32 (scaled to unit norm), then u += d
            const double sc = 1.0 / std::sqrt(rr);
            launch_begin(K_SOLVE, c.s);
            k_mask_copy<double, float><<<c.grid, kBlock, 0, c.s>>>(N, c.m[0], c.m[1], m2, c.dim, rd, sc, b32);
            launch_end(K_SOLVE, c.s);
            cudaMemsetAsync(d32, 0, N * sizeof(float), c.s);
            int it = 0;
            double inner_rel = 0.0;
            e = cg_core<float, float>(c, b32, d32, r32, p32, q32, 1e-4, maxit - total, 10, &it, &inner_rel);
            if (e != cudaSuccess) break;
            total += it;
            launch_begin(K_SOLVE, c.s);
            k_add_scaled<<<c.grid, kBlock, 0, c.s>>>(N, d32, 1.0 / sc, u);
            launch_end(K_SOLVE, c.s);
            ++outer;
        }
        *iters = total;
        *relres = (ff > 0.0) ? rel : 0.0;
    }
    cudaError_t fe = cudaFreeAsync(buf, c.s);
    cudaError_t se = cudaStreamSynchronize(c.s);
    if (e == cudaSuccess) e = fe;
    if (e == cudaSuccess) e = se;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return iga::report_error(IGA_ECUDA, cudaGetErrorString(e));
    return IGA_OK;
}
