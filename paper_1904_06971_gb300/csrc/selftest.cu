// Self-test of the double-float elementary functions used by the coefficient
// kernel (dfmath.cuh) against CUDA's FP64 sincospi / exp on their domains.
#include <cstring>

#include "dfmath.cuh"
#include "iga_internal.cuh"

namespace iga {

// err[0]: max |sin - ref| / 1 over |pi y| <= 0.5; err[1]: same for cos;
// err[2]: max |exp - ref| / ref over |x| <= 1.  Reduced with atomicMax on the bit
// patterns of non-negative doubles (monotone as unsigned integers).
__global__ void k_selftest_dfmath(int n, unsigned long long* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double y = (0.5 / 3.14159265358979323846) * (2.0 * i / (n - 1) - 1.0);
    df2 s, c;
    df_sincospi_small(df_from_double(y), s, c);
    double rs, rc;
    sincospi(y, &rs, &rc);
    const double es = fabs(df_to_double(s) - rs), ec = fabs(df_to_double(c) - rc);
    const double x = 2.0 * i / (n - 1) - 1.0;
    const double re = exp(x);
    const double ee = fabs(df_to_double(df_exp_small(df_from_double(x))) - re) / re;
    atomicMax(&err[0], (unsigned long long)__double_as_longlong(es));
    atomicMax(&err[1], (unsigned long long)__double_as_longlong(ec));
    atomicMax(&err[2], (unsigned long long)__double_as_longlong(ee));
}

}  // namespace iga

// Library self-test: maximum errors of the double-float sin / cos / exp against
// CUDA's FP64 functions on n points (errors[0..2] = sin, cos, exp).  Synchronous.
extern "C" int iga_selftest_dfmath(int n, double* errors)
{
    if (n < 2 || !errors) return iga::report_error(IGA_EINVAL, "iga_selftest_dfmath: need n >= 2 and an output array");
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 3 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(d, 0, 3 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        iga::k_selftest_dfmath<<<(n + 255) / 256, 256>>>(n, d);
        e = cudaGetLastError();
    }
    unsigned long long h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return iga::report_error(IGA_ECUDA, cudaGetErrorString(e));
    for (int k = 0; k < 3; ++k) memcpy(&errors[k], &h[k], sizeof(double));
    return IGA_OK;
}
