// Cubic B-splines with open uniform knots on [0, 1] (the B-spline diffusion
// coefficient IGA_KAPPA_BSPLINE3): the four functions first..first+3 that are
// nonzero at x, by the triangular Cox-de Boor recursion.  Knot j is kp(j)/ne
// with kp(j) = clamp(j - 3, 0, ne); every denominator of the recursion is a
// knot difference c/ne with c in {1, 2, 3}, so it is a multiplication by ne/c.
#pragma once

#include <cuda_runtime.h>

#include "dfmath.cuh"

namespace iga {

__device__ __forceinline__ int cubic_knot_pos(int j, int ne) { return j <= 3 ? 0 : (j >= ne + 3 ? ne : j - 3); }

__device__ __forceinline__ void cubic_open_basis(int ne, double x, int& first, double N[4])
{
    int e = (int)(x * ne);
    e = e < 0 ? 0 : (e > ne - 1 ? ne - 1 : e);
    const int mu = e + 3;
    const double rne = 1.0 / (double)ne, fne = (double)ne;
    double left[4], right[4];
    N[0] = 1.0;
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        left[k] = x - cubic_knot_pos(mu + 1 - k, ne) * rne;
        right[k] = cubic_knot_pos(mu + k, ne) * rne - x;
        double saved = 0.0;
#pragma unroll
        for (int r = 0; r < k; ++r) {
            const int cnt = cubic_knot_pos(mu + r + 1, ne) - cubic_knot_pos(mu + 1 - k + r, ne);
            const double rc = cnt == 1 ? 1.0 : (cnt == 2 ? 0.5 : 1.0 / 3.0);
            const double tmp = N[r] * (fne * rc);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[k - r] * tmp;
        }
        N[k] = saved;
    }
    first = e;
}

// The same four values in double-float arithmetic on the FP32 pipe (dfmath.cuh):
// in the scaled coordinate t = x ne the knots are the integers kp(j) and every
// denominator of the recursion is 1, 2 or 3, so a step is a multiplication by
// 1, 1/2 or 1/3 (the last as a double-float constant).  first comes from the
// FP64 x exactly as in cubic_open_basis (cubic_open_basis_df), or is given
// (cubic_open_basis_df_span: a span chosen from a rounded x may be the
// neighbouring one at a knot, where both pieces agree to C^2); x_df is x as a
// float pair.
__device__ __forceinline__ void cubic_open_basis_df_span(int ne, int e, df2 x_df, df2 N[4])
{
    const int mu = e + 3;
    const df2 t = df_mul(x_df, df2{(float)ne, 0.f});
    const df2 third = df2{0.333333343267f, -9.93410742e-09f};     // 1/3 = hi + lo
    df2 left[4], right[4];
    N[0] = df2{1.f, 0.f};
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        left[k] = df_sub(t, df2{(float)cubic_knot_pos(mu + 1 - k, ne), 0.f});
        right[k] = df_sub(df2{(float)cubic_knot_pos(mu + k, ne), 0.f}, t);
        df2 saved = df2{0.f, 0.f};
#pragma unroll
        for (int r = 0; r < k; ++r) {
            const int cnt = cubic_knot_pos(mu + r + 1, ne) - cubic_knot_pos(mu + 1 - k + r, ne);
            const df2 tmp = cnt == 1 ? N[r] : (cnt == 2 ? df2{0.5f * N[r].h, 0.5f * N[r].l} : df_mul(N[r], third));
            N[r] = df_add(saved, df_mul(right[r + 1], tmp));
            saved = df_mul(left[k - r], tmp);
        }
        N[k] = saved;
    }
}

__device__ __forceinline__ void cubic_open_basis_df(int ne, double x, df2 x_df, int& first, df2 N[4])
{
    int e = (int)(x * ne);
    e = e < 0 ? 0 : (e > ne - 1 ? ne - 1 : e);
    cubic_open_basis_df_span(ne, e, x_df, N);
    first = e;
}

}  // namespace iga
