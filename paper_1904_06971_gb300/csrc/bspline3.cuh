// Cubic B-splines with open uniform knots on [0, 1] (the B-spline diffusion
// coefficient IGA_KAPPA_BSPLINE3): the four functions first..first+3 that are
// nonzero at x, by the triangular Cox-de Boor recursion.  Knot j is kp(j)/ne
// with kp(j) = clamp(j - 3, 0, ne); every denominator of the recursion is a
// knot difference c/ne with c in {1, 2, 3}, so it is a multiplication by ne/c.
#pragma once

#include <cuda_runtime.h>

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

}  // namespace iga
