// FP64 evaluation of a sample's kernel-function table (g1 = B'', g2 = (r B'' - B')/r^3,
// Eq. BrV): Chebyshev degree F64_DEG on panels of u = 1 + r^2/delta^2 indexed by the
// double's exponent (octave) and top F64_SUB_LOG2 mantissa bits; g2's coefficients start P
// panels after g1's.  Clenshaw recurrence.
#pragma once

#include "common.cuh"

static __device__ __forceinline__ void kern_f64(const double *__restrict__ tab, int P, int pmax, double u, double &g1,
                                         double &g2) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(u);
    unsigned long long p = (bits >> (52 - F64_SUB_LOG2)) - (1023ull << F64_SUB_LOG2);
    if (p > (unsigned long long)pmax) p = pmax;
    double f = __longlong_as_double(0x3ff0000000000000LL | (long long)((bits << F64_SUB_LOG2) & 0x000fffffffffffffull)) - 1.0;
    double t = 2.0 * f - 1.0, t2 = 2.0 * t;
    const double *c1 = tab + p * F64_NODES;
    const double *c2 = tab + ((size_t)P + p) * F64_NODES;
    double a1 = 0.0, a2 = 0.0, b1 = 0.0, b2 = 0.0;
#pragma unroll
    for (int k = F64_DEG; k >= 1; --k) {
        double a0 = fma(t2, a1, c1[k] - a2);
        a2 = a1;
        a1 = a0;
        double b0 = fma(t2, b1, c2[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    g1 = fma(t, a1, c1[0] - a2);
    g2 = fma(t, b1, c2[0] - b2);
}
