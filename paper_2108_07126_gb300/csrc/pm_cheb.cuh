// Chebyshev expansion of exp(-i G) (Sec. 2.1, Eq. chebychev_series, Algorithm 1):
// with the spectrum of G in [-beta, beta],
//   exp(-i G) ~ a_0 I + 2 sum_{k=1}^{m} a_k T_k(G / beta),  a_k = (-i)^k J_k(beta),
// evaluated by the Clenshaw recurrence D_k = a_k I + 2 X D_{k+1} - D_{k+2},
// exp(-i G) ~ D_0 - D_2.  The degree m is the smallest one whose truncation
// bound (Sec. 2.1, Eq. error_chebychev, with beta - alpha = 2 beta) is below u.
#pragma once

#include <cmath>

namespace pm {

constexpr int kMaxChebDegree = 48;

// eps(r, m) = 4 (exp(1 - y^2) y)^(m+1), y = r / (4m + 4), r = beta - alpha (Eq. error_chebychev)
__host__ __device__ inline double cheb_error_bound(double r, int m) {
    const double y = r / (4.0 * m + 4.0);
    return 4.0 * pow(exp(1.0 - y * y) * y, (double)(m + 1));
}

// largest half-width beta with eps(2 beta, m) < u (the bound increases with beta for y < 1/sqrt(2))
__host__ __device__ inline double cheb_theta(int m, double u) {
    double lo = 0.0, hi = (4.0 * m + 4.0) * 0.70710678118654752 * 0.5;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (cheb_error_bound(2.0 * mid, m) < u) lo = mid; else hi = mid;
    }
    return lo;
}

// J_0(x) .. J_n(x) for x >= 0 (Miller's backward recurrence J_{k-1} = (2k/x) J_k - J_{k+1},
// normalised by J_0 + 2 (J_2 + J_4 + ...) = 1); out has n + 1 entries
__host__ __device__ inline void bessel_j_seq(double x, int n, double *out) {
    for (int k = 0; k <= n; ++k) out[k] = (k == 0) ? 1.0 : 0.0;
    if (!(x > 0.0)) return;
    int start = n + 24 + (int)(2.0 * x);
    start += start & 1;  // even start
    double jp1 = 0.0, j = 1e-300, norm = 0.0;
    for (int k = start; k >= 1; --k) {
        const double jm1 = (2.0 * k / x) * j - jp1;
        jp1 = j;
        j = jm1;  // j = J_{k-1} (unnormalised)
        if (k - 1 <= n) out[k - 1] = j;
        if ((k - 1) % 2 == 0 && k - 1 > 0) norm += 2.0 * j;
        if (fabs(j) > 1e250) {  // rescale to stay finite
            j *= 1e-250;
            jp1 *= 1e-250;
            norm *= 1e-250;
            for (int q = k - 1; q <= n; ++q) out[q] *= 1e-250;
        }
    }
    norm += j;  // J_0
    for (int k = 0; k <= n; ++k) out[k] /= norm;
}

}  // namespace pm
