// Device helpers of the linewidth kernels: mesh arithmetic and the occupation/smearing
// weight of Eq. (gamma) with Eq. (broadening) (decay + absorption counting over ordered
// partner pairs, window |df| < window*sigma, partners below f_min skipped).
#pragma once
#include "common.h"

__device__ __forceinline__ int phx_third_index(int iq, int qp, int m1, int m2, int m3) {
    const int a1 = iq / (m2 * m3), a2 = (iq / m3) % m2, a3 = iq % m3;
    const int b1 = qp / (m2 * m3), b2 = (qp / m3) % m2, b3 = qp % m3;
    const int c1 = (2 * m1 - a1 - b1) % m1, c2 = (2 * m2 - a2 - b2) % m2, c3 = (2 * m3 - a3 - b3) % m3;
    return (c1 * m2 + c2) * m3 + c3;
}

__device__ __forceinline__ double phx_broad(double x, const GammaParams& gp) {
    const double s = gp.sigma;
    if (!(fabs(x) < gp.window * s)) return 0.0;
    if (gp.shape == PHX_GAUSS) {
        const double u = x / s;
        return exp(-u * u) / (1.7724538509055160273 * s);
    }
    const double h = 0.5 * s;
    return h / (phx::kPi * (x * x + h * h));
}

// Weight per |V|^2 in ps^4: [(1+n1+n2) g(f0-f1-f2) + 2(n1-n2) g(f0+f1-f2)] / (2 pi w0 w1 w2).
__device__ __forceinline__ double phx_pair_weight(double f0, double f1, double f2, double n1,
                                                  double n2, const GammaParams& gp) {
    if (!(f0 >= gp.f_min && f1 >= gp.f_min && f2 >= gp.f_min)) return 0.0;
    const double gd = phx_broad(f0 - f1 - f2, gp);
    const double ga = phx_broad(f0 + f1 - f2, gp);
    if (gd == 0.0 && ga == 0.0) return 0.0;
    const double tp3 = phx::kTwoPi * phx::kTwoPi * phx::kTwoPi;
    return ((1.0 + n1 + n2) * gd + 2.0 * (n1 - n2) * ga) / phx::kTwoPi / (tp3 * f0 * f1 * f2);
}
