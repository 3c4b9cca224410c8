// FP64 RPY blocks of one pair of segments (Sec. 2.7.1), shared by the J0
// kernels: far form for r >= 2a, the overlapping-sphere form below, the self
// values at r = 0.
#pragma once

#include "quat.cuh"

namespace fil {

// RPY blocks of one pair, scaled by 8 pi eta (see rpy.cu for the formulas):
// Mtt v = A v + B (d.v) d, Mrr w = C w + D (d.w) d, Mtr w = G (w x d),
// Mrt v = G (v x d). The self pair and r = 0 take the r -> 0 limit.
struct PairCoef {
    double A, B, C, D, G;
};

__device__ __forceinline__ PairCoef pair_coef(V3 d, double a) {
    const double r2 = dot(d, d);
    PairCoef k;
    if (r2 < 4.0 * a * a) {
        const double r = sqrt(r2);
        const double rinv = r > 0.0 ? 1.0 / r : 0.0;
        const double ia3 = 1.0 / (a * a * a);
        k.A = (4.0 / (3.0 * a)) * (1.0 - 9.0 * r / (32.0 * a));
        k.B = rinv / (8.0 * a * a);
        k.C = ia3 * (1.0 - 27.0 * r / (32.0 * a) + 5.0 * r * r2 / (64.0 * a * a * a));
        k.D = ia3 * (9.0 * rinv / (32.0 * a) - 3.0 * r / (64.0 * a * a * a));
        k.G = 0.5 * ia3 * (1.0 - 3.0 * r / (8.0 * a));
    } else {
        const double rinv = rsqrt(r2);
        const double rinv2 = rinv * rinv, rinv3 = rinv * rinv2, rinv5 = rinv3 * rinv2;
        k.A = rinv + (2.0 * a * a / 3.0) * rinv3;
        k.B = rinv3 - 2.0 * a * a * rinv5;
        k.C = -0.5 * rinv3;
        k.D = 1.5 * rinv5;
        k.G = rinv3;
    }
    return k;
}

// (V, Omega) += M_nm (v, w) in units of 1/(8 pi eta)
__device__ __forceinline__ void apply_pair(const PairCoef &k, V3 d, V3 v, V3 w, V3 &V, V3 &W) {
    V = V + k.A * v + (k.B * dot(d, v)) * d + k.G * cross(w, d);
    W = W + k.G * cross(v, d) + k.C * w + (k.D * dot(d, w)) * d;
}

}  // namespace fil
