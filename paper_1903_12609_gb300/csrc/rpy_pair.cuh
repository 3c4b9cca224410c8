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

// (V, Omega) += M_nm (v, w) in units of 1/(8 pi eta), as fused multiply-adds
// (35 FP64 operations: the two dot products, e = G d, and four terms per
// component; GB300 runs FP64 at 1/64 of the FP32 rate, so the count matters)
__device__ __forceinline__ void apply_pair(const PairCoef &k, V3 d, V3 v, V3 w, V3 &V, V3 &W) {
    const double bdv = k.B * fma(d.x, v.x, fma(d.y, v.y, d.z * v.z));
    const double ddw = k.D * fma(d.x, w.x, fma(d.y, w.y, d.z * w.z));
    const double ex = k.G * d.x, ey = k.G * d.y, ez = k.G * d.z;
    V.x = fma(k.A, v.x, fma(bdv, d.x, fma(w.y, ez, fma(-w.z, ey, V.x))));
    V.y = fma(k.A, v.y, fma(bdv, d.y, fma(w.z, ex, fma(-w.x, ez, V.y))));
    V.z = fma(k.A, v.z, fma(bdv, d.z, fma(w.x, ey, fma(-w.y, ex, V.z))));
    W.x = fma(k.C, w.x, fma(ddw, d.x, fma(v.y, ez, fma(-v.z, ey, W.x))));
    W.y = fma(k.C, w.y, fma(ddw, d.y, fma(v.z, ex, fma(-v.x, ez, W.y))));
    W.z = fma(k.C, w.z, fma(ddw, d.z, fma(v.x, ey, fma(-v.y, ex, W.z))));
}

}  // namespace fil
