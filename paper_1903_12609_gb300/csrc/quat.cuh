// FP64 quaternion / Lie-group helpers for device code (paper Sec. 2.9, App. A).
#pragma once

#include <cuda_runtime.h>

namespace fil {

struct Q4 {
    double w, x, y, z;   // (q0, q1, q2, q3), scalar first
};

struct V3 {
    double x, y, z;
};

__device__ __forceinline__ V3 v3(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm(V3 a) { return sqrt(dot(a, a)); }

__device__ __forceinline__ V3 ld3(const double *p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ void st3(double *p, V3 v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }
__device__ __forceinline__ Q4 ld4(const double *p) { return {p[0], p[1], p[2], p[3]}; }
__device__ __forceinline__ void st4(double *p, Q4 q) { p[0] = q.w; p[1] = q.x; p[2] = q.y; p[3] = q.z; }

// Product (p0 q0 - p.q, p0 q + q0 p + p x q), Sec. 2.9.1.
__device__ __forceinline__ Q4 qmul(Q4 p, Q4 q) {
    return {p.w * q.w - (p.x * q.x + p.y * q.y + p.z * q.z),
            p.w * q.x + q.w * p.x + (p.y * q.z - p.z * q.y),
            p.w * q.y + q.w * p.y + (p.z * q.x - p.x * q.z),
            p.w * q.z + q.w * p.z + (p.x * q.y - p.y * q.x)};
}
__device__ __forceinline__ Q4 qconj(Q4 q) { return {q.w, -q.x, -q.y, -q.z}; }

// Square root of a unit quaternion, App. A.1 (special case p0 = -1):
// ((p0 + 1)/s, p/s) with s = sqrt(2 (p0 + 1)), using one reciprocal square
// root (sqrt((p0 + 1)/2) = (p0 + 1)/s).
__device__ __forceinline__ Q4 qsqrt(Q4 p) {
    if (p.w == -1.0) return {0.0, 0.0, 0.0, 1.0};
    const double r = rsqrt(2.0 * (p.w + 1.0));
    return {(p.w + 1.0) * r, p.x * r, p.y * r, p.z * r};
}

// exp(u) = (cos(|u|/2), sin(|u|/2) u/|u|), Sec. 2.9.3. Rotation increments
// are small (|u| < 1/4 in practice), where the Taylor series in x^2 of
// cos(x/2) = sum_k (-1)^k x^2k / (4^k (2k)!) and of
// sin(x/2)/x = sum_k (-1)^k x^2k / (2 4^k (2k+1)!), cut after the x^10 term,
// are exact to ~1e-19 -- far cheaper in FP64 than a sine and a cosine; larger
// angles use sincos.
__device__ __forceinline__ Q4 qexp(V3 u) {
    const double t2 = dot(u, u);
    double c, f;
    if (t2 < 0.0625) {
        c = 1.0 + t2 * (-1.0 / 8.0 + t2 * (1.0 / 384.0 + t2 * (-1.0 / 46080.0 +
            t2 * (1.0 / 10321920.0 + t2 * (-1.0 / 3715891200.0)))));
        f = 0.5 + t2 * (-1.0 / 48.0 + t2 * (1.0 / 3840.0 + t2 * (-1.0 / 645120.0 +
            t2 * (1.0 / 185794560.0 + t2 * (-1.0 / 81749606400.0)))));
    } else {
        const double ith = rsqrt(t2);
        double s;
        sincos(0.5 * t2 * ith, &s, &c);
        f = s * ith;
    }
    return {c, f * u.x, f * u.y, f * u.z};
}

// Columns of R(q) (eq. quaternion_rotation_matrix): tangent, mu, nu.
__device__ __forceinline__ V3 frame_t(Q4 q) {
    return {1.0 - 2.0 * (q.y * q.y + q.z * q.z), 2.0 * (q.x * q.y + q.z * q.w),
            2.0 * (q.x * q.z - q.y * q.w)};
}
__device__ __forceinline__ V3 frame_mu(Q4 q) {
    return {2.0 * (q.x * q.y - q.z * q.w), 1.0 - 2.0 * (q.x * q.x + q.z * q.z),
            2.0 * (q.z * q.y + q.x * q.w)};
}
__device__ __forceinline__ V3 frame_nu(Q4 q) {
    return {2.0 * (q.x * q.z + q.y * q.w), 2.0 * (q.z * q.y - q.x * q.w),
            1.0 - 2.0 * (q.y * q.y + q.x * q.x)};
}
// R(q) v
__device__ __forceinline__ V3 rotate(Q4 q, V3 v) {
    V3 t = frame_t(q), m = frame_mu(q), n = frame_nu(q);
    return {t.x * v.x + m.x * v.y + n.x * v.z, t.y * v.x + m.y * v.y + n.y * v.z,
            t.z * v.x + m.z * v.y + n.z * v.z};
}

// dexpinv_u(W) = W - (u x W)/2 - c(|u|) u x (u x W), eq. dexpinv_definition,
// c(x) = (x cot(x/2) - 2)/(2x^2). From (x/2) cot(x/2) = sum_k (-1)^k B_2k x^2k / (2k)!
// (B_2k the Bernoulli numbers), c = sum_{k>=1} (-1)^k B_2k x^(2k-2) / (2k)!
//   = -1/12 - x^2/720 - x^4/30240 - x^6/1209600 - x^8/47900160 - 691 x^10/1307674368000 - ...,
// used below x = 1/4 (truncation < 1e-18 relative); tan above.
__device__ __forceinline__ V3 dexpinv(V3 u, V3 W) {
    const double t2 = dot(u, u);
    double c;
    if (t2 < 0.0625) {
        c = -1.0 / 12.0 + t2 * (-1.0 / 720.0 + t2 * (-1.0 / 30240.0 + t2 * (-1.0 / 1209600.0 +
            t2 * (-1.0 / 47900160.0 + t2 * (-691.0 / 1307674368000.0)))));
    } else {
        const double th = sqrt(t2);
        c = (th / tan(0.5 * th) - 2.0) / (2.0 * t2);
    }
    V3 uw = cross(u, W);
    V3 uuw = cross(u, uw);
    return {W.x - 0.5 * uw.x - c * uuw.x, W.y - 0.5 * uw.y - c * uuw.y,
            W.z - 0.5 * uw.z - c * uuw.z};
}

// Internal moment between neighbouring segments, eq. quaternionM:
// q_h = (q_b q_a^*)^{1/2} q_a,
// M = R(q_h) D (2 [q_h^* (q_b - q_a)/dL]_R3 - (gamma0, kappa_mu, kappa_nu)),
// D = diag(KT, KB, KB).
__device__ __forceinline__ V3 internal_moment(Q4 qa, Q4 qb, double dL, double KB, double KT,
                                              double g0, double kmu, double knu) {
    Q4 qh = qmul(qsqrt(qmul(qb, qconj(qa))), qa);
    const double idL = 1.0 / dL;
    Q4 dq = {(qb.w - qa.w) * idL, (qb.x - qa.x) * idL, (qb.y - qa.y) * idL, (qb.z - qa.z) * idL};
    Q4 s = qmul(qconj(qh), dq);
    V3 strain = {KT * (2.0 * s.x - g0), KB * (2.0 * s.y - kmu), KB * (2.0 * s.z - knu)};
    return rotate(qh, strain);
}

}  // namespace fil
