// 3x3 matrix helpers and the App. B.2 moment derivatives shared by the
// banded (drag mobility) and dense (filament RPY mobility) J0 kernels.
#pragma once

#include <cuda_runtime.h>

#include "quat.cuh"

namespace fil {

struct M33 {
    double m[9];
};

__device__ __forceinline__ M33 mzero() {
    M33 r;
#pragma unroll
    for (int i = 0; i < 9; ++i) r.m[i] = 0.0;
    return r;
}
__device__ __forceinline__ M33 meye() {
    M33 r = mzero();
    r.m[0] = r.m[4] = r.m[8] = 1.0;
    return r;
}
// [v x]: [v x] w = v x w
__device__ __forceinline__ M33 skew(V3 v) {
    M33 r;
    r.m[0] = 0.0;   r.m[1] = -v.z; r.m[2] = v.y;
    r.m[3] = v.z;   r.m[4] = 0.0;  r.m[5] = -v.x;
    r.m[6] = -v.y;  r.m[7] = v.x;  r.m[8] = 0.0;
    return r;
}
// [x v] = -[v x]: [x v] w = w x v
__device__ __forceinline__ M33 rskew(V3 v) { return skew(v3(-v.x, -v.y, -v.z)); }
__device__ __forceinline__ M33 mmul(const M33 &a, const M33 &b) {
    M33 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            r.m[3 * i + j] = a.m[3 * i] * b.m[j] + a.m[3 * i + 1] * b.m[3 + j] +
                             a.m[3 * i + 2] * b.m[6 + j];
    return r;
}
__device__ __forceinline__ M33 madd(const M33 &a, const M33 &b, double s = 1.0) {
    M33 r;
#pragma unroll
    for (int i = 0; i < 9; ++i) r.m[i] = a.m[i] + s * b.m[i];
    return r;
}
__device__ __forceinline__ M33 mscale(const M33 &a, double s) {
    M33 r;
#pragma unroll
    for (int i = 0; i < 9; ++i) r.m[i] = s * a.m[i];
    return r;
}
__device__ __forceinline__ M33 outer(V3 a, V3 b) {
    M33 r;
    r.m[0] = a.x * b.x; r.m[1] = a.x * b.y; r.m[2] = a.x * b.z;
    r.m[3] = a.y * b.x; r.m[4] = a.y * b.y; r.m[5] = a.y * b.z;
    r.m[6] = a.z * b.x; r.m[7] = a.z * b.y; r.m[8] = a.z * b.z;
    return r;
}

struct J0Params {
    double dL, KB, KT, g0, kmu, knu, ct, cr;
};

// Derivatives of the frame-vector moment of joint (a, b) with respect to u_a
// (Da) and u_b (Db), App. B.2.
__device__ __forceinline__ void moment_derivs(const J0Params &p, Q4 qa, Q4 qb, M33 &Da, M33 &Db) {
    const V3 ta = frame_t(qa), tb = frame_t(qb);
    const V3 ma = frame_mu(qa), mb = frame_mu(qb);
    const V3 na = frame_nu(qa), nb = frame_nu(qb);
    const double beta = (dot(mb, na) - dot(ma, nb)) / (2.0 * p.dL) - p.g0;
    const V3 w = cross(na, mb) - cross(ma, nb);
    const M33 tw = mscale(outer(ta + tb, w), 1.0 / (2.0 * p.dL));
    // Da = KB([x tb][x ta]/dL - kmu/2 [x ma] - knu/2 [x na]) + KT/2 (beta [x ta] + tw)
    M33 bend = mscale(mmul(rskew(tb), rskew(ta)), 1.0 / p.dL);
    bend = madd(bend, rskew(ma), -0.5 * p.kmu);
    bend = madd(bend, rskew(na), -0.5 * p.knu);
    Da = madd(mscale(bend, p.KB), madd(mscale(rskew(ta), beta), tw), 0.5 * p.KT);
    // Db = KB([ta x][x tb]/dL - kmu/2 [x mb] - knu/2 [x nb]) + KT/2 (beta [x tb] - tw)
    bend = mscale(mmul(skew(ta), rskew(tb)), 1.0 / p.dL);
    bend = madd(bend, rskew(mb), -0.5 * p.kmu);
    bend = madd(bend, rskew(nb), -0.5 * p.knu);
    Db = madd(mscale(bend, p.KB), madd(mscale(rskew(tb), beta), tw, -1.0), 0.5 * p.KT);
}

}  // namespace fil
