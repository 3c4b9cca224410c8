// Learned warm start of the implicit step (include/fil_mlp.h): the per-filament
// network's inputs and training targets, and the assembly of its prediction
// into the unknowns X = (Y_1, u, Lambda) of the step (Sec. 3.3 extrapolates
// X_0 from past steps; the prediction is a second candidate).
//
// Frame of filament i: origin Y_1, axes t, mu, nu of q_1 (the columns of
// R(q_1)), so the network sees each filament in its own frame:
//   input  (per segment n): R1^T (Y_n - Y_1), q_1^* q_n, R1^T F_n, R1^T T_n,
//          then R1^T (X_ex - X^j) per 3-vector of the unknowns (X^j the
//          current state), the extrapolated increment, and R1^T corr, corr
//          = X* - X_ex of the previous step (lab frame, zero if unknown)
//   output: R1^T (X* - X_ex) per 3-vector of the filament's unknowns, the
//           correction of the extrapolated X_0 (a zero network reproduces it)
// One warp per filament, lane n = segment n (the network is defined for
// filaments of FIL_MLP_SEG = 32 segments; other rows are zero / unused).
#include <cuda_runtime.h>

#include "../../include/fil_mlp.h"
#include "fil_internal.cuh"
#include "quat.cuh"

namespace fil {
namespace {

constexpr int kSeg = FIL_MLP_SEG;
constexpr int kIn = FIL_MLP_IN, kOut = FIL_MLP_OUT;

__device__ __forceinline__ V3 to_frame(V3 t, V3 m, V3 n, V3 v) { return {dot(t, v), dot(m, v), dot(n, v)}; }
__device__ __forceinline__ V3 from_frame(V3 t, V3 m, V3 n, V3 v) {
    return v.x * t + v.y * m + v.z * n;
}

// X of the current state: (Y_1^j, u = 0, Lambda^j).
__global__ void current_X_kernel(Layout lay, const double *__restrict__ Y,
                                 const double *__restrict__ lam, double *__restrict__ X) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= lay.S) return;
    const int i = lay.fil_of[g];
    const int s0 = lay.off[i];
    const int N = lay.off[i + 1] - s0;
    const int n = (int)(g - s0);
    double *Xf = X + 6 * (int64_t)s0;
    if (n == 0) st3(Xf, ld3(Y + 3 * g));
    st3(Xf + 3 + 3 * n, v3(0, 0, 0));
    if (n <= N - 2) st3(Xf + 3 + 3 * N + 3 * n, ld3(lam + 3 * (int64_t)(s0 - i + n)));
}

// Network inputs of every 32-segment filament (row i of feat; other rows 0).
// FT holds the loads (F, T) of the current state Xc; Xex the extrapolated X_0.
__global__ void features_kernel(Layout lay, const double *__restrict__ Y, const double *__restrict__ q,
                                const double *__restrict__ FT, const double *__restrict__ Xc,
                                const double *__restrict__ Xex, const double *__restrict__ corr,
                                float *__restrict__ feat) {
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= lay.M) return;
    const int s0 = lay.off[i];
    const int N = lay.off[i + 1] - s0;
    float *row = feat + (int64_t)i * kIn;
    if (N != kSeg) {
        for (int c = lane; c < kIn; c += 32) row[c] = 0.f;
        return;
    }
    const Q4 q1 = ld4(q + 4 * (int64_t)s0);
    const V3 t = frame_t(q1), m = frame_mu(q1), nn = frame_nu(q1);
    const int64_t g = s0 + lane;
    const V3 p = to_frame(t, m, nn, ld3(Y + 3 * g) - ld3(Y + 3 * (int64_t)s0));
    const Q4 qr = qmul(qconj(q1), ld4(q + 4 * g));
    const V3 F = to_frame(t, m, nn, ld3(FT + 6 * g));
    const V3 T = to_frame(t, m, nn, ld3(FT + 6 * g + 3));
    float *o = row + 13 * lane;
    o[0] = (float)p.x; o[1] = (float)p.y; o[2] = (float)p.z;
    o[3] = (float)qr.w; o[4] = (float)qr.x; o[5] = (float)qr.y; o[6] = (float)qr.z;
    o[7] = (float)F.x; o[8] = (float)F.y; o[9] = (float)F.z;
    o[10] = (float)T.x; o[11] = (float)T.y; o[12] = (float)T.z;
    const double *xc = Xc + 6 * (int64_t)s0;
    const double *xe = Xex + 6 * (int64_t)s0;
    float *ox = row + 13 * kSeg;
    for (int v = lane; v < 2 * N; v += 32) {
        const V3 d = to_frame(t, m, nn, ld3(xe + 3 * v) - ld3(xc + 3 * v));
        ox[3 * v] = (float)d.x; ox[3 * v + 1] = (float)d.y; ox[3 * v + 2] = (float)d.z;
    }
    float *oc = ox + 6 * kSeg;
    for (int v = lane; v < 2 * N; v += 32) {
        const V3 d = corr ? to_frame(t, m, nn, ld3(corr + 6 * (int64_t)s0 + 3 * v)) : v3(0, 0, 0);
        oc[3 * v] = (float)d.x; oc[3 * v + 1] = (float)d.y; oc[3 * v + 2] = (float)d.z;
    }
}

// corr = X* - X_ex (the correction of the step being committed).
__global__ void diff_kernel(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                            double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i];
}

// Training targets of the step just committed: R1^T (X* - X_ex) per 3-vector
// of the filament's unknowns (Y_1, u_0..u_{N-1}, Lambda_0..Lambda_{N-2}), X*
// the converged unknowns and X_ex the extrapolated X_0 of that step, in the
// frame of the state the step started from: q_1^j = exp(-u_1) q_1^{j+1}.
__global__ void targets_kernel(Layout lay, const double *__restrict__ q,
                               const double *__restrict__ Xs, const double *__restrict__ Xex,
                               float *__restrict__ targ) {
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= lay.M) return;
    const int s0 = lay.off[i];
    const int N = lay.off[i + 1] - s0;
    float *row = targ + (int64_t)i * kOut;
    if (N != kSeg) {
        for (int c = lane; c < kOut; c += 32) row[c] = 0.f;
        return;
    }
    const double *xs = Xs + 6 * (int64_t)s0;
    const double *xe = Xex + 6 * (int64_t)s0;
    const V3 u1 = ld3(xs + 3);
    const Q4 q1 = qmul(qexp(v3(-u1.x, -u1.y, -u1.z)), ld4(q + 4 * (int64_t)s0));
    const V3 t = frame_t(q1), m = frame_mu(q1), nn = frame_nu(q1);
    for (int v = lane; v < 2 * N; v += 32) {     // 2N 3-vectors per filament
        const V3 d = to_frame(t, m, nn, ld3(xs + 3 * v) - ld3(xe + 3 * v));
        row[3 * v] = (float)d.x; row[3 * v + 1] = (float)d.y; row[3 * v + 2] = (float)d.z;
    }
}

// X_pred = X_ex + R1 y per 3-vector (y the network output in raw units, the
// frame that of the current state); filaments the network does not cover keep X_ex.
__global__ void predict_kernel(Layout lay, const double *__restrict__ q, const float *__restrict__ yout,
                               const double *__restrict__ Xex, double *__restrict__ Xp) {
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= lay.M) return;
    const int s0 = lay.off[i];
    const int N = lay.off[i + 1] - s0;
    const double *xe = Xex + 6 * (int64_t)s0;
    double *xp = Xp + 6 * (int64_t)s0;
    if (N != kSeg) {
        for (int c = lane; c < 6 * N; c += 32) xp[c] = xe[c];
        return;
    }
    const float *y = yout + (int64_t)i * kOut;
    const Q4 q1 = ld4(q + 4 * (int64_t)s0);
    const V3 t = frame_t(q1), m = frame_mu(q1), nn = frame_nu(q1);
    for (int v = lane; v < 2 * N; v += 32)
        st3(xp + 3 * v, ld3(xe + 3 * v) + from_frame(t, m, nn, v3(y[3 * v], y[3 * v + 1], y[3 * v + 2])));
}

unsigned warps(int M, int threads) { return (unsigned)(((int64_t)M * 32 + threads - 1) / threads); }

}  // namespace

// Xex: the extrapolated X_0 (null: computed here into stage_b).
cudaError_t warm_features(fil_ctx *c, const double *Xex, float *feat) {
    if (!Xex) {
        cudaError_t e = extrapolate_guess(c, c->stage_b);
        if (e != cudaSuccess) return e;
        Xex = c->stage_b;
    }
    current_X_kernel<<<(unsigned)((c->lay.S + 255) / 256), 256, 0, c->stream>>>(c->lay, c->Y, c->lam,
                                                                               c->stage_c);
    cudaError_t e = unpack_forces(c, c->stage_c, 1);
    if (e != cudaSuccess) return e;
    features_kernel<<<warps(c->lay.M, 128), 128, 0, c->stream>>>(
        c->lay, c->Y, c->q, c->FT, c->stage_c, Xex, c->warm_corr_ok ? c->warm_corr : nullptr, feat);
    c->n_launches += 2;
    return cudaGetLastError();
}

cudaError_t warm_record_correction(fil_ctx *c) {
    const int64_t n = c->lay.nX;
    diff_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->Xk, c->warm_xex,
                                                                    c->warm_corr);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t warm_targets(fil_ctx *c, float *targ) {
    targets_kernel<<<warps(c->lay.M, 128), 128, 0, c->stream>>>(c->lay, c->q, c->Xk, c->warm_xex,
                                                                targ);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t warm_predict(fil_ctx *c, const double *Xex, double *Xpred) {
    cudaError_t e = warm_features(c, Xex, c->warm_feat);
    if (e != cudaSuccess) return e;
    e = mlp_forward_async(c->warm_net, c->warm_feat, c->warm_out, c->lay.M, c->stream,
                          &c->n_launches);
    if (e != cudaSuccess) return e;
    predict_kernel<<<warps(c->lay.M, 128), 128, 0, c->stream>>>(c->lay, c->q, c->warm_out, Xex,
                                                                Xpred);
    c->n_launches += 1;
    return cudaGetLastError();
}

}  // namespace fil
