// Tethered and clamped filaments (Sec. 5.2.1; eqs. tethering_constraint,
// tethered_rotation_constraint, tethering_constraint_force_and_torque).
//
// A tethered filament's base position Y_1 and the rotation u_1 of its first
// segment over the step are prescribed; the slots of X that held them carry
// the multipliers lambda_1 (a force on segment 1) and lambda_2 (the torque
// D^T lambda_2 on segment 1, D v = dexpinv_{u_1}(v)). The update equations of
// the first segment keep their form with the prescribed values substituted.
//
// On the device:
//   * the residual runs on X_r, a copy of X with the prescribed values in the
//     slots, and the multiplier loads are added to the segment loads;
//   * J0 of a tethered filament is the free J0 at X_r with the six slot
//     columns replaced by the derivatives with respect to the multipliers.
//     The free J0 is built and solved as for any filament; the replacement
//     is a rank-6 change per filament, applied by the Sherman-Morrison-
//     Woodbury identity: with Z = J0_free^{-1} U (U the six new columns,
//     packed for all tethered filaments into six vectors, since J0 is block
//     diagonal over filaments) and C = Z restricted to the filament's slots,
//     J0^{-1} b = y - Z w + E w, y = J0_free^{-1} b, w = C^{-1} y_slots
//     (E the unit vectors of the slots: J0_free^{-1} maps the free slot
//     columns to them);
//   * initial guess: the multipliers extrapolated from the last two steps.
#include <cuda_runtime.h>

#include "fil_internal.cuh"
#include "quat.cuh"
#include "rpy_pair.cuh"

namespace fil {
namespace {

__device__ __forceinline__ int fil_of_entry(const Layout &lay, int64_t e) {
    return lay.fil_of[e / 6];     // entry e of X lies in segment e / 6's filament block
}

// D^T w with D v = dexpinv_u(v) = v - (u x v)/2 - c u x (u x v):
// D^T w = w + (u x w)/2 - c u x (u x w).
__device__ __forceinline__ V3 dexpinv_T(V3 u, V3 w) {
    const V3 d = dexpinv(u, w);          // w - (u x w)/2 - c u x (u x w)
    return d + cross(u, w);              // flips the sign of the (u x w)/2 term
}

__global__ void resolve_kernel(Layout lay, const double *__restrict__ X,
                               const int *__restrict__ tmask, const double *__restrict__ tY1,
                               const double *__restrict__ tu1, double *__restrict__ Xr) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= lay.nX) return;
    const int i = fil_of_entry(lay, e);
    const int64_t l = e - 6 * (int64_t)lay.off[i];
    double v = X[e];
    if (tmask[i] && l < 6) v = l < 3 ? tY1[3 * i + l] : tu1[3 * i + l - 3];
    Xr[e] = v;
}

// F_1 += lambda_1, T_1 += D^T lambda_2 (X holds the multipliers in the slots)
__global__ void loads_kernel(Layout lay, const double *__restrict__ X,
                             const int *__restrict__ tmask, const double *__restrict__ tu1,
                             const int *__restrict__ active, double *__restrict__ FT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lay.M || !tmask[i]) return;
    const int64_t s0 = lay.off[i];
    if (active && !active[lay.sys_of[s0]]) return;
    const double *x = X + 6 * s0;
    double *ft = FT + 6 * s0;
    const V3 T = dexpinv_T(ld3(tu1 + 3 * i), ld3(x + 3));
    ft[0] += x[0];
    ft[1] += x[1];
    ft[2] += x[2];
    ft[3] += T.x;
    ft[4] += T.y;
    ft[5] += T.z;
}

// Multiplier slots of X0: 2 lam^j - lam^{j-1} (two committed steps), lam^j
// (one), else zero.
__global__ void guess_kernel(Layout lay, const int *__restrict__ tmask,
                             const double *__restrict__ tlam, const double *__restrict__ tlam_prev,
                             int hist, double *__restrict__ X0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lay.M || !tmask[i]) return;
    double *x = X0 + 6 * (int64_t)lay.off[i];
    for (int l = 0; l < 6; ++l) {
        double v = 0.0;
        if (hist >= 2) v = 2.0 * tlam[6 * i + l] - tlam_prev[6 * i + l];
        else if (hist == 1) v = tlam[6 * i + l];
        x[l] = v;
    }
}

// lam^{j-1} <- lam^j, lam^j <- slots of the converged X
__global__ void record_kernel(Layout lay, const int *__restrict__ tmask,
                              const double *__restrict__ X, double *__restrict__ tlam,
                              double *__restrict__ tlam_prev) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lay.M) return;
    const double *x = X + 6 * (int64_t)lay.off[i];
    for (int l = 0; l < 6; ++l) {
        tlam_prev[6 * i + l] = tlam[6 * i + l];
        tlam[6 * i + l] = tmask[i] ? x[l] : 0.0;
    }
}

// The six multiplier columns of every tethered filament's J0, packed into six
// vectors of length nX (column c of filament i in filament i's rows of
// vector c). Row of segment k: position row (k = 0: the Y_1 row, else the
// f^3_k row) -bdt V_k, rotation row -bdt A_k Omega_k, where (V_k, Omega_k) is
// the response of segment k to the unit load of the column on segment 0
// (lambda_1: F_0 = e_c; lambda_2: T_0 = D^T e_c) through the filament's
// mobility (drag: the self term only; filament RPY: every pair block with
// segment 0) and A_k = I - [u_k x]/2 + [u_k x]^2/12.
__global__ void columns_kernel(Layout lay, const int *__restrict__ tmask,
                               const double *__restrict__ tu1, const double *__restrict__ Xr,
                               const double *__restrict__ Yc, double a, double inv8pieta,
                               double bdt, int rpy_model, double *__restrict__ U) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= lay.S) return;
    const int i = lay.fil_of[g];
    if (!tmask[i]) return;
    const int64_t s0 = lay.off[i];
    const int N = lay.off[i + 1] - (int)s0;
    const int k = (int)(g - s0);
    if (!rpy_model && k > 0) return;                  // drag: no coupling between segments
    const V3 d = ld3(Yc + 3 * g) - ld3(Yc + 3 * s0);
    const PairCoef pc = pair_coef(d, a);
    const V3 u1 = ld3(tu1 + 3 * i);
    const V3 uk = ld3(Xr + 6 * s0 + 3 + 3 * k);
    const int64_t base = 6 * s0;
    const int64_t prow = base + (k == 0 ? 0 : 3 + 3 * N + 3 * (k - 1));
    const int64_t rrow = base + 3 + 3 * k;
    for (int col = 0; col < 6; ++col) {
        const V3 e = v3(col % 3 == 0, col % 3 == 1, col % 3 == 2);
        V3 v = v3(0, 0, 0), w = v3(0, 0, 0);
        if (col < 3) v = e;
        else w = dexpinv_T(u1, e);
        V3 V = v3(0, 0, 0), W = v3(0, 0, 0);
        apply_pair(pc, d, v, w, V, W);
        V = (-bdt * inv8pieta) * V;
        W = (-bdt * inv8pieta) * W;
        // A_k W = W - (u x W)/2 + u x (u x W)/12
        const V3 uW = cross(uk, W);
        W = W - 0.5 * uW + (1.0 / 12.0) * cross(uk, uW);
        double *Uc = U + (int64_t)col * lay.nX;
        st3(Uc + prow, V);
        st3(Uc + rrow, W);
    }
}

// Per tethered filament: C = (Z_c)_slots (6 x 6), inverted by Gauss-Jordan
// elimination with partial pivoting; a zero pivot flags J0 as singular.
__global__ void capacitance_kernel(Layout lay, const int *__restrict__ tmask,
                                   const double *__restrict__ Z, double *__restrict__ Cinv,
                                   int *__restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lay.M || !tmask[i]) return;
    const int64_t base = 6 * (int64_t)lay.off[i];
    double A[6][12];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) {
            A[r][c] = Z[(int64_t)c * lay.nX + base + r];
            A[r][6 + c] = r == c ? 1.0 : 0.0;
        }
    for (int p = 0; p < 6; ++p) {
        int piv = p;
        for (int r = p + 1; r < 6; ++r)
            if (fabs(A[r][p]) > fabs(A[piv][p])) piv = r;
        if (!(A[piv][p] != 0.0)) {
            atomicOr(flags + 1, 1);
            return;
        }
        if (piv != p)
            for (int c = 0; c < 12; ++c) {
                const double t = A[p][c];
                A[p][c] = A[piv][c];
                A[piv][c] = t;
            }
        const double inv = 1.0 / A[p][p];
        for (int c = 0; c < 12; ++c) A[p][c] *= inv;
        for (int r = 0; r < 6; ++r) {
            if (r == p) continue;
            const double f = A[r][p];
            if (f != 0.0)
                for (int c = 0; c < 12; ++c) A[r][c] -= f * A[p][c];
        }
    }
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) Cinv[36 * (int64_t)i + 6 * r + c] = A[r][6 + c];
}

// w = C^{-1} y_slots per tethered filament
__global__ void weights_kernel(Layout lay, const int *__restrict__ tmask,
                               const double *__restrict__ Cinv, const double *__restrict__ y,
                               double *__restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lay.M || !tmask[i]) return;
    const double *ys = y + 6 * (int64_t)lay.off[i];
    const double *C = Cinv + 36 * (int64_t)i;
    for (int r = 0; r < 6; ++r) {
        double s = 0.0;
        for (int c = 0; c < 6; ++c) s = fma(C[6 * r + c], ys[c], s);
        w[6 * i + r] = s;
    }
}

// x = y - sum_c Z_c w_c (+ w in the slots), in the rows of tethered filaments
__global__ void correct_kernel(Layout lay, const int *__restrict__ tmask,
                               const double *__restrict__ Z, const double *__restrict__ w,
                               double *__restrict__ x) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= lay.nX) return;
    const int i = fil_of_entry(lay, e);
    if (!tmask[i]) return;
    const int64_t l = e - 6 * (int64_t)lay.off[i];
    double v = x[e];
    for (int c = 0; c < 6; ++c) v = fma(-Z[(int64_t)c * lay.nX + e], w[6 * i + c], v);
    if (l < 6) v += w[6 * i + l];
    x[e] = v;
}

unsigned grid_of(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t tether_resolve(fil_ctx *c, const double *X, double *Xr) {
    resolve_kernel<<<grid_of(c->lay.nX, 256), 256, 0, c->stream>>>(c->lay, X, c->tmask, c->tY1,
                                                                   c->tu1, Xr);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t tether_loads(fil_ctx *c, const double *X, bool active_only) {
    loads_kernel<<<grid_of(c->lay.M, 128), 128, 0, c->stream>>>(
        c->lay, X, c->tmask, c->tu1, active_only ? c->d_active : nullptr, c->FT);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t tether_guess(fil_ctx *c, double *X0) {
    guess_kernel<<<grid_of(c->lay.M, 128), 128, 0, c->stream>>>(c->lay, c->tmask, c->tlam,
                                                                c->tlam_prev, c->thist, X0);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t tether_record(fil_ctx *c, const double *X) {
    record_kernel<<<grid_of(c->lay.M, 128), 128, 0, c->stream>>>(c->lay, c->tmask, X, c->tlam,
                                                                 c->tlam_prev);
    c->n_launches += 1;
    if (c->thist < 2) c->thist += 1;
    return cudaGetLastError();
}

// After the free J0 was built at the resolved X0 (held in c->txr, positions in
// c->Yc): the multiplier columns, Z = J0_free^{-1} U and the inverse
// capacitance of every tethered filament.
cudaError_t tether_j0_setup(fil_ctx *c, cudaError_t (*free_solve)(fil_ctx *, const double *,
                                                                  double *)) {
    const int64_t nX = c->lay.nX;
    cudaError_t e = cudaMemsetAsync(c->tU, 0, sizeof(double) * 6 * nX, c->stream);
    if (e != cudaSuccess) return e;
    const double bdt = (c->have_prev ? 2.0 / 3.0 : 1.0) * c->dt;
    columns_kernel<<<grid_of(c->lay.S, 128), 128, 0, c->stream>>>(
        c->lay, c->tmask, c->tu1, c->txr, c->Yc, c->a, 1.0 / (8.0 * kPi * c->eta), bdt,
        c->j0_model == FIL_J0_FILAMENT_RPY ? 1 : 0, c->tU);
    c->n_launches += 1;
    e = cudaGetLastError();
    for (int col = 0; col < 6 && e == cudaSuccess; ++col)
        e = free_solve(c, c->tU + col * nX, c->tZ + col * nX);
    if (e != cudaSuccess) return e;
    capacitance_kernel<<<grid_of(c->lay.M, 64), 64, 0, c->stream>>>(c->lay, c->tmask, c->tZ,
                                                                    c->tCinv, c->d_flags);
    c->n_launches += 1;
    return cudaGetLastError();
}

// x = J0^{-1} b for the tethered J0, given x = J0_free^{-1} b.
cudaError_t tether_j0_correct(fil_ctx *c, double *x) {
    weights_kernel<<<grid_of(c->lay.M, 128), 128, 0, c->stream>>>(c->lay, c->tmask, c->tCinv, x,
                                                                  c->tw);
    correct_kernel<<<grid_of(c->lay.nX, 256), 256, 0, c->stream>>>(c->lay, c->tmask, c->tZ, c->tw,
                                                                   x);
    c->n_launches += 2;
    return cudaGetLastError();
}

}  // namespace fil
