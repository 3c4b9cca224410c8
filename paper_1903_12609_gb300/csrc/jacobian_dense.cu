// J0 with each filament's own RPY mobility, dense per filament.
//
// J0 = d f_0 / dX where f_0 is the residual with (V, Omega) = M_f (F, T):
// M_f holds every RPY block between segments of the same filament (held
// fixed at X, no dM/dY term), the loads are the internal constraint and
// elastic ones, and the derivative approximations are those of App. B.2
// (d t / d u = [x t], frame-vector moments, three-term dexpinv). Rows, in the
// order of f, and columns, in the order of X:
//   position row n : I on Y_1 + (dL/2) w_nk [x t_k] on u_k (k <= n, n >= 1)
//                    - b dt (M_f G)_{V_n}
//   rotation row n : I on u_n - b dt A_n (M_f G)_{Omega_n}
//                    - b dt (-[x Om_n]/2 + ([x (u_n x Om_n)] + [u_n x][x Om_n])/12) on u_n
// with G = d(F, T)/dX, A_n = I - [u_n x]/2 + [u_n x]^2/12 and Om_n the
// angular velocity of the internal loads. With M_f reduced to the self
// mobility this is exactly the J0 of App. B.2 (the banded path in
// jacobian.cu); keeping the whole filament block captures the hydrodynamic
// coupling along a filament, which the drag model drops and which makes
// Broyden need O(number of filaments) iterations in dense suspensions.
//
// Storage: row-major (6N)^2 FP64 block per filament at jofs[i]; factored in
// place by Gaussian elimination with partial pivoting (one CTA per filament),
// solved by one warp per filament.
#include <cuda_runtime.h>

#include <algorithm>

#include "fil_internal.cuh"
#include "j0_common.cuh"
#include "quat.cuh"

namespace fil {
namespace {

constexpr int kAsmThreads = 256;
constexpr int kLuThreads = 256;

struct DenseParams {
    J0Params jp;
    double bdt;            // (scheme weight) * dt
    double inv8pieta;      // 1 / (8 pi eta)
    double near2;          // (2a)^2
    double a;
};

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
        const double rinv = 1.0 / sqrt(r2);
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

__device__ __forceinline__ V3 col(const M33 &m, int c) { return {m.m[c], m.m[3 + c], m.m[6 + c]}; }

// Per-segment data staged in shared memory for one filament.
struct SegSmem {
    double *Y, *t, *u, *Ls, *Fi, *Ti, *Om;   // 3N each
    double *Q;                                // 4N
};

__global__ void __launch_bounds__(kAsmThreads)
j0_dense_assemble_kernel(Layout lay, const int64_t *__restrict__ jofs, const double *__restrict__ X,
                         const double *__restrict__ qc, const double *__restrict__ Yc,
                         const double *__restrict__ Tint, DenseParams dp,
                         double *__restrict__ J_all) {
    extern __shared__ double sm[];
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    const int N = lay.off[f + 1] - s0;
    const int n6 = 6 * N;
    double *J = J_all + jofs[f];
    SegSmem g;
    g.Y = sm;
    g.t = sm + 3 * N;
    g.u = sm + 6 * N;
    g.Ls = sm + 9 * N;
    g.Fi = sm + 12 * N;
    g.Ti = sm + 15 * N;
    g.Om = sm + 18 * N;
    g.Q = sm + 21 * N;
    const double *Xf = X + 6 * (int64_t)s0;
    const double *Lam = Xf + 3 + 3 * N;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int64_t gg = s0 + n;
        const Q4 q = ld4(qc + 4 * gg);
        st4(g.Q + 4 * n, q);
        st3(g.Y + 3 * n, ld3(Yc + 3 * gg));
        st3(g.t + 3 * n, frame_t(q));
        st3(g.u + 3 * n, ld3(Xf + 3 + 3 * n));
        const V3 Lr = (n <= N - 2) ? ld3(Lam + 3 * n) : v3(0, 0, 0);
        const V3 Ll = (n >= 1) ? ld3(Lam + 3 * (n - 1)) : v3(0, 0, 0);
        st3(g.Ls + 3 * n, Lr + Ll);
        st3(g.Fi + 3 * n, Lr - Ll);
        st3(g.Ti + 3 * n, ld3(Tint + 3 * gg));
    }
    for (int64_t e = threadIdx.x; e < (int64_t)n6 * n6; e += blockDim.x) J[e] = 0.0;
    __syncthreads();
    // angular velocity of the internal loads, filament block only
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        V3 V = v3(0, 0, 0), W = v3(0, 0, 0);
        const V3 Yn = ld3(g.Y + 3 * n);
        for (int m = 0; m < N; ++m) {
            const V3 d = Yn - ld3(g.Y + 3 * m);
            const PairCoef k = pair_coef(d, dp.a);
            apply_pair(k, d, ld3(g.Fi + 3 * m), ld3(g.Ti + 3 * m), V, W);
        }
        st3(g.Om + 3 * n, dp.inv8pieta * W);
    }
    __syncthreads();

    // tasks: (row segment n, column block x), x = 0..N-1 -> u_x, x = N..2N-2 -> Lam_{x-N}
    const int ncol = 2 * N - 1;
    for (int task = threadIdx.x; task < N * ncol; task += blockDim.x) {
        const int n = task / ncol;
        const int x = task - n * ncol;
        const V3 Yn = ld3(g.Y + 3 * n);
        V3 MV[3] = {v3(0, 0, 0), v3(0, 0, 0), v3(0, 0, 0)};
        V3 MW[3] = {v3(0, 0, 0), v3(0, 0, 0), v3(0, 0, 0)};
        int colX;
        if (x < N) {
            // d T_m / d u_k, m = k-1, k, k+1 (App. B.2)
            const int k = x;
            colX = 3 + 3 * k;
            const Q4 qk = ld4(g.Q + 4 * k);
            M33 Da_k, Db_k, Da_km, Db_km;
            if (k <= N - 2) moment_derivs(dp.jp, qk, ld4(g.Q + 4 * (k + 1)), Da_k, Db_k);
            if (k >= 1) moment_derivs(dp.jp, ld4(g.Q + 4 * (k - 1)), qk, Da_km, Db_km);
            for (int mm = -1; mm <= 1; ++mm) {
                const int m = k + mm;
                if (m < 0 || m > N - 1) continue;
                M33 Gt;
                if (mm == -1) {
                    Gt = Db_km;
                } else if (mm == 0) {
                    Gt = mscale(mmul(rskew(ld3(g.Ls + 3 * k)), rskew(ld3(g.t + 3 * k))),
                                0.5 * dp.jp.dL);
                    if (k <= N - 2) Gt = madd(Gt, Da_k);
                    if (k >= 1) Gt = madd(Gt, Db_km, -1.0);
                } else {
                    Gt = mscale(Da_k, -1.0);
                }
                const V3 d = Yn - ld3(g.Y + 3 * m);
                const PairCoef kc = pair_coef(d, dp.a);
                for (int c = 0; c < 3; ++c) apply_pair(kc, d, v3(0, 0, 0), col(Gt, c), MV[c], MW[c]);
            }
        } else {
            // d(F_m, T_m)/d Lam_j for m = j (F += I) and m = j+1 (F -= I); T: (dL/2)[t_m x]
            const int j = x - N;
            colX = 3 + 3 * N + 3 * j;
            for (int mm = 0; mm <= 1; ++mm) {
                const int m = j + mm;
                const M33 Gt = mscale(skew(ld3(g.t + 3 * m)), 0.5 * dp.jp.dL);
                const double sF = mm == 0 ? 1.0 : -1.0;
                const V3 d = Yn - ld3(g.Y + 3 * m);
                const PairCoef kc = pair_coef(d, dp.a);
                for (int c = 0; c < 3; ++c) {
                    V3 e = v3(c == 0 ? sF : 0.0, c == 1 ? sF : 0.0, c == 2 ? sF : 0.0);
                    apply_pair(kc, d, e, col(Gt, c), MV[c], MW[c]);
                }
            }
        }
        // rows of segment n
        const int prow = (n == 0) ? 0 : 3 + 3 * N + 3 * (n - 1);
        const int rrow = 3 + 3 * n;
        const V3 un = ld3(g.u + 3 * n);
        const M33 ux = skew(un);
        const M33 A = madd(madd(meye(), ux, -0.5), mmul(ux, ux), 1.0 / 12.0);
        const double s = -dp.bdt * dp.inv8pieta;
        for (int c = 0; c < 3; ++c) {
            const V3 w = v3(A.m[0] * MW[c].x + A.m[1] * MW[c].y + A.m[2] * MW[c].z,
                            A.m[3] * MW[c].x + A.m[4] * MW[c].y + A.m[5] * MW[c].z,
                            A.m[6] * MW[c].x + A.m[7] * MW[c].y + A.m[8] * MW[c].z);
            double *Jp = J + (int64_t)prow * n6 + colX + c;
            Jp[0] = s * MV[c].x;
            Jp[n6] = s * MV[c].y;
            Jp[2 * n6] = s * MV[c].z;
            double *Jr = J + (int64_t)rrow * n6 + colX + c;
            Jr[0] = s * w.x;
            Jr[n6] = s * w.y;
            Jr[2 * n6] = s * w.z;
        }
        if (x < N) {
            const int k = x;
            // robot-arm term of position row n >= 1 on u_k: (dL/2) w [x t_k]
            if (n >= 1 && k <= n) {
                const double wgt = (k == 0 || k == n) ? 1.0 : 2.0;
                const M33 arm = mscale(rskew(ld3(g.t + 3 * k)), 0.5 * dp.jp.dL * wgt);
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c)
                        J[(int64_t)(prow + r) * n6 + colX + c] += arm.m[3 * r + c];
            }
            if (k == n) {
                const V3 Om = ld3(g.Om + 3 * n);
                const M33 xO = rskew(Om);
                M33 dd = madd(mscale(xO, -0.5),
                              madd(rskew(cross(un, Om)), mmul(ux, xO)), 1.0 / 12.0);
                dd = madd(meye(), dd, -dp.bdt);
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c)
                        J[(int64_t)(rrow + r) * n6 + colX + c] += dd.m[3 * r + c];
            }
        }
    }
    // Y_1 column: identity on every position row
    for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) {
        const int n = e / 3, r = e % 3;
        const int prow = (n == 0) ? 0 : 3 + 3 * N + 3 * (n - 1);
        J[(int64_t)(prow + r) * n6 + r] = 1.0;
    }
}

// In-place LU with partial pivoting of each filament's block (LAPACK getf2
// order: the whole pivot row is swapped, then the trailing rank-1 update).
__global__ void __launch_bounds__(kLuThreads)
dense_lu_kernel(Layout lay, const int64_t *__restrict__ jofs, double *__restrict__ J_all,
                int *__restrict__ piv_all, int *__restrict__ flags) {
    __shared__ double red_v[kLuThreads / 32];
    __shared__ int red_i[kLuThreads / 32];
    __shared__ int s_piv;
    extern __shared__ double prow[];   // pivot row (n doubles)
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    const int n = 6 * (lay.off[f + 1] - s0);
    double *A = J_all + jofs[f];
    int *piv = piv_all + 6 * (int64_t)s0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int j = 0; j < n; ++j) {
        double v = -1.0;
        int idx = j;
        for (int i = j + tid; i < n; i += blockDim.x) {
            const double a = fabs(A[(int64_t)i * n + j]);
            if (a > v) {
                v = a;
                idx = i;
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, v, d);
            const int oi = __shfl_down_sync(0xffffffffu, idx, d);
            if (ov > v || (ov == v && oi < idx)) {
                v = ov;
                idx = oi;
            }
        }
        if (lane == 0) {
            red_v[wid] = v;
            red_i[wid] = idx;
        }
        __syncthreads();
        if (tid == 0) {
            double bv = red_v[0];
            int bi = red_i[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bi)) {
                    bv = red_v[w];
                    bi = red_i[w];
                }
            s_piv = bi;
            piv[j] = bi;
            if (!(bv > 0.0)) atomicOr(flags + 1, 1);
        }
        __syncthreads();
        const int p = s_piv;
        if (p != j) {
            for (int c = tid; c < n; c += blockDim.x) {
                const double tmp = A[(int64_t)j * n + c];
                A[(int64_t)j * n + c] = A[(int64_t)p * n + c];
                A[(int64_t)p * n + c] = tmp;
            }
            __syncthreads();
        }
        const double piv_inv = 1.0 / A[(int64_t)j * n + j];
        for (int c = j + 1 + tid; c < n; c += blockDim.x) prow[c] = A[(int64_t)j * n + c];
        for (int i = j + 1 + tid; i < n; i += blockDim.x) A[(int64_t)i * n + j] *= piv_inv;
        __syncthreads();
        const int w = n - j - 1;
        for (int64_t e = tid; e < (int64_t)w * w; e += blockDim.x) {
            const int i = j + 1 + (int)(e / w);
            const int c = j + 1 + (int)(e % w);
            A[(int64_t)i * n + c] -= A[(int64_t)i * n + j] * prow[c];
        }
        __syncthreads();
    }
}

// x = J0^{-1} b, one warp per filament: row interchanges, unit-lower forward,
// upper backward substitution; rows are read with coalesced loads.
__global__ void dense_solve_kernel(Layout lay, const int64_t *__restrict__ jofs,
                                   const double *__restrict__ J_all, const int *__restrict__ piv_all,
                                   const double *b, double *x, int zmax) {
    extern __shared__ double zs[];
    const int wib = threadIdx.x >> 5;
    const int f = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= lay.M) return;
    double *z = zs + (int64_t)wib * zmax;
    const int s0 = lay.off[f];
    const int n = 6 * (lay.off[f + 1] - s0);
    const double *A = J_all + jofs[f];
    const int *piv = piv_all + 6 * (int64_t)s0;
    const double *bf = b + 6 * (int64_t)s0;
    double *xf = x + 6 * (int64_t)s0;
    for (int i = lane; i < n; i += 32) z[i] = bf[i];
    __syncwarp();
    if (lane == 0)
        for (int j = 0; j < n; ++j) {
            const int p = piv[j];
            if (p != j) {
                const double t = z[j];
                z[j] = z[p];
                z[p] = t;
            }
        }
    __syncwarp();
    for (int i = 1; i < n; ++i) {
        const double *row = A + (int64_t)i * n;
        double t = 0.0;
        for (int c = lane; c < i; c += 32) t += row[c] * z[c];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
        if (lane == 0) z[i] -= t;
        __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
        const double *row = A + (int64_t)i * n;
        double t = 0.0;
        for (int c = i + 1 + lane; c < n; c += 32) t += row[c] * z[c];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
        if (lane == 0) z[i] = (z[i] - t) / row[i];
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) xf[i] = z[i];
}

}  // namespace

cudaError_t j0_dense_build_factor(fil_ctx *c, const double *X) {
    const double beta = c->have_prev ? 2.0 / 3.0 : 1.0;
    DenseParams dp;
    dp.jp = J0Params{c->dL, c->KB, c->KT, c->g0, c->kmu, c->knu, 0.0, 0.0};
    dp.bdt = beta * c->dt;
    dp.inv8pieta = 1.0 / (8.0 * kPi * c->eta);
    dp.near2 = 4.0 * c->a * c->a;
    dp.a = c->a;
    const size_t smem_asm = (size_t)25 * c->lay.maxN * sizeof(double);
    if (smem_asm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(j0_dense_assemble_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_asm);
        if (e != cudaSuccess) return e;
    }
    j0_dense_assemble_kernel<<<c->lay.M, kAsmThreads, smem_asm, c->stream>>>(
        c->lay, c->jofs, X, c->qc, c->Yc, c->Tint, dp, c->jdense);
    const size_t smem_lu = (size_t)6 * c->lay.maxN * sizeof(double);
    if (smem_lu > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(dense_lu_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_lu);
        if (e != cudaSuccess) return e;
    }
    dense_lu_kernel<<<c->lay.M, kLuThreads, smem_lu, c->stream>>>(c->lay, c->jofs, c->jdense,
                                                                   c->piv, c->d_flags);
    c->n_launches += 2;
    return cudaGetLastError();
}

cudaError_t j0_dense_solve(fil_ctx *c, const double *b, double *x) {
    const int zmax = 6 * c->lay.maxN;
    const size_t per_warp = (size_t)zmax * sizeof(double);
    int warps = (int)std::min<size_t>(4, kSolveSmemMax / per_warp);
    if (warps < 1) return cudaErrorInvalidValue;
    const size_t smem = warps * per_warp;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(dense_solve_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = 32 * warps;
    const unsigned grid = (unsigned)(((int64_t)c->lay.M * 32 + threads - 1) / threads);
    dense_solve_kernel<<<grid, threads, smem, c->stream>>>(c->lay, c->jofs, c->jdense, c->piv, b,
                                                           x, zmax);
    c->n_launches += 1;
    return cudaGetLastError();
}

}  // namespace fil
