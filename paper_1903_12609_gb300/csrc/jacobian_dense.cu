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
// Storage: row-major (6N)^2 FP64 block per filament at jofs[i] (kept for the
// refinement residuals) and its inverse in FP32 at the same offsets, computed
// by Gauss-Jordan elimination with partial pivoting in shared memory (one CTA
// per filament; FP32 runs at 64x the FP64 rate on this part). A solve applies
// the FP32 inverse and then kJ0Refine steps of iterative refinement with FP64
// residuals b - J0 x, which brings x to FP64 accuracy (each step multiplies
// the error by ~cond(J0) * 2^-24).
#include <cuda_runtime.h>

#include <algorithm>

#include "fil_internal.cuh"
#include "j0_common.cuh"
#include "quat.cuh"

namespace fil {
namespace {

constexpr int kAsmThreads = 256;
constexpr int kInvThreads = 512;
constexpr int kMaxInvN = 6 * kMaxDenseSeg;   // rows of the largest inverted block

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
    // per-pair RPY coefficients and per-joint moment derivatives, computed once
    PairCoef *pc = reinterpret_cast<PairCoef *>(sm + 25 * N);      // N*N entries
    M33 *DaJ = reinterpret_cast<M33 *>(sm + 25 * N + 5 * N * N);    // N-1 joints
    M33 *DbJ = DaJ + (N > 1 ? N - 1 : 0);
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int n = e / N, m = e - (e / N) * N;
        pc[e] = pair_coef(ld3(g.Y + 3 * n) - ld3(g.Y + 3 * m), dp.a);
    }
    for (int jn = threadIdx.x; jn < N - 1; jn += blockDim.x)
        moment_derivs(dp.jp, ld4(g.Q + 4 * jn), ld4(g.Q + 4 * (jn + 1)), DaJ[jn], DbJ[jn]);
    __syncthreads();
    // angular velocity of the internal loads, filament block only
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        V3 V = v3(0, 0, 0), W = v3(0, 0, 0);
        const V3 Yn = ld3(g.Y + 3 * n);
        for (int m = 0; m < N; ++m) {
            const V3 d = Yn - ld3(g.Y + 3 * m);
            apply_pair(pc[n * N + m], d, ld3(g.Fi + 3 * m), ld3(g.Ti + 3 * m), V, W);
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
            for (int mm = -1; mm <= 1; ++mm) {
                const int m = k + mm;
                if (m < 0 || m > N - 1) continue;
                M33 Gt;
                if (mm == -1) {
                    Gt = DbJ[k - 1];
                } else if (mm == 0) {
                    Gt = mscale(mmul(rskew(ld3(g.Ls + 3 * k)), rskew(ld3(g.t + 3 * k))),
                                0.5 * dp.jp.dL);
                    if (k <= N - 2) Gt = madd(Gt, DaJ[k]);
                    if (k >= 1) Gt = madd(Gt, DbJ[k - 1], -1.0);
                } else {
                    Gt = mscale(DaJ[k], -1.0);
                }
                const V3 d = Yn - ld3(g.Y + 3 * m);
                const PairCoef kc = pc[n * N + m];
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
                const PairCoef kc = pc[n * N + m];
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

// Inverse of each filament's J0 in FP32 by Gauss-Jordan elimination with
// partial pivoting, in place in shared memory (one CTA per filament). Step k:
//   (1) save column k (colk) and zero it in the matrix;
//   (2) one warp finds the pivot row p (first maximal |a_ik|, i >= k);
//   (3) form the scaled pivot row pr = row p / pivot with entry k = 1/pivot,
//       and keep row k (krow) if it is displaced (p != k);
//   (4) row k <- pr; every other row i <- row - a_ik pr, where row p starts
//       from krow and uses the old a_kk (the swap), which also leaves
//       -a_ik / pivot in column k.
// Four barriers per step. Row swaps are undone as column swaps at the end.
// Threads own column chunks c = lane + 32 jj (jj < NCH, pr in registers) and
// rows i = warp + nwarps * r.
template <int NCH>
__global__ void __launch_bounds__(kInvThreads)
gauss_jordan_inverse_kernel(Layout lay, const int64_t *__restrict__ jofs,
                            const double *__restrict__ J_all, float *__restrict__ inv_all,
                            int *__restrict__ flags) {
    extern __shared__ float Asm[];                  // n rows of stride ld = n + 1
    __shared__ float colk[kMaxInvN];
    __shared__ float pr_s[kMaxInvN];
    __shared__ float krow[kMaxInvN];
    __shared__ int perm[kMaxInvN];
    __shared__ int pos[kMaxInvN];
    __shared__ int s_p;
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    const int n = 6 * (lay.off[f + 1] - s0);
    const double *J = J_all + jofs[f];
    float *out = inv_all + jofs[f];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = (int)(blockDim.x >> 5);
    const int ld = n + 1;   // odd stride: column accesses hit distinct banks
    for (int i = wid; i < n; i += nw)
        for (int c = lane; c < n; c += 32) Asm[i * ld + c] = (float)J[(int64_t)i * n + c];
    bool valid[NCH];
#pragma unroll
    for (int jj = 0; jj < NCH; ++jj) valid[jj] = (lane + 32 * jj) < n;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        for (int i = tid; i < n; i += blockDim.x) {
            colk[i] = Asm[i * ld + k];
            Asm[i * ld + k] = 0.f;
        }
        __syncthreads();
        if (wid == 0) {
            float v = -1.f;
            int idx = 0x7fffffff;
            for (int i = k + lane; i < n; i += 32) {
                const float x = fabsf(colk[i]);
                if (x > v) { v = x; idx = i; }
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const float ov = __shfl_down_sync(0xffffffffu, v, d);
                const int oi = __shfl_down_sync(0xffffffffu, idx, d);
                if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
            }
            if (lane == 0) {
                s_p = idx;
                perm[k] = idx;
                if (!(v > 0.f)) atomicOr(flags + 1, 1);
            }
        }
        __syncthreads();
        const int p = s_p;
        const float pinv = 1.f / colk[p];
        for (int c = tid; c < n; c += blockDim.x) {
            pr_s[c] = (c == k) ? pinv : Asm[p * ld + c] * pinv;
            krow[c] = Asm[k * ld + c];
        }
        __syncthreads();
        float pr[NCH];
#pragma unroll
        for (int jj = 0; jj < NCH; ++jj) pr[jj] = valid[jj] ? pr_s[lane + 32 * jj] : 0.f;
        for (int i = wid; i < n; i += nw) {
            float *row = Asm + i * ld + lane;
            if (i == k) {
#pragma unroll
                for (int jj = 0; jj < NCH; ++jj)
                    if (valid[jj]) row[32 * jj] = pr[jj];
            } else if (i == p) {
                const float mf = -colk[k];
#pragma unroll
                for (int jj = 0; jj < NCH; ++jj)
                    if (valid[jj]) row[32 * jj] = fmaf(mf, pr[jj], krow[lane + 32 * jj]);
            } else {
                const float mf = -colk[i];
#pragma unroll
                for (int jj = 0; jj < NCH; ++jj)
                    if (valid[jj]) row[32 * jj] = fmaf(mf, pr[jj], row[32 * jj]);
            }
        }
        __syncthreads();
    }
    // row interchanges undone as column interchanges, last first: column c of
    // the result is column idx[c] of the current matrix; pos is its inverse
    if (tid == 0) {
        for (int c = 0; c < n; ++c) krow[c] = __int_as_float(c);
        for (int k = n - 1; k >= 0; --k) {
            const float t = krow[k];
            krow[k] = krow[perm[k]];
            krow[perm[k]] = t;
        }
        for (int c = 0; c < n; ++c) pos[__float_as_int(krow[c])] = c;
    }
    __syncthreads();
    for (int i = wid; i < n; i += nw)
        for (int c = lane; c < n; c += 32) out[(int64_t)i * n + pos[c]] = Asm[i * ld + c];
}

// Register-resident Gauss-Jordan inverse for blocks of n <= 192 (N <= 32),
// with implicit pivoting. Thread (w, l) of 16 warps holds rows i = w + 16 r
// (r < 12) and columns c = l + 32 j (j < 6) in registers. Step k pivots column
// k on the unused row p of largest |a_pk| (recorded, never swapped) and applies
//   a_i <- s_i a_i + t_i pr,   pr = row p / a_pk with entry k = 1/a_pk,
// with (s, t) = (0, 1) for row p and (1, -a_ik) otherwise, after column k has
// been zeroed -- the in-place Gauss-Jordan update, uniform over all rows. The
// step loop is unrolled over the six 32-column chunks so that column k has a
// static register index. The result is A^{-1} with rows and columns permuted:
// A^{-1}[k][m] = S[p_k][q(m)], p_k the pivot row of column k and q its inverse.
constexpr int kGjWarps = 16, kGjRows = 12, kGjCols = 6, kGjMaxN = 32 * kGjCols;  // 192

__global__ void __launch_bounds__(32 * kGjWarps, 1)
gauss_jordan_inverse_reg_kernel(Layout lay, const int64_t *__restrict__ jofs,
                                const double *__restrict__ J_all, float *__restrict__ inv_all,
                                int *__restrict__ flags) {
    __shared__ float colk[kGjMaxN];
    __shared__ float prow[kGjMaxN];
    __shared__ int used[kGjMaxN];
    __shared__ int pivrow[kGjMaxN];
    __shared__ int qinv[kGjMaxN];
    __shared__ int s_p;
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    const int n = 6 * (lay.off[f + 1] - s0);
    const double *J = J_all + jofs[f];
    float *out = inv_all + jofs[f];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float a[kGjRows][kGjCols];
#pragma unroll
    for (int r = 0; r < kGjRows; ++r)
#pragma unroll
        for (int j = 0; j < kGjCols; ++j) {
            const int i = wid + kGjWarps * r, c = lane + 32 * j;
            a[r][j] = (i < n && c < n) ? (float)J[(int64_t)i * n + c] : 0.f;
        }
    for (int i = tid; i < kGjMaxN; i += blockDim.x) used[i] = (i < n) ? 0 : 1;
    __syncthreads();
#pragma unroll
    for (int kj = 0; kj < kGjCols; ++kj) {
        for (int kl = 0; kl < 32; ++kl) {
            const int k = 32 * kj + kl;
            if (k >= n) break;
            // (1) column k -> colk (held by lane kl), then zero it
            if (lane == kl) {
#pragma unroll
                for (int r = 0; r < kGjRows; ++r) {
                    colk[wid + kGjWarps * r] = a[r][kj];
                    a[r][kj] = 0.f;
                }
            }
            __syncthreads();
            // (2) pivot: unused row of largest |a_ik| (first such), by warp 0
            if (wid == 0) {
                float v = -1.f;
                int idx = 0x7fffffff;
                for (int i = lane; i < n; i += 32) {
                    const float x = used[i] ? -1.f : fabsf(colk[i]);
                    if (x > v) { v = x; idx = i; }
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    const float ov = __shfl_down_sync(0xffffffffu, v, d);
                    const int oi = __shfl_down_sync(0xffffffffu, idx, d);
                    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
                }
                if (lane == 0) {
                    s_p = idx;
                    pivrow[k] = idx;
                    used[idx] = 1;
                    if (!(v > 0.f)) atomicOr(flags + 1, 1);
                }
            }
            __syncthreads();
            const int p = s_p;
            // (3) row p -> prow (its owner warp; static registers, predicated stores)
            if (wid == p % kGjWarps) {
                const int pr = p / kGjWarps;
#pragma unroll
                for (int r = 0; r < kGjRows; ++r)
                    if (r == pr)
#pragma unroll
                        for (int j = 0; j < kGjCols; ++j) prow[lane + 32 * j] = a[r][j];
            }
            __syncthreads();
            // (4) a_i <- s_i a_i + t_i pr for every row
            const float pinv = 1.f / colk[p];
            float pr_r[kGjCols];
#pragma unroll
            for (int j = 0; j < kGjCols; ++j) {
                const int c = lane + 32 * j;
                pr_r[j] = (c == k) ? pinv : prow[c] * pinv;
            }
#pragma unroll
            for (int r = 0; r < kGjRows; ++r) {
                const int i = wid + kGjWarps * r;
                const float sc = (i == p) ? 0.f : 1.f;
                const float t = (i == p) ? 1.f : -colk[i];
#pragma unroll
                for (int j = 0; j < kGjCols; ++j) a[r][j] = fmaf(t, pr_r[j], sc * a[r][j]);
            }
            __syncthreads();
        }
    }
    // A^{-1}[k][m] = S[p_k][q(m)]: element S[i][c] goes to out[q(i)][p_c]
    for (int k = tid; k < n; k += blockDim.x) qinv[pivrow[k]] = k;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kGjRows; ++r)
#pragma unroll
        for (int j = 0; j < kGjCols; ++j) {
            const int i = wid + kGjWarps * r, c = lane + 32 * j;
            if (i < n && c < n) out[(int64_t)qinv[i] * n + pivrow[c]] = a[r][j];
        }
}

// Refined solve, as grid-wide GEMV phases over every row of every filament
// (one warp per row, lanes stride the columns with coalesced loads):
//   x = Inv b;  then kJ0Refine times:  r = b - J0 x (FP64);  x += Inv r.
__global__ void inv_apply_kernel(Layout lay, const int64_t *__restrict__ jofs,
                                 const float *__restrict__ inv_all, const float *__restrict__ r,
                                 double *__restrict__ x, int accumulate) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= lay.nX) return;
    const int f = lay.fil_of[row / 6];
    const int64_t r0 = 6 * (int64_t)lay.off[f];
    const int n = (int)(6 * (int64_t)lay.off[f + 1] - r0);
    const int i = (int)(row - r0);
    const float *A = inv_all + jofs[f] + (int64_t)i * n;
    const float *rf = r + r0;
    float t = 0.f;
    for (int c = lane; c < n; c += 32) t = fmaf(A[c], rf[c], t);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
    if (lane == 0) x[row] = accumulate ? x[row] + (double)t : (double)t;
}

__global__ void to_float_kernel(int64_t n, const double *__restrict__ b, double *__restrict__ bb,
                                float *__restrict__ r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = b[i];
        bb[i] = v;
        r[i] = (float)v;
    }
}

__global__ void residual_gemv_kernel(Layout lay, const int64_t *__restrict__ jofs,
                                     const double *__restrict__ J_all, const double *__restrict__ b,
                                     const double *__restrict__ x, float *__restrict__ r) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= lay.nX) return;
    const int f = lay.fil_of[row / 6];
    const int64_t r0 = 6 * (int64_t)lay.off[f];
    const int n = (int)(6 * (int64_t)lay.off[f + 1] - r0);
    const int i = (int)(row - r0);
    const double *A = J_all + jofs[f] + (int64_t)i * n;
    const double *xf = x + r0;
    double t = 0.0;
    for (int c = lane; c < n; c += 32) t = fma(A[c], xf[c], t);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
    if (lane == 0) r[row] = (float)(b[row] - t);
}

}  // namespace

template <int NCH>
cudaError_t launch_gj(fil_ctx *c, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(gauss_jordan_inverse_kernel<NCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gauss_jordan_inverse_kernel<NCH><<<c->lay.M, kInvThreads, smem, c->stream>>>(
        c->lay, c->jofs, c->jdense, c->jinv, c->d_flags);
    return cudaGetLastError();
}

cudaError_t launch_gauss_jordan(fil_ctx *c, int nch, size_t smem) {
    switch (nch) {
        case 1: return launch_gj<1>(c, smem);
        case 2: return launch_gj<2>(c, smem);
        case 3: return launch_gj<3>(c, smem);
        case 4: return launch_gj<4>(c, smem);
        case 5: return launch_gj<5>(c, smem);
        case 6: return launch_gj<6>(c, smem);
        case 7: return launch_gj<7>(c, smem);
        case 8: return launch_gj<8>(c, smem);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t j0_dense_build_factor(fil_ctx *c, const double *X) {
    const double beta = c->have_prev ? 2.0 / 3.0 : 1.0;
    DenseParams dp;
    dp.jp = J0Params{c->dL, c->KB, c->KT, c->g0, c->kmu, c->knu, 0.0, 0.0};
    dp.bdt = beta * c->dt;
    dp.inv8pieta = 1.0 / (8.0 * kPi * c->eta);
    dp.near2 = 4.0 * c->a * c->a;
    dp.a = c->a;
    const int N = c->lay.maxN;
    const size_t smem_asm = (size_t)(25 * N + 5 * N * N) * sizeof(double) +
                            (size_t)2 * (N > 1 ? N - 1 : 0) * sizeof(M33);
    cudaError_t e = cudaFuncSetAttribute(j0_dense_assemble_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_asm);
    if (e != cudaSuccess) return e;
    j0_dense_assemble_kernel<<<c->lay.M, kAsmThreads, smem_asm, c->stream>>>(
        c->lay, c->jofs, X, c->qc, c->Yc, c->Tint, dp, c->jdense);
#ifndef FIL_GJ_SHARED_ONLY
    if (6 * N <= kGjMaxN) {
        gauss_jordan_inverse_reg_kernel<<<c->lay.M, 32 * kGjWarps, 0, c->stream>>>(
            c->lay, c->jofs, c->jdense, c->jinv, c->d_flags);
        e = cudaGetLastError();
    } else
#endif
    {
        const size_t smem_inv = (size_t)6 * N * (6 * N + 1) * sizeof(float);
        e = launch_gauss_jordan(c, (6 * N + 31) / 32, smem_inv);
    }
    if (e != cudaSuccess) return e;
    c->n_launches += 2;
    return cudaGetLastError();
}

cudaError_t j0_dense_solve(fil_ctx *c, const double *b, double *x) {
    // b and x may alias: b is copied into the refinement scratch first
    const int64_t nX = c->lay.nX;
    const unsigned grid = (unsigned)((nX * 32 + 255) / 256);
    double *bb = c->j0_rhs, *xx = c->j0_x;
    float *rr = reinterpret_cast<float *>(c->j0_res);
    to_float_kernel<<<(unsigned)((nX + 255) / 256), 256, 0, c->stream>>>(nX, b, bb, rr);
    inv_apply_kernel<<<grid, 256, 0, c->stream>>>(c->lay, c->jofs, c->jinv, rr, xx, 0);
    for (int it = 0; it < kJ0Refine; ++it) {
        residual_gemv_kernel<<<grid, 256, 0, c->stream>>>(c->lay, c->jofs, c->jdense, bb, xx, rr);
        inv_apply_kernel<<<grid, 256, 0, c->stream>>>(c->lay, c->jofs, c->jinv, rr, xx, 1);
    }
    cudaError_t e = cudaMemcpyAsync(x, xx, sizeof(double) * nX, cudaMemcpyDeviceToDevice,
                                    c->stream);
    c->n_launches += 2 + 2 * kJ0Refine;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

size_t j0_dense_smem_needed(int maxN) {
    const size_t a = (size_t)(25 * maxN + 5 * maxN * maxN) * sizeof(double) +
                     (size_t)2 * maxN * sizeof(M33);
    const size_t b = (size_t)6 * maxN * (6 * maxN + 1) * sizeof(float);
    return a > b ? a : b;
}

}  // namespace fil
