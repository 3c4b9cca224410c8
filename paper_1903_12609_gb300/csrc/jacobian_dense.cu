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
// Per step and filament:
//   1. j0_precompute_kernel (FP64): frames, Lambda sums, dexpinv matrices A_n,
//      the u-diagonal dexpinv terms Du_n, the load derivatives dT_m/du_m, the
//      joint moment derivatives Da, Db, the angular velocity of the internal
//      loads and every pair's RPY coefficients -> a per-filament aux block.
//   2. j0_assemble32_kernel (FP32): the (6N)^2 matrix J0 from the aux block,
//      written into the inverse buffer and inverted there in FP32 by
//      Gauss-Jordan elimination (FP32 runs at 64x the FP64 rate on this part).
// A solve (j0_solve_fused_kernel, one CTA per filament, the FP32 inverse
// streamed from global memory) applies the inverse and then, in FP64 mode,
// kJ0Refine steps of iterative refinement x += Inv (b - J0 x), with b - J0 x
// evaluated matrix-free in FP64 from the aux block -- the same operator as the
// dense definition -- so x reaches FP64 accuracy (each step multiplies the
// error by ~cond(J0) * 2^-24). In mixed mode (FP32 pair sums, Broyden
// tolerances of ~1e-4) the FP32 solve (relative error ~1e-7, far below the
// error of J0 as an approximation of the Jacobian) is used as it is.
#include <cuda_runtime.h>

#include <algorithm>

#include "fil_internal.cuh"
#include "j0_common.cuh"
#include "quat.cuh"
#include "rpy_pair.cuh"


namespace fil {
namespace {

constexpr int kAsmThreads = 256;
constexpr int kGemvRows = 4;   // rows per warp in flight in the streamed inverse apply
constexpr int kInvThreads = 512;
constexpr int kMaxInvN = 6 * kMaxDenseSeg;   // rows of the largest inverted block

struct DenseParams {
    J0Params jp;
    double bdt;            // (scheme weight) * dt
    double inv8pieta;      // 1 / (8 pi eta)
    double near2;          // (2a)^2
    double a;
};

// Aux block of one filament with N segments, 60 N + 5 N^2 doubles, offsets in units of N:
//   t 3N | Ls 3N | u 3N | Om 3N | Y 3N | A 9N | Du 9N | dTmm 9N | Da 9N | Db 9N | pc 5N^2
// (everything at the X where J0 was built: the solves of later iterates must
// apply the same operator)
// (Da, Db: joint m between segments m and m+1; pc[n N + m] = A,B,C,D,G of the
// pair (n, m) in units of 1/(8 pi eta)).
struct AuxView {
    double *t, *Ls, *u, *Om, *Y, *A, *Du, *dT, *Da, *Db, *pc;
};
__device__ __forceinline__ AuxView aux_view(double *base, int N) {
    AuxView v;
    v.t = base; v.Ls = base + 3 * N; v.u = base + 6 * N; v.Om = base + 9 * N;
    v.Y = base + 12 * N; v.A = base + 15 * N; v.Du = base + 24 * N; v.dT = base + 33 * N;
    v.Da = base + 42 * N; v.Db = base + 51 * N; v.pc = base + 60 * N;
    return v;
}
__device__ __forceinline__ void st33(double *p, const M33 &m) {
#pragma unroll
    for (int i = 0; i < 9; ++i) p[i] = m.m[i];
}
__device__ __forceinline__ M33 ld33(const double *p) {
    M33 m;
#pragma unroll
    for (int i = 0; i < 9; ++i) m.m[i] = p[i];
    return m;
}
__device__ __forceinline__ V3 mv(const M33 &m, V3 v) {
    return {m.m[0] * v.x + m.m[1] * v.y + m.m[2] * v.z, m.m[3] * v.x + m.m[4] * v.y + m.m[5] * v.z,
            m.m[6] * v.x + m.m[7] * v.y + m.m[8] * v.z};
}

// FP32 forms of pair_coef / apply_pair for the mixed mode's J0 (same branches).
struct PairCoef32 {
    float A, B, C, D, G;
};

__device__ __forceinline__ PairCoef32 pair_coef32(float dx, float dy, float dz, float a) {
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    PairCoef32 k;
    if (r2 < 4.f * a * a) {
        const float r = sqrtf(r2);
        const float rinv = r > 0.f ? 1.f / r : 0.f;
        const float ia3 = 1.f / (a * a * a);
        k.A = (4.f / (3.f * a)) * (1.f - 9.f * r / (32.f * a));
        k.B = rinv / (8.f * a * a);
        k.C = ia3 * (1.f - 27.f * r / (32.f * a) + 5.f * r * r2 / (64.f * a * a * a));
        k.D = ia3 * (9.f * rinv / (32.f * a) - 3.f * r / (64.f * a * a * a));
        k.G = 0.5f * ia3 * (1.f - 3.f * r / (8.f * a));
    } else {
        const float rinv = rsqrtf(r2);
        const float rinv2 = rinv * rinv, rinv3 = rinv * rinv2, rinv5 = rinv3 * rinv2;
        k.A = rinv + (2.f * a * a / 3.f) * rinv3;
        k.B = rinv3 - 2.f * a * a * rinv5;
        k.C = -0.5f * rinv3;
        k.D = 1.5f * rinv5;
        k.G = rinv3;
    }
    return k;
}

// Separation component of segments i, j from positions relative to segment 0
// split into FP32 hi + lo parts: the hi difference is exact for nearby
// segments, so d carries the rounding of d itself, not of |Y - Y_0|.
__device__ __forceinline__ float dif_hl(const float *h, const float *l, int i, int j) {
    return __fadd_rn(__fsub_rn(h[i], h[j]), __fsub_rn(l[i], l[j]));
}

// FP64 work per filament (one CTA per filament). fast (the mixed mode, whose
// J0 is used only through its FP32 assembly): the two N^2 loops -- pair
// coefficients and the angular velocity of the internal loads -- in FP32.
__global__ void __launch_bounds__(kAsmThreads)
j0_precompute_kernel(Layout lay, const int64_t *__restrict__ auxofs, const double *__restrict__ X,
                     const double *__restrict__ qc, const double *__restrict__ Yc,
                     const double *__restrict__ Tint, DenseParams dp, double *__restrict__ aux_all,
                     int fast) {
    // F_int 3N | Yrel 3N (doubles), then for fast: Y hi 3N | Y lo 3N | F_int 3N | T_int 3N |
    // pc 5N^2 (floats)
    extern __shared__ double sm[];
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    const int N = lay.off[f + 1] - s0;
    AuxView g = aux_view(aux_all + auxofs[f], N);
    double *Fi = sm, *Yf = sm + 3 * N;
    float *Y32 = reinterpret_cast<float *>(sm + 6 * N), *Yl32 = Y32 + 3 * N, *F32 = Yl32 + 3 * N,
          *T32 = F32 + 3 * N, *pc32 = T32 + 3 * N;
    const double *Xf = X + 6 * (int64_t)s0;
    const double *Lam = Xf + 3 + 3 * N;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int64_t gg = s0 + n;
        st3(g.t + 3 * n, frame_t(ld4(qc + 4 * gg)));
        const V3 u = ld3(Xf + 3 + 3 * n);
        st3(g.u + 3 * n, u);
        const V3 Lr = (n <= N - 2) ? ld3(Lam + 3 * n) : v3(0, 0, 0);
        const V3 Ll = (n >= 1) ? ld3(Lam + 3 * (n - 1)) : v3(0, 0, 0);
        st3(g.Ls + 3 * n, Lr + Ll);
        st3(Fi + 3 * n, Lr - Ll);
        st3(Yf + 3 * n, ld3(Yc + 3 * gg));
        st3(g.Y + 3 * n, ld3(Yc + 3 * gg));
        const M33 ux = skew(u);
        st33(g.A + 9 * n, madd(madd(meye(), ux, -0.5), mmul(ux, ux), 1.0 / 12.0));
        if (n <= N - 2) {
            M33 Da, Db;
            moment_derivs(dp.jp, ld4(qc + 4 * gg), ld4(qc + 4 * (gg + 1)), Da, Db);
            st33(g.Da + 9 * n, Da);
            st33(g.Db + 9 * n, Db);
        }
    }
    __syncthreads();
    if (fast) {
        for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) {
            const double yr = Yf[e] - Yf[e % 3];         // relative to segment 0
            Y32[e] = (float)yr;
            Yl32[e] = (float)(yr - (double)Y32[e]);
            F32[e] = (float)Fi[e];
            T32[e] = (float)Tint[3 * (int64_t)s0 + e];
        }
        __syncthreads();
        const float a32 = (float)dp.a;
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int n = e / N, m = e - (e / N) * N;
            if (m < n) continue;
            const PairCoef32 k = pair_coef32(dif_hl(Y32, Yl32, 3 * n, 3 * m),
                                             dif_hl(Y32, Yl32, 3 * n + 1, 3 * m + 1),
                                             dif_hl(Y32, Yl32, 3 * n + 2, 3 * m + 2), a32);
            const float v[5] = {k.A, k.B, k.C, k.D, k.G};
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                pc32[5 * e + c] = v[c];
                g.pc[5 * (int64_t)e + c] = (double)v[c];
            }
            if (m != n) {
                const int et = m * N + n;
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    pc32[5 * et + c] = v[c];
                    g.pc[5 * (int64_t)et + c] = (double)v[c];
                }
            }
        }
        __syncthreads();
        for (int base = 0; base < N; base += (int)blockDim.x / 8) {
            const int n = base + (int)threadIdx.x / 8;
            const int sub = threadIdx.x & 7;
            float Wx = 0.f, Wy = 0.f, Wz = 0.f;
            if (n < N) {
                for (int m = sub; m < N; m += 8) {
                    const float *pc = pc32 + 5 * (n * N + m);
                    const float dx = dif_hl(Y32, Yl32, 3 * n, 3 * m),
                                dy = dif_hl(Y32, Yl32, 3 * n + 1, 3 * m + 1),
                                dz = dif_hl(Y32, Yl32, 3 * n + 2, 3 * m + 2);
                    const float vx = F32[3 * m], vy = F32[3 * m + 1], vz = F32[3 * m + 2];
                    const float wx = T32[3 * m], wy = T32[3 * m + 1], wz = T32[3 * m + 2];
                    // Omega += G (v x d) + C w + D (d.w) d
                    const float dw = pc[3] * fmaf(dx, wx, fmaf(dy, wy, dz * wz));
                    Wx += pc[4] * (vy * dz - vz * dy) + pc[2] * wx + dw * dx;
                    Wy += pc[4] * (vz * dx - vx * dz) + pc[2] * wy + dw * dy;
                    Wz += pc[4] * (vx * dy - vy * dx) + pc[2] * wz + dw * dz;
                }
            }
#pragma unroll
            for (int d = 4; d > 0; d >>= 1) {
                Wx += __shfl_xor_sync(0xffffffffu, Wx, d);
                Wy += __shfl_xor_sync(0xffffffffu, Wy, d);
                Wz += __shfl_xor_sync(0xffffffffu, Wz, d);
            }
            if (n < N && sub == 0) st3(g.Om + 3 * n, dp.inv8pieta * v3(Wx, Wy, Wz));
        }
        __syncthreads();
    } else {
    // the coefficients depend on r only: each unordered pair once, stored twice
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int n = e / N, m = e - (e / N) * N;
        if (m < n) continue;
        const PairCoef k = pair_coef(ld3(Yf + 3 * n) - ld3(Yf + 3 * m), dp.a);
        double *pc = g.pc + 5 * (int64_t)e;
        pc[0] = k.A; pc[1] = k.B; pc[2] = k.C; pc[3] = k.D; pc[4] = k.G;
        if (m != n) {
            double *pt = g.pc + 5 * ((int64_t)m * N + n);
            pt[0] = k.A; pt[1] = k.B; pt[2] = k.C; pt[3] = k.D; pt[4] = k.G;
        }
    }
    __syncthreads();
    // angular velocity of the internal loads within the filament: 8 lanes per
    // target, reduced with shuffles in a fixed order
    for (int base = 0; base < N; base += (int)blockDim.x / 8) {
        const int n = base + (int)threadIdx.x / 8;
        const int sub = threadIdx.x & 7;
        V3 W = v3(0, 0, 0);
        if (n < N) {
            V3 V = v3(0, 0, 0);
            const V3 Yn = ld3(Yf + 3 * n);
            for (int m = sub; m < N; m += 8) {
                const double *pc = g.pc + 5 * ((int64_t)n * N + m);
                const PairCoef k{pc[0], pc[1], pc[2], pc[3], pc[4]};
                apply_pair(k, Yn - ld3(Yf + 3 * m), ld3(Fi + 3 * m),
                           ld3(Tint + 3 * (int64_t)(s0 + m)), V, W);
            }
        }
#pragma unroll
        for (int d = 4; d > 0; d >>= 1) {
            W.x += __shfl_xor_sync(0xffffffffu, W.x, d);
            W.y += __shfl_xor_sync(0xffffffffu, W.y, d);
            W.z += __shfl_xor_sync(0xffffffffu, W.z, d);
        }
        if (n < N && sub == 0) st3(g.Om + 3 * n, dp.inv8pieta * W);
    }
    __syncthreads();
    }
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        // dT_n/du_n = (dL/2)[x Ls][x t] + Da(n) - Db(n-1)
        M33 dT = mscale(mmul(rskew(ld3(g.Ls + 3 * n)), rskew(ld3(g.t + 3 * n))), 0.5 * dp.jp.dL);
        if (n <= N - 2) dT = madd(dT, ld33(g.Da + 9 * n));
        if (n >= 1) dT = madd(dT, ld33(g.Db + 9 * (n - 1)), -1.0);
        st33(g.dT + 9 * n, dT);
        const V3 Om = ld3(g.Om + 3 * n);
        const V3 u = ld3(g.u + 3 * n);
        const M33 ux = skew(u), xO = rskew(Om);
        st33(g.Du + 9 * n, madd(mscale(xO, -0.5), madd(rskew(cross(u, Om)), mmul(ux, xO)), 1.0 / 12.0));
    }
}

// FP32 helpers for the assembly.
struct F3 {
    float x, y, z;
};
__device__ __forceinline__ F3 f3v(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ float fdot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ F3 fcross(F3 a, F3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ F3 fmad3(float s, F3 a, F3 b) {
    return {fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z)};
}
// (V, W) += M_nm (v, w) with FP32 coefficients (units of 1/(8 pi eta))
__device__ __forceinline__ void apply_pair32(const float *c, F3 d, F3 v, F3 w, F3 &V, F3 &W) {
    const float A = c[0], B = c[1], C = c[2], D = c[3], G = c[4];
    V = fmad3(A, v, V);
    V = fmad3(B * fdot(d, v), d, V);
    V = fmad3(G, fcross(w, d), V);
    W = fmad3(G, fcross(v, d), W);
    W = fmad3(C, w, W);
    W = fmad3(D * fdot(d, w), d, W);
}
__device__ __forceinline__ F3 mcol(const float *m9, int c) { return {m9[c], m9[3 + c], m9[6 + c]}; }

// J0 in FP32 from the aux block, written into the inverse buffer (row-major).
__global__ void __launch_bounds__(kAsmThreads)
j0_assemble32_kernel(Layout lay, const int64_t *__restrict__ jofs,
                     const int64_t *__restrict__ auxofs, DenseParams dp, const double *__restrict__ aux_all, float *__restrict__ J_all) {
    extern __shared__ float smf[];     // pc 5N^2 | Yrel hi 3N | lo 3N | t 3N | A, Du, dT, Da, Db 45N
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    const int N = lay.off[f + 1] - s0;
    const int n6 = 6 * N;
    const AuxView g = aux_view(const_cast<double *>(aux_all) + auxofs[f], N);
    float *pcs = smf, *Ys = smf + 5 * N * N, *Yl = Ys + 3 * N, *ts = Yl + 3 * N, *m32 = ts + 3 * N;
    float *A32 = m32, *Du32 = m32 + 9 * N, *dT32 = m32 + 18 * N, *Da32 = m32 + 27 * N,
          *Db32 = m32 + 36 * N;
    float *J = J_all + jofs[f];
    const double *Y0 = g.Y;
    for (int e = threadIdx.x; e < 5 * N * N; e += blockDim.x) pcs[e] = (float)g.pc[e];
    for (int e = threadIdx.x; e < 45 * N; e += blockDim.x) m32[e] = (float)g.A[e];   // A..Db
    for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) {
        const double yr = Y0[e] - Y0[e % 3];    // positions relative to segment 0, hi + lo
        Ys[e] = (float)yr;
        Yl[e] = (float)(yr - (double)Ys[e]);
        ts[e] = (float)g.t[e];
    }
    for (int64_t e = threadIdx.x; e < (int64_t)n6 * n6; e += blockDim.x) J[e] = 0.f;
    __syncthreads();
    const float s = (float)(-dp.bdt * dp.inv8pieta);
    const float hdL = (float)(0.5 * dp.jp.dL);
    const int ncol = 2 * N - 1;
    for (int task = threadIdx.x; task < N * ncol; task += blockDim.x) {
        const int n = task / ncol;
        const int x = task - n * ncol;
        F3 MV[3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        F3 MW[3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        int colX;
        if (x < N) {
            const int k = x;
            colX = 3 + 3 * k;
            for (int mm = -1; mm <= 1; ++mm) {
                const int m = k + mm;
                if (m < 0 || m > N - 1) continue;
                // d T_m / d u_k: Db(k-1) for m = k-1, dT_k for m = k, -Da(k) for m = k+1
                const float *Gt = (mm == -1) ? Db32 + 9 * (k - 1) : (mm == 0) ? dT32 + 9 * k : Da32 + 9 * k;
                const float sg = (mm == 1) ? -1.f : 1.f;
                const F3 d = f3v(dif_hl(Ys, Yl, 3 * n, 3 * m), dif_hl(Ys, Yl, 3 * n + 1, 3 * m + 1),
                                 dif_hl(Ys, Yl, 3 * n + 2, 3 * m + 2));
                const float *c5 = pcs + 5 * (n * N + m);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    F3 w = mcol(Gt, c);
                    w = {sg * w.x, sg * w.y, sg * w.z};
                    apply_pair32(c5, d, f3v(0, 0, 0), w, MV[c], MW[c]);
                }
            }
        } else {
            // d(F_m, T_m)/d Lam_j: F += I (m = j), F -= I (m = j+1); T: (dL/2)[t_m x]
            const int j = x - N;
            colX = 3 + 3 * N + 3 * j;
            for (int mm = 0; mm <= 1; ++mm) {
                const int m = j + mm;
                const F3 tm = f3v(ts[3 * m], ts[3 * m + 1], ts[3 * m + 2]);
                const float sF = mm == 0 ? 1.f : -1.f;
                const F3 d = f3v(dif_hl(Ys, Yl, 3 * n, 3 * m), dif_hl(Ys, Yl, 3 * n + 1, 3 * m + 1),
                                 dif_hl(Ys, Yl, 3 * n + 2, 3 * m + 2));
                const float *c5 = pcs + 5 * (n * N + m);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const F3 e = f3v(c == 0 ? sF : 0.f, c == 1 ? sF : 0.f, c == 2 ? sF : 0.f);
                    // column c of (dL/2)[t_m x] is (dL/2) t_m x e_c
                    const F3 ec = f3v(c == 0 ? 1.f : 0.f, c == 1 ? 1.f : 0.f, c == 2 ? 1.f : 0.f);
                    F3 w = fcross(tm, ec);
                    w = {hdL * w.x, hdL * w.y, hdL * w.z};
                    apply_pair32(c5, d, e, w, MV[c], MW[c]);
                }
            }
        }
        const int prow = (n == 0) ? 0 : 3 + 3 * N + 3 * (n - 1);
        const int rrow = 3 + 3 * n;
        const float *An = A32 + 9 * n;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float *Jp = J + (int64_t)prow * n6 + colX + c;
            Jp[0] = s * MV[c].x;
            Jp[n6] = s * MV[c].y;
            Jp[2 * n6] = s * MV[c].z;
            float *Jr = J + (int64_t)rrow * n6 + colX + c;
#pragma unroll
            for (int r = 0; r < 3; ++r)
                Jr[r * n6] = s * (An[3 * r] * MW[c].x + An[3 * r + 1] * MW[c].y +
                                  An[3 * r + 2] * MW[c].z);
        }
        if (x < N) {
            const int k = x;
            if (n >= 1 && k <= n) {
                // robot-arm term (dL/2) w [x t_k], w = 1 at k = 0 and k = n, else 2
                const float wgt = (k == 0 || k == n) ? hdL : 2.f * hdL;
                const F3 tk = f3v(ts[3 * k], ts[3 * k + 1], ts[3 * k + 2]);
                // [x t] = -[t x]: rows (0, tz, -ty), (-tz, 0, tx), (ty, -tx, 0)
                const float arm[9] = {0.f, tk.z, -tk.y, -tk.z, 0.f, tk.x, tk.y, -tk.x, 0.f};
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c)
                        J[(int64_t)(prow + r) * n6 + colX + c] += wgt * arm[3 * r + c];
            }
            if (k == n) {
                const float *Du = Du32 + 9 * n;
                const float bdt = (float)dp.bdt;
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c)
                        J[(int64_t)(rrow + r) * n6 + colX + c] +=
                            (r == c ? 1.f : 0.f) - bdt * Du[3 * r + c];
            }
        }
    }
    // Y_1 column: identity on every position row
    for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) {
        const int n = e / 3, r = e % 3;
        const int prow = (n == 0) ? 0 : 3 + 3 * N + 3 * (n - 1);
        J[(int64_t)(prow + r) * n6 + r] = 1.f;
    }
}

constexpr int kMfLanes = 16;   // lanes per target in the matrix-free pair sums

// r = b - J0 x for the filament of this CTA, matrix-free in FP64 from the
// aux block (every thread of the CTA calls it; it ends with a barrier):
//   (F, T) = G x, (V, W) = M_f (F, T) (the filament's RPY blocks), then
//   position rows  x_Y1 + arm_n(x_u) - b dt V_n,
//   rotation rows  x_u_n - b dt (A_n W_n + Du_n x_u_n);
// the result is stored in FP32 (it feeds the FP32 inverse). x, b: the
// filament's 6N entries; FT, VW (6N) and Ys (3N) are shared-memory scratch.
__device__ void residual_mf_cta(const AuxView &g, int N, const DenseParams &dp,
                                const double *xf, const double *bf, float *rf, double *FT,
                                double *VW, double *Ys) {
    const double *xu = xf + 3, *xL = xf + 3 + 3 * N;
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        const V3 Lr = (m <= N - 2) ? ld3(xL + 3 * m) : v3(0, 0, 0);
        const V3 Ll = (m >= 1) ? ld3(xL + 3 * (m - 1)) : v3(0, 0, 0);
        V3 T = (0.5 * dp.jp.dL) * cross(ld3(g.t + 3 * m), Lr + Ll);
        T = T + mv(ld33(g.dT + 9 * m), ld3(xu + 3 * m));
        if (m <= N - 2) T = T + mv(ld33(g.Db + 9 * m), ld3(xu + 3 * (m + 1)));
        if (m >= 1) T = T - mv(ld33(g.Da + 9 * (m - 1)), ld3(xu + 3 * (m - 1)));
        st3(FT + 6 * m, Lr - Ll);
        st3(FT + 6 * m + 3, T);
        st3(Ys + 3 * m, ld3(g.Y + 3 * m));
    }
    __syncthreads();
    // pair sums: kMfLanes lanes per target, reduced with shuffles in fixed order
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < N; base += (int)blockDim.x / kMfLanes) {
        const int n = base + (int)threadIdx.x / kMfLanes;
        const int sub = threadIdx.x & (kMfLanes - 1);
        V3 V = v3(0, 0, 0), W = v3(0, 0, 0);
        if (n < N) {
            const V3 Yn = ld3(Ys + 3 * n);
            for (int m = sub; m < N; m += kMfLanes) {
                const double *pc = g.pc + 5 * ((int64_t)n * N + m);
                const PairCoef k{pc[0], pc[1], pc[2], pc[3], pc[4]};
                apply_pair(k, Yn - ld3(Ys + 3 * m), ld3(FT + 6 * m), ld3(FT + 6 * m + 3), V, W);
            }
        }
#pragma unroll
        for (int d = kMfLanes / 2; d > 0; d >>= 1) {
            V.x += __shfl_xor_sync(0xffffffffu, V.x, d);
            V.y += __shfl_xor_sync(0xffffffffu, V.y, d);
            V.z += __shfl_xor_sync(0xffffffffu, V.z, d);
            W.x += __shfl_xor_sync(0xffffffffu, W.x, d);
            W.y += __shfl_xor_sync(0xffffffffu, W.y, d);
            W.z += __shfl_xor_sync(0xffffffffu, W.z, d);
        }
        if (n < N && sub == 0) {
            st3(VW + 6 * n, dp.inv8pieta * V);
            st3(VW + 6 * n + 3, dp.inv8pieta * W);
        }
    }
    __syncthreads();
    // rotation rows
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const V3 un = ld3(xu + 3 * n);
        const V3 rot = un - dp.bdt * (mv(ld33(g.A + 9 * n), ld3(VW + 6 * n + 3)) +
                                      mv(ld33(g.Du + 9 * n), un));
        const V3 bb = ld3(bf + 3 + 3 * n);
        rf[3 + 3 * n] = (float)(bb.x - rot.x);
        rf[3 + 3 * n + 1] = (float)(bb.y - rot.y);
        rf[3 + 3 * n + 2] = (float)(bb.z - rot.z);
    }
    // position rows: arm_n = (dL/2) sum_{k=1}^{n} (x_{k-1} x t_{k-1} + x_k x t_k), by warp 0
    if (threadIdx.x < 32) {
        V3 carry = v3(0, 0, 0), cprev = v3(0, 0, 0);
        const V3 xY = ld3(xf);
        for (int base = 0; base < N; base += 32) {
            const int n = base + lane;
            const bool act = n < N;
            const V3 cn = act ? cross(ld3(xu + 3 * n), ld3(g.t + 3 * n)) : v3(0, 0, 0);
            V3 cp = v3(__shfl_up_sync(0xffffffffu, cn.x, 1), __shfl_up_sync(0xffffffffu, cn.y, 1),
                       __shfl_up_sync(0xffffffffu, cn.z, 1));
            if (lane == 0) cp = cprev;
            V3 inc = (act && n > 0) ? (0.5 * dp.jp.dL) * (cp + cn) : v3(0, 0, 0);
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const V3 o = v3(__shfl_up_sync(0xffffffffu, inc.x, d),
                                __shfl_up_sync(0xffffffffu, inc.y, d),
                                __shfl_up_sync(0xffffffffu, inc.z, d));
                if (lane >= d) inc = inc + o;
            }
            const V3 arm = carry + inc;
            if (act) {
                const V3 pos = xY + arm - dp.bdt * ld3(VW + 6 * n);
                const int prow = (n == 0) ? 0 : 3 + 3 * N + 3 * (n - 1);
                const V3 bb = ld3(bf + prow);
                rf[prow] = (float)(bb.x - pos.x);
                rf[prow + 1] = (float)(bb.y - pos.y);
                rf[prow + 2] = (float)(bb.z - pos.z);
            }
            carry = v3(__shfl_sync(0xffffffffu, arm.x, 31), __shfl_sync(0xffffffffu, arm.y, 31),
                       __shfl_sync(0xffffffffu, arm.z, 31));
            cprev = v3(__shfl_sync(0xffffffffu, cn.x, 31), __shfl_sync(0xffffffffu, cn.y, 31),
                       __shfl_sync(0xffffffffu, cn.z, 31));
        }
    }
    __syncthreads();
}

// x (+)= Inv r for one filament, Inv (n x n, row-major) and r in shared
// memory: warp per row, lanes stride the columns (conflict-free).
// Each warp takes kGemvRows rows at a time, so that a lane has the loads of
// several rows in flight; every row is summed in the same order as one row
// at a time (lane-strided FMAs, then a butterfly over the lanes).
template <int ROWS = kGemvRows>
__device__ __forceinline__ void inv_gemv_cta(const float *Inv, const float *r, double *x, int n,
                                             bool accumulate) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i0 = wid * ROWS; i0 < n; i0 += nw * ROWS) {
        float t[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) t[u] = 0.f;
#pragma unroll 2
        for (int c = lane; c < n; c += 32) {
            const float rc = r[c];
#pragma unroll
            for (int u = 0; u < ROWS; ++u)
                if (i0 + u < n) t[u] = fmaf(Inv[(int64_t)(i0 + u) * n + c], rc, t[u]);
        }
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) t[u] += __shfl_xor_sync(0xffffffffu, t[u], d);
            if (lane == 0 && i0 + u < n) x[i0 + u] = accumulate ? x[i0 + u] + (double)t[u]
                                                               : (double)t[u];
        }
    }
}

// x = Inv b without refinement (the mixed mode): the inverse is read once, so it
// is streamed from global memory instead of being staged in shared memory, and
// small CTAs keep many rows in flight per SM. Same summation order as the first
// product of the fused solve. b and x may alias.
constexpr int kApplyThreads = 256;
__global__ void __launch_bounds__(kApplyThreads)
j0_apply_inverse_kernel(Layout lay, const int64_t *__restrict__ jofs,
                        const float *__restrict__ inv_all, const double *b, double *x,
                        const int *__restrict__ active) {
    __shared__ float rs[6 * kMaxDenseSeg];
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    if (active && !active[lay.sys_of[s0]]) return;   // converged system: rows not needed
    const int n = 6 * (lay.off[f + 1] - s0);
    const double *bg = b + 6 * (int64_t)s0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rs[i] = (float)bg[i];
    __syncthreads();
    inv_gemv_cta<kGemvRows>(inv_all + jofs[f], rs, x + 6 * (int64_t)s0, n, false);
}

// J0 solve, one CTA per filament:  x = Inv b;  `refine` times { r = b - J0 x
// (FP64, matrix-free); x += Inv r }.  The FP32 inverse is read from global
// memory by both products (the second read mostly hits L2) rather than staged
// in shared memory: the CTA then needs a few KB of shared memory, several
// run per SM, and the FP64 residual of one filament overlaps the inverse
// products of others (staging the 147 KB inverse of a 32-segment filament
// allowed one CTA per SM and serialised the two). b and x may alias.
constexpr int kSolveThreads = 256;

__global__ void __launch_bounds__(kSolveThreads)
j0_solve_fused_kernel(Layout lay, const int64_t *__restrict__ jofs,
                      const int64_t *__restrict__ auxofs, DenseParams dp,
                      const double *__restrict__ aux_all, const float *__restrict__ inv_all,
                      const double *b, double *x, const int *__restrict__ active,
                      int refine) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    if (active && !active[lay.sys_of[s0]]) return;   // converged system: rows not needed
    const int N = lay.off[f + 1] - s0;
    const int n = 6 * N;
    const float *Inv = inv_all + jofs[f];
    double *bs = reinterpret_cast<double *>(smraw);
    double *xs = bs + n, *FT = xs + n, *VW = FT + 6 * N, *Ys = VW + 6 * N;
    float *rs = reinterpret_cast<float *>(Ys + 3 * N);
    const AuxView g = aux_view(const_cast<double *>(aux_all) + auxofs[f], N);
    const double *bg = b + 6 * (int64_t)s0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = bg[i];
        bs[i] = v;
        rs[i] = (float)v;
    }
    __syncthreads();
    inv_gemv_cta(Inv, rs, xs, n, false);
    __syncthreads();
    for (int it = 0; it < refine; ++it) {
        residual_mf_cta(g, N, dp, xs, bs, rs, FT, VW, Ys);
        inv_gemv_cta(Inv, rs, xs, n, true);
        __syncthreads();
    }
    double *xg = x + 6 * (int64_t)s0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xg[i] = xs[i];
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
                            const float *J_all, float *inv_all,
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
    const float *J = J_all + jofs[f];   // J0 in FP32, inverted in place
    float *out = inv_all + jofs[f];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = (int)(blockDim.x >> 5);
    const int ld = n + 1;   // odd stride: column accesses hit distinct banks
    for (int i = wid; i < n; i += nw)
        for (int c = lane; c < n; c += 32) Asm[i * ld + c] = J[(int64_t)i * n + c];
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

// Register-resident Gauss-Jordan inverse for blocks of n <= 192 (N <= 32):
// 16 warps per block.
constexpr int kGjWarps = 16, kGjMaxN = 192;

// The in-place Gauss-Jordan inverse with the matrix distributed by
// columns: warp w holds columns w + 16 q (q < 12), lane l rows l + 32 j
// (j < 6), as pairs of columns (w + 32 t, w + 32 t + 16) for the packed FP32
// FMA. The pivot search of step k is one warp's reduction over its column: a
// redux.sync over 32-bit keys, |a_ik| with its 8 low mantissa bits replaced by
// 255 - i, so the first of the rows whose magnitudes agree to 15 significant
// bits wins. The owner of column k publishes the negated column (each entry
// twice, the packed multipliers of the update), the pivot row and 1/pivot;
// after the single CTA barrier of the step every warp takes its part of the
// pivot row from the lane that holds row p, through shared memory, and updates
// its 72 entries. Column and pivot are double buffered.
constexpr int kGcSlots = 6, kGcPairs = 6;    // row slots per lane, column pairs per warp
constexpr int kGcThreads = 32 * kGjWarps;
constexpr int kGcLoad = kGjMaxN * kGjMaxN / kGcThreads;   // elements per thread, load / store
static_assert(32 * kGcSlots == kGjMaxN && kGjWarps * 2 * kGcPairs == kGjMaxN &&
              kGcLoad * kGcThreads == kGjMaxN * kGjMaxN,
              "column-layout Gauss-Jordan covers 192 x 192");

// Row slot j (warp-uniform at run time) of the register array, as a static index.
#define FIL_GC_SLOT_SWITCH(jp, BODY)           \
    switch (jp) {                              \
        case 0: { constexpr int J = 0; BODY } break; \
        case 1: { constexpr int J = 1; BODY } break; \
        case 2: { constexpr int J = 2; BODY } break; \
        case 3: { constexpr int J = 3; BODY } break; \
        case 4: { constexpr int J = 4; BODY } break; \
        default: { constexpr int J = 5; BODY } break; \
    }

__global__ void __launch_bounds__(kGcThreads, 1)
gauss_jordan_inverse_col_kernel(Layout lay, const int64_t *__restrict__ jofs, float *inv_all,
                                int *__restrict__ flags) {
    extern __shared__ float St[];                     // n x (n + 1): staging of the load / store
    __shared__ float4 colk[2][32][kGcSlots / 2];      // -a_{l+32j,k} twice, j = 2 e, 2 e + 1
    __shared__ float4 prow[kGjWarps][kGcPairs / 2];   // pivot row, this warp's column pairs
    __shared__ float2 s_piv[2];                       // (p as bits, 1/pivot)
    __shared__ int pivrow[kGjMaxN];
    __shared__ int qinv[kGjMaxN];
    const int f = blockIdx.x;
    const int s0 = lay.off[f];
    const int n = 6 * (lay.off[f + 1] - s0);
    float *A = inv_all + jofs[f];   // J0 in FP32 on entry, its inverse on exit
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    {
        // element e = tid + kGcThreads r of the row-major matrix is (row, col),
        // stepped by (dq, dr) from r to r + 1
        const int nn = n * n, ld = n + 1;
        const int dq = kGcThreads / n, dr = kGcThreads - dq * n;
        int row = tid / n, col = tid - (tid / n) * n;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            constexpr int kH = kGcLoad / 2;
            float tmp[kH];            // a batch of loads in flight before its stores
#pragma unroll
            for (int r = 0; r < kH; ++r) {
                const int e = tid + kGcThreads * (kH * h + r);
                tmp[r] = e < nn ? A[e] : 0.f;
            }
#pragma unroll
            for (int r = 0; r < kH; ++r) {
                if (tid + kGcThreads * (kH * h + r) < nn) St[row * ld + col] = tmp[r];
                row += dq;
                col += dr;
                if (col >= n) { col -= n; ++row; }
            }
        }
    }
    __syncthreads();
    float2 a[kGcSlots][kGcPairs];     // a[j][t] = (column wid + 32 t, column wid + 32 t + 16)
    unsigned used = 0;                // bit j: row lane + 32 j pivoted, or padding
#pragma unroll
    for (int j = 0; j < kGcSlots; ++j) {
        const int i = lane + 32 * j, ld = n + 1;
        if (i >= n) used |= 1u << j;
#pragma unroll
        for (int t = 0; t < kGcPairs; ++t) {
            const int c0 = wid + 32 * t, c1 = c0 + 16;
            a[j][t].x = (i < n && c0 < n) ? St[i * ld + c0] : 0.f;
            a[j][t].y = (i < n && c1 < n) ? St[i * ld + c1] : 0.f;
        }
    }
    // column k = wid + 16 q  <->  pair t = q / 2, half q & 1
#pragma unroll
    for (int q = 0; q < 2 * kGcPairs; ++q) {
        for (int wk = 0; wk < kGjWarps; ++wk) {
            const int k = wk + 16 * q;
            if (k >= n) break;
            const int buf = k & 1;
            if (wid == wk) {
                unsigned key = 0;
#pragma unroll
                for (int j = 0; j < kGcSlots; ++j) {
                    const float v = (q & 1) ? a[j][q >> 1].y : a[j][q >> 1].x;
                    const unsigned kj =
                        (__float_as_uint(v) & 0x7fffff00u) | (255u - (unsigned)(lane + 32 * j));
                    if (!((used >> j) & 1u)) key = max(key, kj);
                }
                key = __reduce_max_sync(0xffffffffu, key);
                const int p = 255 - (int)(key & 255u);
                // publish the negated column, then zero it
#pragma unroll
                for (int e = 0; e < kGcSlots / 2; ++e) {
                    const float m0 = -((q & 1) ? a[2 * e][q >> 1].y : a[2 * e][q >> 1].x);
                    const float m1 = -((q & 1) ? a[2 * e + 1][q >> 1].y : a[2 * e + 1][q >> 1].x);
                    colk[buf][lane][e] = make_float4(m0, m0, m1, m1);
                }
#pragma unroll
                for (int j = 0; j < kGcSlots; ++j) {
                    if (q & 1) a[j][q >> 1].y = 0.f;
                    else a[j][q >> 1].x = 0.f;
                }
                if (lane == (p & 31)) {
                    float2 *cp = reinterpret_cast<float2 *>(&colk[buf][lane][0]) + (p >> 5);
                    const float v = -cp->x;           // written by this lane just above
                    if (!(fabsf(v) > 0.f)) atomicOr(flags + 1, 1);
                    s_piv[buf] = make_float2(__int_as_float(p), fabsf(v) > 0.f ? __frcp_rn(v) : 0.f);
                    *cp = make_float2(1.f, 1.f);      // multiplier +1: the pivot row becomes pr
                    pivrow[k] = p;
                }
            }
            __syncthreads();
            const float2 piv = s_piv[buf];
            const int p = __float_as_int(piv.x);
            const float2 vinv2 = make_float2(piv.y, piv.y);
            const int src = p & 31, jp = p >> 5;
            if (lane == src) {
                FIL_GC_SLOT_SWITCH(jp,
                    _Pragma("unroll") for (int e = 0; e < kGcPairs / 2; ++e) {
                        prow[wid][e] = make_float4(a[J][2 * e].x, a[J][2 * e].y,
                                                   a[J][2 * e + 1].x, a[J][2 * e + 1].y);
                        a[J][2 * e] = make_float2(0.f, 0.f);
                        a[J][2 * e + 1] = make_float2(0.f, 0.f);
                    })
                used |= 1u << jp;
            }
            __syncwarp();
            // this warp's part of the pivot row, scaled; entry k is 1/pivot
            float2 pr[kGcPairs];
#pragma unroll
            for (int e = 0; e < kGcPairs / 2; ++e) {
                const float4 r4 = prow[wid][e];
                pr[2 * e] = __fmul2_rn(make_float2(r4.x, r4.y), vinv2);
                pr[2 * e + 1] = __fmul2_rn(make_float2(r4.z, r4.w), vinv2);
            }
            if (wid == wk) {
                if (q & 1) pr[q >> 1].y = piv.y;
                else pr[q >> 1].x = piv.y;
            }
            // a_i <- a_i + m_i pr: m_i = -a_ik before the step, +1 for the pivot row
#pragma unroll
            for (int e = 0; e < kGcSlots / 2; ++e) {
                const float4 m4 = colk[buf][lane][e];
                const float2 m0 = make_float2(m4.x, m4.y), m1 = make_float2(m4.z, m4.w);
#pragma unroll
                for (int t = 0; t < kGcPairs; ++t) {
                    a[2 * e][t] = __ffma2_rn(m0, pr[t], a[2 * e][t]);
                    a[2 * e + 1][t] = __ffma2_rn(m1, pr[t], a[2 * e + 1][t]);
                }
            }
        }
    }
    // A^{-1}[R][C] = S[pivrow[R]][qinv[C]], i.e. S[i][c] -> A^{-1}[qinv[i]][pivrow[c]]:
    // scatter S into the staging buffer, then write rows coalesced
    __syncthreads();
    for (int k = tid; k < n; k += kGcThreads) qinv[pivrow[k]] = k;
    __syncthreads();
    const int nn = n * n, ld = n + 1;
#pragma unroll
    for (int j = 0; j < kGcSlots; ++j) {
        const int i = lane + 32 * j;
        if (i < n) {
            const int R = qinv[i];
#pragma unroll
            for (int t = 0; t < kGcPairs; ++t) {
                const int c0 = wid + 32 * t, c1 = c0 + 16;
                if (c0 < n) St[R * ld + pivrow[c0]] = a[j][t].x;
                if (c1 < n) St[R * ld + pivrow[c1]] = a[j][t].y;
            }
        }
    }
    __syncthreads();
    const int dq = kGcThreads / n, dr = kGcThreads - dq * n;
    int row = tid / n, col = tid - (tid / n) * n;
#pragma unroll 8
    for (int r = 0; r < kGcLoad; ++r) {
        const int e = tid + kGcThreads * r;
        if (e < nn) A[e] = St[row * ld + col];
        row += dq;
        col += dr;
        if (col >= n) { col -= n; ++row; }
    }
}
#undef FIL_GC_SLOT_SWITCH

}  // namespace

template <int NCH>
cudaError_t launch_gj(fil_ctx *c, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(gauss_jordan_inverse_kernel<NCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gauss_jordan_inverse_kernel<NCH><<<c->lay.M, kInvThreads, smem, c->stream>>>(
        c->lay, c->jofs, c->jinv, c->jinv, c->d_flags);
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
    c->j0_dp_bdt = dp.bdt;
    const int N = c->lay.maxN;
    const int fast = fast_mixed(c) ? 1 : 0;
    const size_t smem_pre = (size_t)6 * N * sizeof(double) +
                            (fast ? (size_t)(12 * N + 5 * N * N) * sizeof(float) : 0);
    if (smem_pre > 48 * 1024) {
        cudaError_t ea = cudaFuncSetAttribute(j0_precompute_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem_pre);
        if (ea != cudaSuccess) return ea;
    }
    j0_precompute_kernel<<<c->lay.M, kAsmThreads, smem_pre, c->stream>>>(
        c->lay, c->auxofs, X, c->qc, c->Yc, c->Tint, dp, c->aux, fast);
    const size_t smem_asm = (size_t)(5 * N * N + 54 * N) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(j0_assemble32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_asm);
    if (e != cudaSuccess) return e;
    j0_assemble32_kernel<<<c->lay.M, kAsmThreads, smem_asm, c->stream>>>(
        c->lay, c->jofs, c->auxofs, dp, c->aux, c->jinv);
    if (6 * N <= kGjMaxN) {
        const size_t smem_gc = (size_t)6 * N * (6 * N + 1) * sizeof(float);
        e = cudaFuncSetAttribute(gauss_jordan_inverse_col_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_gc);
        if (e != cudaSuccess) return e;
        gauss_jordan_inverse_col_kernel<<<c->lay.M, kGcThreads, smem_gc, c->stream>>>(
            c->lay, c->jofs, c->jinv, c->d_flags);
        e = cudaGetLastError();
    } else {
        const size_t smem_inv = (size_t)6 * N * (6 * N + 1) * sizeof(float);
        e = launch_gauss_jordan(c, (6 * N + 31) / 32, smem_inv);
    }
    if (e != cudaSuccess) return e;
    c->n_launches += 3;
    return cudaGetLastError();
}

size_t j0_solve_smem(int maxN) {
    const size_t n = 6 * (size_t)maxN;
    return (2 * n + 15 * (size_t)maxN) * sizeof(double) + n * sizeof(float);
}

cudaError_t j0_dense_solve(fil_ctx *c, const double *b, double *x, const int *active) {
    if (fast_mixed(c)) {
        j0_apply_inverse_kernel<<<c->lay.M, kApplyThreads, 0, c->stream>>>(c->lay, c->jofs,
                                                                          c->jinv, b, x, active);
        c->n_launches += 1;
        return cudaGetLastError();
    }
    DenseParams dp;
    dp.jp = J0Params{c->dL, c->KB, c->KT, c->g0, c->kmu, c->knu, 0.0, 0.0};
    dp.bdt = c->j0_dp_bdt;
    dp.inv8pieta = 1.0 / (8.0 * kPi * c->eta);
    dp.near2 = 4.0 * c->a * c->a;
    dp.a = c->a;
    const size_t smem = j0_solve_smem(c->lay.maxN);
    cudaError_t e = cudaFuncSetAttribute(j0_solve_fused_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    j0_solve_fused_kernel<<<c->lay.M, kSolveThreads, smem, c->stream>>>(
        c->lay, c->jofs, c->auxofs, dp, c->aux, c->jinv, b, x, active,
        kJ0Refine);
    c->n_launches += 1;
    return cudaGetLastError();
}

}  // namespace fil
