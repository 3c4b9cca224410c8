// Per-filament kernels of the residual f(X) (paper Sec. 2.5, 2.9.3):
//   unpack  : q_n = exp(u_n) q_n^j, t_n = R(q_n) e_x, robot-arm positions
//             Y_n = Y_1 + (dL/2) sum_{m=2}^n (t_{m-1} + t_m)  (positionSubstitution-3d)
//   forces  : F_n = Lam_{n+1/2} - Lam_{n-1/2} + external,
//             T_n = M_{n+1/2} - M_{n-1/2} + (dL/2) t_n x (Lam_{n+1/2} + Lam_{n-1/2}) + external
//             (constraint-force, constraint-torque, elastic-torque, quaternionM)
//   residual: position rows Y_n - a1 Y^j_n - a0 Y^{j-1}_n - b dt V_n and rotation rows
//             u_n - g u^j_n - b dt dexpinv_{u_n}(Omega_n) (RA-3d-system).
// One warp per filament for the scans along the filament (the robot-arm prefix
// sum uses warp shuffles, 32 segments per pass with a carry); one thread per
// segment for the element-wise residual rows.
#include <cuda_runtime.h>

#include <vector>

#include "fil_internal.cuh"
#include "quat.cuh"

namespace fil {
namespace {

__device__ __forceinline__ V3 shfl_up3(V3 v, int d) {
    return {__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
            __shfl_up_sync(0xffffffffu, v.z, d)};
}
__device__ __forceinline__ V3 shfl3(V3 v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
            __shfl_sync(0xffffffffu, v.z, src)};
}

struct ForceParams {
    double dL, KB, KT, g0, kmu, knu;
};

// Warp-wide robot-arm positions for one filament: given t_n per lane (one pass
// of up to 32 segments), carry = Y of the segment before the pass and the
// tangent before the pass. Returns Y_n for the lane; updates the carries.
__device__ __forceinline__ V3 robot_arm_pass(V3 t, bool active, int n, double dL, V3 &carry_Y,
                                             V3 &carry_t, int lane) {
    V3 tprev = shfl_up3(t, 1);
    if (lane == 0) tprev = carry_t;
    V3 inc = (active && n > 0) ? (0.5 * dL) * (tprev + t) : v3(0, 0, 0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        V3 o = shfl_up3(inc, d);
        if (lane >= d) inc = inc + o;
    }
    V3 Yn = carry_Y + inc;
    carry_Y = shfl3(Yn, 31);
    carry_t = shfl3(t, 31);
    return Yn;
}

// unpack (+ forces): one warp per filament.
__global__ void unpack_forces_kernel(Layout lay, const double *__restrict__ X,
                                     const double *__restrict__ qj, ForceParams fp,
                                     const double *__restrict__ Fext,
                                     const double *__restrict__ Text,
                                     const double *__restrict__ follower, int with_forces,
                                     const int *__restrict__ active, double *__restrict__ qc,
                                     double *__restrict__ Yc, double *__restrict__ FT,
                                     double *__restrict__ Tint) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= lay.M) return;
    const int s0 = lay.off[warp];
    if (active && !active[lay.sys_of[s0]]) return;   // a converged system keeps its unpack
    const int N = lay.off[warp + 1] - s0;
    const double *Xf = X + 6 * (int64_t)s0;

    V3 carry_Y = ld3(Xf);
    V3 carry_t = v3(0, 0, 0);
    for (int base = 0; base < N; base += 32) {
        const int n = base + lane;
        const bool active = n < N;
        Q4 q = {1, 0, 0, 0};
        V3 t = v3(0, 0, 0);
        if (active) {
            q = qmul(qexp(ld3(Xf + 3 + 3 * n)), ld4(qj + 4 * (int64_t)(s0 + n)));
            t = frame_t(q);
        }
        V3 Yn = robot_arm_pass(t, active, n, fp.dL, carry_Y, carry_t, lane);
        if (active) {
            st4(qc + 4 * (int64_t)(s0 + n), q);
            st3(Yc + 3 * (int64_t)(s0 + n), Yn);
        }
    }
    if (!with_forces) return;
    __syncwarp();

    const double *Lam = Xf + 3 + 3 * N;   // Lambda_{j+3/2}, j = 0..N-2
    const double follow = follower ? follower[warp] : 0.0;
    // each joint moment M_{n+1/2} once, by lane n; M_{n-1/2} from the lane below
    V3 Mcarry = v3(0, 0, 0);               // M of the joint before this pass
    for (int base = 0; base < N; base += 32) {
        const int n = base + lane;
        const bool act = n < N;
        const int64_t g = s0 + n;
        Q4 q = {1, 0, 0, 0};
        if (act) q = ld4(qc + 4 * g);
        V3 Mr = v3(0, 0, 0);
        if (act && n <= N - 2)
            Mr = internal_moment(q, ld4(qc + 4 * (g + 1)), fp.dL, fp.KB, fp.KT, fp.g0, fp.kmu,
                                 fp.knu);
        V3 Ml = shfl_up3(Mr, 1);
        if (lane == 0) Ml = Mcarry;
        Mcarry = shfl3(Mr, 31);
        if (!act) continue;
        const V3 t = frame_t(q);
        const V3 Lr = (n <= N - 2) ? ld3(Lam + 3 * n) : v3(0, 0, 0);
        const V3 Ll = (n >= 1) ? ld3(Lam + 3 * (n - 1)) : v3(0, 0, 0);
        V3 F = Lr - Ll;
        V3 Ti = (Mr - Ml) + (0.5 * fp.dL) * cross(t, Lr + Ll);
        if (Fext) F = F + ld3(Fext + 3 * g);
        if (n == N - 1) F = F - follow * t;
        V3 T = Ti;
        if (Text) T = T + ld3(Text + 3 * g);
        st3(FT + 6 * g, F);
        st3(FT + 6 * g + 3, T);
        if (Tint) st3(Tint + 3 * g, Ti);
    }
}

struct Scheme {
    double a1, a0, bdt, g;   // f = Y - a1 Y^j - a0 Y^{j-1} - bdt V ; u - g u^j - bdt dexpinv
};

// One thread per segment: both 3-rows of the residual, plus ||f||_inf of the
// segment's system (as the maximum of the IEEE bit patterns of |f|; a NaN
// compares above every number).
__global__ void residual_rows_kernel(Layout lay, const double *__restrict__ X,
                                     const double *__restrict__ Yc,
                                     const double *__restrict__ VW,
                                     const double *__restrict__ Yj,
                                     const double *__restrict__ Yjm1,
                                     const double *__restrict__ uj, Scheme sc,
                                     const int *__restrict__ active,
                                     const double *__restrict__ fprev, double *__restrict__ f,
                                     unsigned long long *__restrict__ finf_bits) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    bool eval = g < lay.S;
    if (eval && active && !active[lay.sys_of[g]]) {
        // a converged system keeps its residual (its iterate is frozen)
        const int i = lay.fil_of[g];
        const int s0 = lay.off[i];
        const int N = lay.off[i + 1] - s0;
        const int n = (int)(g - s0);
        const int64_t r = 6 * (int64_t)s0;
        const int64_t pr = r + (n == 0 ? 0 : 3 + 3 * N + 3 * (n - 1));
        const int64_t rr = r + 3 + 3 * n;
        for (int k = 0; k < 3; ++k) {
            f[pr + k] = fprev[pr + k];
            f[rr + k] = fprev[rr + k];
        }
        eval = false;
    }
    if (eval) {
        const int i = lay.fil_of[g];
        const int s0 = lay.off[i];
        const int N = lay.off[i + 1] - s0;
        const int n = (int)(g - s0);
        const double *Xf = X + 6 * (int64_t)s0;
        double *ff = f + 6 * (int64_t)s0;
        const V3 u = ld3(Xf + 3 + 3 * n);
        const V3 V = ld3(VW + 6 * g), W = ld3(VW + 6 * g + 3);
        V3 pos = ld3(Yc + 3 * g) - sc.a1 * ld3(Yj + 3 * g) - sc.bdt * V;
        if (sc.a0 != 0.0) pos = pos - sc.a0 * ld3(Yjm1 + 3 * g);
        V3 rot = u - sc.bdt * dexpinv(u, W);
        if (sc.g != 0.0) rot = rot - sc.g * ld3(uj + 3 * g);
        st3(ff + 3 + 3 * n, rot);
        st3(n == 0 ? ff : ff + 3 + 3 * N + 3 * (n - 1), pos);
        m = fmax(fmax(fmax(fabs(pos.x), fabs(pos.y)), fmax(fabs(pos.z), fabs(rot.x))),
                 fmax(fabs(rot.y), fabs(rot.z)));
        if (isnan(pos.x + pos.y + pos.z + rot.x + rot.y + rot.z)) m = __longlong_as_double(
            0x7ff8000000000000ll);
    }
    unsigned long long bits = (unsigned long long)__double_as_longlong(m);
    const int sid = g < lay.S ? lay.sys_of[g] : -1;
    const int sid0 = __shfl_sync(0xffffffffu, sid, 0);
    if (__all_sync(0xffffffffu, sid == sid0 || sid < 0)) {
        // the warp's segments belong to one system (the usual case)
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            unsigned long long o = __shfl_down_sync(0xffffffffu, bits, d);
            bits = o > bits ? o : bits;
        }
        if ((threadIdx.x & 31) == 0 && sid0 >= 0) atomicMax(finf_bits + sid0, bits);
    } else if (sid >= 0) {
        atomicMax(finf_bits + sid, bits);
    }
}

// Straight filaments from (base, t, mu) with the App. A.1 construction and an
// optional perturbation q <- exp(xi) q; one warp per filament.
__global__ void init_straight_kernel(Layout lay, const double *__restrict__ base,
                                     const double *__restrict__ tt,
                                     const double *__restrict__ mu,
                                     const double *__restrict__ xi, double dL,
                                     double *__restrict__ Y, double *__restrict__ q) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= lay.M) return;
    const int s0 = lay.off[warp];
    const int N = lay.off[warp + 1] - s0;
    const V3 t = ld3(tt + 3 * warp), m = ld3(mu + 3 * warp);
    // p1 = (e_x . t, e_x x t)^{1/2} = (t1, 0, -t3, t2)^{1/2}
    const Q4 p1 = qsqrt(Q4{t.x, 0.0, -t.z, t.y});
    // n' = R(p1) e_y, p2 = (n'.mu, n' x mu)^{1/2}, q = p2 p1
    const V3 np = frame_mu(p1);
    const V3 c = cross(np, m);
    const Q4 p2 = qsqrt(Q4{dot(np, m), c.x, c.y, c.z});
    const Q4 qf = qmul(p2, p1);
    V3 carry_Y = ld3(base + 3 * warp);
    V3 carry_t = v3(0, 0, 0);
    for (int b = 0; b < N; b += 32) {
        const int n = b + lane;
        const bool active = n < N;
        Q4 qn = qf;
        if (active && xi) qn = qmul(qexp(ld3(xi + 3 * (int64_t)(s0 + n))), qf);
        const V3 tn = active ? frame_t(qn) : v3(0, 0, 0);
        const V3 Yn = robot_arm_pass(tn, active, n, dL, carry_Y, carry_t, lane);
        if (active) {
            st4(q + 4 * (int64_t)(s0 + n), qn);
            st3(Y + 3 * (int64_t)(s0 + n), Yn);
        }
    }
}

// Value at the next step of the polynomial through the last ord + 1 committed
// values x^j (x0), x^{j-1} (x1), x^{j-2} (x2): ord 0 keeps x^j, ord 1 gives
// 2 x^j - x^{j-1}, ord 2 gives 3 x^j - 3 x^{j-1} + x^{j-2}.
__device__ __forceinline__ V3 extrapolated(V3 x0, const double *x1, const double *x2, int ord) {
    if (ord == 1) return 2.0 * x0 - ld3(x1);
    if (ord == 2) return 3.0 * (x0 - ld3(x1)) + ld3(x2);
    return x0;
}

// Fraction theta of the second difference in the adaptive guess of one block:
// P / Q from its fit statistics (P, Q), clipped to [0, 1]; 0 before a fit.
__device__ __forceinline__ double fit_theta(const double *pq) {
    const double P = pq[0], Q = pq[1];
    if (!(Q > 0.0)) return 0.0;
    return fmin(fmax(P / Q, 0.0), 1.0);
}

// Guess of one 3-vector: extrapolated at order ord (<= 1), or with three
// values either quadratic (theta < 0) or the linear guess plus theta times
// the second difference (the adaptive form).
__device__ __forceinline__ V3 guess(V3 x0, const double *x1, const double *x2, int ord,
                                    double theta) {
    if (ord < 2 || theta < 0.0) return extrapolated(x0, x1, x2, ord);
    const V3 a = ld3(x1);
    return (2.0 * x0 - a) + theta * ((x0 - 2.0 * a) + ld3(x2));
}

// X_0 of a step: each unknown extrapolated from the committed steps, Y_1 with
// order y_ord from its BDF2 history (Y^j, Y^{j-1}, Y^{j-2}), u and Lambda with
// order u_ord from (u^j, u^{j-1}, u^{j-2}) and (Lambda^j, ...); u_ord < 0
// before the first step: u = 0, Lambda = Lambda^j. With xfit (the adaptive
// form) an order-2 block takes its fitted theta (xfit[6i + 2b], b = 0: Y_1,
// 1: u, 2: Lambda). One thread per segment.
__global__ void extrapolate_kernel(Layout lay, const double *__restrict__ Y,
                                   const double *__restrict__ Yprev,
                                   const double *__restrict__ Yprev2,
                                   const double *__restrict__ uprev,
                                   const double *__restrict__ uprev2,
                                   const double *__restrict__ uprev3,
                                   const double *__restrict__ lam,
                                   const double *__restrict__ lamprev,
                                   const double *__restrict__ lamprev2, int y_ord, int u_ord,
                                   const double *__restrict__ xfit, double *__restrict__ X0) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= lay.S) return;
    const int i = lay.fil_of[g];
    const int s0 = lay.off[i];
    const int N = lay.off[i + 1] - s0;
    const int n = (int)(g - s0);
    const double *fit = xfit ? xfit + 6 * (int64_t)i : nullptr;
    double *Xf = X0 + 6 * (int64_t)s0;
    if (n == 0)
        st3(Xf, guess(ld3(Y + 3 * g), Yprev + 3 * g, Yprev2 + 3 * g, y_ord,
                      fit ? fit_theta(fit) : -1.0));
    V3 u0 = v3(0, 0, 0);
    if (u_ord >= 0)
        u0 = guess(ld3(uprev + 3 * g), uprev2 + 3 * g, uprev3 + 3 * g, u_ord,
                   fit ? fit_theta(fit + 2) : -1.0);
    st3(Xf + 3 + 3 * n, u0);
    if (n <= N - 2) {
        const int64_t li = 3 * (int64_t)(s0 - i + n);
        st3(Xf + 3 + 3 * N + 3 * n, guess(ld3(lam + li), lamprev + li, lamprev2 + li,
                                          u_ord > 0 ? u_ord : 0, fit ? fit_theta(fit + 4) : -1.0));
    }
}

// Terms of the adaptive fit of one 3-vector: with l = 2 x^j - x^{j-1} and
// d = x^j - 2 x^{j-1} + x^{j-2}, pq[0] += <x* - l, d> and pq[1] += <d, d>.
__device__ __forceinline__ void fit_terms(const double *xs, const double *x0, const double *x1,
                                          const double *x2, double pq[2]) {
    const V3 a = ld3(x0), b = ld3(x1);
    const V3 d = (a - 2.0 * b) + ld3(x2);
    const V3 r = ld3(xs) - (2.0 * a - b);
    pq[0] += dot(r, d);
    pq[1] += dot(d, d);
}

// Adaptive fit at a commit (before the history shift): for each filament and
// block (Y_1, u, Lambda) whose last three values exist (y_ok, u_ok),
// P <- kFitDecay P + <x* - l, d>, Q <- kFitDecay Q + <d, d> over the block's
// 3-vectors, x* the committed solution X; filaments of a system that took no
// Broyden iteration this step (iterated[system] = 0: x* is the guess itself and
// says nothing about its error) keep their fit. One warp per filament, lane
// sums combined by a fixed shuffle tree.
constexpr double kFitDecay = 0.7;

__global__ void extrap_fit_kernel(Layout lay, const double *__restrict__ X,
                                  const double *__restrict__ Y, const double *__restrict__ Yprev,
                                  const double *__restrict__ Yprev2,
                                  const double *__restrict__ uprev,
                                  const double *__restrict__ uprev2,
                                  const double *__restrict__ uprev3,
                                  const double *__restrict__ lam,
                                  const double *__restrict__ lamprev,
                                  const double *__restrict__ lamprev2, int y_ok, int u_ok,
                                  const int *__restrict__ iterated, double *__restrict__ xfit) {
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= lay.M) return;
    const int s0 = lay.off[i];
    if (!iterated[lay.sys_of[s0]]) return;     // the whole warp leaves together
    const int N = lay.off[i + 1] - s0;
    const double *Xf = X + 6 * (int64_t)s0;
    double fu[2] = {0, 0}, fl[2] = {0, 0};
    if (u_ok) {
        for (int n = lane; n < N; n += 32) {
            const int64_t g = s0 + n;
            fit_terms(Xf + 3 + 3 * n, uprev + 3 * g, uprev2 + 3 * g, uprev3 + 3 * g, fu);
            if (n <= N - 2) {
                const int64_t li = 3 * (int64_t)(s0 - i + n);
                fit_terms(Xf + 3 + 3 * N + 3 * n, lam + li, lamprev + li, lamprev2 + li, fl);
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            fu[0] += __shfl_xor_sync(0xffffffffu, fu[0], d);
            fu[1] += __shfl_xor_sync(0xffffffffu, fu[1], d);
            fl[0] += __shfl_xor_sync(0xffffffffu, fl[0], d);
            fl[1] += __shfl_xor_sync(0xffffffffu, fl[1], d);
        }
    }
    if (lane == 0) {
        double *f = xfit + 6 * (int64_t)i;
        if (y_ok) {
            double fy[2] = {0, 0};
            const int64_t g = s0;
            fit_terms(Xf, Y + 3 * g, Yprev + 3 * g, Yprev2 + 3 * g, fy);
            f[0] = kFitDecay * f[0] + fy[0];
            f[1] = kFitDecay * f[1] + fy[1];
        }
        if (u_ok) {
            f[2] = kFitDecay * f[2] + fu[0];
            f[3] = kFitDecay * f[3] + fu[1];
            f[4] = kFitDecay * f[4] + fl[0];
            f[5] = kFitDecay * f[5] + fl[1];
        }
    }
}

// History shift after convergence (qc, Yc hold the unpack of X).
__global__ void commit_kernel(Layout lay, const double *__restrict__ X,
                              const double *__restrict__ qc, const double *__restrict__ Yc,
                              double *__restrict__ Y, double *__restrict__ Yprev,
                              double *__restrict__ Yprev2, double *__restrict__ q,
                              double *__restrict__ uprev, double *__restrict__ uprev2,
                              double *__restrict__ uprev3, double *__restrict__ lam,
                              double *__restrict__ lamprev, double *__restrict__ lamprev2) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= lay.S) return;
    const int i = lay.fil_of[g];
    const int s0 = lay.off[i];
    const int N = lay.off[i + 1] - s0;
    const int n = (int)(g - s0);
    const double *Xf = X + 6 * (int64_t)s0;
    st3(Yprev2 + 3 * g, ld3(Yprev + 3 * g));
    st3(Yprev + 3 * g, ld3(Y + 3 * g));
    st3(Y + 3 * g, ld3(Yc + 3 * g));
    st4(q + 4 * g, ld4(qc + 4 * g));
    st3(uprev3 + 3 * g, ld3(uprev2 + 3 * g));
    st3(uprev2 + 3 * g, ld3(uprev + 3 * g));
    st3(uprev + 3 * g, ld3(Xf + 3 + 3 * n));
    if (n <= N - 2) {
        const int64_t li = 3 * (int64_t)(s0 - i + n);
        st3(lamprev2 + li, ld3(lamprev + li));
        st3(lamprev + li, ld3(lam + li));
        st3(lam + li, ld3(Xf + 3 + 3 * N + 3 * n));
    }
}

unsigned warp_grid(int M, int threads) { return (unsigned)(((int64_t)M * 32 + threads - 1) / threads); }
unsigned seg_grid(int64_t S, int threads) { return (unsigned)((S + threads - 1) / threads); }

}  // namespace

cudaError_t unpack_forces(fil_ctx *c, const double *X, int with_forces, bool active_only) {
    ForceParams fp{c->dL, c->KB, c->KT, c->g0, c->kmu, c->knu};
    unpack_forces_kernel<<<warp_grid(c->lay.M, 128), 128, 0, c->stream>>>(
        c->lay, X, c->q, fp, c->has_Fext ? c->Fext : nullptr, c->has_Text ? c->Text : nullptr,
        c->has_follower ? c->follower : nullptr, with_forces, active_only ? c->d_active : nullptr,
        c->qc, c->Yc, c->FT, with_forces == 2 ? c->Tint : nullptr);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t residual_rows(fil_ctx *c, const double *X, double *f, const double *fprev) {
    Scheme sc;
    if (c->have_prev) {
        sc = {4.0 / 3.0, -1.0 / 3.0, 2.0 / 3.0 * c->dt, 1.0 / 3.0};
    } else {
        sc = {1.0, 0.0, c->dt, 0.0};
    }
    cudaError_t e = cudaMemsetAsync(c->d_finf, 0, sizeof(unsigned long long) * c->n_sys, c->stream);
    if (e != cudaSuccess) return e;
    residual_rows_kernel<<<seg_grid(c->lay.S, 256), 256, 0, c->stream>>>(
        c->lay, X, c->Yc, c->VW, c->Y, c->Yprev, c->uprev, sc, fprev ? c->d_active : nullptr,
        fprev, f, c->d_finf);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t init_straight(fil_ctx *c, const double *base, const double *t, const double *mu,
                          const double *xi) {
    init_straight_kernel<<<warp_grid(c->lay.M, 128), 128, 0, c->stream>>>(c->lay, base, t, mu, xi,
                                                                          c->dL, c->Y, c->q);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t extrapolate_guess(fil_ctx *c, double *X0) {
    // order of each unknown's polynomial: as high as the committed history and
    // the chosen order allow (Y_1 has one level more than u and Lambda: the
    // BDF2 history holds Y^{j-1} from the first step on); the adaptive form
    // replaces the quadratic one by its fitted blend per filament and block
    const bool adaptive = c->extrap_order == FIL_EXTRAP_ADAPTIVE;
    const int cap = adaptive ? 2 : c->extrap_order;
    const int y_ord = c->ylev < cap ? c->ylev : cap;
    const int u_lev = c->have_prev ? (c->hist >= 3 ? 2 : c->hist >= 2 ? 1 : 0) : -1;
    const int u_ord = u_lev < cap ? u_lev : cap;
    extrapolate_kernel<<<seg_grid(c->lay.S, 256), 256, 0, c->stream>>>(
        c->lay, c->Y, c->Yprev, c->Yprev2, c->uprev, c->uprev2, c->uprev3, c->lam, c->lamprev,
        c->lamprev2, y_ord, u_ord, adaptive ? c->xfit : nullptr, X0);
    c->n_launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c->tether_on) e = tether_guess(c, X0);
    return e;
}

cudaError_t commit_state(fil_ctx *c, const double *X) {
    cudaError_t e = unpack_forces(c, X, 0);
    if (e != cudaSuccess) return e;
    if (c->extrap_order == FIL_EXTRAP_ADAPTIVE) {
        // the fit needs the three values before this commit: Y_1 once two past
        // levels are held, u and Lambda once three steps were committed; and
        // which systems iterated this step
        std::vector<int> iterated(c->n_sys);
        for (int s = 0; s < c->n_sys; ++s) iterated[s] = c->sys_iters_h[s] > 0 ? 1 : 0;
        e = cudaMemcpyAsync(c->d_iterated, iterated.data(), sizeof(int) * c->n_sys,
                            cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return e;
        extrap_fit_kernel<<<warp_grid(c->lay.M, 128), 128, 0, c->stream>>>(
            c->lay, X, c->Y, c->Yprev, c->Yprev2, c->uprev, c->uprev2, c->uprev3, c->lam,
            c->lamprev, c->lamprev2, c->ylev >= 2 ? 1 : 0, c->hist >= 3 ? 1 : 0, c->d_iterated,
            c->xfit);
        c->n_launches += 1;
    }
    commit_kernel<<<seg_grid(c->lay.S, 256), 256, 0, c->stream>>>(
        c->lay, X, c->qc, c->Yc, c->Y, c->Yprev, c->Yprev2, c->q, c->uprev, c->uprev2, c->uprev3,
        c->lam, c->lamprev, c->lamprev2);
    c->n_launches += 1;
    return cudaGetLastError();
}

}  // namespace fil
