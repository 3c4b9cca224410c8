// Approximate Jacobian J0 of App. B.2 and its solve, one filament per warp.
//
// Per filament, J0 = [[I, 0, J13], [0, J22, J23], [I, J32, J33]] acting on
// (Y_1, u_0..u_{N-1}, Lam_0..Lam_{N-2}) (0-based segments; Lam_j joins segments
// j and j+1). Its blocks are those of App. B.2 (J13, J33 as in App. B.1):
//   J13 = -c_t I on Lam_0;  J33: c_t (Lam_{s-1} - Lam_s) in the row of segment s;
//   J32: (dL/2) w [x t_n] with w = 1 at the ends of the cumulative sum, 2 inside;
//   J22, J23 from the Taylor-truncated dexpinv and the frame-vector moments;
//   c_t = b dt/(6 pi eta a), c_r = b dt/(8 pi eta a^3), b = 2/3 (BDF2) or 1.
//
// The paper factors each 6N x 6N block densely (O(N^3)). Here the same linear
// system is solved exactly in O(N): row 1 gives Y_1 = b1 + c_t Lam_0; subtracting
// consecutive constraint rows (row_{s+1} - row_s, and row_1 - row of Y_1) removes
// Y_1 and turns the cumulative J32 into two neighbour terms. With the unknowns
// interleaved as (u_0, Lam_0, u_1, Lam_1, ..., Lam_{N-2}, u_{N-1}) the remaining
// (6N-3) x (6N-3) matrix is block-pentadiagonal in 3x3 blocks, i.e. banded with
// 8 sub- and 8 super-diagonals, and is factored by Gaussian elimination with
// partial pivoting inside the band (U gains up to 8 more super-diagonals).
//
// Band storage: row-major windows, A(i, c) at band[i * kBandW + (c - i + kBandKL)]
// for c - i in [-8, 16]; filament f starts at row 6 off[f] - 3 f.
#include <cuda_runtime.h>

#include <algorithm>

#include "fil_internal.cuh"
#include "j0_common.cuh"
#include "quat.cuh"

namespace fil {
namespace {

template <typename TO>
__device__ __forceinline__ void put_block(TO *band, int64_t row_block, int64_t col_block,
                                          const M33 &B) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int64_t i = 3 * row_block + r;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const int64_t col = 3 * col_block + cc;
            band[i * kBandW + (col - i + kBandKL)] = (TO)B.m[3 * r + cc];
        }
    }
}

// Assemble the band of each filament (one warp per filament), computed in
// FP64 and stored in the precision TO of the factors.
template <typename TO>
__global__ void j0_build_kernel(Layout lay, const double *__restrict__ X,
                                const double *__restrict__ qc, const double *__restrict__ Tint,
                                J0Params p, TO *__restrict__ band_all) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= lay.M) return;
    const int s0 = lay.off[warp];
    const int N = lay.off[warp + 1] - s0;
    const int64_t nrow = 6 * (int64_t)N - 3;
    TO *band = band_all + (6 * (int64_t)s0 - 3 * (int64_t)warp) * kBandW;
    for (int64_t i = lane; i < nrow * kBandW; i += 32) band[i] = TO(0);
    __syncwarp();
    const double *Xf = X + 6 * (int64_t)s0;
    const double *Lam = Xf + 3 + 3 * N;
    const M33 I3 = meye();
    for (int s = lane; s < N; s += 32) {
        const int64_t g = s0 + s;
        const Q4 qs = ld4(qc + 4 * g);
        const V3 ts = frame_t(qs);
        const V3 u = ld3(Xf + 3 + 3 * s);
        const V3 T = ld3(Tint + 3 * g);
        const V3 Lsum = ((s <= N - 2) ? ld3(Lam + 3 * s) : v3(0, 0, 0)) +
                        ((s >= 1) ? ld3(Lam + 3 * (s - 1)) : v3(0, 0, 0));
        M33 Da_r, Db_r, Da_l, Db_l;   // joint s (right) and joint s-1 (left)
        if (s <= N - 2) moment_derivs(p, qs, ld4(qc + 4 * (g + 1)), Da_r, Db_r);
        if (s >= 1) moment_derivs(p, ld4(qc + 4 * (g - 1)), qs, Da_l, Db_l);
        const M33 ux = skew(u);
        const M33 ux2 = mmul(ux, ux);
        // A_s = I - [u x]/2 + [u x]^2/12
        const M33 A = madd(madd(I3, ux, -0.5), ux2, 1.0 / 12.0);
        // dT_s/du_s
        M33 dT = mscale(mmul(rskew(Lsum), rskew(ts)), 0.5 * p.dL);
        if (s <= N - 2) dT = madd(dT, Da_r);
        if (s >= 1) dT = madd(dT, Db_l, -1.0);
        // J22_ss = I - c_r { dT - ([x T] + [u x] dT)/2 + ([x (u x T)] + [u x][x T] + [u x]^2 dT)/12 }
        const M33 xT = rskew(T);
        M33 inner = madd(dT, madd(xT, mmul(ux, dT)), -0.5);
        M33 third = madd(madd(rskew(cross(u, T)), mmul(ux, xT)), mmul(ux2, dT));
        inner = madd(inner, third, 1.0 / 12.0);
        const int64_t rb = 2 * s;   // block row of the rotation rows of segment s
        put_block(band, rb, 2 * s, madd(I3, inner, -p.cr));
        if (s <= N - 2) put_block(band, rb, 2 * s + 2, mscale(mmul(A, Db_r), -p.cr));
        if (s >= 1) put_block(band, rb, 2 * s - 2, mscale(mmul(A, Da_l), p.cr));
        // J23: -c_r A (dL/2) [t_s x] on Lam_{s-1} and Lam_s
        const M33 G = mscale(mmul(A, skew(ts)), -p.cr * 0.5 * p.dL);
        if (s >= 1) put_block(band, rb, 2 * s - 1, G);
        if (s <= N - 2) put_block(band, rb, 2 * s + 1, G);
        // differenced constraint rows of joint j = s:
        // (dL/2)([x t_s] u_s + [x t_{s+1}] u_{s+1}) + c_t(-Lam_{s-1} + 2 Lam_s - Lam_{s+1})
        if (s <= N - 2) {
            const int64_t cb = 2 * s + 1;
            const V3 tn = frame_t(ld4(qc + 4 * (g + 1)));
            put_block(band, cb, 2 * s, mscale(rskew(ts), 0.5 * p.dL));
            put_block(band, cb, 2 * s + 2, mscale(rskew(tn), 0.5 * p.dL));
            put_block(band, cb, 2 * s + 1, mscale(I3, 2.0 * p.ct));
            if (s >= 1) put_block(band, cb, 2 * s - 1, mscale(I3, -p.ct));
            if (s + 1 <= N - 2) put_block(band, cb, 2 * s + 3, mscale(I3, -p.ct));
        }
    }
}

constexpr int kJ0Threads = 128;
constexpr int kLuRing = 16;    // band rows a warp keeps in shared memory
constexpr int kLuAhead = 13;   // column j requests row j + kLuAhead

// One element of a band row, global -> shared, asynchronously (cp.async).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(kPending) : "memory");
}

// In-place banded LU with partial pivoting (one warp per filament), in the
// precision T of the stored factors. Column j reads and writes rows j .. j+8
// only, and row j is final once column j is done, so each warp keeps a ring
// of kLuRing band rows in shared memory: row j + kLuAhead is requested with
// cp.async at column j (into the slot of row j - 3, already written back),
// waited for five columns later, and row j is written back, with its pivot
// replaced by the reciprocal the solves multiply by, when column j is done.
template <typename T>
__global__ void __launch_bounds__(kJ0Threads)
band_lu_kernel(Layout lay, T *__restrict__ band_all, int *__restrict__ piv_all,
               int *__restrict__ flags) {
    static_assert(kLuAhead < kLuRing, "a requested row reuses the slot of a written-back row");
    __shared__ T ring_all[kJ0Threads / 32][kLuRing * kBandW];
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= lay.M) return;
    const int s0 = lay.off[warp];
    const int N = lay.off[warp + 1] - s0;
    const int n = 6 * N - 3;
    const int64_t row0 = 6 * (int64_t)s0 - 3 * (int64_t)warp;
    T *G = band_all + row0 * kBandW;
    T *R = ring_all[threadIdx.x >> 5];
    int *piv = piv_all + row0;
#define RB(i, c) R[((i) & (kLuRing - 1)) * kBandW + ((c) - (i) + kBandKL)]
    for (int r = 0; r < kLuAhead && r < n; ++r)
        if (lane < kBandW) cp_async_elem(&R[r * kBandW + lane], G + (int64_t)r * kBandW + lane);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    for (int j = 0; j < n; ++j) {
        {
            const int r = j + kLuAhead;
            if (r < n && lane < kBandW)
                cp_async_elem(&R[(r & (kLuRing - 1)) * kBandW + lane], G + (int64_t)r * kBandW + lane);
            cp_async_commit();
        }
        // rows up to j + 8, requested at column j + 8 - kLuAhead or before, have landed
        cp_async_wait<kLuAhead - kBandKL>();
        __syncwarp();
        const int last = min(n - 1, j + kBandKL);
        // pivot: first row of maximal |A(i, j)|, i in [j, last]
        T v = T(-1);
        int idx = j;
        if (j + lane <= last && lane <= kBandKL) {
            v = fabs(RB(j + lane, j));
            idx = j + lane;
        }
#pragma unroll
        for (int d = 8; d > 0; d >>= 1) {
            const T ov = __shfl_down_sync(0xffffffffu, v, d);
            const int oi = __shfl_down_sync(0xffffffffu, idx, d);
            if (ov > v || (ov == v && oi < idx)) {
                v = ov;
                idx = oi;
            }
        }
        const int p = __shfl_sync(0xffffffffu, idx, 0);
        const T pv = __shfl_sync(0xffffffffu, v, 0);
        if (lane == 0) piv[j] = p;
        const int cmax = min(n - 1, j + kBandKL + kBandKU);
        if (p != j) {
            const int c = j + lane;
            if (c <= cmax) {
                const T t = RB(j, c);
                RB(j, c) = RB(p, c);
                RB(p, c) = t;
            }
        }
        __syncwarp();
        if (pv == T(0)) {
            if (lane == 0) atomicOr(flags + 1, 1);
        } else {
            const T inv = T(1) / RB(j, j);
            if (lane >= 1 && j + lane <= last) RB(j + lane, j) = RB(j + lane, j) * inv;
            __syncwarp();
            // rank-1 update of rows j+1..last (lane / 16 + 2k), columns j+1..cmax (lane % 16)
            const int c = j + 1 + (lane & 15);
            if (c <= cmax) {
                const T ujc = RB(j, c);
#pragma unroll
                for (int k = 0; k < kBandKL / 2; ++k) {
                    const int i = j + 1 + (lane >> 4) + 2 * k;
                    if (i <= last) RB(i, c) -= RB(i, j) * ujc;
                }
            }
        }
        __syncwarp();
        // row j is final: write it back (the solves multiply by the reciprocal pivot)
        if (lane < kBandW) {
            T e = R[(j & (kLuRing - 1)) * kBandW + lane];
            if (lane == kBandKL) e = e != T(0) ? T(1) / e : T(0);
            G[(int64_t)j * kBandW + lane] = e;
        }
    }
#undef RB
}

constexpr int kSolvePf = 8;   // rows of factors loaded ahead by the band solve

// x = J0^{-1} b for every filament (b and x in the X / f layout; may alias),
// with the factors and the working vector in precision T.
template <typename T>
__global__ void band_solve_kernel(Layout lay, const T *__restrict__ band_all,
                                  const int *__restrict__ piv_all, double ct,
                                  const double *b, double *x, int zmax,
                                  const int *__restrict__ active) {
    extern __shared__ __align__(16) unsigned char zraw[];
    const int wib = threadIdx.x >> 5;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= lay.M) return;
    T *z = reinterpret_cast<T *>(zraw) + (int64_t)wib * zmax;
    const int s0 = lay.off[warp];
    if (active && !active[lay.sys_of[s0]]) return;   // converged system: rows not needed
    const int N = lay.off[warp + 1] - s0;
    const int n = 6 * N - 3;
    const int64_t row0 = 6 * (int64_t)s0 - 3 * (int64_t)warp;
    const T *A = band_all + row0 * kBandW;
    const int *piv = piv_all + row0;
    const double *bf = b + 6 * (int64_t)s0;
    double *xf = x + 6 * (int64_t)s0;
#define BAND(i, c) A[(int64_t)(i) * kBandW + ((c) - (i) + kBandKL)]
    // gather the right-hand side in band order
    for (int e = lane; e < 3 * N; e += 32) {
        const int s = e / 3, r = e % 3;
        z[6 * s + r] = (T)bf[3 + 3 * s + r];   // rotation rows of segment s
        if (s <= N - 2) {
            const double b3n = bf[3 + 3 * N + 3 * s + r];                      // f3 of segment s+1
            const double b3p = (s == 0) ? bf[r] : bf[3 + 3 * N + 3 * (s - 1) + r];
            z[6 * s + 3 + r] = (T)(b3n - b3p);
        }
    }
    const double b1x = bf[0], b1y = bf[1], b1z = bf[2];
    __syncwarp();
    // The factors a row step needs do not depend on z, so each lane loads them
    // kSolvePf rows ahead into a register queue: the loads of the next block are
    // in flight while the current block's dependency chain runs through shared
    // memory. Lane l's entries sit at a fixed offset of consecutive rows:
    // forward L(j + 1 + l, j), backward U(j - 1 - l, j) and the reciprocal U_jj.
    // forward: L with row interchanges applied in elimination order
    T zprev = T(0);   // lane 0: the finished entry of the previous row / column
    {
        T lq[kSolvePf];
        int pq[kSolvePf];
#pragma unroll
        for (int u = 0; u < kSolvePf; ++u) {
            const int j = u;
            lq[u] = (lane < kBandKL && j + 1 + lane < n) ? BAND(j + 1 + lane, j) : T(0);
            pq[u] = j < n ? piv[j] : j;
        }
        for (int jb = 0; jb < n; jb += kSolvePf) {
            T ln[kSolvePf];
            int pn[kSolvePf];
#pragma unroll
            for (int u = 0; u < kSolvePf; ++u) {
                const int j = jb + kSolvePf + u;
                ln[u] = (lane < kBandKL && j + 1 + lane < n) ? BAND(j + 1 + lane, j) : T(0);
                pn[u] = j < n ? piv[j] : j;
            }
#pragma unroll
            for (int u = 0; u < kSolvePf; ++u) {
                const int j = jb + u;
                if (j < n) {
                    // row j after the interchange with row p (p in j .. j+8): every lane
                    // reads both entries; the lane of row p takes the old z_j as its own
                    // entry; z_j itself is stored one row later, when no lane reads it
                    const int p = pq[u];
                    const T zold = z[j], zp = z[p];
                    const T zj = (p != j) ? zp : zold;
                    const int i = j + 1 + lane;
                    if (lane < kBandKL && i < n) z[i] = ((i == p) ? zold : z[i]) - lq[u] * zj;
                    if (lane == 0) {
                        if (j > 0) z[j - 1] = zprev;
                        zprev = zj;
                    }
                    __syncwarp();
                }
            }
#pragma unroll
            for (int u = 0; u < kSolvePf; ++u) {
                lq[u] = ln[u];
                pq[u] = pn[u];
            }
        }
    }
    if (lane == 0) z[n - 1] = zprev;
    __syncwarp();
    // backward, column by column: z_j *= 1/U_jj (stored reciprocal), then the
    // kl + ku rows above take their U_ij z_j
    {
        T uq[kSolvePf], dq[kSolvePf];
#pragma unroll
        for (int u = 0; u < kSolvePf; ++u) {
            const int j = n - 1 - u;
            uq[u] = (lane < kBandKL + kBandKU && j - 1 - lane >= 0) ? BAND(j - 1 - lane, j) : T(0);
            dq[u] = j >= 0 ? BAND(j, j) : T(0);
        }
        for (int jb = n - 1; jb >= 0; jb -= kSolvePf) {
            T un[kSolvePf], dn[kSolvePf];
#pragma unroll
            for (int u = 0; u < kSolvePf; ++u) {
                const int j = jb - kSolvePf - u;
                un[u] = (lane < kBandKL + kBandKU && j - 1 - lane >= 0) ? BAND(j - 1 - lane, j)
                                                                         : T(0);
                dn[u] = j >= 0 ? BAND(j, j) : T(0);
            }
#pragma unroll
            for (int u = 0; u < kSolvePf; ++u) {
                const int j = jb - u;
                if (j >= 0) {
                    const T zj = z[j] * dq[u];
                    const int i = j - 1 - lane;
                    if (lane < kBandKL + kBandKU && i >= 0) z[i] -= uq[u] * zj;
                    if (lane == 0) {
                        if (j < n - 1) z[j + 1] = zprev;
                        zprev = zj;
                    }
                    __syncwarp();
                }
            }
#pragma unroll
            for (int u = 0; u < kSolvePf; ++u) {
                uq[u] = un[u];
                dq[u] = dn[u];
            }
        }
    }
    if (lane == 0) z[0] = zprev;
    __syncwarp();
    // scatter back: u_s, Lam_j, and Y_1 = b1 + c_t Lam_0
    for (int e = lane; e < 3 * N; e += 32) {
        const int s = e / 3, r = e % 3;
        xf[3 + 3 * s + r] = (double)z[6 * s + r];
        if (s <= N - 2) xf[3 + 3 * N + 3 * s + r] = (double)z[6 * s + 3 + r];
    }
    if (lane == 0) {
        const double l0 = (N >= 2) ? (double)z[3] : 0.0, l1 = (N >= 2) ? (double)z[4] : 0.0,
                     l2 = (N >= 2) ? (double)z[5] : 0.0;
        xf[0] = b1x + ct * l0;
        xf[1] = b1y + ct * l1;
        xf[2] = b1z + ct * l2;
    }
#undef BAND
}


J0Params make_params(const fil_ctx *c) {
    const double beta = c->have_prev ? 2.0 / 3.0 : 1.0;
    return J0Params{c->dL, c->KB, c->KT, c->g0, c->kmu, c->knu,
                    beta * c->dt / (6.0 * kPi * c->eta * c->a),
                    beta * c->dt / (8.0 * kPi * c->eta * c->a * c->a * c->a)};
}

}  // namespace

cudaError_t j0_build_factor(fil_ctx *c, const double *X) {
    const unsigned grid = (unsigned)(((int64_t)c->lay.M * 32 + kJ0Threads - 1) / kJ0Threads);
    const J0Params p = make_params(c);
    if (c->band32) {
        // mixed precision: the band is stored, factored and solved in FP32 (J0 is an
        // approximation of the Jacobian far coarser than FP32 rounding; FP64 issues at
        // 1/64 of the FP32 rate on this GPU); its entries are still computed in FP64
        j0_build_kernel<float><<<grid, kJ0Threads, 0, c->stream>>>(c->lay, X, c->qc, c->Tint, p,
                                                                   c->band32);
        band_lu_kernel<float><<<grid, kJ0Threads, 0, c->stream>>>(c->lay, c->band32, c->piv,
                                                                  c->d_flags);
    } else {
        j0_build_kernel<double><<<grid, kJ0Threads, 0, c->stream>>>(c->lay, X, c->qc, c->Tint, p,
                                                                    c->band);
        band_lu_kernel<double><<<grid, kJ0Threads, 0, c->stream>>>(c->lay, c->band, c->piv,
                                                                   c->d_flags);
    }
    c->n_launches += 2;
    return cudaGetLastError();
}

cudaError_t j0_solve(fil_ctx *c, const double *b, double *x, const int *active) {
    // one warp per filament; up to 4 warps per CTA, fewer for long filaments so
    // that each warp's right-hand side fits in shared memory
    const int zmax = 6 * c->lay.maxN;
    const size_t per_warp = (size_t)zmax * sizeof(double);
    int warps = (int)std::min<size_t>(4, kSolveSmemMax / per_warp);
    if (warps < 1) return cudaErrorInvalidValue;
    const size_t smem = warps * per_warp;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(band_solve_kernel<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(band_solve_kernel<float>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = 32 * warps;
    const unsigned grid = (unsigned)(((int64_t)c->lay.M * 32 + threads - 1) / threads);
    if (c->band32)
        band_solve_kernel<float><<<grid, threads, smem, c->stream>>>(
            c->lay, c->band32, c->piv, make_params(c).ct, b, x, zmax, active);
    else
        band_solve_kernel<double><<<grid, threads, smem, c->stream>>>(
            c->lay, c->band, c->piv, make_params(c).ct, b, x, zmax, active);
    c->n_launches += 1;
    return cudaGetLastError();
}

}  // namespace fil
