// Vector kernels of the limited-memory bad Broyden iteration (Algorithm 2).
//
// With w_k = H_k f_k held from the previous iteration, one pass is
//   X_{k+1} = X_k - w_k,   f_{k+1} = f(X_{k+1}),   df = f_{k+1} - f_k,
//   g = H_k f_{k+1} = J0^{-1} f_{k+1} + sum_i c_i (d_i . f_{k+1}),
//   c_{k+1} = -g / ||df||,  d_{k+1} = df / ||df||,
//   w_{k+1} = H_{k+1} f_{k+1} = g + c_{k+1} (d_{k+1} . f_{k+1}),
// which is the algorithm's update with H_k f_{k+1} computed once and reused
// for the next step (one J0 solve per iteration).
//
// Dot products are reduced deterministically: a fixed grid writes one partial
// per block and output, and a single block adds the partials in block order.
#include <cuda_runtime.h>

#include "fil_internal.cuh"

namespace fil {
namespace {

constexpr int kRedThreads = 256;
constexpr int kDotGroup = 4;   // outputs accumulated per pass over the vectors

__global__ void axpy_neg_kernel(int64_t n, const double *__restrict__ x,
                                const double *__restrict__ w, double *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i] - w[i];
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    return s;
}

// Outputs o = 0..k-1: d_o . fn;  o = k: |fn - fk|^2;  o = k+1: (fn - fk) . fn.
__global__ void dots_partial_kernel(int64_t n, const double *__restrict__ fn,
                                    const double *__restrict__ fk, const double *__restrict__ D,
                                    int k, double *__restrict__ part) {
    __shared__ double sh[kRedThreads / 32];
    const int nout = k + 2;
    for (int o0 = 0; o0 < nout; o0 += kDotGroup) {
        double acc[kDotGroup];
#pragma unroll
        for (int j = 0; j < kDotGroup; ++j) acc[j] = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double f = fn[i];
            const double df = f - fk[i];
#pragma unroll
            for (int j = 0; j < kDotGroup; ++j) {
                const int o = o0 + j;
                if (o < k)
                    acc[j] += D[(int64_t)o * n + i] * f;
                else if (o == k)
                    acc[j] += df * df;
                else if (o == k + 1)
                    acc[j] += df * f;
            }
        }
#pragma unroll
        for (int j = 0; j < kDotGroup; ++j) {
            const double s = block_sum(acc[j], sh);
            if (threadIdx.x == 0 && o0 + j < nout) part[(int64_t)(o0 + j) * gridDim.x + blockIdx.x] = s;
        }
    }
}

__global__ void dots_final_kernel(int nout, int nblocks, const double *__restrict__ part,
                                  double *__restrict__ out) {
    // one warp per output, lanes stride the partials, fixed-order tree
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (o >= nout) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += part[(int64_t)o * nblocks + b];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) out[o] = s;
}

// g += sum_i c_i alpha_i; history pair k; w = g + c_k (df . fn)/|df|.
__global__ void update_kernel(int64_t n, int k, const double *__restrict__ scal,
                              const double *__restrict__ fn, const double *__restrict__ fk,
                              double *__restrict__ g, double *__restrict__ C,
                              double *__restrict__ D, double *__restrict__ w,
                              int *__restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double ndf2 = scal[k];
    if (i == 0 && !(ndf2 > 0.0)) flags[0] = 1;
    if (i >= n) return;
    double gi = g[i];
    for (int l = 0; l < k; ++l) gi += C[(int64_t)l * n + i] * scal[l];
    const double ndf = sqrt(ndf2);
    const double c = -gi / ndf;
    const double d = (fn[i] - fk[i]) / ndf;
    C[(int64_t)k * n + i] = c;
    D[(int64_t)k * n + i] = d;
    w[i] = gi + c * (scal[k + 1] / ndf);
}

}  // namespace

cudaError_t broyden_axpy_step(fil_ctx *c) {
    const int64_t n = c->lay.nX;
    axpy_neg_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->Xk, c->w, c->Xn);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t broyden_dots(fil_ctx *c) {
    const int64_t n = c->lay.nX;
    dots_partial_kernel<<<c->red_blocks, kRedThreads, 0, c->stream>>>(n, c->fn, c->fk, c->D, c->k,
                                                                       c->red_part);
    const int nout = c->k + 2;
    dots_final_kernel<<<(nout + 7) / 8, 256, 0, c->stream>>>(nout, c->red_blocks, c->red_part,
                                                             c->scal);
    c->n_launches += 2;
    return cudaGetLastError();
}

cudaError_t broyden_update(fil_ctx *c) {
    const int64_t n = c->lay.nX;
    update_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
        n, c->k, c->scal, c->fn, c->fk, c->g, c->C, c->D, c->w, c->d_flags);
    c->n_launches += 1;
    return cudaGetLastError();
}

}  // namespace fil
