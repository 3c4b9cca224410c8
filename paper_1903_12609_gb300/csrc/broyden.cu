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
// Dot products and norms are taken per system (ensembles of independent
// systems; one system otherwise) and reduced deterministically: every block
// covers a slice of one system and writes one partial per output, and a warp
// per (system, output) adds the system's partials in block order. Systems that
// have converged (active = 0) keep their iterate: their step w is zero and
// their history is not updated.
#include <cuda_runtime.h>

#include "fil_internal.cuh"

namespace fil {
namespace {

constexpr int kRedThreads = 256;
constexpr int kDotGroup = 8;   // outputs accumulated per pass over the vectors

__global__ void axpy_neg_kernel(int64_t n, const double *__restrict__ x,
                                const double *__restrict__ w, double *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i] - w[i];
}


// Sums of G per-thread values over the block, written to part[o_j * nb + b]
// (fixed order: warp shuffles, then the warps in order).
template <int G>
__device__ __forceinline__ void block_reduce_write(double (&acc)[G], double *sh, const int *o,
                                                   int nb, double *part) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < G; ++j) {
        double v = acc[j];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
        if (lane == 0) sh[j * 32 + wid] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < G) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[threadIdx.x * 32 + w];
        part[(int64_t)o[threadIdx.x] * nb + blockIdx.x] = s;
    }
    __syncthreads();
}

// d_{o0+j} . fn for j < G over [i0, i1)
// (H = float: the mixed mode's FP32 history, products and the per-thread
// partial sums in FP32, the block sums in FP64)
template <int G, typename H>
__device__ __forceinline__ void dots_group(const H *__restrict__ D, int64_t n, int o0,
                                           const double *__restrict__ fn, int64_t i0, int64_t i1,
                                           double *sh, int nb, double *part) {
    H acc[G];
#pragma unroll
    for (int j = 0; j < G; ++j) acc[j] = H(0);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const H f = (H)fn[i];
#pragma unroll
        for (int j = 0; j < G; ++j) acc[j] = fma(D[(int64_t)(o0 + j) * n + i], f, acc[j]);
    }
    double accd[G];
    int o[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        accd[j] = (double)acc[j];
        o[j] = o0 + j;
    }
    block_reduce_write<G>(accd, sh, o, nb, part);
}

// Outputs o = 0..k-1: d_o . fn;  o = k: |fn - fk|^2;  o = k+1: (fn - fk) . fn,
// over the X slice [blk_beg[b], blk_beg[b+1]) of block column b. Row y = 0 of
// the grid takes the last two, row y >= 1 the outputs 8(y-1) .. 8(y-1)+7 (rows
// past k leave at once), so a long history is read by many blocks at a time;
// each output's sum is the same whichever row computes it. Outputs are taken
// in compile-time groups so that every FP64 instruction is useful work.
template <typename H>
__global__ void dots_partial_kernel(int64_t n, const double *__restrict__ fn,
                                    const double *__restrict__ fk, const H *__restrict__ D,
                                    const int *__restrict__ dk, const int64_t *__restrict__ blk_beg,
                                    const int *__restrict__ blk_sys,
                                    const int *__restrict__ active, double *__restrict__ part) {
    __shared__ double sh[kDotGroup * 32];
    if (active && !active[blk_sys[blockIdx.x]]) return;   // a converged system: not needed
    const int k = *dk;
    const int nb = gridDim.x;
    const int64_t i0 = blk_beg[blockIdx.x], i1 = blk_beg[blockIdx.x + 1];
    if (blockIdx.y == 0) {
        double acc[2] = {0.0, 0.0};
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const double f = fn[i];
            const double df = f - fk[i];
            acc[0] = fma(df, df, acc[0]);
            acc[1] = fma(df, f, acc[1]);
        }
        const int o[2] = {k, k + 1};
        block_reduce_write<2>(acc, sh, o, nb, part);
        return;
    }
    const int o0 = (int)(blockIdx.y - 1) * kDotGroup;
    if (o0 >= k) return;
    switch (k - o0 < kDotGroup ? k - o0 : kDotGroup) {
        case 1: dots_group<1, H>(D, n, o0, fn, i0, i1, sh, nb, part); break;
        case 2: dots_group<2, H>(D, n, o0, fn, i0, i1, sh, nb, part); break;
        case 3: dots_group<3, H>(D, n, o0, fn, i0, i1, sh, nb, part); break;
        case 4: dots_group<4, H>(D, n, o0, fn, i0, i1, sh, nb, part); break;
        case 5: dots_group<5, H>(D, n, o0, fn, i0, i1, sh, nb, part); break;
        case 6: dots_group<6, H>(D, n, o0, fn, i0, i1, sh, nb, part); break;
        case 7: dots_group<7, H>(D, n, o0, fn, i0, i1, sh, nb, part); break;
        default: dots_group<kDotGroup, H>(D, n, o0, fn, i0, i1, sh, nb, part); break;
    }
}

__global__ void dots_final_kernel(int n_sys, int max_out, const int *__restrict__ dk, int nblocks,
                                  const int *__restrict__ sys_blk, const double *__restrict__ part,
                                  int sstride, double *__restrict__ out,
                                  float *__restrict__ out32) {
    // one warp per (system, output), lanes stride the system's partials, fixed-order tree
    const int64_t job = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (job >= (int64_t)n_sys * max_out) return;
    const int sy = (int)(job / max_out), o = (int)(job - (int64_t)sy * max_out);
    if (o >= *dk + 2) return;
    double s = 0.0;
    for (int b = sys_blk[sy] + lane; b < sys_blk[sy + 1]; b += 32) s += part[(int64_t)o * nblocks + b];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) {
        out[(int64_t)sy * sstride + o] = s;
        if (out32) out32[(int64_t)sy * sstride + o] = (float)s;   // for the FP32 history sums
        // |df|^2: also 1/|df| in slot k + 2 (free until the next iteration), so
        // that the update multiplies instead of dividing in every entry
        if (o == *dk) out[(int64_t)sy * sstride + o + 2] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    }
}

// g += sum_i c_i alpha_i; history pair k; w = g + c_k (df . fn)/|df|, with the
// scalars of entry i's system; w = 0 in systems that have converged.
template <typename H>
__global__ void update_kernel(int64_t n, const int *__restrict__ dk,
                              const double *__restrict__ scal_all, const float *__restrict__ scal32,
                              int sstride, const int *__restrict__ sys_of,
                              const int *__restrict__ active, const double *__restrict__ fn,
                              const double *__restrict__ fk, double *__restrict__ g,
                              H *__restrict__ C, H *__restrict__ D, double *__restrict__ w,
                              int *__restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sy = sys_of[i / 6];
    const int k = *dk;
    if (!active[sy]) {
        // a converged system takes no step and no history pair (zero rows, so
        // that carried pairs hold nothing stale for it)
        w[i] = 0.0;
        C[(int64_t)k * n + i] = (H)0;
        D[(int64_t)k * n + i] = (H)0;
        return;
    }
    const double *scal = scal_all + (int64_t)sy * sstride;
    const double ndf2 = scal[k];
    if (!(ndf2 > 0.0)) flags[0] = 1;
    double gi = g[i];
    if (sizeof(H) == sizeof(double)) {
        for (int l = 0; l < k; ++l) gi += (double)C[(int64_t)l * n + i] * scal[l];
    } else {
        // the history sum in FP32 (mixed mode), added to g once
        const float *sc32 = scal32 + (int64_t)sy * sstride;
        float h = 0.f;
        for (int l = 0; l < k; ++l) h = fmaf((float)C[(int64_t)l * n + i], sc32[l], h);
        gi += (double)h;
    }
    const double indf = scal[k + 2];            // 1/|df|
    const double c = -gi * indf;
    const double d = (fn[i] - fk[i]) * indf;
    C[(int64_t)k * n + i] = (H)c;
    D[(int64_t)k * n + i] = (H)d;
    w[i] = gi + c * (scal[k + 1] * indf);
}

__global__ void k_advance_kernel(int *dk) { *dk += 1; }
__global__ void k_set_kernel(int *dk, int k) { *dk = k; }

// w += sum_{l<k} c_l alpha_l (alpha_l = d_l . f in the scalars of entry i's
// system): the carried part of H_0 f at the start of a step.
template <typename H>
__global__ void history_apply_kernel(int64_t n, const int *__restrict__ dk,
                                     const double *__restrict__ scal_all, int sstride,
                                     const int *__restrict__ sys_of, const H *__restrict__ C,
                                     double *__restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = *dk;
    const double *scal = scal_all + (int64_t)sys_of[i / 6] * sstride;
    double s = w[i];
    for (int l = 0; l < k; ++l) s += (double)C[(int64_t)l * n + i] * scal[l];
    w[i] = s;
}

__global__ void mask_inactive_kernel(int64_t n, const int *__restrict__ sys_of,
                                     const int *__restrict__ active, double *__restrict__ v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !active[sys_of[i / 6]]) v[i] = 0.0;
}

// Grid of dots_partial_kernel: a column per X slice, a row for the two
// step outputs and one per group of kDotGroup history outputs (the history
// holds at most hist_cap pairs; rows past the current k leave at once).
dim3 dots_grid(const fil_ctx *c) {
    return dim3((unsigned)c->red_blocks, (unsigned)(1 + (c->hist_cap + kDotGroup - 1) / kDotGroup));
}

}  // namespace

cudaError_t broyden_mask_inactive(fil_ctx *c, double *v) {
    if (c->n_sys == 1) return cudaSuccess;      // the one system is active inside a step
    const int64_t n = c->lay.nX;
    mask_inactive_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->lay.sys_of,
                                                                             c->d_active, v);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t broyden_axpy_step(fil_ctx *c) {
    const int64_t n = c->lay.nX;
    axpy_neg_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->Xk, c->w, c->Xn);
    c->n_launches += 1;
    return cudaGetLastError();
}

cudaError_t broyden_dots(fil_ctx *c) {
    const int64_t n = c->lay.nX;
    if (c->C32)
        dots_partial_kernel<float><<<dots_grid(c), kRedThreads, 0, c->stream>>>(
            n, c->fn, c->fk, c->D32, c->d_k, c->blk_beg, c->blk_sys,
            c->n_sys > 1 ? c->d_active : nullptr, c->red_part);
    else
        dots_partial_kernel<double><<<dots_grid(c), kRedThreads, 0, c->stream>>>(
            n, c->fn, c->fk, c->D, c->d_k, c->blk_beg, c->blk_sys,
            c->n_sys > 1 ? c->d_active : nullptr, c->red_part);
    const int max_out = c->hist_cap + 2;
    const int64_t jobs = (int64_t)c->n_sys * max_out;
    dots_final_kernel<<<(unsigned)((jobs + 7) / 8), 256, 0, c->stream>>>(
        c->n_sys, max_out, c->d_k, c->red_blocks, c->sys_blk_off, c->red_part, c->sstride, c->scal,
        c->C32 ? c->scal32 : nullptr);
    c->n_launches += 2;
    return cudaGetLastError();
}

cudaError_t broyden_update(fil_ctx *c) {
    const int64_t n = c->lay.nX;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (c->C32)
        update_kernel<float><<<grid, 256, 0, c->stream>>>(
            n, c->d_k, c->scal, c->scal32, c->sstride, c->lay.sys_of, c->d_active, c->fn, c->fk,
            c->g, c->C32, c->D32, c->w, c->d_flags);
    else
        update_kernel<double><<<grid, 256, 0, c->stream>>>(
            n, c->d_k, c->scal, nullptr, c->sstride, c->lay.sys_of, c->d_active, c->fn, c->fk,
            c->g, c->C, c->D, c->w, c->d_flags);
    k_advance_kernel<<<1, 1, 0, c->stream>>>(c->d_k);     // the next history slot
    c->n_launches += 2;
    return cudaGetLastError();
}

cudaError_t broyden_carry(fil_ctx *c, int from, int m, const double *f, double *w) {
    const int64_t n = c->lay.nX;
    const size_t vb = (size_t)n * (c->C32 ? sizeof(float) : sizeof(double));
    char *C = c->C32 ? (char *)c->C32 : (char *)c->C;
    char *D = c->D32 ? (char *)c->D32 : (char *)c->D;
    // pair from + i -> i in increasing i: each copy reads a slot above the one
    // it writes, never one already written
    for (int i = 0; from > 0 && i < m; ++i) {
        cudaError_t e = cudaMemcpyAsync(C + i * vb, C + (size_t)(from + i) * vb, vb,
                                        cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(D + i * vb, D + (size_t)(from + i) * vb, vb,
                                cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
    }
    k_set_kernel<<<1, 1, 0, c->stream>>>(c->d_k, m);
    // alpha_i = d_i . f (outputs k and k + 1 come out zero with fn = fk = f)
    if (c->C32)
        dots_partial_kernel<float><<<dots_grid(c), kRedThreads, 0, c->stream>>>(
            n, f, f, c->D32, c->d_k, c->blk_beg, c->blk_sys, nullptr, c->red_part);
    else
        dots_partial_kernel<double><<<dots_grid(c), kRedThreads, 0, c->stream>>>(
            n, f, f, c->D, c->d_k, c->blk_beg, c->blk_sys, nullptr, c->red_part);
    const int max_out = c->hist_cap + 2;
    const int64_t jobs = (int64_t)c->n_sys * max_out;
    dots_final_kernel<<<(unsigned)((jobs + 7) / 8), 256, 0, c->stream>>>(
        c->n_sys, max_out, c->d_k, c->red_blocks, c->sys_blk_off, c->red_part, c->sstride,
        c->scal, c->C32 ? c->scal32 : nullptr);
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (c->C32)
        history_apply_kernel<float><<<grid, 256, 0, c->stream>>>(n, c->d_k, c->scal, c->sstride,
                                                                  c->lay.sys_of, c->C32, w);
    else
        history_apply_kernel<double><<<grid, 256, 0, c->stream>>>(n, c->d_k, c->scal, c->sstride,
                                                                   c->lay.sys_of, c->C, w);
    c->n_launches += 4;
    return cudaGetLastError();
}

}  // namespace fil
