// Steric barrier force between segments (Sec. 2.6, eqn barrier-force):
//   F^B_n = sum_m F^S ((4a^2 chi^2 - r^2) / (4a^2 (chi^2 - 1)))^4 r_nm / (2a),  r < 2 chi a,
// over m in the same system, m != n, excluding the neighbours n +- 1 of the
// same filament; added to the force of the mobility problem's right-hand side.
//
// A cutoff pass on a hashed uniform grid of cell size h = 2 chi a: every
// segment's cell (plus its system, so that the systems of an ensemble do not
// share buckets) hashes into a power-of-two table of fixed-capacity buckets;
// a segment then scans the buckets of its 27 neighbouring cells (each distinct
// bucket once). The candidates within range are put in increasing segment
// order before they are summed, so the result does not depend on the order in
// which the buckets were filled. A bucket or candidate list that overflows
// sets status flag 2 (the residual evaluation then fails with FIL_EOVERFLOW).
//
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the scan
// works on integer cells and FP32 positions within the cell (exact to ~1e-7 a
// whatever the size of the box), computed once per segment by the binning
// kernel; only entries that pass the FP32 range test with a 0.1% margin are
// tested again, and summed, in FP64.
#include <cuda_runtime.h>

#include "fil_internal.cuh"
#include "quat.cuh"

namespace fil {
namespace {

constexpr int kStericWarps = 8;   // warps (segments) per CTA of the force kernel

__device__ __forceinline__ uint32_t cell_hash(int ix, int iy, int iz, int sys, uint32_t mask) {
    const uint32_t h = (uint32_t)ix * 73856093u ^ (uint32_t)iy * 19349663u ^
                       (uint32_t)iz * 83492791u ^ (uint32_t)sys * 2654435761u;
    return h & mask;
}

// cell, position within the cell, and the bucket entry of every segment
__global__ void steric_bin_kernel(int64_t S, const double *__restrict__ Y,
                                  const int *__restrict__ sys_of, double h, double inv_h,
                                  uint32_t mask, int cap, int *__restrict__ count,
                                  int *__restrict__ bucket, int4 *__restrict__ cell,
                                  float4 *__restrict__ frac, int *__restrict__ flags) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S) return;
    const double x = Y[3 * g], y = Y[3 * g + 1], z = Y[3 * g + 2];
    const double cx = floor(x * inv_h), cy = floor(y * inv_h), cz = floor(z * inv_h);
    const int sys = sys_of[g];
    const int4 c = make_int4((int)cx, (int)cy, (int)cz, sys);
    cell[g] = c;
    frac[g] = make_float4((float)(x - cx * h), (float)(y - cy * h), (float)(z - cz * h), 0.f);
    const uint32_t b = cell_hash(c.x, c.y, c.z, sys, mask);
    const int slot = atomicAdd(count + b, 1);
    if (slot < cap) bucket[(int64_t)b * cap + slot] = (int)g;
    else atomicOr(flags + 2, 1);
}

// One warp per segment: lane c < 27 takes neighbour cell c (dx, dy, dz) =
// (c / 9 - 1, c / 3 % 3 - 1, c % 3 - 1); lanes whose cell hashes to a bucket
// that a lower lane already holds skip it. Candidates within range go to a
// per-warp list in shared memory, which is then put in increasing segment
// order (rank of each entry); lane k evaluates the k-th and (k+32)-th
// candidates and a fixed shuffle tree sums the lanes, so the sum does not
// depend on the order in which the buckets were filled.
__global__ void __launch_bounds__(32 * kStericWarps)
steric_force_kernel(Layout lay, const double *__restrict__ Y, float hf, uint32_t mask, int cap,
                    const int *__restrict__ count, const int *__restrict__ bucket,
                    const int4 *__restrict__ cell, const float4 *__restrict__ frac, double a,
                    double FS, double chi, const int *__restrict__ active,
                    double *__restrict__ FT, int *__restrict__ flags) {
    static_assert(kStericNbrMax <= 64, "two candidates per lane");
    __shared__ int s_cand[kStericWarps][kStericNbrMax];
    __shared__ int s_sorted[kStericWarps][kStericNbrMax];
    __shared__ int s_n[kStericWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // warp-uniform
    if (n >= lay.S) return;
    const int4 cn = cell[n];
    const int sys = cn.w;
    if (active && !active[sys]) return;
    const float4 pn = frac[n];
    const int fn = lay.fil_of[n];
    const double rc2 = 4.0 * a * a * chi * chi;
    const float rc2_pre = (float)(rc2 * 1.001);
    if (lane == 0) s_n[w] = 0;
    __syncwarp();
    uint32_t b = 0xffffffffu;
    if (lane < 27)
        b = cell_hash(cn.x + lane / 9 - 1, cn.y + lane / 3 % 3 - 1, cn.z + lane % 3 - 1, sys,
                      mask);
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (lane < 27 && __ffs(peers) - 1 == lane) {
        const int cnt = min(count[b], cap);
        for (int e = 0; e < cnt; ++e) {
            const int m = bucket[(int64_t)b * cap + e];
            if (m == n) continue;
            const int4 cm = cell[m];
            if (cm.w != sys) continue;
            if ((m == n + 1 || m == n - 1) && lay.fil_of[m] == fn) continue;
            const float4 pm = frac[m];
            const float dx = fmaf((float)(cn.x - cm.x), hf, pn.x - pm.x);
            const float dy = fmaf((float)(cn.y - cm.y), hf, pn.y - pm.y);
            const float dz = fmaf((float)(cn.z - cm.z), hf, pn.z - pm.z);
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= rc2_pre) continue;
            const V3 d = ld3(Y + 3 * n) - ld3(Y + 3 * (int64_t)m);
            if (dot(d, d) >= rc2) continue;
            const int slot = atomicAdd(&s_n[w], 1);
            if (slot < kStericNbrMax) s_cand[w][slot] = m;
            else atomicOr(flags + 2, 1);
        }
    }
    __syncwarp();
    const int nc = min(s_n[w], kStericNbrMax);
    if (nc == 0) return;
    // increasing segment order: an entry's rank is the number of smaller entries
    for (int e = lane; e < nc; e += 32) {
        const int v = s_cand[w][e];
        int r = 0;
        for (int j = 0; j < nc; ++j) r += s_cand[w][j] < v;
        s_sorted[w][r] = v;
    }
    __syncwarp();
    const V3 yn = ld3(Y + 3 * n);
    const double inv = 1.0 / (4.0 * a * a * (chi * chi - 1.0));
    const double fs = FS / (2.0 * a);
    V3 F = v3(0, 0, 0);
    for (int e = lane; e < nc; e += 32) {
        const V3 d = yn - ld3(Y + 3 * (int64_t)s_sorted[w][e]);
        const double x = (rc2 - dot(d, d)) * inv;
        const double x2 = x * x;
        F = F + (fs * x2 * x2) * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        F.x += __shfl_xor_sync(0xffffffffu, F.x, o);
        F.y += __shfl_xor_sync(0xffffffffu, F.y, o);
        F.z += __shfl_xor_sync(0xffffffffu, F.z, o);
    }
    if (lane == 0) {
        double *f = FT + 6 * n;
        f[0] += F.x;
        f[1] += F.y;
        f[2] += F.z;
    }
}

}  // namespace

cudaError_t steric_forces(fil_ctx *c, bool active_only) {
    if (!(c->steric_FS != 0.0)) return cudaSuccess;
    const int64_t S = c->lay.S;
    const double h = 2.0 * c->steric_chi * c->a;
    const uint32_t mask = (uint32_t)(c->steric_buckets - 1);
    cudaError_t e = cudaMemsetAsync(c->steric_count, 0, sizeof(int) * c->steric_buckets, c->stream);
    if (e != cudaSuccess) return e;
    steric_bin_kernel<<<(unsigned)((S + 255) / 256), 256, 0, c->stream>>>(
        S, c->Yc, c->lay.sys_of, h, 1.0 / h, mask, kStericCap, c->steric_count, c->steric_bucket,
        c->steric_cell, c->steric_frac, c->d_flags);
    steric_force_kernel<<<(unsigned)((S + kStericWarps - 1) / kStericWarps), 32 * kStericWarps, 0,
                          c->stream>>>(
        c->lay, c->Yc, (float)h, mask, kStericCap, c->steric_count, c->steric_bucket,
        c->steric_cell, c->steric_frac, c->a, c->steric_FS, c->steric_chi,
        active_only ? c->d_active : nullptr, c->FT, c->d_flags);
    c->n_launches += 2;
    return cudaGetLastError();
}

}  // namespace fil
