// Steric barrier force between segments (Sec. 2.6, eqn barrier-force):
//   F^B_n = sum_m F^S ((4a^2 chi^2 - r^2) / (4a^2 (chi^2 - 1)))^4 r_nm / (2a),  r < 2 chi a,
// over m in the same system, m != n, excluding the neighbours n +- 1 of the
// same filament; added to the force of the mobility problem's right-hand side.
//
// A cutoff pass on a hashed uniform grid of cell size h = 2 chi a: every
// segment's cell (plus its system, so that the systems of an ensemble do not
// share buckets) hashes into a power-of-two table of fixed-capacity buckets;
// a segment then scans the buckets of its 27 neighbouring cells (each distinct
// bucket once). The candidates within range are summed in increasing segment
// order, so the result does not depend on the order in which the buckets were
// filled. A bucket or candidate list that overflows sets status flag 2 (the
// residual evaluation then fails with FIL_EOVERFLOW).
#include <cuda_runtime.h>

#include "fil_internal.cuh"
#include "quat.cuh"

namespace fil {
namespace {

__device__ __forceinline__ uint32_t cell_hash(int64_t ix, int64_t iy, int64_t iz, int sys,
                                              uint32_t mask) {
    const uint32_t h = (uint32_t)ix * 73856093u ^ (uint32_t)iy * 19349663u ^
                       (uint32_t)iz * 83492791u ^ (uint32_t)sys * 2654435761u;
    return h & mask;
}

__device__ __forceinline__ int64_t cell_of(double x, double inv_h) {
    return (int64_t)floor(x * inv_h);
}

__global__ void steric_bin_kernel(int64_t S, const double *__restrict__ Y,
                                  const int *__restrict__ sys_of, double inv_h, uint32_t mask,
                                  int cap, int *__restrict__ count, int *__restrict__ bucket,
                                  int *__restrict__ flags) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S) return;
    const uint32_t b = cell_hash(cell_of(Y[3 * g], inv_h), cell_of(Y[3 * g + 1], inv_h),
                                 cell_of(Y[3 * g + 2], inv_h), sys_of[g], mask);
    const int slot = atomicAdd(count + b, 1);
    if (slot < cap) bucket[(int64_t)b * cap + slot] = (int)g;
    else atomicOr(flags + 2, 1);
}

__global__ void steric_force_kernel(Layout lay, const double *__restrict__ Y, double inv_h,
                                    uint32_t mask, int cap, const int *__restrict__ count,
                                    const int *__restrict__ bucket, double a, double FS,
                                    double chi, const int *__restrict__ active,
                                    double *__restrict__ FT, int *__restrict__ flags) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= lay.S) return;
    const int sys = lay.sys_of[n];
    if (active && !active[sys]) return;
    const V3 yn = ld3(Y + 3 * n);
    const int fn = lay.fil_of[n];
    const double rc2 = 4.0 * a * a * chi * chi;
    const int64_t cx = cell_of(yn.x, inv_h), cy = cell_of(yn.y, inv_h), cz = cell_of(yn.z, inv_h);
    int cand[kStericNbrMax];
    int nc = 0;
    uint32_t seen[27];
    int ns = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                const uint32_t b = cell_hash(cx + dx, cy + dy, cz + dz, sys, mask);
                bool dup = false;
                for (int k = 0; k < ns; ++k) dup |= seen[k] == b;
                if (dup) continue;
                seen[ns++] = b;
                const int cnt = min(count[b], cap);
                for (int e = 0; e < cnt; ++e) {
                    const int m = bucket[(int64_t)b * cap + e];
                    if (m == n || lay.sys_of[m] != sys) continue;
                    if (lay.fil_of[m] == fn && (m == n + 1 || m == n - 1)) continue;
                    const V3 d = yn - ld3(Y + 3 * (int64_t)m);
                    if (dot(d, d) >= rc2) continue;
                    if (nc < kStericNbrMax) {
                        // insert m in increasing order
                        int k = nc++;
                        while (k > 0 && cand[k - 1] > m) {
                            cand[k] = cand[k - 1];
                            --k;
                        }
                        cand[k] = m;
                    } else {
                        atomicOr(flags + 2, 1);
                    }
                }
            }
    if (nc == 0) return;
    const double inv = 1.0 / (4.0 * a * a * (chi * chi - 1.0));
    V3 F = v3(0, 0, 0);
    for (int k = 0; k < nc; ++k) {
        const V3 d = yn - ld3(Y + 3 * (int64_t)cand[k]);
        const double x = (rc2 - dot(d, d)) * inv;
        const double x2 = x * x;
        F = F + (FS * x2 * x2 / (2.0 * a)) * d;
    }
    double *f = FT + 6 * n;
    f[0] += F.x;
    f[1] += F.y;
    f[2] += F.z;
}

}  // namespace

cudaError_t steric_forces(fil_ctx *c, bool active_only) {
    if (!(c->steric_FS != 0.0)) return cudaSuccess;
    const int64_t S = c->lay.S;
    const double inv_h = 1.0 / (2.0 * c->steric_chi * c->a);
    const uint32_t mask = (uint32_t)(c->steric_buckets - 1);
    cudaError_t e = cudaMemsetAsync(c->steric_count, 0, sizeof(int) * c->steric_buckets, c->stream);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((S + 255) / 256);
    steric_bin_kernel<<<grid, 256, 0, c->stream>>>(S, c->Yc, c->lay.sys_of, inv_h, mask,
                                                   kStericCap, c->steric_count, c->steric_bucket,
                                                   c->d_flags);
    steric_force_kernel<<<grid, 256, 0, c->stream>>>(c->lay, c->Yc, inv_h, mask, kStericCap,
                                                     c->steric_count, c->steric_bucket, c->a,
                                                     c->steric_FS, c->steric_chi,
                                                     active_only ? c->d_active : nullptr, c->FT,
                                                     c->d_flags);
    c->n_launches += 2;
    return cudaGetLastError();
}

}  // namespace fil
