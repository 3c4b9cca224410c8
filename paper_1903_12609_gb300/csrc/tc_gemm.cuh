// BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_100 family):
//   C[M x N] = A[M x K] . B[N x K]^T      (A, B row-major BF16, K contiguous)
// with FP32 accumulation in tensor memory and a fused epilogue. It is the
// contraction of the per-filament warm-start MLP (inference and training).
//
// One CTA computes a 128 x Nt tile (Nt = min(N, 256), a multiple of 32):
//   * K is consumed in stages of 64 (one 128-byte swizzle atom of BF16);
//     128 threads copy the A and B stage tiles from global memory into shared
//     memory in the 128-byte-swizzled K-major layout (16-byte chunk c of row r
//     stored at chunk c ^ (r % 8), 1024-byte aligned tiles);
//   * one thread issues four tcgen05.mma (M = 128, N = Nt, K = 16 each, the
//     shared-memory descriptors advanced by 32 bytes inside the atom) into an
//     FP32 accumulator of Nt tensor-memory columns, then tcgen05.commit to an
//     mbarrier that every thread waits on (bounded) before the stage buffers
//     are reused;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns rows
//     32w..32w+31, i.e. tensor-memory lanes 32w..) and applies bias, ReLU or
//     a ReLU mask, storing FP32 and/or BF16 (row-major and transposed).
// Rows past M read as zero and are not stored; N must be a multiple of 32 and
// K a multiple of 64 (callers pad with zeros).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fil {
namespace tc {

constexpr int kTileM = 128;
constexpr int kTileK = 64;
constexpr int kMaxTileN = 256;
constexpr int kThreads = 128;
constexpr int kTmemCols = 256;
// dynamic shared memory: A and B stage tiles + alignment slack; sized so that
// at most two CTAs share an SM (2 x 256 tensor-memory columns = all 512)
constexpr int kSmemBytes = 100 * 1024;

struct Epilogue {
    float *c_f32;              // [M x ldc] FP32 out (nullable)
    int ldc;
    __nv_bfloat16 *c_bf16;     // [M x ldh] BF16 out (nullable)
    int ldh;
    __nv_bfloat16 *c_bf16_t;   // [N x ldt] BF16 out, transposed (nullable)
    int ldt;
    const float *bias;         // [N] added before the activation (nullable)
    int relu;                  // 1: max(x, 0)
    const __nv_bfloat16 *mask; // [M x ldm]: x *= (mask > 0) (nullable; ReLU derivative)
    int ldm;
    float alpha;               // acc scale (applied first)
    int n_valid;               // columns >= n_valid are not stored (multiples of 32)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), leading byte offset unused (16 B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address, 16-byte units
    d |= (uint64_t)(16 >> 4) << 16;                      // leading byte offset
    d |= (uint64_t)(1024 >> 4) << 32;                    // stride byte offset
    d |= (uint64_t)1 << 46;                              // descriptor version (tcgen05)
    d |= (uint64_t)2 << 61;                              // swizzle: 128 B
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4)                        // D format F32
           | (1u << 7)                      // A format BF16
           | (1u << 10)                     // B format BF16
           | ((uint32_t)(n >> 3) << 17)     // N / 8
           | ((uint32_t)(kTileM >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :
                 : "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(mbar), "r"(count) : "memory");
}

// Bounded wait for phase `parity` of the mbarrier (try_wait suspends for a
// bounded time per call): false if it did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int i = 0; i < (1 << 22); ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kThreads)
gemm_bf16_kernel(const __nv_bfloat16 *__restrict__ A, int lda, const __nv_bfloat16 *__restrict__ B,
                 int ldb, int M, int N, int K, Epilogue ep, int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *sA = base;                              // 128 rows x 128 B
    unsigned char *sB = base + kTileM * 128;               // <= 256 rows x 128 B
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;
    const int n0 = blockIdx.y * kMaxTileN;
    const int nt = min(kMaxTileN, N - n0);
    const uint32_t mb = smem_u32(&mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_u32(&tmem_slot)), "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_bf16(nt);

    uint32_t phase = 0;
    bool failed = false;
    for (int k0 = 0; k0 < K; k0 += kTileK) {
        // stage tiles, 16-byte chunks, 128-byte swizzle
        for (int c = tid; c < kTileM * 8; c += kThreads) {
            const int r = c >> 3, ch = c & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + r < M)
                v = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + k0 + 8 * ch);
            *reinterpret_cast<uint4 *>(sA + r * 128 + ((ch ^ (r & 7)) << 4)) = v;
        }
        for (int c = tid; c < nt * 8; c += kThreads) {
            const int r = c >> 3, ch = c & 7;
            const uint4 v =
                *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * ldb + k0 + 8 * ch);
            *reinterpret_cast<uint4 *>(sB + r * 128 + ((ch ^ (r & 7)) << 4)) = v;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            fence_after();
#pragma unroll
            for (int kk = 0; kk < kTileK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(smem_u32(sA) + 32 * kk), sw128_desc(smem_u32(sB) + 32 * kk),
                         idesc, (k0 > 0 || kk > 0) ? 1u : 0u);
            mma_commit(mb);
        }
        const bool ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
    }
    if (failed) {
        if (tid == 0) atomicExch(err, 1);
        mbar_wait(mb, phase ^ 1u);      // the copies in flight, bounded
    } else {
        // epilogue: thread = row m0 + 32 warp + lane
        const int row = m0 + 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c0 = 0; c0 < nt; c0 += 32) {
            float v[32];
            tmem_ld32(trow + (uint32_t)c0, v);
            const int nb = n0 + c0;
            if (row < M && nb < ep.n_valid) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float x = ep.alpha * v[j];
                    if (ep.bias) x += ep.bias[nb + j];
                    if (ep.relu) x = fmaxf(x, 0.f);
                    if (ep.mask && !(__bfloat162float(ep.mask[(size_t)row * ep.ldm + nb + j]) > 0.f))
                        x = 0.f;
                    v[j] = x;
                }
                if (ep.c_f32) {
                    float4 *o = reinterpret_cast<float4 *>(ep.c_f32 + (size_t)row * ep.ldc + nb);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
                if (ep.c_bf16) {
                    __nv_bfloat162 *o =
                        reinterpret_cast<__nv_bfloat162 *>(ep.c_bf16 + (size_t)row * ep.ldh + nb);
#pragma unroll
                    for (int j = 0; j < 16; ++j) o[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                }
                if (ep.c_bf16_t) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        ep.c_bf16_t[(size_t)(nb + j) * ep.ldt + row] = __float2bfloat16_rn(v[j]);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :
                     : "r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

}  // namespace tc
}  // namespace fil
