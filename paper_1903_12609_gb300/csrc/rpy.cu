// Rotne-Prager-Yamakawa mobility apply on sm_103a (paper Sec. 2.7.1).
//
//   V_n     = sum_m Mtt_nm F_m + Mtr_nm T_m
//   Omega_n = sum_m Mrt_nm F_m + Mrr_nm T_m      over all S^2 ordered pairs.
//
// With d = Y_n - Y_m, r = |d| and every block scaled by 8 pi eta, a pair adds
//   V     += A F + B (d.F) d + G (T x d)
//   Omega += C T + D (d.T) d + G (F x d)
// far form (r >= 2a):  A = 1/r + (2a^2/3)/r^3, B = 1/r^3 - 2a^2/r^5,
//                      C = -1/(2 r^3), D = 3/(2 r^5), G = 1/r^3;
// overlapping spheres (r < 2a, equal-radius form of Wajnryb et al., which the
// paper cites for this case):
//                      A = (4/(3a)) (1 - 9r/(32a)),  B = 1/(8 a^2 r),
//                      C = (1 - 27r/(32a) + 5r^3/(64a^3)) / a^3,
//                      D = (9/(32 a r) - 3r/(64 a^3)) / a^3,
//                      G = (1 - 3r/(8a)) / (2 a^3);
// at r = 0 (the self pair, or coincident distinct segments) the d-terms vanish
// and A, C give the self mobilities 1/(6 pi eta a), 1/(8 pi eta a^3).
//
// Kernel design (GB300, one GPU):
//  * No tensor cores: the pair sum is not a dense contraction. The bound is the
//    FP32 (or FP64) FMA pipe; a pair costs ~51 FP32 operations + 1 MUFU.
//  * Each thread owns kRpyTargetsPerThread targets in registers; a CTA owns a
//    tile of kRpyTile targets and streams sources through double-buffered
//    shared memory in chunks of kRpyChunk; all lanes read the same source
//    (broadcast), so shared-memory traffic is 3 LDS.128 per source per thread.
//  * Packed FP32x2 arithmetic: a thread evaluates its target
//    against two sources at once, lane x of every float2 holding the even
//    source and lane y the odd one; the records of a source pair are stored
//    interleaved so that each loaded float2 is an operand. This halves the
//    issued FP32 instructions (the scheduler, not the FMA pipe, limited the
//    one-source form).
//  * Stream-K persistent grid: the (tile, chunk) work units are split evenly
//    over G = #SMs x resident-CTAs; a CTA writes one partial per tile it
//    touches into slot (cta + tile), and the CTA that completes a tile (a
//    counter per tile) sums its partials in CTA order and writes the tile's
//    rows, in the same launch. The order of the sums never depends on timing:
//    results are bitwise reproducible.
//  * Mixed precision: positions are stored as FP32 hi/lo pairs (hi = fl32(Y),
//    lo = fl32(Y - hi)). The inner loop forms d from the hi parts alone,
//    which carries the rounding of the coordinates (~ulp(|Y|)) and is
//    accurate for pairs that are far apart compared with that; a group of
//    kRpyComp sources in which a warp met a pair closer than R_c = 4a is
//    recomputed with d = (t_hi - s_hi) + (t_lo - s_lo), which keeps ~2 ulp of
//    relative accuracy for close pairs. Each target sums kRpyComp pair terms
//    in FP32 and folds them into a (hi, lo) compensated accumulator (TwoSum);
//    the tile's sum adds the partials in FP64.
//  * The inner loop is branch-free (far form only, tracking the smallest r^2);
//    close pairs are rare. A recomputed group in which a warp met an
//    overlapping pair (r < 2a) is computed once more with the exact far /
//    overlap branches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <vector>
#include <mutex>
#include <type_traits>
#include <utility>

#include "fil_internal.cuh"

namespace fil {
namespace {

constexpr float kFarPad = 1.0e5f;   // position of padding sources (they carry no load)

struct RpyConst32 {
    float near2;       // (2a)^2
    float close2;      // R_c^2 = (4a)^2: groups with a pair this close use hi/lo differences
    float k23a2;       // 2a^2/3
    float k2a2;        // 2a^2
    float ov_A0, ov_A1;          // A = ov_A0 - ov_A1 r
    float ov_B;                  // B = ov_B / r
    float ov_C0, ov_C1, ov_C3;   // C = ov_C0 - ov_C1 r + ov_C3 r^3
    float ov_D0, ov_D1;          // D = ov_D0 / r - ov_D1 r
    float ov_G0, ov_G1;          // G = ov_G0 - ov_G1 r
};

struct RpyConst64 {
    double near2, k23a2, k2a2;
    double ov_A0, ov_A1, ov_B, ov_C0, ov_C1, ov_C3, ov_D0, ov_D1, ov_G0, ov_G1;
};

template <typename T, typename K>
__host__ K make_const(double a) {
    K k;
    k.near2 = (T)(4.0 * a * a);
    if constexpr (sizeof(T) == 4) k.close2 = (T)(16.0 * a * a);
    k.k23a2 = (T)(2.0 * a * a / 3.0);
    k.k2a2 = (T)(2.0 * a * a);
    k.ov_A0 = (T)(4.0 / (3.0 * a));
    k.ov_A1 = (T)(4.0 / (3.0 * a) * 9.0 / (32.0 * a));
    k.ov_B = (T)(1.0 / (8.0 * a * a));
    double ia3 = 1.0 / (a * a * a);
    k.ov_C0 = (T)ia3;
    k.ov_C1 = (T)(ia3 * 27.0 / (32.0 * a));
    k.ov_C3 = (T)(ia3 * 5.0 / (64.0 * a * a * a));
    k.ov_D0 = (T)(ia3 * 9.0 / (32.0 * a));
    k.ov_D1 = (T)(ia3 * 3.0 / (64.0 * a * a * a));
    k.ov_G0 = (T)(0.5 * ia3);
    k.ov_G1 = (T)(0.5 * ia3 * 3.0 / (8.0 * a));
    return k;
}

// ---------------------------------------------------------------------------
// Ensembles of independent systems: every system is padded to whole target
// tiles (kRpyTile) in the source/target layout, so that a work unit (tile,
// source chunk) never mixes systems and the apply stays one persistent launch.
// System s owns padded positions [pad_off[s], pad_off[s+1]); its tiles come
// in order, each with ceil(S_s / kRpyChunk) source chunks, and padding records
// sit far away with zero load. With null tables there is one system whose
// padded position equals the segment index (tile = u / n_chunks).
// ---------------------------------------------------------------------------
struct SysMap {
    const int64_t *tile_unit_off;  // [n_tiles + 1] first unit of each listed tile
    const int64_t *tile_src;       // [n_tiles] padded position of the tile's first source
    const int64_t *tile_nsrc;      // [n_tiles] real sources of the tile's system (null: n_src)
    const int *tile_id;            // [n_tiles] padded tile of each listed tile (null: same)
    const int *slot_of;            // [all tiles] list index of a padded tile, -1 if not listed
    const int64_t *pos_of_seg;     // [S] padded position of each segment
    const int *pad_map;            // [Spad] segment at a padded position, or -1
    int64_t n_tiles, n_chunks;     // listed tiles; n_chunks: the one-system case
    int64_t n_src;                 // real sources of the one-system case
    // non-null: {listed tiles, work units} read on the device, so that a captured
    // launch stays valid when the list of active tiles is rewritten
    const int64_t *dyn = nullptr;
};

// The listed tiles and the unit count of a launch (from the device when dynamic).
__device__ __forceinline__ void resolve_dyn(SysMap &m, int64_t &W) {
    if (m.dyn) {
        m.n_tiles = m.dyn[0];
        W = m.dyn[1];
    }
}

__device__ __forceinline__ int64_t tile_unit_begin(const SysMap &m, int64_t tile) {
    return m.tile_unit_off ? m.tile_unit_off[tile] : tile * m.n_chunks;
}

// Tile of work unit u, the tile's first unit and chunk count, and its first source.
__device__ __forceinline__ void locate_unit(const SysMap &m, int64_t u, int64_t &tile,
                                            int64_t &ubeg, int64_t &nch, int64_t &src0) {
    if (!m.tile_unit_off) {
        tile = u / m.n_chunks;
        ubeg = tile * m.n_chunks;
        nch = m.n_chunks;
        src0 = 0;
        return;
    }
    int64_t lo = 0, hi = m.n_tiles;      // tile_unit_off[lo] <= u < tile_unit_off[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (m.tile_unit_off[mid] <= u) lo = mid;
        else hi = mid;
    }
    tile = lo;
    ubeg = m.tile_unit_off[lo];
    nch = m.tile_unit_off[lo + 1] - ubeg;
    src0 = m.tile_src[lo];
}

__device__ __forceinline__ int64_t segment_at(const SysMap &m, int64_t P, int64_t S) {
    return m.pad_map ? (int64_t)m.pad_map[P] : (P < S ? P : -1);
}

// ---------------------------------------------------------------------------
// Pack: FP64 (Y, FT) -> padded FP32 source records of 12 values per segment.
// Positions are taken relative to the first segment, y = Y - Y_0 (the apply is
// translation invariant, and the FP32 rounding of y then depends on the extent
// of the suspension, not on where it sits), hi = fl32(y), lo = fl32(y - hi),
// negated:
//   -hi_x -hi_y -hi_z  F_x F_y F_z  T_x T_y T_z  -lo_z -lo_x -lo_y
// Sources 2p and 2p+1 share the kRpyPairF4 float4 at src + kRpyPairF4 p;
// value c of source h sits at float 2c + h, so each float2 holds one
// component of both (even, odd) and the far-form loop, which needs no lo
// part, reads the first 4.5 float4 of a record.
// Padding records sit far away with zero load, so they add exactly zero.
// ---------------------------------------------------------------------------
__global__ void pack32_kernel(const double *__restrict__ Y, const double *__restrict__ FT,
                              int64_t S, int64_t Spad, SysMap sm, float4 *__restrict__ src) {
    const int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= Spad) return;
    const int64_t i = segment_at(sm, P, S);
    constexpr int kV = 2 * kRpyPairF4;
    float v[kV];
    if (i >= 0) {
        const double y0 = Y[3 * i] - Y[0], y1 = Y[3 * i + 1] - Y[1], y2 = Y[3 * i + 2] - Y[2];
        const float h0 = __double2float_rn(y0), h1 = __double2float_rn(y1),
                    h2 = __double2float_rn(y2);
        const double *f = FT + 6 * i;
        v[0] = -h0; v[1] = -h1; v[2] = -h2;
#pragma unroll
        for (int c = 0; c < 6; ++c) v[3 + c] = __double2float_rn(f[c]);
        v[9] = -__double2float_rn(y2 - (double)h2);
        v[10] = -__double2float_rn(y0 - (double)h0);
        v[11] = -__double2float_rn(y1 - (double)h1);
    } else {
        v[0] = v[1] = v[2] = -kFarPad;
#pragma unroll
        for (int c = 3; c < kV; ++c) v[c] = 0.f;
    }
    float *o = reinterpret_cast<float *>(src + kRpyPairF4 * (P >> 1)) + (P & 1);
#pragma unroll
    for (int c = 0; c < kV; ++c) o[2 * c] = v[c];
}

// FP64 records: 9 doubles per segment (Y, F, T); padding far away, no load.
__global__ void pack64_kernel(const double *__restrict__ Y, const double *__restrict__ FT,
                              int64_t S, int64_t Spad, SysMap sm, double *__restrict__ src) {
    const int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= Spad) return;
    const int64_t i = segment_at(sm, P, S);
    double *o = src + 9 * P;
    if (i >= 0) {
        o[0] = Y[3 * i];
        o[1] = Y[3 * i + 1];
        o[2] = Y[3 * i + 2];
        for (int k = 0; k < 6; ++k) o[3 + k] = FT[6 * i + k];
    } else {
        o[0] = o[1] = o[2] = (double)kFarPad;
        for (int k = 0; k < 6; ++k) o[3 + k] = 0.0;
    }
}

// Error-free transformation s + e = a + b (Knuth's TwoSum), with the adds
// kept out of FMA contraction and reassociation.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// 1/sqrt(x): one MUFU operation (PTX rsqrt.approx.ftz.f32, max relative error
// 2^-22.9 for normal x). Its results are kept only for r^2 >= (2a)^2.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

// sqrt(x) and 1/x: one MUFU operation each (PTX sqrt.approx.ftz.f32,
// rcp.approx.ftz.f32; a few ulp at most, no slow path).
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exact coefficients of one pair (one lane): the far form for r^2 >= (2a)^2,
// the overlapping-sphere form below it and the self values at r = 0, chosen
// without a branch (both are evaluated; this runs in recomputed groups only).
__device__ __forceinline__ void coef_exact(float r2, const RpyConst32 &k, float &A, float &B,
                                           float &C, float &D, float &G) {
    const bool ov = r2 < k.near2;
    const float rinv = rsqrt_approx(fmaxf(r2, k.near2));   // the far form's, finite everywhere
    const float rinv2 = rinv * rinv;
    const float rinv3 = rinv * rinv2;
    const float rinv5 = rinv3 * rinv2;
    const float r = sqrt_approx(r2);
    const float ri = r > 0.f ? rcp_approx(r) : 0.f;
    A = ov ? fmaf(-k.ov_A1, r, k.ov_A0) : fmaf(k.k23a2, rinv3, rinv);
    B = ov ? k.ov_B * ri : fmaf(-k.k2a2, rinv5, rinv3);
    C = ov ? fmaf(k.ov_C3 * r2, r, fmaf(-k.ov_C1, r, k.ov_C0)) : -0.5f * rinv3;
    D = ov ? fmaf(k.ov_D0, ri, -k.ov_D1 * r) : 1.5f * rinv5;
    G = ov ? fmaf(-k.ov_G1, r, k.ov_G0) : rinv3;
}

// How a group of sources is evaluated (pair32x2's MODE).
enum PairMode { kFarHi = 0, kFarHiLo = 1, kExact = 2 };

// The pair terms of one target and the two sources of a packed record (q),
// lane x = even source, lane y = odd source, tracking the smallest r^2 seen.
//  kFarHi (the inner loop): d from the hi parts only and the far form for every
//    pair, branch-free; whatever it produces for close, overlapping or
//    coincident pairs (Inf or NaN at r = 0) is discarded by the caller, which
//    evaluates such groups again.
//  kFarHiLo: d = (t_hi - s_hi) + (t_lo - s_lo), far form; source jx (jx + 1
//    for lane y) equal to self_j is the target itself: its term is zero (d = 0
//    and 1/r taken as 0) and it is left out of the smallest r^2.
//  kExact: hi/lo differences and the exact coefficients of every pair
//    (coef_exact; the self pair takes the self values).
template <int MODE>
__device__ __forceinline__ void pair32x2(const float2 *th, const float2 *tl, const float4 *q,
                                         const RpyConst32 &k, float2 k23, float2 nk2,
                                         float2 *acc, float &rmin2, int self_j = -1,
                                         int jx = 0) {
    const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    const float2 q4 = reinterpret_cast<const float2 *>(q + 4)[0];
    float2 dx = __fadd2_rn(th[0], f2(q0.x, q0.y));
    float2 dy = __fadd2_rn(th[1], f2(q0.z, q0.w));
    float2 dz = __fadd2_rn(th[2], f2(q1.x, q1.y));
    if (MODE != kFarHi) {
        const float4 q5 = q[5];
        const float2 lz = reinterpret_cast<const float2 *>(q + 4)[1];
        dx = __fadd2_rn(dx, __fadd2_rn(tl[0], f2(q5.x, q5.y)));
        dy = __fadd2_rn(dy, __fadd2_rn(tl[1], f2(q5.z, q5.w)));
        dz = __fadd2_rn(dz, __fadd2_rn(tl[2], lz));
    }
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    float2 A, B, C, D, G;
    if (MODE != kExact) {
        float2 rinv = f2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        if (MODE == kFarHiLo) {
            const bool sx = (jx == self_j), sy = (jx + 1 == self_j);
            rinv.x = sx ? 0.f : rinv.x;
            rinv.y = sy ? 0.f : rinv.y;
            rmin2 = fminf(rmin2, fminf(sx ? k.close2 : r2.x, sy ? k.close2 : r2.y));
        } else {
            rmin2 = fminf(rmin2, fminf(r2.x, r2.y));
        }
        const float2 rinv2 = __fmul2_rn(rinv, rinv);
        const float2 rinv3 = __fmul2_rn(rinv, rinv2);
        const float2 rinv5 = __fmul2_rn(rinv3, rinv2);
        A = __ffma2_rn(k23, rinv3, rinv);
        B = __ffma2_rn(nk2, rinv5, rinv3);
        C = __fmul2_rn(f2(-0.5f, -0.5f), rinv3);
        D = __fmul2_rn(f2(1.5f, 1.5f), rinv5);
        G = rinv3;
    } else {
        coef_exact(r2.x, k, A.x, B.x, C.x, D.x, G.x);
        coef_exact(r2.y, k, A.y, B.y, C.y, D.y, G.y);
    }
    const float2 Fx = f2(q1.z, q1.w), Fy = f2(q2.x, q2.y), Fz = f2(q2.z, q2.w);
    const float2 Tx = f2(q3.x, q3.y), Ty = f2(q3.z, q3.w), Tz = q4;
    const float2 bF = __fmul2_rn(B, __ffma2_rn(dx, Fx, __ffma2_rn(dy, Fy, __fmul2_rn(dz, Fz))));
    const float2 dT = __fmul2_rn(D, __ffma2_rn(dx, Tx, __ffma2_rn(dy, Ty, __fmul2_rn(dz, Tz))));
    const float2 ex = __fmul2_rn(G, dx), ey = __fmul2_rn(G, dy), ez = __fmul2_rn(G, dz);
    // (negated operands fold into the packed FMA)
    const float2 nTx = neg2(Tx), nTy = neg2(Ty), nTz = neg2(Tz);
    const float2 nFx = neg2(Fx), nFy = neg2(Fy), nFz = neg2(Fz);
    acc[0] = __ffma2_rn(A, Fx, __ffma2_rn(bF, dx, __ffma2_rn(Ty, ez, __ffma2_rn(nTz, ey, acc[0]))));
    acc[1] = __ffma2_rn(A, Fy, __ffma2_rn(bF, dy, __ffma2_rn(Tz, ex, __ffma2_rn(nTx, ez, acc[1]))));
    acc[2] = __ffma2_rn(A, Fz, __ffma2_rn(bF, dz, __ffma2_rn(Tx, ey, __ffma2_rn(nTy, ex, acc[2]))));
    acc[3] = __ffma2_rn(C, Tx, __ffma2_rn(dT, dx, __ffma2_rn(Fy, ez, __ffma2_rn(nFz, ey, acc[3]))));
    acc[4] = __ffma2_rn(C, Ty, __ffma2_rn(dT, dy, __ffma2_rn(Fz, ex, __ffma2_rn(nFx, ez, acc[4]))));
    acc[5] = __ffma2_rn(C, Tz, __ffma2_rn(dT, dz, __ffma2_rn(Fx, ey, __ffma2_rn(nFy, ex, acc[5]))));
}

// Scalar record ((hi, F_x), (lo, F_y), (T, F_z)) of source h (0 even, 1 odd) of
// a packed record.
__device__ __forceinline__ void unpack_source(const float4 *q, int h, float4 &s0, float4 &s1,
                                              float4 &s2) {
    const float *f = reinterpret_cast<const float *>(q) + h;
    s0 = make_float4(-f[0], -f[2], -f[4], f[6]);
    s1 = make_float4(-f[20], -f[22], -f[18], f[8]);
    s2 = make_float4(f[12], f[14], f[16], f[10]);
}

// One pair in FP64 (record layout: Y, F, T).
__device__ __forceinline__ void pair64(double tx, double ty, double tz, const double *s,
                                       const RpyConst64 &k, double *acc) {
    const double dx = tx - s[0], dy = ty - s[1], dz = tz - s[2];
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    double A, B, C, D, G;
    if (__builtin_expect(r2 < k.near2, 0)) {
        const double r = sqrt(r2);
        const double rinv = r > 0.0 ? 1.0 / r : 0.0;
        A = fma(-k.ov_A1, r, k.ov_A0);
        B = k.ov_B * rinv;
        C = fma(k.ov_C3 * r2, r, fma(-k.ov_C1, r, k.ov_C0));
        D = fma(k.ov_D0, rinv, -k.ov_D1 * r);
        G = fma(-k.ov_G1, r, k.ov_G0);
    } else {
        const double rinv = rsqrt(r2);
        const double rinv2 = rinv * rinv;
        const double rinv3 = rinv * rinv2;
        const double rinv5 = rinv3 * rinv2;
        A = fma(k.k23a2, rinv3, rinv);
        B = fma(-k.k2a2, rinv5, rinv3);
        C = -0.5 * rinv3;
        D = 1.5 * rinv5;
        G = rinv3;
    }
    const double Fx = s[3], Fy = s[4], Fz = s[5], Tx = s[6], Ty = s[7], Tz = s[8];
    const double bF = B * fma(dx, Fx, fma(dy, Fy, dz * Fz));
    const double dT = D * fma(dx, Tx, fma(dy, Ty, dz * Tz));
    const double ex = G * dx, ey = G * dy, ez = G * dz;
    acc[0] = fma(A, Fx, fma(bF, dx, fma(Ty, ez, fma(-Tz, ey, acc[0]))));
    acc[1] = fma(A, Fy, fma(bF, dy, fma(Tz, ex, fma(-Tx, ez, acc[1]))));
    acc[2] = fma(A, Fz, fma(bF, dz, fma(Tx, ey, fma(-Ty, ex, acc[2]))));
    acc[3] = fma(C, Tx, fma(dT, dx, fma(Fy, ez, fma(-Fz, ey, acc[3]))));
    acc[4] = fma(C, Ty, fma(dT, dy, fma(Fz, ex, fma(-Fx, ez, acc[4]))));
    acc[5] = fma(C, Tz, fma(dT, dz, fma(Fx, ey, fma(-Fy, ex, acc[5]))));
}

// Asynchronous copy of one chunk of source records (kRec float4) from global to
// shared memory, 16 bytes per cp.async, spread over the CTA's threads; the
// copies land when cp_async_wait_all returns (plus a barrier for the others').
template <int kRec, int kThreads>
__device__ __forceinline__ void stage_chunk(float4 *dst, const float4 *__restrict__ g, int tid) {
#pragma unroll
    for (int i = tid; i < kRec; i += kThreads) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + i);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(g + i) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Unit range of CTA b in the stream-K split of W units over G CTAs.
__device__ __forceinline__ int64_t unit_start(int64_t b, int64_t W, int64_t G) {
    return (b * W) / G;
}

// ---------------------------------------------------------------------------
// Completion of a tile: the stream-K partials of its targets are summed and
// scaled by 1/(8 pi eta) inside the pair kernel, by the CTA that finishes the
// tile's last work unit, so that no separate reduce launch follows the pair
// kernel and the sums of early tiles overlap the pair work of late ones.
// Every CTA that wrote a partial of the tile adds the units it covered to the
// tile's counter (one acquire-release atomic after a barrier, which orders
// the whole CTA's stores before it); the CTA whose addition completes
// the tile's unit count reads the partials of all the tile's CTAs (from L2),
// adds them in CTA order -- the same order whichever CTA came last, so results
// do not depend on timing -- writes the targets' rows of VW and sets the
// counter back to zero for the next launch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cta_range_of_tile(const SysMap &sm, int64_t tile, int64_t W,
                                                  int64_t G, int64_t &u0, int64_t &u1,
                                                  int64_t &b0, int64_t &b1) {
    // CTA b owns units [floor(bW/G), floor((b+1)W/G)); the CTA that holds unit
    // u is ceil((u+1)G/W) - 1.
    u0 = tile_unit_begin(sm, tile);
    u1 = tile_unit_begin(sm, tile + 1) - 1;
    b0 = ((u0 + 1) * G + W - 1) / W - 1;
    b1 = ((u1 + 1) * G + W - 1) / W - 1;
}

// fetch-and-add with acquire-release semantics at GPU scope: its release
// covers the writes the CTA's threads made before the preceding barrier, its
// acquire the reads they make after the following one
__device__ __forceinline__ int fetch_add_acq_rel(int *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

template <typename PT, int NPART, int TPT>
__device__ __forceinline__ void finish_tile(const PT *part, const SysMap &smap, int64_t tile,
                                            int64_t ptile, int64_t units, int64_t n_chunks,
                                            int64_t W, int64_t G, int *__restrict__ cnt,
                                            double scale, double *__restrict__ VW,
                                            bool worker = true) {
    constexpr int kTile = kRpyThreads * TPT;
    __shared__ int s_last;
    const int tid = threadIdx.x;
    __syncthreads();   // the CTA's partial is written before it is counted
    if (tid == 0)
        s_last = fetch_add_acq_rel(cnt + tile, (int)units) + (int)units == (int)n_chunks;
    __syncthreads();
    // (`worker`: false for the second half of a source-split CTA, which holds no targets)
    if (!s_last || !worker) return;
    int64_t u0, u1, b0, b1;
    cta_range_of_tile(smap, tile, W, G, u0, u1, b0, b1);
    // With G > W (a fixed grid over a short active list) a CTA owns at most one
    // unit and some own none: the tile's CTAs are then the owners of its units.
    const bool by_unit = G > W;
    const int64_t n_parts = by_unit ? u1 - u0 + 1 : b1 - b0 + 1;
    // FP32 partials (hi, lo) are added in float-float arithmetic (TwoSum of the
    // hi parts, the lo parts added to its error, renormalised by a second
    // TwoSum: ~2^-44 relative, far below the 2^-24 of the pair terms) and
    // converted to FP64 once per target: the whole tile's sum runs on one SM,
    // and on GB300 the FP64 pipe has 1/64 of the FP32 rate.
    // FP64 partials are added in FP64.
    using Acc = typename std::conditional<NPART == 2, float, double>::type;
    Acc ah[TPT][6], al[TPT][6];
#pragma unroll
    for (int t = 0; t < TPT; ++t)
#pragma unroll
        for (int c = 0; c < 6; ++c) ah[t][c] = al[t][c] = (Acc)0;
#pragma unroll 4
    for (int64_t i = 0; i < n_parts; ++i) {
        const int64_t cb = by_unit ? ((u0 + i + 1) * G + W - 1) / W - 1 : b0 + i;
        const PT *p = part + (size_t)(cb + tile) * (6 * NPART) * kTile;
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int local = t * kRpyThreads + tid;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                if constexpr (NPART == 2) {
                    const float h = __ldcg(p + c * kTile + local);
                    const float l = __ldcg(p + (6 + c) * kTile + local);
                    float sh, e;
                    two_sum(ah[t][c], h, sh, e);
                    e = __fadd_rn(e, __fadd_rn(al[t][c], l));
                    two_sum(sh, e, ah[t][c], al[t][c]);
                } else {
                    ah[t][c] += (double)__ldcg(p + c * kTile + local);
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t n = segment_at(smap, ptile * kTile + t * kRpyThreads + tid, smap.n_src);
        if (n >= 0) {
#pragma unroll
            for (int c = 0; c < 6; ++c)
                VW[6 * n + c] = ((double)ah[t][c] + (double)al[t][c]) * scale;
        }
    }
    if (tid == 0) cnt[tile] = 0;
}

// ---------------------------------------------------------------------------
// Mixed-precision pair kernel. A CTA of kRpyThreads threads owns a tile of
// kRpyThreads * TPT targets, TPT per thread; their pair terms are summed in
// registers over groups of kRpyComp sources with the branch-free far form and
// the group sums folded (TwoSum) into (hi, lo) accumulators.
//  * TPT = 2, 256-target tiles (large systems): a group in which the warp met
//    a pair closer than R_c is evaluated again with hi/lo differences and the
//    exact coefficients.
//  * TPT = 1, 128-target tiles (small systems: less padding, finer units; a
//    warp's own segments then sit in one of every few dozen groups): the
//    group holding the warp's own segments is recognised by index and
//    evaluated once with hi/lo differences and the self pair masked, other
//    close groups again with hi/lo differences in the far form, and exactly
//    only when distinct segments overlap.
// Measured on GB300, each structure is the faster one for its tile size.
// SPLIT = 2 (128-target tiles only) gives a CTA twice the warps on the same
// targets: the two halves take alternate 32-source groups of every chunk and
// their sums are added (float-float, in half order) before the partial is
// written, so a work unit is done by eight warps instead of four -- more
// warps at work on small problems, whose few units leave SMs short of them.
// ---------------------------------------------------------------------------
template <int TPT, int SPLIT = 1>
__global__ void __launch_bounds__(kRpyThreads * SPLIT,
                                  TPT == 2 ? kRpyMinBlocksTpt2
                                           : (SPLIT == 1 ? kRpyMinBlocksTpt1 : kRpyMinBlocksSplit2))
rpy_pair32_kernel(const float4 *__restrict__ src, SysMap smap, int64_t W, int G, RpyConst32 k,
                  float *__restrict__ part, int *__restrict__ cnt, double scale,
                  double *__restrict__ VW) {
    constexpr int kRec = kRpyPairF4 * (kRpyChunk / 2);   // float4 per chunk
    constexpr int kT = TPT;                               // targets per thread
    constexpr int kTile = kRpyThreads * TPT;              // targets per tile
    static_assert(SPLIT == 1 || (SPLIT == 2 && TPT == 1), "source split: 128-target tiles only");
    __shared__ float4 sm[2][kRec];
    // target slot, and which of the SPLIT sets of source groups the thread takes
    // (both compile-time for SPLIT = 1, so the unsplit kernels are unchanged)
    const int tid = SPLIT == 1 ? (int)threadIdx.x : (int)(threadIdx.x % kRpyThreads);
    const int half = SPLIT == 1 ? 0 : (int)(threadIdx.x / kRpyThreads);
    const int64_t b = blockIdx.x;
    resolve_dyn(smap, W);
    int64_t u = unit_start(b, W, G);
    const int64_t u_end = unit_start(b + 1, W, G);

    while (u < u_end) {
        int64_t tile, ubeg, n_chunks, src0;
        locate_unit(smap, u, tile, ubeg, n_chunks, src0);
        const int64_t c_begin = u - ubeg;
        const int64_t c_end = min(n_chunks, c_begin + (u_end - u));
        const float4 *srcs = src + kRec * (src0 / kRpyChunk);   // this tile's system
        const int64_t ptile = smap.tile_id ? smap.tile_id[tile] : tile;   // padded tile
        // groups of the system's last chunk that hold padding only are skipped
        const int64_t nsrc = smap.tile_nsrc ? smap.tile_nsrc[tile] : smap.n_src;

        // target positions (hi parts) broadcast to both lanes; the lo parts are
        // read again only when a group is recomputed
        // record of target t: trec + t * kTRecStep
        constexpr int kTRecStep = kRpyPairF4 * (kRpyThreads / 2);
        const float4 *trec = src + kRpyPairF4 * ((ptile * kTile + tid) >> 1);
        float2 thb[kT][3];
#pragma unroll
        for (int t = 0; t < kT; ++t) {
            const int64_t n = ptile * kTile + t * kRpyThreads + tid;
            float4 a0, a1, a2;
            unpack_source(src + kRpyPairF4 * (n >> 1), (int)(n & 1), a0, a1, a2);
            thb[t][0] = f2(a0.x, a0.x);
            thb[t][1] = f2(a0.y, a0.y);
            thb[t][2] = f2(a0.z, a0.z);
        }
        const int tpar = tid & 1;   // even / odd record slot of every target of this thread
        [[maybe_unused]] const int lane = tid & 31;
        // first target of this warp (slot 0), for the own-group test of 128-target tiles
        [[maybe_unused]] const int64_t wbase = ptile * kTile + (tid & ~31);
        // 128-target tiles (small systems): a warp whose targets are all padding (in a
        // system's last tile) computes nothing; the reduce never reads those rows
        bool idle = false;
        if constexpr (TPT == 1) idle = wbase - src0 >= nsrc;
        const float2 k23 = f2(k.k23a2, k.k23a2), nk2 = f2(-k.k2a2, -k.k2a2);
        float hi[kT][6], lo[kT][6];
#pragma unroll
        for (int t = 0; t < kT; ++t)
#pragma unroll
            for (int c = 0; c < 6; ++c) hi[t][c] = lo[t][c] = 0.f;

        // first chunk -> buffer 0
        stage_chunk<kRec, kRpyThreads * SPLIT>(sm[0], srcs + kRec * c_begin, threadIdx.x);
        cp_async_wait_all();
        __syncthreads();

        for (int64_t ch = c_begin; ch < c_end; ++ch) {
            const int buf = (int)((ch - c_begin) & 1);
            // the next chunk streams into the other buffer while this one is computed
            // (that buffer was last read before the barrier that ended the previous chunk)
            const bool has_next = (ch + 1 < c_end);
            if (has_next)
                stage_chunk<kRec, kRpyThreads * SPLIT>(sm[buf ^ 1], srcs + kRec * (ch + 1),
                                                       threadIdx.x);
            const float4 *s = sm[buf];
            const int n_grp = (int)min((int64_t)(kRpyChunk / kRpyComp),
                                       (nsrc - ch * kRpyChunk + kRpyComp - 1) / kRpyComp);
#pragma unroll 1
            for (int grp = half; grp < (idle ? 0 : n_grp); grp += SPLIT) {
                const float4 *qg = s + kRpyPairF4 * (grp * (kRpyComp / 2));
                float acc[kT][6];
                if constexpr (TPT == 1) {
                    // the group that holds this warp's own segments (slot t's targets
                    // wbase + t kRpyThreads + lane are sources g0 + lane): one per warp and slot
                    const int64_t g0 = src0 + ch * kRpyChunk + grp * kRpyComp;
                    int own = 0;
#pragma unroll
                    for (int t = 0; t < kT; ++t) own |= (g0 == wbase + t * kRpyThreads) ? (1 << t) : 0;
                    float2 acc2[kT][6];
#pragma unroll
                    for (int t = 0; t < kT; ++t)
#pragma unroll
                        for (int c = 0; c < 6; ++c) acc2[t][c] = f2(0.f, 0.f);
                    float rmin2 = k.close2;
                    bool hilo = own != 0;
                    if (!hilo) {
#pragma unroll (kRpyUnroll / 2)
                        for (int jp = 0; jp < kRpyComp / 2; ++jp) {
#pragma unroll
                            for (int t = 0; t < kT; ++t)
                                pair32x2<kFarHi>(thb[t], thb[t], qg + kRpyPairF4 * jp, k, k23, nk2,
                                                 acc2[t], rmin2);
                        }
                        // a pair closer than R_c: the group again with hi/lo differences
                        hilo = __any_sync(0xffffffffu, rmin2 < k.close2);
                    }
                    if (hilo) {
                        rmin2 = k.close2;
#pragma unroll
                        for (int t = 0; t < kT; ++t) {   // one target at a time (fewer live registers)
                            float4 a0, a1, a2;
                            unpack_source(trec + t * kTRecStep, tpar, a0, a1, a2);
                            const float2 tlb[3] = {f2(a1.x, a1.x), f2(a1.y, a1.y), f2(a1.z, a1.z)};
                            const int self_j = (own >> t) & 1 ? lane : -1;
#pragma unroll
                            for (int c = 0; c < 6; ++c) acc2[t][c] = f2(0.f, 0.f);
#pragma unroll 1
                            for (int jp = 0; jp < kRpyComp / 2; ++jp)
                                pair32x2<kFarHiLo>(thb[t], tlb, qg + kRpyPairF4 * jp, k, k23, nk2,
                                                   acc2[t], rmin2, self_j, 2 * jp);
                        }
                    }
                    // overlapping distinct segments (r < 2a): the exact coefficients
                    const bool exact = hilo && __any_sync(0xffffffffu, rmin2 < k.near2);
                    if (exact) {
#pragma unroll
                        for (int t = 0; t < kT; ++t) {
                            float4 a0, a1, a2;
                            unpack_source(trec + t * kTRecStep, tpar, a0, a1, a2);
                            const float2 tlb[3] = {f2(a1.x, a1.x), f2(a1.y, a1.y), f2(a1.z, a1.z)};
#pragma unroll
                            for (int c = 0; c < 6; ++c) acc2[t][c] = f2(0.f, 0.f);
#pragma unroll 1
                            for (int jp = 0; jp < kRpyComp / 2; ++jp)
                                pair32x2<kExact>(thb[t], tlb, qg + kRpyPairF4 * jp, k, k23, nk2,
                                                 acc2[t], rmin2);
                        }
                    }
#pragma unroll
                    for (int t = 0; t < kT; ++t)
#pragma unroll
                        for (int c = 0; c < 6; ++c) acc[t][c] = __fadd_rn(acc2[t][c].x, acc2[t][c].y);
                    if (own && !exact) {
                        // the self term of the targets whose own segment is in this group
                        // (left out of the far-form pass above): 4/(3a) F_n and T_n / a^3
                        float4 s0, s1, s2;
                        unpack_source(qg + kRpyPairF4 * (lane >> 1), lane & 1, s0, s1, s2);
#pragma unroll
                        for (int t = 0; t < kT; ++t)
                            if ((own >> t) & 1) {
                                acc[t][0] = fmaf(k.ov_A0, s0.w, acc[t][0]);
                                acc[t][1] = fmaf(k.ov_A0, s1.w, acc[t][1]);
                                acc[t][2] = fmaf(k.ov_A0, s2.w, acc[t][2]);
                                acc[t][3] = fmaf(k.ov_C0, s2.x, acc[t][3]);
                                acc[t][4] = fmaf(k.ov_C0, s2.y, acc[t][4]);
                                acc[t][5] = fmaf(k.ov_C0, s2.z, acc[t][5]);
                            }
                    }
                } else {
                    // 256-target tiles (large systems): a far pass with hi-only
                    // differences; a group in which a warp met a pair closer than R_c
                    // (own segments included) is evaluated again exactly
                    float2 acc2[kT][6];
#pragma unroll
                    for (int t = 0; t < kT; ++t)
#pragma unroll
                        for (int c = 0; c < 6; ++c) acc2[t][c] = f2(0.f, 0.f);
                    float rmin2 = k.close2;
#pragma unroll (kRpyUnroll / 2)
                    for (int jp = 0; jp < kRpyComp / 2; ++jp) {
#pragma unroll
                        for (int t = 0; t < kT; ++t)
                            pair32x2<kFarHi>(thb[t], thb[t], qg + kRpyPairF4 * jp, k, k23, nk2,
                                             acc2[t], rmin2);
                    }
                    if (__any_sync(0xffffffffu, rmin2 < k.close2)) {
#pragma unroll
                        for (int t = 0; t < kT; ++t) {   // one target at a time (fewer live registers)
                            float4 a0, a1, a2;
                            unpack_source(trec + t * kTRecStep, tpar, a0, a1, a2);
                            const float2 tlb[3] = {f2(a1.x, a1.x), f2(a1.y, a1.y), f2(a1.z, a1.z)};
#pragma unroll
                            for (int c = 0; c < 6; ++c) acc2[t][c] = f2(0.f, 0.f);
#pragma unroll 1
                            for (int jp = 0; jp < kRpyComp / 2; ++jp)
                                pair32x2<kExact>(thb[t], tlb, qg + kRpyPairF4 * jp, k, k23, nk2,
                                                 acc2[t], rmin2);
                        }
                    }
#pragma unroll
                    for (int t = 0; t < kT; ++t)
#pragma unroll
                        for (int c = 0; c < 6; ++c)
                            acc[t][c] = __fadd_rn(acc2[t][c].x, acc2[t][c].y);
                }
#pragma unroll
                for (int t = 0; t < kT; ++t)
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        float sh, e;
                        two_sum(hi[t][c], acc[t][c], sh, e);
                        hi[t][c] = sh;
                        lo[t][c] = __fadd_rn(lo[t][c], e);
                    }
            }
            if (has_next) cp_async_wait_all();
            __syncthreads();
        }

        if constexpr (SPLIT > 1) {
            // the second half's sums join the first's (TwoSum of the hi parts, the lo
            // parts into its error, renormalised); the buffer is next written after
            // the next segment's first chunk barrier
            __shared__ float xs[12][kRpyThreads];
            if (half == 1) {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    xs[c][tid] = hi[0][c];
                    xs[6 + c][tid] = lo[0][c];
                }
            }
            __syncthreads();
            if (half == 0) {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    float sh, e;
                    two_sum(hi[0][c], xs[c][tid], sh, e);
                    e = __fadd_rn(e, __fadd_rn(lo[0][c], xs[6 + c][tid]));
                    two_sum(sh, e, hi[0][c], lo[0][c]);
                }
            }
        }
        // partial of this CTA for this tile -> slot (b + tile)
        if (half == 0) {
            float *p = part + (size_t)(b + tile) * 12 * kTile;
#pragma unroll
            for (int t = 0; t < kT; ++t) {
                const int local = t * kRpyThreads + tid;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    p[c * kTile + local] = hi[t][c];
                    p[(6 + c) * kTile + local] = lo[t][c];
                }
            }
        }
        finish_tile<float, 2, TPT>(part, smap, tile, ptile, c_end - c_begin, n_chunks, W, G, cnt,
                                   scale, VW, SPLIT == 1 || half == 0);
        u = ubeg + c_end;
    }
}

// ---------------------------------------------------------------------------
// FP64 pair kernel (same stream-K scaffolding).
// ---------------------------------------------------------------------------
template <int TPT>
__global__ void __launch_bounds__(kRpyThreads)
rpy_pair64_kernel(const double *__restrict__ src, SysMap smap, int64_t W, int G, RpyConst64 k,
                  double *__restrict__ part, int *__restrict__ cnt, double scale,
                  double *__restrict__ VW) {
    constexpr int kRec = 9 * kRpyChunk;
    constexpr int kTile = kRpyThreads * TPT;
    __shared__ double sm[2][kRec];
    const int tid = threadIdx.x;
    const int64_t b = blockIdx.x;
    resolve_dyn(smap, W);
    int64_t u = unit_start(b, W, G);
    const int64_t u_end = unit_start(b + 1, W, G);

    while (u < u_end) {
        int64_t tile, ubeg, n_chunks, src0;
        locate_unit(smap, u, tile, ubeg, n_chunks, src0);
        const int64_t c_begin = u - ubeg;
        const int64_t c_end = min(n_chunks, c_begin + (u_end - u));
        const double *srcs = src + 9 * src0;
        const int64_t ptile = smap.tile_id ? smap.tile_id[tile] : tile;
        // real sources of the tile's system (its padding follows them): padded
        // sources carry no load and padded targets are never read, so both are
        // left out (a small system would otherwise cost a whole padded tile x
        // chunk at the FP64 rate)
        const int64_t nsrc = smap.tile_nsrc ? smap.tile_nsrc[tile] : smap.n_src;
        // A tile whose real targets fit in one warp (a system of <= 32 segments)
        // would leave three of the four warps idle, and one warp issues FP64
        // only through its own sub-partition's share of the SM's small FP64
        // rate: then every warp takes the first warp's targets and every fourth
        // source, and the four sums are added in warp order before the partial.
        const bool narrow = nsrc - (ptile * kTile - src0) <= 32;
        const int wid = tid >> 5;

        double ty[TPT][3];
        bool live[TPT];
        bool any = false;
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int64_t n = ptile * kTile + t * kRpyThreads + (narrow ? (tid & 31) : tid);
            ty[t][0] = src[9 * n];
            ty[t][1] = src[9 * n + 1];
            ty[t][2] = src[9 * n + 2];
            live[t] = (!narrow || t == 0) && n - src0 < nsrc;
            any = any || live[t];
        }
        double acc[TPT][6];
#pragma unroll
        for (int t = 0; t < TPT; ++t)
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[t][c] = 0.0;

        {
            const double *g = srcs + 9 * (c_begin * kRpyChunk);
            for (int i = tid; i < kRec; i += kRpyThreads) sm[0][i] = g[i];
        }
        __syncthreads();
        for (int64_t ch = c_begin; ch < c_end; ++ch) {
            const int buf = (int)((ch - c_begin) & 1);
            double pre[(kRec + kRpyThreads - 1) / kRpyThreads];
            const bool has_next = (ch + 1 < c_end);
            if (has_next) {
                const double *g = srcs + 9 * ((ch + 1) * kRpyChunk);
#pragma unroll
                for (int r = 0; r < (kRec + kRpyThreads - 1) / kRpyThreads; ++r) {
                    const int i = tid + r * kRpyThreads;
                    pre[r] = (i < kRec) ? g[i] : 0.0;
                }
            }
            const double *s = sm[buf];
            const int jmax = any ? (int)min((int64_t)kRpyChunk, nsrc - ch * kRpyChunk) : 0;
            const int jstep = narrow ? kRpyThreads / 32 : 1;
#pragma unroll 2
            for (int j = narrow ? wid : 0; j < jmax; j += jstep) {
#pragma unroll
                for (int t = 0; t < TPT; ++t)
                    if (live[t]) pair64(ty[t][0], ty[t][1], ty[t][2], s + 9 * j, k, acc[t]);
            }
            if (has_next) {
#pragma unroll
                for (int r = 0; r < (kRec + kRpyThreads - 1) / kRpyThreads; ++r) {
                    const int i = tid + r * kRpyThreads;
                    if (i < kRec) sm[buf ^ 1][i] = pre[r];
                }
            }
            __syncthreads();
        }
        if (narrow) {
            // the other warps' sums join the first warp's; their own slots (and
            // the second slot of every thread) are padding and stay zero. The
            // buffer is next written after the next segment's first barrier.
            __shared__ double red64[kRpyThreads / 32 - 1][6][32];
            if (wid > 0) {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    red64[wid - 1][c][tid & 31] = acc[0][c];
                    acc[0][c] = 0.0;
                }
            }
            __syncthreads();
            if (wid == 0) {
                for (int w = 0; w < kRpyThreads / 32 - 1; ++w)
#pragma unroll
                    for (int c = 0; c < 6; ++c) acc[0][c] += red64[w][c][tid];
            }
        }
        double *p = part + (size_t)(b + tile) * 6 * kTile;
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int local = t * kRpyThreads + tid;
#pragma unroll
            for (int c = 0; c < 6; ++c) p[c * kTile + local] = acc[t][c];
        }
        finish_tile<double, 1, TPT>(part, smap, tile, ptile, c_end - c_begin, n_chunks, W, G, cnt,
                                    scale, VW);
        u = ubeg + c_end;
    }
}

SysMap sys_map(const fil_ctx *c, bool active_only) {
    SysMap m;
    m.n_src = c->lay.S;
    m.pos_of_seg = c->pos_of_seg_d;
    m.pad_map = c->pad_map_d;
    m.n_chunks = 0;
    if (active_only) {
        m.tile_unit_off = c->act_unit_off_d;
        m.tile_src = c->act_src_d;
        m.tile_nsrc = c->act_nsrc_d;
        m.tile_id = c->act_tile_d;
        m.slot_of = c->act_slot_d;
        m.n_tiles = c->act_tiles;
        m.dyn = c->act_dyn_d;
    } else {
        m.tile_unit_off = c->tile_unit_off_d;
        m.tile_src = c->tile_src_d;
        m.tile_nsrc = c->tile_nsrc_d;
        m.tile_id = c->tile_id_d;
        m.slot_of = c->slot_d;
        m.n_tiles = c->rpy_tiles;
    }
    return m;
}

constexpr int kRpyPad = 256;   // systems start at multiples of this in the padded layout

int64_t count_tiles(const fil_ctx *c, int T) {
    int64_t n = 0;
    for (int s = 0; s < c->n_sys; ++s)
        n += (c->sys_seg_off_h[s + 1] - c->sys_seg_off_h[s] + T - 1) / T;
    return n;
}

// Tiles of T targets of every system (only tiles that hold real targets),
// each with ceil(S_s / chunk) source chunks.
void build_tiles(fil_ctx *c) {
    const int T = rpy_tile(c);
    c->tile_unit_off_h.assign(1, 0);
    c->tile_src_h.clear();
    c->tile_nsrc_h.clear();
    c->tile_sys_h.clear();
    c->tile_id_h.clear();
    for (int s = 0; s < c->n_sys; ++s) {
        const int64_t Ss = c->sys_seg_off_h[s + 1] - c->sys_seg_off_h[s];
        const int64_t tiles = (Ss + T - 1) / T;
        const int64_t chunks = (Ss + kRpyChunk - 1) / kRpyChunk;
        for (int64_t t = 0; t < tiles; ++t) {
            c->tile_unit_off_h.push_back(c->tile_unit_off_h.back() + chunks);
            c->tile_src_h.push_back(c->sys_pad_off_h[s]);
            c->tile_nsrc_h.push_back(Ss);
            c->tile_sys_h.push_back(s);
            c->tile_id_h.push_back((int)(c->sys_pad_off_h[s] / T + t));
        }
    }
    c->rpy_tiles = (int64_t)c->tile_src_h.size();
    c->rpy_units = c->tile_unit_off_h.back();
}

template <typename K>
int occupancy(K kernel, int threads = kRpyThreads) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess)
        return 1;
    return std::max(1, occ);
}

void set_grids(fil_ctx *c) {
    c->rpy_grid32 = c->rpy_ctas * c->num_sms;
    c->rpy_grid64 = c->rpy_ctas * c->num_sms;
}

// Resident CTAs per SM of the pair kernel of a schedule (targets per thread,
// source split; the split exists for the FP32 kernel with one target per thread).
int pair_occupancy(const fil_ctx *c, int tpt, int split) {
    if (!pair32_on(c))
        return tpt == 1 ? occupancy(rpy_pair64_kernel<1>) : occupancy(rpy_pair64_kernel<2>);
    if (tpt == 2) return occupancy(rpy_pair32_kernel<2>);
    return split == 2 ? occupancy(rpy_pair32_kernel<1, 2>, 2 * kRpyThreads)
                      : occupancy(rpy_pair32_kernel<1>);
}

}  // namespace

cudaError_t rpy_setup(fil_ctx *c) {
    c->rpy_tpt = kRpyTargetsPerThread;
    c->rpy_threads = kRpyThreads;
    int occ = pair32_on(c) ? occupancy(rpy_pair32_kernel<kRpyTargetsPerThread>)
                                   : occupancy(rpy_pair64_kernel<kRpyTargetsPerThread>);
    c->rpy_ctas = occ;
    c->rpy_split = 1;
    c->rpy_ctas_max = std::max({occ, occupancy(rpy_pair32_kernel<1>), occupancy(rpy_pair32_kernel<2>),
                                occupancy(rpy_pair32_kernel<1, 2>, 2 * kRpyThreads),
                                occupancy(rpy_pair64_kernel<1>), occupancy(rpy_pair64_kernel<2>)});
    set_grids(c);
    // padded layout: system s occupies [pad_off[s], pad_off[s+1]), a multiple of kRpyPad
    const int ns = c->n_sys;
    c->sys_pad_off_h.assign(ns + 1, 0);
    c->pairs_all = 0.0;
    for (int s = 0; s < ns; ++s) {
        const int64_t Ss = c->sys_seg_off_h[s + 1] - c->sys_seg_off_h[s];
        c->sys_pad_off_h[s + 1] = c->sys_pad_off_h[s] + (Ss + kRpyPad - 1) / kRpyPad * kRpyPad;
        c->pairs_all += (double)Ss * (double)Ss;
    }
    c->pairs_act = c->pairs_all;
    c->Spad = c->sys_pad_off_h[ns];
    c->pos_of_seg_h.resize(c->lay.S);
    c->pad_map_h.assign(c->Spad, -1);
    for (int s = 0; s < ns; ++s)
        for (int64_t g = c->sys_seg_off_h[s]; g < c->sys_seg_off_h[s + 1]; ++g) {
            const int64_t P = c->sys_pad_off_h[s] + (g - c->sys_seg_off_h[s]);
            c->pos_of_seg_h[g] = P;
            c->pad_map_h[P] = (int)g;
        }
    c->rpy_tiles_max = std::max(count_tiles(c, kRpyThreads), count_tiles(c, 2 * kRpyThreads));
    build_tiles(c);
    return cudaSuccess;
}

// Tile tables of the current tile size (after the arena exists, and after a retune).
cudaError_t upload_tiles(fil_ctx *c) {
    std::vector<int> slot(c->Spad / kRpyThreads, -1);
    for (int64_t t = 0; t < c->rpy_tiles; ++t) slot[c->tile_id_h[t]] = (int)t;
    cudaError_t e = cudaMemcpyAsync(c->tile_unit_off_d, c->tile_unit_off_h.data(),
                                    sizeof(int64_t) * c->tile_unit_off_h.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->tile_src_d, c->tile_src_h.data(), sizeof(int64_t) * c->tile_src_h.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->tile_nsrc_d, c->tile_nsrc_h.data(),
                            sizeof(int64_t) * c->tile_nsrc_h.size(), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->tile_id_d, c->tile_id_h.data(), sizeof(int) * c->tile_id_h.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->slot_d, slot.data(), sizeof(int) * slot.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // slot goes out of scope
    return e;
}

cudaError_t rpy_upload_tables(fil_ctx *c) {
    cudaError_t e = upload_tiles(c);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->pos_of_seg_d, c->pos_of_seg_h.data(),
                            sizeof(int64_t) * c->pos_of_seg_h.size(), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->pad_map_d, c->pad_map_h.data(), sizeof(int) * c->pad_map_h.size(),
                            cudaMemcpyHostToDevice, c->stream);
    return e;
}

size_t rpy_partial_bytes(const fil_ctx *c) {
    // slots b + tile for b < G and listed tiles; 12 floats = 6 doubles per target;
    // the largest over the tile sizes and grids the autotuner may choose
    const int64_t G = (int64_t)c->rpy_ctas_max * c->num_sms;
    size_t most = 0;
    for (int tpt = 1; tpt <= 2; ++tpt) {
        const int T = kRpyThreads * tpt;
        const size_t b = (size_t)(G + count_tiles(c, T)) * T * 12 * sizeof(float);
        most = std::max(most, b);
    }
    return most;
}

// The tiles of the systems still iterating (c->active_h), listed for the
// stream-K split of the next applies with active_only.
cudaError_t rpy_set_active(fil_ctx *c) {
    std::vector<int64_t> uoff(1, 0), src, nsrc;
    std::vector<int> tid, slot(c->Spad / kRpyThreads, -1);
    for (int64_t t = 0; t < c->rpy_tiles; ++t) {
        if (!c->active_h[c->tile_sys_h[t]]) continue;
        slot[c->tile_id_h[t]] = (int)tid.size();
        tid.push_back(c->tile_id_h[t]);
        src.push_back(c->tile_src_h[t]);
        nsrc.push_back(c->tile_nsrc_h[t]);
        uoff.push_back(uoff.back() + (c->tile_unit_off_h[t + 1] - c->tile_unit_off_h[t]));
    }
    c->act_tiles = (int64_t)tid.size();
    c->act_units = uoff.back();
    c->pairs_act = 0.0;
    for (int s = 0; s < c->n_sys; ++s)
        if (c->active_h[s]) {
            const double Ss = (double)(c->sys_seg_off_h[s + 1] - c->sys_seg_off_h[s]);
            c->pairs_act += Ss * Ss;
        }
    cudaError_t e = cudaMemcpyAsync(c->act_unit_off_d, uoff.data(), sizeof(int64_t) * uoff.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !tid.empty())
        e = cudaMemcpyAsync(c->act_src_d, src.data(), sizeof(int64_t) * src.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !tid.empty())
        e = cudaMemcpyAsync(c->act_nsrc_d, nsrc.data(), sizeof(int64_t) * nsrc.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !tid.empty())
        e = cudaMemcpyAsync(c->act_tile_d, tid.data(), sizeof(int) * tid.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->act_slot_d, slot.data(), sizeof(int) * slot.size(),
                            cudaMemcpyHostToDevice, c->stream);
    const int64_t dyn[2] = {c->act_tiles, c->act_units};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->act_dyn_d, dyn, sizeof(dyn), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // host vectors go out of scope
    return e;
}

namespace {

// A timing event on the context stream; while the stream is being captured the
// record becomes an event-record node of the graph, so that the events hold
// the kernel's times of each replay.
void prof_record(fil_ctx *c, cudaEvent_t ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    cudaEventRecordWithFlags(ev, c->stream, cs == cudaStreamCaptureStatusActive
                                                ? cudaEventRecordExternal
                                                : cudaEventRecordDefault);
}

}  // namespace

cudaError_t rpy_apply(fil_ctx *c, const double *Y, const double *FT, double *VW,
                      bool active_only) {
    const int64_t S = c->lay.S;
    const double scale = 1.0 / (8.0 * kPi * c->eta);
    const int pb = 256;
    const unsigned pgrid = (unsigned)((c->Spad + pb - 1) / pb);
    const bool timed = c->prof_on && c->prof_n < kProfMax;
    const SysMap sm = sys_map(c, active_only);
    const int64_t W = active_only ? c->act_units : c->rpy_units;
    if (W == 0) return cudaSuccess;
    // the active-tile list changes between applies: its launches keep a fixed grid
    // (and read the unit count from the device), so captured graphs stay valid
    if (pair32_on(c)) {
        const int G = (int)(active_only ? c->rpy_grid32 : std::min<int64_t>(c->rpy_grid32, W));
        pack32_kernel<<<pgrid, pb, 0, c->stream>>>(Y, FT, S, c->Spad, sm, c->src32);
        if (c->tune_ev) cudaEventRecord(c->tune_ev[0], c->stream);
        if (timed) prof_record(c, c->prof_ev[2 * c->prof_n]);
        const RpyConst32 k = make_const<float, RpyConst32>(c->a);
        if (c->rpy_tpt == 1 && c->rpy_split == 2)
            rpy_pair32_kernel<1, 2><<<G, 2 * kRpyThreads, 0, c->stream>>>(
                c->src32, sm, W, G, k, (float *)c->partials, c->tile_cnt, scale, VW);
        else if (c->rpy_tpt == 1)
            rpy_pair32_kernel<1><<<G, kRpyThreads, 0, c->stream>>>(
                c->src32, sm, W, G, k, (float *)c->partials, c->tile_cnt, scale, VW);
        else
            rpy_pair32_kernel<2><<<G, kRpyThreads, 0, c->stream>>>(
                c->src32, sm, W, G, k, (float *)c->partials, c->tile_cnt, scale, VW);
        if (timed) prof_record(c, c->prof_ev[2 * c->prof_n + 1]);
        if (c->tune_ev) cudaEventRecord(c->tune_ev[1], c->stream);
    } else {
        const int G = (int)(active_only ? c->rpy_grid64 : std::min<int64_t>(c->rpy_grid64, W));
        pack64_kernel<<<pgrid, pb, 0, c->stream>>>(Y, FT, S, c->Spad, sm, c->src64);
        if (c->tune_ev) cudaEventRecord(c->tune_ev[0], c->stream);
        if (timed) prof_record(c, c->prof_ev[2 * c->prof_n]);
        const RpyConst64 k = make_const<double, RpyConst64>(c->a);
        if (c->rpy_tpt == 1)
            rpy_pair64_kernel<1><<<G, kRpyThreads, 0, c->stream>>>(
                c->src64, sm, W, G, k, (double *)c->partials, c->tile_cnt, scale, VW);
        else
            rpy_pair64_kernel<2><<<G, kRpyThreads, 0, c->stream>>>(
                c->src64, sm, W, G, k, (double *)c->partials, c->tile_cnt, scale, VW);
        if (timed) prof_record(c, c->prof_ev[2 * c->prof_n + 1]);
        if (c->tune_ev) cudaEventRecord(c->tune_ev[1], c->stream);
    }
    if (timed) c->prof_n += 1;
    c->n_applies += 1;
    c->n_pairs += active_only ? c->pairs_act : c->pairs_all;
    c->n_launches += 2;
    return cudaGetLastError();
}


// Autotuner of the pair kernel: times every (targets per thread, resident CTAs
// per SM) candidate on `reps` applies of (Y, FT) and keeps the fastest. An idle
// GPU runs at a low clock for some tens of milliseconds after work arrives, so
// the applies first run for kSpinUpMs of wall time, and the candidates are then
// swept twice, each keeping the faster of its two times: a candidate measured
// while the clock still climbs is not chosen against or for that reason.
cudaError_t rpy_autotune(fil_ctx *c, const double *Y, const double *FT, double *VW, int reps,
                         double *best_ms) {
    constexpr double kSpinUpMs = 50.0;
    constexpr int kSweeps = 2;
    const int64_t a0 = c->n_applies, l0 = c->n_launches;
    const double p0 = c->n_pairs;
    // each rep's pair kernel is timed by its own pair of events, so
    // that host launch gaps between applies (which dominate tiny problems) do not
    // enter the comparison
    std::vector<cudaEvent_t> ev(2 * (size_t)std::max(1, reps), nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    struct cand { int tpt, split, ctas; float ms; };
    std::vector<cand> cands;
    for (int tpt = 1; tpt <= 2; ++tpt) {
        for (int split = 1; split <= (tpt == 1 && pair32_on(c) ? 2 : 1); ++split) {
            const int occ = pair_occupancy(c, tpt, split);
            for (int ctas = 1; ctas <= std::min(occ, c->rpy_ctas_max); ++ctas)
                cands.push_back({tpt, split, ctas, 1e30f});
        }
    }
    const auto t0 = std::chrono::steady_clock::now();
    while (e == cudaSuccess) {
        for (int r = 0; r < 4 && e == cudaSuccess; ++r) e = rpy_apply(c, Y, FT, VW);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        const std::chrono::duration<double, std::milli> dt = std::chrono::steady_clock::now() - t0;
        if (dt.count() >= kSpinUpMs) break;
    }
    for (int sweep = 0; sweep < kSweeps && e == cudaSuccess; ++sweep) {
        for (cand &k : cands) {
            if (e != cudaSuccess) break;
            c->rpy_tpt = k.tpt;
            c->rpy_split = k.split;
            c->rpy_threads = kRpyThreads;
            c->rpy_ctas = k.ctas;
            set_grids(c);
            build_tiles(c);
            e = upload_tiles(c);
            if (e == cudaSuccess) e = rpy_apply(c, Y, FT, VW);       // warm-up
            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                c->tune_ev = &ev[2 * r];
                e = rpy_apply(c, Y, FT, VW);
                c->tune_ev = nullptr;
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            float ms = 0.f;
            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                float one = 0.f;
                e = cudaEventElapsedTime(&one, ev[2 * r], ev[2 * r + 1]);
                ms += one;
            }
            if (e == cudaSuccess) k.ms = std::min(k.ms, ms);
        }
    }
    c->tune_ev = nullptr;
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    float best = 1e30f;
    int best_tpt = c->rpy_tpt, best_split = c->rpy_split, best_ctas = c->rpy_ctas;
    for (const cand &k : cands)
        if (k.ms < best) {
            best = k.ms;
            best_tpt = k.tpt;
            best_split = k.split;
            best_ctas = k.ctas;
        }
    c->rpy_tpt = best_tpt;
    c->rpy_split = best_split;
    c->rpy_threads = kRpyThreads;
    c->rpy_ctas = best_ctas;
    set_grids(c);
    build_tiles(c);
    if (e == cudaSuccess) e = upload_tiles(c);
    c->n_applies = a0;
    c->n_launches = l0;
    c->n_pairs = p0;
    if (best_ms) *best_ms = best / std::max(1, reps);
    return e;
}

// A given pair schedule (targets per thread, threads per CTA, resident CTAs per
// SM for the stream-K grid); false if the kernel has no such schedule or the
// CTA count exceeds its occupancy.
bool rpy_schedule_valid(const fil_ctx *c, int tpt, int threads, int ctas, int split) {
    if (threads != kRpyThreads || (tpt != 1 && tpt != 2)) return false;
    if (split != 1 && !(split == 2 && tpt == 1 && pair32_on(c))) return false;
    const int occ = pair_occupancy(c, tpt, split);
    return ctas >= 1 && ctas <= std::min(occ, c->rpy_ctas_max);
}

cudaError_t rpy_set_schedule(fil_ctx *c, int tpt, int threads, int ctas, int split) {
    c->rpy_tpt = tpt;
    c->rpy_split = split;
    c->rpy_threads = threads;
    c->rpy_ctas = ctas;
    set_grids(c);
    build_tiles(c);
    return upload_tiles(c);
}

// ---------------------------------------------------------------------------
// Allocation-free mobility apply (fil_rpy_apply_noalloc).
//
// For callers that cannot allocate device memory themselves -- code running
// where cudaMalloc is unavailable or forbidden, e.g. inside another
// framework's memory pool or a process whose allocations are owned by
// someone else -- this variant of the mixed-precision apply uses no context
// and allocates nothing: its scratch (packed FP32 sources, the stream-K
// partial sums and the tiles' completion counters) is the file-scope arrays
// below, which every GPU that loads the library holds until the process exits. The caller passes the inputs and
// the output in device memory.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxSeg = 32768;     // largest S accepted
// The context path runs the stream-K split over (resident CTAs per SM) x SMs
// CTAs. The scratch holds the partial sums of at most kNoAllocMaxSMs SMs at
// the pair kernel's compiled residency (GB300 has 152 SMs); on a larger part
// the grid is capped here, and the results then differ from
// fil_mobility_apply's in rounding only (another summation order).
constexpr int kNoAllocMaxSMs = 152;
constexpr int kNoAllocMaxGrid = kRpyMinBlocksTpt2 * kNoAllocMaxSMs;   // stream-K CTAs at most
constexpr int64_t kNoAllocMaxTiles = (kNoAllocMaxSeg + kRpyTile - 1) / kRpyTile;
constexpr int64_t kNoAllocMaxChunks = (kNoAllocMaxSeg + kRpyChunk - 1) / kRpyChunk;
constexpr int64_t kNoAllocMaxSpad = (kNoAllocMaxTiles * kRpyTile > kNoAllocMaxChunks * kRpyChunk)
                                        ? kNoAllocMaxTiles * kRpyTile
                                        : kNoAllocMaxChunks * kRpyChunk;
constexpr size_t kNoAllocSrcBytes = (size_t)kRpyPairF4 * (kNoAllocMaxSpad / 2) * sizeof(float4);
constexpr size_t kNoAllocPartBytes =
    (size_t)(kNoAllocMaxGrid + kNoAllocMaxTiles) * 12 * kRpyTile * sizeof(float);
constexpr size_t kNoAllocBytes = kNoAllocSrcBytes + kNoAllocPartBytes;   // ~10.6 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
// per-tile completion counters of the pair kernel: zero at load, and every
// launch leaves them zero
static __device__ int g_noalloc_cnt[kNoAllocMaxTiles] = {0};

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[kNoAllocMaxDevices];   // device address of the array, per device
int *g_noalloc_cnt_ptr[kNoAllocMaxDevices];         // and of the counters
int g_noalloc_grid[kNoAllocMaxDevices];

// Once per device, with that device current: the device addresses of the
// arrays (their names are only host-side stand-ins) and the stream-K grid size.
cudaError_t noalloc_setup(int dev, unsigned char **ptr, int **cnt, int *grid) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr, *q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&q, g_noalloc_cnt);
        if (e != cudaSuccess) return e;
        g_noalloc_cnt_ptr[dev] = static_cast<int *>(q);
        int occ = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rpy_pair32_kernel<kRpyTargetsPerThread>,
                                                          kRpyThreads, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_noalloc_grid[dev] = std::max(1, std::min(kNoAllocMaxGrid, std::max(1, occ) * sms));
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *ptr = g_noalloc_ptr[dev];
    *cnt = g_noalloc_cnt_ptr[dev];
    *grid = g_noalloc_grid[dev];
    return cudaSuccess;
}

// Memory the kernels may read on device `dev`: device memory of that device,
// or managed memory. Host memory and memory of another GPU (which these
// kernels could only reach through peer access) are rejected.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // the error of this query only
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// A launch whose own status is returned (cudaGetLastError would also report
// an earlier, unrelated failure of the caller's).
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st,
                   Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace

}  // namespace fil

extern "C" fil_status fil_rpy_apply_noalloc(int64_t n_seg, const double *Y, const double *FT,
                                            double *VW, double a, double eta, void *stream) {
    using namespace fil;
    if (n_seg < 1 || n_seg > kNoAllocMaxSeg) return FIL_EINVAL;
    if (!(a > 0) || !(eta > 0) || !Y || !FT || !VW) return FIL_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return FIL_ECUDA;
    if (!on_device(Y, dev) || !on_device(FT, dev) || !on_device(VW, dev)) return FIL_EINVAL;
    unsigned char *base = nullptr;
    int *cnt = nullptr;
    int grid_max = 1;
    if (noalloc_setup(dev, &base, &cnt, &grid_max) != cudaSuccess) return FIL_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t tiles = (n_seg + kRpyTile - 1) / kRpyTile;
    const int64_t n_chunks = (n_seg + kRpyChunk - 1) / kRpyChunk;
    const int64_t Spad = std::max(tiles * kRpyTile, n_chunks * kRpyChunk);
    const int64_t W = tiles * n_chunks;
    const int G = (int)std::min<int64_t>(grid_max, W);
    float4 *src = reinterpret_cast<float4 *>(base);
    float *part = reinterpret_cast<float *>(base + kNoAllocSrcBytes);
    // every source record up to Spad and every partial slot a tile's sum reads
    // is written below; the tile counters are zero between launches
    const int pb = 256;
    SysMap sm{};                       // one system, no tables
    sm.n_tiles = tiles;
    sm.n_chunks = n_chunks;
    sm.n_src = n_seg;
    cudaError_t e = launch(pack32_kernel, (unsigned)((Spad + pb - 1) / pb), pb, st, Y, FT, n_seg,
                           Spad, sm, src);
    if (e == cudaSuccess)
        e = launch(rpy_pair32_kernel<kRpyTargetsPerThread>, (unsigned)G, kRpyThreads, st,
                   (const float4 *)src, sm, W, G, make_const<float, RpyConst32>(a), part, cnt,
                   1.0 / (8.0 * kPi * eta), VW);
    return e == cudaSuccess ? FIL_OK : FIL_ECUDA;
}
