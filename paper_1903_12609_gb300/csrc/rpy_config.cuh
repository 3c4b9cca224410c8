// Tile shape of the RPY pair kernels (shared by the launcher and the kernels).
#pragma once

namespace fil {

// ----------------------------------------------------------------------------
// RPY pair-kernel geometry (shared by the launcher and the kernels).
// ----------------------------------------------------------------------------
// Tile shape of the FP32 pair kernel; the defaults are the tuned values and the
// macros only exist so that tile-shape sweeps can rebuild the library.
#ifndef FIL_RPY_TPT
#define FIL_RPY_TPT 2
#endif
#ifndef FIL_RPY_UNROLL
#define FIL_RPY_UNROLL 8
#endif
// Resident CTAs per SM the FP32 pair kernel is compiled for, by targets per
// thread: caps the registers (65536 / (128 threads x CTAs)) so that this many
// CTAs fit.
#ifndef FIL_RPY_MINB_TPT2
#define FIL_RPY_MINB_TPT2 4
#endif
#ifndef FIL_RPY_MINB_TPT1
#define FIL_RPY_MINB_TPT1 4
#endif
// 1: the FP32 pair kernel works on two sources at once with packed FP32x2
// arithmetic (sm_100 family); 0: one source at a time.
#ifndef FIL_RPY_PACKED
#define FIL_RPY_PACKED 1
#endif
#ifndef FIL_RPY_THREADS
#define FIL_RPY_THREADS 128
#endif
// resident CTAs per SM assumed by the stream-K grid (0: the occupancy API's)
#ifndef FIL_RPY_OCC
#define FIL_RPY_OCC 0
#endif
constexpr int kRpyThreads = FIL_RPY_THREADS;   // threads per CTA
constexpr int kRpyUnroll = FIL_RPY_UNROLL;     // unroll of the per-source loop
constexpr int kRpyTargetsPerThread = FIL_RPY_TPT;   // register-blocked targets
constexpr int kRpyTile = kRpyThreads * kRpyTargetsPerThread;   // targets per tile
constexpr int kRpyChunk = 128;                 // sources per shared-memory chunk
constexpr int kRpyComp = 32;                   // sources per compensated partial (FP32)
// float4 per two FP32 source records
constexpr int kRpyPairF4 = 6;

}  // namespace fil
