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
#ifndef FIL_RPY_MINB
#define FIL_RPY_MINB 1
#endif
constexpr int kRpyThreads = 128;               // threads per CTA
constexpr int kRpyUnroll = FIL_RPY_UNROLL;     // unroll of the per-source loop
constexpr int kRpyTargetsPerThread = FIL_RPY_TPT;   // register-blocked targets
constexpr int kRpyTile = kRpyThreads * kRpyTargetsPerThread;   // targets per tile
constexpr int kRpyChunk = 128;                 // sources per shared-memory chunk
constexpr int kRpyComp = 32;                   // sources per compensated partial (FP32)

}  // namespace fil
