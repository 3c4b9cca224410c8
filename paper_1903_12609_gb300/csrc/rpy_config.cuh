// Tile shape of the RPY pair kernels (shared by the launcher and the kernels).
#pragma once

namespace fil {

// ----------------------------------------------------------------------------
// RPY pair-kernel geometry (tuned on GB300 at 32 000 segments).
// ----------------------------------------------------------------------------
constexpr int kRpyThreads = 128;               // threads per CTA
constexpr int kRpyUnroll = 16;                 // unroll of the per-source loop
constexpr int kRpyTargetsPerThread = 2;        // register-blocked targets
constexpr int kRpyTile = kRpyThreads * kRpyTargetsPerThread;   // targets per tile
constexpr int kRpyChunk = 128;                 // sources per shared-memory chunk
constexpr int kRpyComp = 32;                   // sources per compensated partial (FP32)
// Resident CTAs per SM the FP32 pair kernel is compiled for, by targets per
// thread: caps the registers (65536 / (128 threads x CTAs)) so that this many
// CTAs fit (2 targets: 128 registers, 4 CTAs; 1 target: 80 registers, 6 CTAs,
// which measured faster on small systems than 4 or 5).
constexpr int kRpyMinBlocksTpt2 = 4;
constexpr int kRpyMinBlocksTpt1 = 6;
// The one-target kernel with its sources split over two halves of a 256-thread
// CTA: 2 resident CTAs (124 registers; at 3 CTAs, 80 registers, it spills).
constexpr int kRpyMinBlocksSplit2 = 2;
// float4 per two FP32 source records (the packed FP32x2 layout)
constexpr int kRpyPairF4 = 6;

}  // namespace fil
