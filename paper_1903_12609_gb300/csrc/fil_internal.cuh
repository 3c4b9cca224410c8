// Internal declarations of the GB300 filament library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fil.h"
#include "../../include/fil_mlp.h"
#include "rpy_config.cuh"

namespace fil {

constexpr double kPi = 3.14159265358979323846;
constexpr int kProfMax = 4096;   // timed pair-kernel launches kept per read

// ----------------------------------------------------------------------------
// J0 band geometry: after eliminating Y_1 and differencing the constraint rows
// the per-filament system is block-pentadiagonal in 3x3 blocks, i.e. a banded
// matrix with 8 sub- and 8 super-diagonals (16 after partial pivoting).
// ----------------------------------------------------------------------------
constexpr int kBandKL = 8;
constexpr int kBandKU = 8;
constexpr int kBandW = 2 * kBandKL + kBandKU + 1;   // row window: c - i in [-8, 16]
constexpr size_t kSolveSmemMax = 200 * 1024;        // shared memory of one band-solve CTA
constexpr int kMaxSegPerFil = (int)(kSolveSmemMax / (6 * sizeof(double)));
// The filament-RPY J0 keeps a filament's block in shared memory for its
// FP32 inverse: (6N)^2 floats <= 200 KB, i.e. N <= 38; refinement steps per solve.
constexpr int kMaxDenseSeg = 38;
constexpr int kJ0Refine = 1;
constexpr int kStericCap = 16;      // segments per bucket of the steric cell grid
constexpr int kStericNbrMax = 48;   // segments within range of one segment

struct Layout {
    int M = 0;           // filaments
    int64_t S = 0;       // segments
    int64_t nX = 0;      // 6S
    int64_t nlam = 0;    // S - M
    int maxN = 0;
    int *N = nullptr;        // [M]
    int *off = nullptr;      // [M+1] segment offsets
    int *fil_of = nullptr;   // [S] filament of a segment
    int *sys_of = nullptr;   // [S] system of a segment (ensembles; one system: all 0)
};

}  // namespace fil

struct fil_ctx;
namespace fil {
// RPY pair sums in FP32 (FIL_MIXED, FIL_PAIR32) rather than FP64.
inline bool pair32_on(const fil_ctx *c);
// J0 factors, solves and the Broyden history in FP32 (FIL_MIXED only).
inline bool fast_mixed(const fil_ctx *c);
}  // namespace fil

struct fil_ctx {
    // parameters
    fil::Layout lay;
    std::vector<int> N_host, off_host;
    double a, eta, dL, KB, KT, g0, kmu, knu, dt, tol;
    int max_iter, prec;
    cudaStream_t stream;
    int device, num_sms;
    std::string err;

    // time-integration state (uprev2, lamprev: u and Lambda one step further
    // back, used by the initial guess once hist >= 2; Yprev2, uprev3, lamprev2
    // one step further still, used by the quadratic initial guess)
    double *Y, *Yprev, *q, *uprev, *lam, *uprev2, *lamprev;
    double *Yprev2, *uprev3, *lamprev2;
    int have_prev;
    int hist;              // steps committed since the last set_state / init
    int ylev;              // past Y levels held (Yprev, Yprev2): 0..2
    int extrap_order = 1;  // FIL_EXTRAP_LINEAR / _QUADRATIC / _ADAPTIVE
    double *xfit;          // adaptive fit (P, Q) per filament and block (Y_1, u, Lambda): 6M
    int *d_iterated;       // [n_sys] whether a system took a Broyden iteration this step
    int64_t steps;

    // external loads
    double *Fext, *Text, *follower;
    int has_Fext, has_Text, has_follower;

    // residual-evaluation buffers
    double *qc, *Yc, *FT, *Tint, *VW, *Mh;

    // independent systems (ensembles): consecutive groups of filaments; the
    // mobility couples segments of the same system only, and each system has
    // its own Broyden scalars and convergence
    int n_sys;
    std::vector<int64_t> sys_seg_off_h;   // [n_sys + 1] segment offsets
    int64_t *sys_xoff;                    // [n_sys + 1] offsets into X (6 x segments)

    // RPY workspace; systems padded to whole target tiles (rpy.cu)
    float4 *src32;        // 3 float4 per (padded) segment, mixed path
    double *src64;        // 12 doubles per (padded) segment, FP64 path
    int64_t Spad;
    void *partials;       // stream-K partial sums
    int *tile_cnt;        // per listed tile: work units whose partial is written (zero between launches)
    int rpy_grid32, rpy_grid64;
    int64_t rpy_tiles, rpy_units;
    std::vector<int64_t> sys_pad_off_h, tile_unit_off_h, tile_src_h, tile_nsrc_h, pos_of_seg_h;
    std::vector<int> pad_map_h, tile_sys_h, tile_id_h;
    int64_t *tile_unit_off_d, *tile_src_d, *tile_nsrc_d, *pos_of_seg_d;
    int *pad_map_d, *tile_id_d, *slot_d;
    int rpy_tpt;           // targets per thread of the pair kernels
    int rpy_split = 1;     // source split of the FP32 one-target kernel (1 or 2 halves per CTA)
    int rpy_threads;       // threads per CTA of the FP32 pair kernel (128, or 64 with tpt 2);
                           // tile = rpy_threads x rpy_tpt targets
    int rpy_ctas;          // resident CTAs per SM of the stream-K grid
    int rpy_ctas_max;
    int64_t rpy_tiles_max; // listed tiles at the smallest tile size
    // the tiles of the systems still iterating (ensembles): applies inside a
    // Broyden iteration only evaluate those
    int64_t act_tiles, act_units;
    double pairs_all, pairs_act;   // sum of S_s^2 over all / the active systems
    double n_pairs;                // pairs evaluated by all applies so far
    int64_t *act_unit_off_d, *act_src_d, *act_nsrc_d;
    int *act_tile_d, *act_slot_d;
    int64_t *act_dyn_d;    // {act_tiles, act_units} on the device

    // Broyden state
    double *Xk, *fk, *Xn, *fn, *w, *g, *C, *D;
    double *scal;          // per system (stride sstride): [alpha_0..alpha_{k-1}, ndf2, dff]
    float *C32, *D32;      // the history in FP32 (mixed mode; C, D are then null)
    float *scal32;         // FP32 copy of scal for the FP32 history sums
    int sstride;
    // Broyden history capacity (pairs; max_iter, or max_iter + keep after
    // fil_set_broyden_memory) and the memory carried across steps
    int hist_cap = 0;
    int bmem_keep = 0;     // pairs kept for the next step (0: reset every step)
    int tether_fresh = 0;  // fil_set_tether was called since J0 was last built
    int bmem_ok = 0;       // the last commit left pairs 0..k_last-1 to carry
    int k_last = 0;
    int k_hold = 0;        // a step that converged on entry keeps k_last (its pairs) for the next
    void *bmem_mem = nullptr;   // the allocation of the larger history, if made
    double *red_part;      // reduction partials, [(max_iter + 2) x red_blocks]
    int red_blocks;        // reduction blocks, each inside one system
    int *blk_sys;          // [red_blocks] system of a block
    int64_t *blk_beg;      // [red_blocks + 1] X range of a block (contiguous per system)
    int *sys_blk_off;      // [n_sys + 1] first block of each system
    std::vector<int> sys_blk_off_h;
    unsigned long long *d_finf;   // [n_sys] atomic max of |f| bits per system
    int *d_flags;          // [0] stall flag, [1] singular J0 flag
    int *d_active;         // [n_sys] system still iterating in the current step
    std::vector<int> active_h, sys_iters_h;   // host copies; iterations per system
    std::vector<int> active_prev_h;           // active_h before the last update
    std::vector<double> finf_h;               // ||f||_inf per system, last read
    double *h_pinned;      // small pinned host buffer
    int k;                 // stored (c, d) pairs of the current step
    int *d_k;              // the same count on the device (read by the Broyden kernels)
    // CUDA graphs of one Broyden iteration (fil_set_graph): one per buffer
    // parity, captured on first use in a step or after the active set changed
    int use_graph;
    cudaStream_t cap_stream;   // private stream the graphs are captured on
    cudaGraphExec_t graph_exec[2];
    const double *graph_xk[2];
    int64_t graph_launches[2], graph_applies[2];
    int in_step;           // a step was begun and not committed
    int iters_step;        // Broyden iterations of the current step
    int conv;              // current iterate satisfies ||f||_inf <= tol * a

    // J0 factors: banded (drag mobility, App. B.2) or dense per filament
    // (filament RPY mobility); piv holds 6S pivots (band rows use 6S - 3M)
    int j0_model;
    double *band;
    float *band32;         // the band in FP32, factored in place (mixed precision; band unused)
    int *piv;
    float *jinv;           // per filament: FP32 J0, then its inverse in place
    int64_t *jofs;         // [M+1] offsets of the (6N)^2 blocks
    int64_t jdense_len;
    double *aux;           // per-filament FP64 data of J0 (matrix-free residual)
    int64_t *auxofs;       // [M+1]
    int64_t aux_len;
    double j0_dp_bdt;      // scheme weight * dt of the current J0
    // J0 reuse across steps (fil_set_j0_reuse): the factors of a step are kept
    // for up to j0_reuse_max steps while the Broyden iteration count stays
    // within one of that of the step that built them
    int j0_reuse_max = 1;
    int j0_age = -1;          // steps committed with the current factors; -1: none
    int j0_iters_ref = 0;     // iterations of the step that built them
    int j0_last_iters = 0;    // iterations of the last committed step
    double j0_weight = 0.0;   // scheme weight * dt the current factors were built with
    int j0_reused = 0;        // the current step runs on factors of an earlier step
    int64_t j0_builds = 0, j0_reuses = 0;

    // staging for host pointers (6S doubles each)
    double *stage_a, *stage_b, *stage_c;

    int64_t n_applies, n_iters;

    // learned warm start (include/fil_mlp.h)
    fil_mlp *warm_net;     // attached network or null
    float *warm_feat;      // [M x FIL_MLP_IN] network inputs
    float *warm_out;       // [M x FIL_MLP_OUT] network outputs
    double *warm_xex;      // [6S] the extrapolated X_0 of the current / last step
    double *warm_corr;     // [6S] X* - X_ex of the last committed step
    int warm_corr_ok;      // warm_corr belongs to the current history
    int warm_mode;         // fil_warm_mode
    int warm_from_pred;    // the current step started from the prediction
    int64_t warm_pred, warm_extrap, warm_restart;   // starts from each candidate, restarts

    // steric barrier (fil_set_steric)
    double steric_FS = 0.0, steric_chi = 1.1;
    int64_t steric_buckets = 0;    // power of two >= 2S
    int *steric_count = nullptr;   // [steric_buckets] segments hashed to each bucket
    int *steric_bucket = nullptr;  // [steric_buckets x kStericCap] their indices
    int4 *steric_cell = nullptr;   // [S] cell (ix, iy, iz) and system of each segment
    float4 *steric_frac = nullptr; // [S] position within its cell, FP32

    // tethered filaments (fil_set_tether)
    int tether_on = 0;             // some filament is tethered
    int *tmask = nullptr;          // [M] tethered
    double *tY1 = nullptr;         // [M x 3] prescribed base position of the step
    double *tu1 = nullptr;         // [M x 3] prescribed rotation of the first segment
    double *tlam = nullptr;        // [M x 6] multipliers of the last committed step
    double *tlam_prev = nullptr;   // [M x 6] of the step before
    int thist = 0;                 // committed steps behind tlam / tlam_prev (0..2)
    double *txr = nullptr;         // [nX] X with the prescribed values in the slots
    double *tU = nullptr;          // [6 x nX] multiplier columns of J0
    double *tZ = nullptr;          // [6 x nX] J0_free^{-1} of them
    double *tCinv = nullptr;       // [M x 36] inverse capacitance matrices
    double *tw = nullptr;          // [M x 6] weights of the current solve
    void *tether_mem = nullptr;    // the allocation holding the arrays above

    void *arena;           // the single device allocation
    size_t arena_bytes;

    int64_t n_launches;    // kernels launched by this library
    int prof_on;           // time RPY pair-kernel launches with CUDA events
    int prof_n;
    cudaEvent_t *prof_ev;  // 2 * kProfMax events, created on first use
    cudaEvent_t *tune_ev = nullptr;   // the autotuner's pair of events for the next apply
};

namespace fil {

inline bool pair32_on(const fil_ctx *c) { return c->prec != FIL_FP64; }
// targets per RPY tile of the current pair-kernel schedule
inline int rpy_tile(const fil_ctx *c) { return c->rpy_threads * c->rpy_tpt; }
inline bool fast_mixed(const fil_ctx *c) { return c->prec == FIL_MIXED; }

// Launchers (all enqueue on c->stream and return a cudaError_t).
cudaError_t rpy_apply(fil_ctx *c, const double *Y, const double *FT, double *VW,
                      bool active_only = false);
cudaError_t rpy_set_active(fil_ctx *c);     // list the active systems' tiles
cudaError_t rpy_autotune(fil_ctx *c, const double *Y, const double *FT, double *VW, int reps,
                         double *best_ms);
cudaError_t rpy_setup(fil_ctx *c);          // grid sizes and padded layout, once at create
bool rpy_schedule_valid(const fil_ctx *c, int tpt, int threads, int ctas, int split);
cudaError_t rpy_set_schedule(fil_ctx *c, int tpt, int threads, int ctas, int split);
cudaError_t rpy_upload_tables(fil_ctx *c);  // the layout tables, after the arena exists
size_t rpy_partial_bytes(const fil_ctx *c);

cudaError_t unpack_forces(fil_ctx *c, const double *X, int with_forces, bool active_only = false);
// fprev non-null: systems that have converged copy their rows from fprev
cudaError_t residual_rows(fil_ctx *c, const double *X, double *f, const double *fprev = nullptr);
// adds the steric barrier forces of the positions Yc to FT (no-op when FS = 0);
// active_only: segments of converged systems are skipped
cudaError_t steric_forces(fil_ctx *c, bool active_only = false);
// tethered filaments (tether.cu)
cudaError_t tether_resolve(fil_ctx *c, const double *X, double *Xr);   // slots <- prescribed
cudaError_t tether_loads(fil_ctx *c, const double *X, bool active_only);   // FT += multipliers
cudaError_t tether_guess(fil_ctx *c, double *X0);                     // multiplier slots of X0
cudaError_t tether_record(fil_ctx *c, const double *X);               // history shift
cudaError_t tether_j0_setup(fil_ctx *c,
                            cudaError_t (*free_solve)(fil_ctx *, const double *, double *));
cudaError_t tether_j0_correct(fil_ctx *c, double *x);                 // Woodbury correction
cudaError_t init_straight(fil_ctx *c, const double *base, const double *t, const double *mu,
                          const double *xi);
cudaError_t extrapolate_guess(fil_ctx *c, double *X0);
cudaError_t commit_state(fil_ctx *c, const double *X);

cudaError_t j0_build_factor(fil_ctx *c, const double *X);
// active non-null: filaments of converged systems are skipped (their rows of x
// are left as they were)
cudaError_t j0_solve(fil_ctx *c, const double *b, double *x, const int *active = nullptr);
cudaError_t j0_dense_build_factor(fil_ctx *c, const double *X);
cudaError_t j0_dense_solve(fil_ctx *c, const double *b, double *x,
                           const int *active = nullptr);

cudaError_t broyden_axpy_step(fil_ctx *c);                 // Xn = Xk - w
cudaError_t broyden_dots(fil_ctx *c);                      // alpha_i, ndf2, dff
cudaError_t broyden_update(fil_ctx *c);
cudaError_t broyden_mask_inactive(fil_ctx *c, double *v);   // v = 0 in converged systems
// carried memory at the start of a step: history pairs [from, from + m) moved
// to [0, m), the device k set to m, and w += sum_{i<m} c_i (d_i . f)
cudaError_t broyden_carry(fil_ctx *c, int from, int m, const double *f, double *w);
cudaError_t warm_features(fil_ctx *c, const double *Xex, float *feat);
cudaError_t warm_targets(fil_ctx *c, float *targ);
cudaError_t warm_record_correction(fil_ctx *c);
cudaError_t warm_predict(fil_ctx *c, const double *Xex, double *Xpred);
// network forward pass on `st` (mlp.cu); launches are added to *launches
cudaError_t mlp_forward_async(fil_mlp *m, const float *x, float *y, int64_t batch,
                              cudaStream_t st, int64_t *launches);
int64_t mlp_max_batch(const fil_mlp *m);                    // history pair, new w

}  // namespace fil
