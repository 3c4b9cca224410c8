// C ABI of the filament library (declared in include/fil.h).
//
// All device memory of a context is one arena allocated in fil_create; the
// other entry points only enqueue kernels and copies on the context stream.
// The timestep loop is host-driven: the single host decision per Broyden
// iteration is the convergence test ||f||_inf <= tol * a, read back together
// with the stall / singular flags in one small copy.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <limits>
#include <cstring>
#include <new>
#include <string>

#include "fil_internal.cuh"

using namespace fil;

namespace {

// Device status: int flags[4] ([0] stall |df| = 0, [1] J0 singular, [2] steric
// cell grid overflow), then
// the bits of ||f||_inf of every system (atomic max). Read back as:
struct StatusBlock {
    int flags[4];
    double fmax;    // max over the systems still iterating (all systems outside a step)
};
constexpr int kRedChunk = 2048;   // X entries per Broyden reduction block

fil_status set_err(fil_ctx *c, fil_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

fil_status cuda_err(fil_ctx *c, cudaError_t e, const char *what) {
    // the failure is reported through the status: clear it from the runtime's
    // last-error slot, where a later launch check of this or another context
    // would otherwise report it a second time (sticky errors stay regardless)
    cudaGetLastError();
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return set_err(c, FIL_ECUDA, buf);
}

#define CK(expr)                                                 \
    do {                                                         \
        cudaError_t e_ = (expr);                                 \
        if (e_ != cudaSuccess) return cuda_err(c, e_, #expr);    \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device view of an input array: the pointer itself, or a copy in `stage`.
cudaError_t input_view(fil_ctx *c, const double *p, int64_t n, double *stage, const double **out) {
    if (is_device_ptr(p)) {
        *out = p;
        return cudaSuccess;
    }
    *out = stage;
    return cudaMemcpyAsync(stage, p, (size_t)n * sizeof(double), cudaMemcpyHostToDevice,
                           c->stream);
}

// Copy a device result to the caller's buffer (host or device) and wait.
cudaError_t output_copy(fil_ctx *c, double *dst, const double *src, int64_t n) {
    if (dst == src) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), cudaMemcpyDefault,
                                    c->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

struct Arena {
    char *base = nullptr;
    size_t used = 0;
    template <typename T>
    T *take(size_t count) {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

void carve(fil_ctx *c, Arena &ar, int red_blocks, size_t partial_bytes) {
    const int64_t S = c->lay.S, nX = c->lay.nX, M = c->lay.M;
    const int64_t nlam = c->lay.nlam;
    const int64_t nband = 6 * S - 3 * M;
    c->lay.N = ar.take<int>(M);
    c->lay.off = ar.take<int>(M + 1);
    c->lay.fil_of = ar.take<int>(S);
    c->lay.sys_of = ar.take<int>(S);
    c->sys_xoff = ar.take<int64_t>(c->n_sys + 1);
    c->tile_unit_off_d = ar.take<int64_t>(c->rpy_tiles_max + 1);
    c->tile_src_d = ar.take<int64_t>(c->rpy_tiles_max);
    c->tile_nsrc_d = ar.take<int64_t>(c->rpy_tiles_max);
    c->tile_id_d = ar.take<int>(c->rpy_tiles_max);
    c->slot_d = ar.take<int>(c->Spad / kRpyThreads);
    c->act_unit_off_d = ar.take<int64_t>(c->rpy_tiles_max + 1);
    c->act_src_d = ar.take<int64_t>(c->rpy_tiles_max);
    c->act_nsrc_d = ar.take<int64_t>(c->rpy_tiles_max);
    c->act_tile_d = ar.take<int>(c->rpy_tiles_max);
    c->act_slot_d = ar.take<int>(c->Spad / kRpyThreads);
    c->act_dyn_d = ar.take<int64_t>(2);
    c->pos_of_seg_d = ar.take<int64_t>(S);
    c->pad_map_d = ar.take<int>(c->Spad);
    c->Y = ar.take<double>(3 * S);
    c->Yprev = ar.take<double>(3 * S);
    c->q = ar.take<double>(4 * S);
    c->uprev = ar.take<double>(3 * S);
    c->lam = ar.take<double>(3 * (nlam > 0 ? nlam : 1));
    c->uprev2 = ar.take<double>(3 * S);
    c->lamprev = ar.take<double>(3 * (nlam > 0 ? nlam : 1));
    c->Yprev2 = ar.take<double>(3 * S);
    c->uprev3 = ar.take<double>(3 * S);
    c->lamprev2 = ar.take<double>(3 * (nlam > 0 ? nlam : 1));
    c->xfit = ar.take<double>(6 * M);
    c->d_iterated = ar.take<int>(c->n_sys);
    c->Fext = ar.take<double>(3 * S);
    c->Text = ar.take<double>(3 * S);
    c->follower = ar.take<double>(M);
    c->qc = ar.take<double>(4 * S);
    c->Yc = ar.take<double>(3 * S);
    c->FT = ar.take<double>(6 * S);
    c->Tint = ar.take<double>(3 * S);
    c->VW = ar.take<double>(6 * S);
    c->Mh = nullptr;
    if (pair32_on(c)) {
        c->src32 = ar.take<float4>((size_t)kRpyPairF4 * (c->Spad / 2));
        c->src64 = nullptr;
    } else {
        c->src64 = ar.take<double>(9 * c->Spad);
        c->src32 = nullptr;
    }
    c->partials = ar.take<char>(partial_bytes);
    c->tile_cnt = ar.take<int>(c->rpy_tiles_max);
    c->Xk = ar.take<double>(nX);
    c->fk = ar.take<double>(nX);
    c->Xn = ar.take<double>(nX);
    c->fn = ar.take<double>(nX);
    c->w = ar.take<double>(nX);
    c->g = ar.take<double>(nX);
    if (fast_mixed(c)) {
        // mixed mode: the Broyden history in FP32 (half the bytes; its sums then
        // need no FP64 work per history vector)
        c->C32 = ar.take<float>((size_t)c->max_iter * nX);
        c->D32 = ar.take<float>((size_t)c->max_iter * nX);
        c->C = c->D = nullptr;
    } else {
        c->C = ar.take<double>((size_t)c->max_iter * nX);
        c->D = ar.take<double>((size_t)c->max_iter * nX);
        c->C32 = c->D32 = nullptr;
    }
    c->scal = ar.take<double>((size_t)c->n_sys * c->sstride);
    c->scal32 = ar.take<float>((size_t)c->n_sys * c->sstride);
    c->red_part = ar.take<double>((size_t)(c->max_iter + 2) * red_blocks);
    c->blk_sys = ar.take<int>(red_blocks);
    c->blk_beg = ar.take<int64_t>(red_blocks + 1);
    c->sys_blk_off = ar.take<int>(c->n_sys + 1);
    c->d_active = ar.take<int>(c->n_sys);
    c->d_k = ar.take<int>(1);
    char *sb = ar.take<char>(16 + 8 * (size_t)c->n_sys);
    c->d_flags = sb ? reinterpret_cast<int *>(sb) : nullptr;
    c->d_finf = sb ? reinterpret_cast<unsigned long long *>(sb + 16) : nullptr;
    if (c->j0_model == FIL_J0_DRAG) {
        c->band = fast_mixed(c) ? nullptr : ar.take<double>((size_t)nband * kBandW);
        c->band32 = fast_mixed(c) ? ar.take<float>((size_t)nband * kBandW) : nullptr;
        c->jinv = nullptr;
        c->jofs = nullptr;
        c->aux = nullptr;
        c->auxofs = nullptr;
    } else {
        c->band = nullptr;
        c->band32 = nullptr;
        c->jinv = ar.take<float>((size_t)c->jdense_len);
        c->jofs = ar.take<int64_t>(M + 1);
        c->aux = ar.take<double>((size_t)c->aux_len);
        c->auxofs = ar.take<int64_t>(M + 1);
    }
    c->piv = ar.take<int>(6 * S);
    c->stage_a = ar.take<double>(nX);
    c->stage_b = ar.take<double>(nX);
    c->stage_c = ar.take<double>(nX);
    c->warm_feat = ar.take<float>((size_t)M * FIL_MLP_IN);
    c->warm_out = ar.take<float>((size_t)M * FIL_MLP_OUT);
    c->warm_xex = ar.take<double>(nX);
    c->warm_corr = ar.take<double>(nX);
}

// Flags and the per-system norms (into c->finf_h); fmax over the systems still
// iterating when `active_only`, else over all.
fil_status read_status(fil_ctx *c, StatusBlock *hs, bool active_only = false) {
    const size_t bytes = 16 + 8 * (size_t)c->n_sys;
    CK(cudaMemcpyAsync(c->h_pinned, c->d_flags, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const char *h = reinterpret_cast<const char *>(c->h_pinned);
    std::memcpy(hs->flags, h, 16);
    if (hs->flags[2]) {
        CK(cudaMemsetAsync(c->d_flags + 2, 0, sizeof(int), c->stream));
        return set_err(c, FIL_EOVERFLOW,
                       "steric barrier: cell grid overflow (too many segments in one bucket or "
                       "within range of one segment)");
    }
    c->finf_h.resize(c->n_sys);
    std::memcpy(c->finf_h.data(), h + 16, 8 * (size_t)c->n_sys);
    double m = 0.0;
    bool nan = false;
    for (int s = 0; s < c->n_sys; ++s) {
        if (active_only && !c->active_h[s]) continue;
        const double v = c->finf_h[s];
        if (!(v == v)) nan = true;
        else if (v > m) m = v;
    }
    hs->fmax = nan ? std::numeric_limits<double>::quiet_NaN() : m;
    return FIL_OK;
}

double finf_of(const StatusBlock &s) { return s.fmax; }

// f(X): unpack + forces (with_forces = 2 also keeps the internal torque for
// J0), steric barrier, RPY mobility, residual rows, ||f||_inf into the status
// block.
// fprev non-null: inside a Broyden iteration of an ensemble, only the
// systems still iterating are evaluated; the others keep fprev's rows.
// Unpack of X and the loads of the mobility problem: with tethered filaments
// the unpack runs on X with the prescribed values in the slots (c->txr, also
// returned in *Xu) and the multipliers join the loads; then the steric barrier.
cudaError_t unpack_all(fil_ctx *c, const double *X, int with_forces, bool act,
                       const double **Xu) {
    *Xu = X;
    cudaError_t e;
    if (c->tether_on) {
        e = tether_resolve(c, X, c->txr);
        if (e != cudaSuccess) return e;
        *Xu = c->txr;
    }
    e = unpack_forces(c, *Xu, with_forces, act);
    if (e != cudaSuccess) return e;
    if (c->tether_on) {
        e = tether_loads(c, X, act);
        if (e != cudaSuccess) return e;
    }
    return steric_forces(c, act);
}

cudaError_t eval_residual(fil_ctx *c, const double *X, double *f, int with_forces,
                          const double *fprev = nullptr) {
    const bool act = fprev != nullptr;
    const double *Xu = X;
    cudaError_t e = unpack_all(c, X, with_forces, act, &Xu);
    if (e != cudaSuccess) return e;
    e = rpy_apply(c, c->Yc, c->FT, c->VW, act);
    if (e != cudaSuccess) return e;
    return residual_rows(c, Xu, f, fprev);
}

cudaError_t j0_apply_free(fil_ctx *c, const double *b, double *x) {
    return c->j0_model == FIL_J0_DRAG ? j0_solve(c, b, x) : j0_dense_solve(c, b, x);
}

// J0^{-1} b (tethered filaments: the free solve and the rank-6 correction).
// active_only: inside the Broyden iterations of an ensemble, the rows of
// converged systems are not computed (the caller masks or ignores them).
cudaError_t j0_apply(fil_ctx *c, const double *b, double *x, bool active_only = false) {
    const int *act = active_only && c->n_sys > 1 ? c->d_active : nullptr;
    cudaError_t e = c->j0_model == FIL_J0_DRAG ? j0_solve(c, b, x, act)
                                               : j0_dense_solve(c, b, x, act);
    if (e == cudaSuccess && c->tether_on) e = tether_j0_correct(c, x);
    return e;
}

}  // namespace

extern "C" {

fil_status fil_create_ensemble(const fil_params *p, int32_t n_sys, const int32_t *fil_per_sys,
                               fil_ctx **out) {
    if (!out) return FIL_EINVAL;
    *out = nullptr;
    if (!p || p->n_fil < 1 || !p->seg_per_fil) return FIL_EINVAL;
    if (n_sys < 1 || !fil_per_sys) return FIL_EINVAL;
    {
        int64_t nf = 0;
        for (int s = 0; s < n_sys; ++s) {
            if (fil_per_sys[s] < 1) return FIL_EINVAL;
            nf += fil_per_sys[s];
        }
        if (nf != p->n_fil) return FIL_EINVAL;
    }
    if (!(p->a > 0) || !(p->eta > 0) || !(p->dL > 0) || !(p->dt > 0) || !(p->tol > 0) ||
        !(p->KB >= 0) || !(p->KT >= 0) || p->max_iter < 1 ||
        (p->precision != FIL_FP64 && p->precision != FIL_MIXED && p->precision != FIL_PAIR32) ||
        (p->j0_model != FIL_J0_DRAG && p->j0_model != FIL_J0_FILAMENT_RPY) ||
        !std::isfinite(p->gamma0) || !std::isfinite(p->kappa_mu) || !std::isfinite(p->kappa_nu))
        return FIL_EINVAL;
    int64_t S = 0;
    int maxN = 0;
    for (int i = 0; i < p->n_fil; ++i) {
        if (p->seg_per_fil[i] < 1) return FIL_EINVAL;
        S += p->seg_per_fil[i];
        if (p->seg_per_fil[i] > maxN) maxN = p->seg_per_fil[i];
    }
    if (S > (int64_t)1 << 30) return FIL_EINVAL;
    // the band solve keeps a filament's right-hand side in shared memory; the
    // filament-RPY J0 inverts each filament block in shared memory
    if (maxN > kMaxSegPerFil) return FIL_EINVAL;
    if (p->j0_model == FIL_J0_FILAMENT_RPY && maxN > kMaxDenseSeg) return FIL_EINVAL;

    fil_ctx *c = new (std::nothrow) fil_ctx();
    if (!c) return FIL_ENOMEM;
    c->lay.M = p->n_fil;
    c->lay.S = S;
    c->lay.nX = 6 * S;
    c->lay.nlam = S - p->n_fil;
    c->lay.maxN = maxN;
    c->N_host.assign(p->seg_per_fil, p->seg_per_fil + p->n_fil);
    c->off_host.resize(p->n_fil + 1);
    c->off_host[0] = 0;
    for (int i = 0; i < p->n_fil; ++i) c->off_host[i + 1] = c->off_host[i] + c->N_host[i];
    c->a = p->a; c->eta = p->eta; c->dL = p->dL; c->KB = p->KB; c->KT = p->KT;
    c->g0 = p->gamma0; c->kmu = p->kappa_mu; c->knu = p->kappa_nu;
    c->dt = p->dt; c->tol = p->tol; c->max_iter = p->max_iter; c->prec = p->precision;
    c->j0_model = p->j0_model;
    c->n_sys = n_sys;
    c->sys_seg_off_h.assign(n_sys + 1, 0);
    std::vector<int> sys_of_seg(S);
    {
        int f = 0;
        for (int s = 0; s < n_sys; ++s) {
            const int f1 = f + fil_per_sys[s];
            c->sys_seg_off_h[s + 1] = c->off_host[f1];
            for (int64_t g = c->off_host[f]; g < c->off_host[f1]; ++g) sys_of_seg[g] = s;
            f = f1;
        }
    }
    c->hist_cap = c->max_iter;
    c->sstride = c->hist_cap + 8;
    c->active_h.assign(n_sys, 0);
    c->sys_iters_h.assign(n_sys, 0);
    c->finf_h.assign(n_sys, 0.0);
    // Broyden reduction blocks: consecutive slices of at most kRedChunk entries inside a system
    std::vector<int> blk_sys;
    std::vector<int64_t> blk_beg;
    c->sys_blk_off_h.assign(n_sys + 1, 0);
    for (int s = 0; s < n_sys; ++s) {
        const int64_t x0 = 6 * c->sys_seg_off_h[s], x1 = 6 * c->sys_seg_off_h[s + 1];
        for (int64_t x = x0; x < x1; x += kRedChunk) {
            blk_sys.push_back(s);
            blk_beg.push_back(x);
        }
        c->sys_blk_off_h[s + 1] = (int)blk_sys.size();
    }
    blk_beg.push_back(6 * S);
    std::vector<int64_t> sys_xoff(n_sys + 1);
    for (int s = 0; s <= n_sys; ++s) sys_xoff[s] = 6 * c->sys_seg_off_h[s];
    std::vector<int64_t> jofs(p->n_fil + 1, 0), auxofs(p->n_fil + 1, 0);
    for (int i = 0; i < p->n_fil; ++i) {
        const int64_t Ni = c->N_host[i];
        jofs[i + 1] = jofs[i] + 36 * Ni * Ni;
        auxofs[i + 1] = auxofs[i] + 60 * Ni + 5 * Ni * Ni;   // layout in jacobian_dense.cu
    }
    c->jdense_len = jofs[p->n_fil];
    c->aux_len = auxofs[p->n_fil];
    c->stream = (cudaStream_t)p->stream;
    c->have_prev = 0; c->ylev = 0; c->hist = 0; c->steps = 0; c->k = 0; c->in_step = 0;
    c->has_Fext = c->has_Text = c->has_follower = 0;
    c->n_applies = c->n_iters = 0;
    c->iters_step = 0; c->conv = 0;
    c->arena = nullptr; c->h_pinned = nullptr;
    c->n_launches = 0; c->prof_on = 0; c->prof_n = 0; c->prof_ev = nullptr;

    auto bail = [&](fil_status s, const char *what, cudaError_t e) {
        if (c->arena) cudaFree(c->arena);
    if (c->tether_mem) cudaFree(c->tether_mem);
    if (c->steric_count) cudaFree(c->steric_count);
    if (c->steric_bucket) cudaFree(c->steric_bucket);
        if (c->h_pinned) cudaFreeHost(c->h_pinned);
        std::fprintf(stderr, "fil_create: %s: %s\n", what, cudaGetErrorString(e));
        delete c;
        return s;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(FIL_ECUDA, "cudaGetDevice", e);
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return bail(FIL_ECUDA, "cudaDeviceGetAttribute", e);
    e = rpy_setup(c);
    if (e != cudaSuccess) return bail(FIL_ECUDA, "rpy_setup", e);
    c->red_blocks = (int)blk_sys.size();
    const size_t pbytes = rpy_partial_bytes(c);

    Arena sizing;
    carve(c, sizing, c->red_blocks, pbytes);
    c->arena_bytes = sizing.used;
    e = cudaMalloc(&c->arena, c->arena_bytes);
    if (e != cudaSuccess) return bail(FIL_ENOMEM, "cudaMalloc", e);
    Arena ar;
    ar.base = (char *)c->arena;
    carve(c, ar, c->red_blocks, pbytes);
    e = cudaMallocHost(&c->h_pinned, std::max<size_t>(256, 16 + 8 * (size_t)n_sys));
    if (e != cudaSuccess) return bail(FIL_ENOMEM, "cudaMallocHost", e);

    // layout tables and a neutral initial state
    std::vector<int> fil_of(S);
    for (int i = 0; i < p->n_fil; ++i)
        for (int n = c->off_host[i]; n < c->off_host[i + 1]; ++n) fil_of[n] = i;
    std::vector<double> q0(4 * S, 0.0);
    for (int64_t n = 0; n < S; ++n) q0[4 * n] = 1.0;
    e = cudaMemsetAsync(c->arena, 0, c->arena_bytes, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->lay.N, c->N_host.data(), sizeof(int) * p->n_fil,
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->lay.off, c->off_host.data(), sizeof(int) * (p->n_fil + 1),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->lay.fil_of, fil_of.data(), sizeof(int) * S,
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->lay.sys_of, sys_of_seg.data(), sizeof(int) * S,
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->sys_xoff, sys_xoff.data(), sizeof(int64_t) * (n_sys + 1),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->blk_sys, blk_sys.data(), sizeof(int) * blk_sys.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->blk_beg, blk_beg.data(), sizeof(int64_t) * blk_beg.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->sys_blk_off, c->sys_blk_off_h.data(), sizeof(int) * (n_sys + 1),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = rpy_upload_tables(c);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->q, q0.data(), sizeof(double) * 4 * S, cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess && c->jofs)
        e = cudaMemcpyAsync(c->jofs, jofs.data(), sizeof(int64_t) * (p->n_fil + 1),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->auxofs)
        e = cudaMemcpyAsync(c->auxofs, auxofs.data(), sizeof(int64_t) * (p->n_fil + 1),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(FIL_ECUDA, "initial upload", e);
    *out = c;
    return FIL_OK;
}

fil_status fil_create(const fil_params *p, fil_ctx **out) {
    if (!p) return FIL_EINVAL;
    const int32_t all = p->n_fil;
    return fil_create_ensemble(p, 1, &all, out);
}

void drop_graphs(fil_ctx *c);

void fil_destroy(fil_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->arena) cudaFree(c->arena);
    if (c->tether_mem) cudaFree(c->tether_mem);
    if (c->steric_count) cudaFree(c->steric_count);
    if (c->steric_bucket) cudaFree(c->steric_bucket);
    if (c->bmem_mem) cudaFree(c->bmem_mem);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->prof_ev) {
        for (int i = 0; i < 2 * kProfMax; ++i) cudaEventDestroy(c->prof_ev[i]);
        delete[] c->prof_ev;
    }
    delete c;
}

const char *fil_last_error(const fil_ctx *c) { return c ? c->err.c_str() : "null context"; }

fil_status fil_sizes(const fil_ctx *c, int64_t *n_seg, int64_t *n_unknowns, int64_t *n_lambda) {
    if (!c) return FIL_EINVAL;
    if (n_seg) *n_seg = c->lay.S;
    if (n_unknowns) *n_unknowns = c->lay.nX;
    if (n_lambda) *n_lambda = c->lay.nlam;
    return FIL_OK;
}

fil_status fil_set_state(fil_ctx *c, const double *Y, const double *q, const double *Yprev,
                         const double *u, const double *Lambda) {
    if (!c) return FIL_EINVAL;
    if (!Y || !q) return set_err(c, FIL_EINVAL, "fil_set_state: Y and q are required");
    if ((Yprev == nullptr) != (u == nullptr))
        return set_err(c, FIL_EINVAL, "fil_set_state: Yprev and u go together");
    CK(cudaSetDevice(c->device));
    const int64_t S = c->lay.S;
    CK(cudaMemcpyAsync(c->Y, Y, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(c->q, q, sizeof(double) * 4 * S, cudaMemcpyDefault, c->stream));
    if (Yprev) {
        CK(cudaMemcpyAsync(c->Yprev, Yprev, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
        CK(cudaMemcpyAsync(c->uprev, u, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
    } else {
        CK(cudaMemsetAsync(c->Yprev, 0, sizeof(double) * 3 * S, c->stream));
        CK(cudaMemsetAsync(c->uprev, 0, sizeof(double) * 3 * S, c->stream));
    }
    if (c->lay.nlam > 0) {
        if (Lambda)
            CK(cudaMemcpyAsync(c->lam, Lambda, sizeof(double) * 3 * c->lay.nlam,
                               cudaMemcpyDefault, c->stream));
        else
            CK(cudaMemsetAsync(c->lam, 0, sizeof(double) * 3 * c->lay.nlam, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemsetAsync(c->xfit, 0, sizeof(double) * 6 * c->lay.M, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->have_prev = Yprev ? 1 : 0;
    c->ylev = Yprev ? 1 : 0;
    c->bmem_ok = 0;
    c->hist = 0;
    c->thist = 0;
    c->warm_corr_ok = 0;
    c->in_step = 0;
    c->j0_age = -1;
    return FIL_OK;
}

fil_status fil_get_state(fil_ctx *c, double *Y, double *q, double *Yprev, double *u,
                         double *Lambda) {
    if (!c) return FIL_EINVAL;
    CK(cudaSetDevice(c->device));
    const int64_t S = c->lay.S;
    if (Y) CK(cudaMemcpyAsync(Y, c->Y, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
    if (q) CK(cudaMemcpyAsync(q, c->q, sizeof(double) * 4 * S, cudaMemcpyDefault, c->stream));
    if (Yprev)
        CK(cudaMemcpyAsync(Yprev, c->Yprev, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
    if (u) CK(cudaMemcpyAsync(u, c->uprev, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
    if (Lambda && c->lay.nlam > 0)
        CK(cudaMemcpyAsync(Lambda, c->lam, sizeof(double) * 3 * c->lay.nlam, cudaMemcpyDefault,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FIL_OK;
}

fil_status fil_init_straight(fil_ctx *c, const double *base, const double *t, const double *mu,
                             const double *xi) {
    if (!c) return FIL_EINVAL;
    if (!base || !t || !mu) return set_err(c, FIL_EINVAL, "fil_init_straight: base, t, mu required");
    CK(cudaSetDevice(c->device));
    const int64_t M = c->lay.M, S = c->lay.S;
    // 3M + 3M doubles in stage_a and 3M in stage_c (each stage holds 6S >= 6M)
    double *sb = c->stage_a, *st = c->stage_a + 3 * M, *sm = c->stage_c;
    CK(cudaMemcpyAsync(sb, base, sizeof(double) * 3 * M, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(st, t, sizeof(double) * 3 * M, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(sm, mu, sizeof(double) * 3 * M, cudaMemcpyDefault, c->stream));
    const double *sxi = nullptr;
    if (xi) {
        CK(cudaMemcpyAsync(c->stage_b, xi, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
        sxi = c->stage_b;
    }
    CK(init_straight(c, sb, st, sm, sxi));
    CK(cudaMemsetAsync(c->Yprev, 0, sizeof(double) * 3 * S, c->stream));
    CK(cudaMemsetAsync(c->uprev, 0, sizeof(double) * 3 * S, c->stream));
    if (c->lay.nlam > 0) CK(cudaMemsetAsync(c->lam, 0, sizeof(double) * 3 * c->lay.nlam, c->stream));
    CK(cudaMemsetAsync(c->xfit, 0, sizeof(double) * 6 * M, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->have_prev = 0;
    c->ylev = 0;
    c->bmem_ok = 0;
    c->hist = 0;
    c->warm_corr_ok = 0;
    c->in_step = 0;
    c->j0_age = -1;
    return FIL_OK;
}

fil_status fil_set_external(fil_ctx *c, const double *Fext, const double *Text,
                            const double *follower) {
    if (!c) return FIL_EINVAL;
    CK(cudaSetDevice(c->device));
    const int64_t S = c->lay.S, M = c->lay.M;
    if (Fext) CK(cudaMemcpyAsync(c->Fext, Fext, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
    if (Text) CK(cudaMemcpyAsync(c->Text, Text, sizeof(double) * 3 * S, cudaMemcpyDefault, c->stream));
    if (follower)
        CK(cudaMemcpyAsync(c->follower, follower, sizeof(double) * M, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->has_Fext = Fext ? 1 : 0;
    c->has_Text = Text ? 1 : 0;
    c->has_follower = follower ? 1 : 0;
    return FIL_OK;
}

fil_status fil_mobility_apply(fil_ctx *c, const double *Y, const double *FT, double *VW) {
    if (!c) return FIL_EINVAL;
    if (!Y || !FT || !VW) return set_err(c, FIL_EINVAL, "fil_mobility_apply: null pointer");
    CK(cudaSetDevice(c->device));
    const int64_t S = c->lay.S;
    const double *dY, *dFT;
    CK(input_view(c, Y, 3 * S, c->stage_a, &dY));
    CK(input_view(c, FT, 6 * S, c->stage_b, &dFT));
    const bool dev_out = is_device_ptr(VW);
    double *dVW = dev_out ? VW : c->stage_c;
    CK(rpy_apply(c, dY, dFT, dVW));
    if (!dev_out) CK(output_copy(c, VW, dVW, 6 * S));
    return FIL_OK;
}

fil_status fil_residual(fil_ctx *c, const double *X, double *f, double *finf) {
    if (!c) return FIL_EINVAL;
    if (!X || !f) return set_err(c, FIL_EINVAL, "fil_residual: null pointer");
    CK(cudaSetDevice(c->device));
    const int64_t nX = c->lay.nX;
    const double *dX;
    CK(input_view(c, X, nX, c->stage_a, &dX));
    const bool dev_out = is_device_ptr(f);
    double *df = dev_out ? f : c->stage_b;
    CK(eval_residual(c, dX, df, 1));
    if (!dev_out) CK(output_copy(c, f, df, nX));
    if (finf) {
        StatusBlock sb;
        fil_status s = read_status(c, &sb);
        if (s != FIL_OK) return s;
        *finf = finf_of(sb);
    }
    return FIL_OK;
}

// X_0 of a step: the extrapolation, or -- with a warm-start network attached
// and use_net set -- the network's prediction: FIL_WARM_BEST_OF_TWO keeps
// whichever of the two has the smaller ||f||_inf, FIL_WARM_PREDICTION_FIRST
// the prediction whenever f is finite there. On return Xk, fk hold X_0,
// f(X_0), and qc, Yc, FT, Tint the unpack of X_0.
fil_status initial_iterate(fil_ctx *c, bool use_net, double *f0) {
    CK(extrapolate_guess(c, c->Xk));
    CK(cudaMemcpyAsync(c->warm_xex, c->Xk, sizeof(double) * c->lay.nX, cudaMemcpyDeviceToDevice,
                       c->stream));
    c->warm_from_pred = 0;
    StatusBlock sb;
    fil_status s;
    if (use_net && c->warm_net && c->warm_mode == FIL_WARM_PREDICTION_FIRST) {
        CK(warm_predict(c, c->Xk, c->Xn));
        CK(eval_residual(c, c->Xn, c->fn, 2));
        s = read_status(c, &sb);
        if (s != FIL_OK) return s;
        const double fp = finf_of(sb);
        if (std::isfinite(fp)) {
            std::swap(c->Xk, c->Xn);
            std::swap(c->fk, c->fn);
            *f0 = fp;
            c->warm_from_pred = 1;
            c->warm_pred += 1;
            return FIL_OK;
        }
        c->warm_extrap += 1;
        use_net = false;
    }
    CK(eval_residual(c, c->Xk, c->fk, 2));
    s = read_status(c, &sb);
    if (s != FIL_OK) return s;
    *f0 = finf_of(sb);
    if (!use_net || !c->warm_net) return FIL_OK;
    const std::vector<double> f_ex = c->finf_h;
    CK(warm_predict(c, c->Xk, c->Xn));
    CK(eval_residual(c, c->Xn, c->fn, 2));
    s = read_status(c, &sb);
    if (s != FIL_OK) return s;
    const double fp = finf_of(sb);
    if (std::isfinite(fp) && fp < *f0) {
        std::swap(c->Xk, c->Xn);
        std::swap(c->fk, c->fn);
        *f0 = fp;
        c->warm_from_pred = 1;
        c->warm_pred += 1;
    } else {
        const double *Xu;
        CK(unpack_all(c, c->Xk, 2, false, &Xu));   // back to the unpack of the extrapolation
        c->finf_h = f_ex;
        c->warm_extrap += 1;
    }
    return FIL_OK;
}

// Systems whose ||f||_inf is within the tolerance stop iterating (host and
// device flags); returns the number still active.
int update_active(fil_ctx *c, bool count_iteration) {
    c->active_prev_h = c->active_h;
    int n = 0;
    for (int sy = 0; sy < c->n_sys; ++sy) {
        if (!c->active_h[sy]) continue;
        if (count_iteration) c->sys_iters_h[sy] += 1;
        if (c->finf_h[sy] <= c->tol * c->a) c->active_h[sy] = 0;
        else ++n;
    }
    return n;
}

cudaError_t upload_active(fil_ctx *c) {
    return cudaMemcpyAsync(c->d_active, c->active_h.data(), sizeof(int) * c->n_sys,
                           cudaMemcpyHostToDevice, c->stream);
}

void drop_graphs(fil_ctx *c) {
    for (int i = 0; i < 2; ++i) {
        if (c->graph_exec[i]) cudaGraphExecDestroy(c->graph_exec[i]);
        c->graph_exec[i] = nullptr;
        c->graph_xk[i] = nullptr;
    }
}

// One Broyden iteration as the device sees it in graph mode: the step, the
// residual of the new iterate, and -- speculatively, before the host has
// checked convergence -- the dot products, the J0 solve and the history update
// (wasted once per step; for systems that have just converged, w is masked
// afterwards).
cudaError_t iteration_body(fil_ctx *c) {
    cudaError_t e = broyden_axpy_step(c);
    if (e == cudaSuccess) e = eval_residual(c, c->Xn, c->fn, 1, c->n_sys > 1 ? c->fk : nullptr);
    if (e == cudaSuccess) e = broyden_dots(c);
    if (e == cudaSuccess) e = j0_apply(c, c->fn, c->g, true);
    if (e == cudaSuccess) e = broyden_update(c);
    return e;
}

// The graph of iteration_body for the current buffers (captured if needed).
cudaError_t graph_for_current(fil_ctx *c, int *slot) {
    for (int i = 0; i < 2; ++i)
        if (c->graph_exec[i] && c->graph_xk[i] == c->Xk) {
            *slot = i;
            return cudaSuccess;
        }
    const int i = c->graph_exec[0] ? 1 : 0;
    const int64_t l0 = c->n_launches, a0 = c->n_applies;
    const double p0 = c->n_pairs;
    cudaGraph_t g = nullptr;
    // captured on the context's private stream (the legacy stream cannot be
    // captured); launched on the context's stream
    const cudaStream_t own = c->stream;
    c->stream = c->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        c->stream = own;
        return e;
    }
    cudaError_t eb = iteration_body(c);
    e = cudaStreamEndCapture(c->stream, &g);
    c->stream = own;
    if (eb != cudaSuccess) e = eb;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec[i], g, 0);
    if (g) cudaGraphDestroy(g);
    // the counters advanced during capture; each launch adds them instead
    c->graph_launches[i] = c->n_launches - l0;
    c->graph_applies[i] = c->n_applies - a0;
    c->n_launches = l0;
    c->n_applies = a0;
    c->n_pairs = p0;
    if (e != cudaSuccess) {
        c->graph_exec[i] = nullptr;
        return e;
    }
    c->graph_xk[i] = c->Xk;
    *slot = i;
    return cudaSuccess;
}

fil_status begin_step(fil_ctx *c, double *finf, bool use_net, bool force_j0 = false) {
    if (!c) return FIL_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), c->stream));
    double f0 = 0.0;
    fil_status s = initial_iterate(c, use_net, &f0);
    if (s != FIL_OK) return s;
    const std::vector<double> f0_sys = c->finf_h;
    const double *Xj = c->Xk;
    if (c->tether_on) {
        CK(tether_resolve(c, c->Xk, c->txr));
        Xj = c->txr;
    }
    // J0 of an earlier step is reused while it is young enough, the scheme
    // weight is unchanged and the iteration count has not risen (J0 only
    // shapes the iterates; the converged X solves f(X) = 0 either way)
    const double weight = (c->have_prev ? 2.0 / 3.0 : 1.0) * c->dt;
    // (with tethers: while their prescription is the one J0 was built with)
    c->j0_reused = !force_j0 && c->j0_reuse_max > 1 && !(c->tether_on && c->tether_fresh) &&
                   c->j0_age >= 1 &&
                   c->j0_age < c->j0_reuse_max && weight == c->j0_weight &&
                   c->j0_last_iters <= c->j0_iters_ref + 1;
    if (!c->j0_reused) {
        if (c->j0_model == FIL_J0_DRAG)
            CK(j0_build_factor(c, Xj));
        else
            CK(j0_dense_build_factor(c, Xj));
        c->j0_age = 0;
        c->j0_weight = weight;
        c->j0_builds += 1;
        c->tether_fresh = 0;
    } else {
        c->j0_reuses += 1;
    }
    if (c->tether_on) CK(tether_j0_setup(c, j0_apply_free));
    StatusBlock sb;
    s = read_status(c, &sb);
    if (s != FIL_OK) return s;
    c->finf_h = f0_sys;
    if (finf) *finf = f0;
    // the previous step's history pairs are kept when this step keeps its J0
    // (they extend that J0's inverse); the last commit's pairs are used once
    const bool carry = c->bmem_keep > 0 && c->bmem_ok && c->j0_reused && c->k_last > 0;
    const int m = carry ? std::min(c->bmem_keep, c->k_last) : 0;
    c->bmem_ok = 0;
    c->k_hold = 0;
    c->k = m;
    if (m == 0) CK(cudaMemsetAsync(c->d_k, 0, sizeof(int), c->stream));
    drop_graphs(c);      // scheme weights, J0 and the active set may have changed
    c->iters_step = 0;
    c->in_step = 0;
    if (sb.flags[1]) return set_err(c, FIL_ENAN, "fil_broyden_begin: J0 is singular");
    if (!std::isfinite(f0)) return set_err(c, FIL_ENAN, "fil_broyden_begin: f(X_0) not finite");
    c->active_h.assign(c->n_sys, 1);
    c->sys_iters_h.assign(c->n_sys, 0);
    const int n_active = update_active(c, false);
    c->conv = n_active == 0 ? 1 : 0;
    if (!c->conv) {
        CK(upload_active(c));
        if (c->n_sys > 1) CK(rpy_set_active(c));
        CK(j0_apply(c, c->fk, c->w, true));
        if (m > 0) CK(broyden_carry(c, c->k_last - m, m, c->fk, c->w));
        CK(broyden_mask_inactive(c, c->w));
    } else if (m > 0) {
        // converged on entry: this step's H_k is its H_0, whose pairs are the
        // ones it would have carried; nothing moved them, so the commit leaves
        // them for the next step (which carries them if it keeps J0 too)
        c->k = 0;
        c->k_hold = c->k_last;
        CK(cudaMemsetAsync(c->d_k, 0, sizeof(int), c->stream));
    }
    c->in_step = 1;
    return FIL_OK;
}

fil_status fil_broyden_begin(fil_ctx *c, double *finf) { return begin_step(c, finf, true); }

fil_status fil_broyden_step(fil_ctx *c, int32_t *converged, double *finf) {
    if (!c) return FIL_EINVAL;
    if (!c->in_step) return set_err(c, FIL_ESTATE, "fil_broyden_step: no step in progress");
    CK(cudaSetDevice(c->device));
    if (c->conv) {
        if (converged) *converged = 1;
        return FIL_OK;
    }
    if (c->iters_step >= c->max_iter)
        return set_err(c, FIL_ENOCONV, "Broyden: max_iter reached without convergence");
    if (c->use_graph && !c->prof_on) {
        int slot = 0;
        CK(graph_for_current(c, &slot));
        CK(cudaGraphLaunch(c->graph_exec[slot], c->stream));
        c->n_launches += c->graph_launches[slot];
        c->n_applies += c->graph_applies[slot];
        // the pairs of the systems active now (the captured count may be stale)
        c->n_pairs += c->graph_applies[slot] * (c->n_sys > 1 ? c->pairs_act : c->pairs_all);
        StatusBlock sb;
        fil_status s = read_status(c, &sb);
        if (s != FIL_OK) return s;
        const double fv = finf_of(sb);
        if (finf) *finf = fv;
        if (!std::isfinite(fv)) return set_err(c, FIL_ENAN, "Broyden: residual not finite");
        c->iters_step += 1;
        c->n_iters += 1;
        if (update_active(c, true) == 0) {
            std::swap(c->Xk, c->Xn);
            std::swap(c->fk, c->fn);
            c->conv = 1;
            if (converged) *converged = 1;
            return FIL_OK;
        }
        if (sb.flags[0]) return set_err(c, FIL_ESTALL, "Broyden: ||df|| = 0 (stalled)");
        if (c->n_sys > 1 && c->active_h != c->active_prev_h) {
            // the graph reads the active set and the active-tile list from the
            // device: rewriting them keeps it valid
            CK(upload_active(c));
            CK(broyden_mask_inactive(c, c->w));
            CK(rpy_set_active(c));
        }
        std::swap(c->Xk, c->Xn);
        std::swap(c->fk, c->fn);
        c->k += 1;
        if (converged) *converged = 0;
        return FIL_OK;
    }
    CK(broyden_axpy_step(c));
    CK(eval_residual(c, c->Xn, c->fn, 1, c->n_sys > 1 ? c->fk : nullptr));
    StatusBlock sb;
    fil_status s = read_status(c, &sb);
    if (s != FIL_OK) return s;
    if (sb.flags[0]) return set_err(c, FIL_ESTALL, "Broyden: ||df|| = 0 (stalled)");
    const double fv = finf_of(sb);
    if (finf) *finf = fv;
    if (!std::isfinite(fv)) return set_err(c, FIL_ENAN, "Broyden: residual not finite");
    c->iters_step += 1;
    c->n_iters += 1;
    if (update_active(c, true) == 0) {
        std::swap(c->Xk, c->Xn);
        std::swap(c->fk, c->fn);
        c->conv = 1;
        if (converged) *converged = 1;
        return FIL_OK;
    }
    if (c->n_sys > 1 && c->active_h != c->active_prev_h) {
        CK(upload_active(c));
        CK(rpy_set_active(c));
    }
    CK(broyden_dots(c));
    CK(j0_apply(c, c->fn, c->g, true));
    CK(broyden_update(c));
    std::swap(c->Xk, c->Xn);
    std::swap(c->fk, c->fn);
    c->k += 1;
    if (converged) *converged = 0;
    return FIL_OK;
}

fil_status fil_get_iterate(fil_ctx *c, double *X, double *f) {
    if (!c) return FIL_EINVAL;
    if (!c->in_step) return set_err(c, FIL_ESTATE, "fil_get_iterate: no step in progress");
    CK(cudaSetDevice(c->device));
    if (X) CK(cudaMemcpyAsync(X, c->Xk, sizeof(double) * c->lay.nX, cudaMemcpyDefault, c->stream));
    if (f) CK(cudaMemcpyAsync(f, c->fk, sizeof(double) * c->lay.nX, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FIL_OK;
}

fil_status fil_j0_solve(fil_ctx *c, const double *b, double *x) {
    if (!c) return FIL_EINVAL;
    if (!b || !x) return set_err(c, FIL_EINVAL, "fil_j0_solve: null pointer");
    if (!c->in_step) return set_err(c, FIL_ESTATE, "fil_j0_solve: J0 exists only inside a step");
    CK(cudaSetDevice(c->device));
    const int64_t nX = c->lay.nX;
    const double *db;
    CK(input_view(c, b, nX, c->stage_a, &db));
    const bool dev_out = is_device_ptr(x);
    double *dx = dev_out ? x : c->stage_b;
    CK(j0_apply(c, db, dx));
    if (!dev_out) CK(output_copy(c, x, dx, nX));
    return FIL_OK;
}

fil_status fil_broyden_commit(fil_ctx *c) {
    if (!c) return FIL_EINVAL;
    if (!c->in_step) return set_err(c, FIL_ESTATE, "fil_broyden_commit: no step in progress");
    CK(cudaSetDevice(c->device));
    const double *Xc = c->Xk;
    if (c->tether_on) {
        CK(tether_record(c, c->Xk));
        CK(tether_resolve(c, c->Xk, c->txr));
        Xc = c->txr;
    }
    CK(commit_state(c, Xc));
    CK(warm_record_correction(c));
    if (c->j0_age == 0) c->j0_iters_ref = c->iters_step;
    if (c->j0_age >= 0) c->j0_age += 1;
    c->j0_last_iters = c->iters_step;
    c->warm_corr_ok = 1;
    c->have_prev = 1;
    c->ylev = c->ylev < 2 ? c->ylev + 1 : 2;
    c->k_last = c->k_hold > 0 ? c->k_hold : c->k;
    c->k_hold = 0;
    c->bmem_ok = 1;
    c->hist += 1;
    c->steps += 1;
    c->in_step = 0;
    return FIL_OK;
}

fil_status fil_step(fil_ctx *c, int32_t *iters) {
    if (!c) return FIL_EINVAL;
    int32_t total = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        // a start from the network's prediction, or on the J0 of an earlier step,
        // that fails restarts from the extrapolation with a J0 built for this step
        fil_status s = begin_step(c, nullptr, attempt == 0, attempt > 0);
        if (s != FIL_OK) return s;
        int32_t conv = c->conv;
        while (!conv && s == FIL_OK) s = fil_broyden_step(c, &conv, nullptr);
        total += c->iters_step;
        if (s == FIL_OK) {
            if (iters) *iters = total;
            return fil_broyden_commit(c);
        }
        c->in_step = 0;
        if (!c->warm_from_pred && !c->j0_reused) return s;
        if (c->warm_from_pred) c->warm_restart += 1;
    }
    return FIL_ECUDA;   // not reached: the second attempt uses neither
}

fil_status fil_set_j0_reuse(fil_ctx *c, int32_t max_age) {
    if (!c) return FIL_EINVAL;
    if (max_age < 1) return set_err(c, FIL_EINVAL, "fil_set_j0_reuse: max_age >= 1");
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_set_j0_reuse: a step is in progress");
    c->j0_reuse_max = max_age;
    return FIL_OK;
}

fil_status fil_j0_stats(const fil_ctx *c, int64_t *builds, int64_t *reuses) {
    if (!c) return FIL_EINVAL;
    if (builds) *builds = c->j0_builds;
    if (reuses) *reuses = c->j0_reuses;
    return FIL_OK;
}

fil_status fil_set_broyden_memory(fil_ctx *c, int32_t keep) {
    if (!c) return FIL_EINVAL;
    if (keep < 0 || keep > c->max_iter)
        return set_err(c, FIL_EINVAL, "fil_set_broyden_memory: keep must be in [0, max_iter]");
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_set_broyden_memory: a step is in progress");
    CK(cudaSetDevice(c->device));
    const int cap = c->max_iter + keep;
    if (cap > c->hist_cap) {
        // a larger history (C, D), its scalars and the dot-product partials
        CK(cudaStreamSynchronize(c->stream));
        const int64_t nX = c->lay.nX;
        const size_t hb = c->C32 ? sizeof(float) : sizeof(double);
        const int sstride = cap + 8;
        auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t bC = up((size_t)cap * nX * hb);
        const size_t bS = up((size_t)c->n_sys * sstride * sizeof(double));
        const size_t bS32 = up((size_t)c->n_sys * sstride * sizeof(float));
        const size_t bR = up((size_t)(cap + 2) * c->red_blocks * sizeof(double));
        char *mem = nullptr;
        if (cudaMalloc(&mem, 2 * bC + bS + bS32 + bR) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, FIL_ENOMEM, "fil_set_broyden_memory: device allocation failed");
        }
        drop_graphs(c);     // captured launches hold the old buffers
        if (c->C32) {
            c->C32 = (float *)mem;
            c->D32 = (float *)(mem + bC);
        } else {
            c->C = (double *)mem;
            c->D = (double *)(mem + bC);
        }
        c->scal = (double *)(mem + 2 * bC);
        c->scal32 = (float *)(mem + 2 * bC + bS);
        c->red_part = (double *)(mem + 2 * bC + bS + bS32);
        if (c->bmem_mem) cudaFree(c->bmem_mem);
        c->bmem_mem = mem;
        c->hist_cap = cap;
        c->sstride = sstride;
        c->bmem_ok = 0;       // the pairs of the last step stayed in the old buffers
    }
    c->bmem_keep = keep;
    return FIL_OK;
}

fil_status fil_set_extrapolation(fil_ctx *c, int32_t order) {
    if (!c) return FIL_EINVAL;
    if (order != FIL_EXTRAP_LINEAR && order != FIL_EXTRAP_QUADRATIC && order != FIL_EXTRAP_ADAPTIVE)
        return set_err(c, FIL_EINVAL, "fil_set_extrapolation: order must be 1, 2 or 3");
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_set_extrapolation: a step is in progress");
    c->extrap_order = order;
    return FIL_OK;
}

fil_status fil_extrapolation(const fil_ctx *c, int32_t *order) {
    if (!c || !order) return FIL_EINVAL;
    *order = c->extrap_order;
    return FIL_OK;
}

fil_status fil_set_dt(fil_ctx *c, double dt) {
    if (!c) return FIL_EINVAL;
    if (!(dt > 0)) return set_err(c, FIL_EINVAL, "fil_set_dt: dt must be > 0");
    c->dt = dt;
    return FIL_OK;
}

fil_status fil_warm_features(fil_ctx *c, float *feat) {
    if (!c) return FIL_EINVAL;
    if (!feat || !is_device_ptr(feat)) return set_err(c, FIL_EINVAL, "fil_warm_features: device array");
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_warm_features: a step is in progress");
    CK(cudaSetDevice(c->device));
    CK(warm_features(c, nullptr, feat));
    CK(cudaStreamSynchronize(c->stream));
    return FIL_OK;
}

fil_status fil_warm_targets(fil_ctx *c, float *targ) {
    if (!c) return FIL_EINVAL;
    if (!targ || !is_device_ptr(targ)) return set_err(c, FIL_EINVAL, "fil_warm_targets: device array");
    if (c->in_step || c->hist < 1)
        return set_err(c, FIL_ESTATE, "fil_warm_targets: needs a step committed since the last set_state");
    CK(cudaSetDevice(c->device));
    CK(warm_targets(c, targ));
    CK(cudaStreamSynchronize(c->stream));
    return FIL_OK;
}

fil_status fil_warm_attach(fil_ctx *c, fil_mlp *net, int32_t mode) {
    if (!c) return FIL_EINVAL;
    if (net && mlp_max_batch(net) < c->lay.M)
        return set_err(c, FIL_EINVAL, "fil_warm_attach: the network's max_batch is below n_fil");
    if (mode != FIL_WARM_BEST_OF_TWO && mode != FIL_WARM_PREDICTION_FIRST)
        return set_err(c, FIL_EINVAL, "fil_warm_attach: unknown mode");
    if (net && c->tether_on)
        return set_err(c, FIL_ESTATE, "fil_warm_attach: not with tethered filaments");
    c->warm_net = net;
    c->warm_mode = mode;
    return FIL_OK;
}

fil_status fil_warm_stats(const fil_ctx *c, int64_t *from_prediction, int64_t *from_extrapolation,
                          int64_t *restarts) {
    if (!c) return FIL_EINVAL;
    if (from_prediction) *from_prediction = c->warm_pred;
    if (from_extrapolation) *from_extrapolation = c->warm_extrap;
    if (restarts) *restarts = c->warm_restart;
    return FIL_OK;
}

fil_status fil_autotune(fil_ctx *c, int32_t reps, int32_t *tile, int32_t *ctas_per_sm,
                        double *ms) {
    if (!c) return FIL_EINVAL;
    if (reps < 1) return set_err(c, FIL_EINVAL, "fil_autotune: reps >= 1");
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_autotune: a step is in progress");
    CK(cudaSetDevice(c->device));
    // the loads of the current state (the unpack of X = (Y_1, 0, Lambda))
    CK(warm_features(c, nullptr, c->warm_feat));
    CK(rpy_autotune(c, c->Yc, c->FT, c->VW, reps, ms));
    drop_graphs(c);
    if (tile) *tile = rpy_tile(c);
    if (ctas_per_sm) *ctas_per_sm = c->rpy_ctas;
    return FIL_OK;
}

fil_status fil_set_pair_schedule(fil_ctx *c, int32_t tile, int32_t targets_per_thread,
                                 int32_t ctas_per_sm) {
    if (!c) return FIL_EINVAL;
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_set_pair_schedule: a step is in progress");
    if (targets_per_thread < 1 || tile % targets_per_thread != 0)
        return set_err(c, FIL_EINVAL, "fil_set_pair_schedule: no such schedule");
    CK(cudaSetDevice(c->device));
    const int threads = tile / targets_per_thread;
    if (!rpy_schedule_valid(c, targets_per_thread, threads, ctas_per_sm, 1))
        return set_err(c, FIL_EINVAL, "fil_set_pair_schedule: no such schedule");
    CK(rpy_set_schedule(c, targets_per_thread, threads, ctas_per_sm, 1));
    drop_graphs(c);
    return FIL_OK;
}

fil_status fil_set_source_split(fil_ctx *c, int32_t split) {
    if (!c) return FIL_EINVAL;
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_set_source_split: a step is in progress");
    CK(cudaSetDevice(c->device));
    if (!rpy_schedule_valid(c, c->rpy_tpt, c->rpy_threads, c->rpy_ctas, split))
        return set_err(c, FIL_EINVAL, "fil_set_source_split: not with the current schedule");
    CK(rpy_set_schedule(c, c->rpy_tpt, c->rpy_threads, c->rpy_ctas, split));
    drop_graphs(c);
    return FIL_OK;
}

fil_status fil_source_split(const fil_ctx *c, int32_t *split) {
    if (!c || !split) return FIL_EINVAL;
    *split = c->rpy_split;
    return FIL_OK;
}

fil_status fil_pair_schedule(const fil_ctx *c, int32_t *tile, int32_t *targets_per_thread,
                             int32_t *ctas_per_sm) {
    if (!c) return FIL_EINVAL;
    if (tile) *tile = rpy_tile(c);
    if (targets_per_thread) *targets_per_thread = c->rpy_tpt;
    if (ctas_per_sm) *ctas_per_sm = c->rpy_ctas;
    return FIL_OK;
}

fil_status fil_set_graph(fil_ctx *c, int32_t enable) {
    if (!c) return FIL_EINVAL;
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_set_graph: a step is in progress");
    CK(cudaSetDevice(c->device));
    drop_graphs(c);
    if (enable && !c->cap_stream)
        CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    c->use_graph = enable ? 1 : 0;
    return FIL_OK;
}

fil_status fil_set_tether(fil_ctx *c, const int32_t *mask, const double *Y1, const double *u1) {
    if (!c) return FIL_EINVAL;
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_set_tether: a step is in progress");
    CK(cudaSetDevice(c->device));
    const int M = c->lay.M;
    if (!mask) {
        if (c->tether_on) drop_graphs(c);
        c->tether_on = 0;
        c->thist = 0;
        return FIL_OK;
    }
    if (!Y1 || !u1) return set_err(c, FIL_EINVAL, "fil_set_tether: Y1 and u1 are required");
    if (c->warm_net)
        return set_err(c, FIL_ESTATE, "fil_set_tether: detach the warm-start network first");
    // the mask as host ints (the argument may be a device array)
    std::vector<int32_t> hm(M);
    CK(cudaMemcpy(hm.data(), mask, sizeof(int32_t) * M, cudaMemcpyDefault));
    int any = 0;
    for (int i = 0; i < M; ++i) {
        hm[i] = hm[i] != 0;
        any |= hm[i];
    }
    if (!c->tether_mem) {
        const int64_t nX = c->lay.nX;
        const size_t doubles = (size_t)M * (3 + 3 + 6 + 6 + 36 + 6) + (size_t)nX * (1 + 6 + 6);
        void *mem = nullptr;
        if (cudaMalloc(&mem, doubles * sizeof(double) + sizeof(int) * (size_t)M) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, FIL_ENOMEM, "fil_set_tether: allocation failed");
        }
        double *d = static_cast<double *>(mem);
        c->tY1 = d; d += 3 * (size_t)M;
        c->tu1 = d; d += 3 * (size_t)M;
        c->tlam = d; d += 6 * (size_t)M;
        c->tlam_prev = d; d += 6 * (size_t)M;
        c->tCinv = d; d += 36 * (size_t)M;
        c->tw = d; d += 6 * (size_t)M;
        c->txr = d; d += nX;
        c->tU = d; d += 6 * (size_t)nX;
        c->tZ = d; d += 6 * (size_t)nX;
        c->tmask = reinterpret_cast<int *>(d);
        c->tether_mem = mem;
        CK(cudaMemsetAsync(c->tmask, 0, sizeof(int) * M, c->stream));
    }
    // a changed mask starts the multipliers' history afresh
    std::vector<int> old(M, 0);
    if (c->tether_on) {
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaMemcpy(old.data(), c->tmask, sizeof(int) * M, cudaMemcpyDeviceToHost));
    }
    bool changed = !c->tether_on;
    for (int i = 0; i < M; ++i) changed |= old[i] != hm[i];
    CK(cudaMemcpyAsync(c->tmask, hm.data(), sizeof(int) * M, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->tY1, Y1, sizeof(double) * 3 * M, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(c->tu1, u1, sizeof(double) * 3 * M, cudaMemcpyDefault, c->stream));
    if (changed) {
        CK(cudaMemsetAsync(c->tlam, 0, sizeof(double) * 6 * M, c->stream));
        CK(cudaMemsetAsync(c->tlam_prev, 0, sizeof(double) * 6 * M, c->stream));
        c->thist = 0;
        drop_graphs(c);
    }
    CK(cudaStreamSynchronize(c->stream));
    c->tether_on = any;
    c->tether_fresh = 1;      // the next step builds J0 for this prescription
    return FIL_OK;
}

fil_status fil_get_tether(fil_ctx *c, double *lam) {
    if (!c || !lam) return FIL_EINVAL;
    CK(cudaSetDevice(c->device));
    const size_t bytes = sizeof(double) * 6 * c->lay.M;
    if (!c->tether_mem) {
        if (is_device_ptr(lam)) CK(cudaMemsetAsync(lam, 0, bytes, c->stream));
        else std::memset(lam, 0, bytes);
    } else {
        CK(cudaMemcpyAsync(lam, c->tlam, bytes, cudaMemcpyDefault, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return FIL_OK;
}

fil_status fil_set_steric(fil_ctx *c, double FS, double chi) {
    if (!c) return FIL_EINVAL;
    if (!(FS >= 0.0) || !std::isfinite(FS) || !(chi > 1.0) || !std::isfinite(chi))
        return set_err(c, FIL_EINVAL, "fil_set_steric: need FS >= 0 finite and chi > 1");
    if (c->in_step) return set_err(c, FIL_ESTATE, "fil_set_steric: a step is in progress");
    CK(cudaSetDevice(c->device));
    if (FS != 0.0 && !c->steric_count) {
        int64_t nb = 1;
        while (nb < 2 * c->lay.S) nb <<= 1;
        int *cnt = nullptr, *bkt = nullptr;
        const size_t table = sizeof(int) * (size_t)nb * kStericCap;   // a multiple of 16 bytes
        const size_t per_seg = (sizeof(int4) + sizeof(float4)) * (size_t)c->lay.S;
        if (cudaMalloc(&cnt, sizeof(int) * nb) != cudaSuccess ||
            cudaMalloc(&bkt, table + per_seg) != cudaSuccess) {
            cudaGetLastError();
            if (cnt) cudaFree(cnt);
            return set_err(c, FIL_ENOMEM, "fil_set_steric: cell grid allocation failed");
        }
        c->steric_count = cnt;
        c->steric_bucket = bkt;
        c->steric_cell = reinterpret_cast<int4 *>(reinterpret_cast<char *>(bkt) + table);
        c->steric_frac = reinterpret_cast<float4 *>(c->steric_cell + c->lay.S);
        c->steric_buckets = nb;
    }
    drop_graphs(c);      // captured residual evaluations hold the old setting
    c->steric_FS = FS;
    c->steric_chi = chi;
    return FIL_OK;
}

fil_status fil_pair_count(const fil_ctx *c, double *pairs) {
    if (!c || !pairs) return FIL_EINVAL;
    *pairs = c->n_pairs;
    return FIL_OK;
}

fil_status fil_sys_stats(const fil_ctx *c, int32_t *iters, double *finf) {
    if (!c) return FIL_EINVAL;
    for (int sy = 0; sy < c->n_sys; ++sy) {
        if (iters) iters[sy] = c->sys_iters_h[sy];
        if (finf) finf[sy] = c->finf_h[sy];
    }
    return FIL_OK;
}

fil_status fil_counters(const fil_ctx *c, int64_t *mobility_applies, int64_t *broyden_iters,
                        int64_t *kernel_launches) {
    if (!c) return FIL_EINVAL;
    if (mobility_applies) *mobility_applies = c->n_applies;
    if (broyden_iters) *broyden_iters = c->n_iters;
    if (kernel_launches) *kernel_launches = c->n_launches;
    return FIL_OK;
}

fil_status fil_profile(fil_ctx *c, int32_t enable) {
    if (!c) return FIL_EINVAL;
    CK(cudaSetDevice(c->device));
    if (enable && !c->prof_ev) {
        c->prof_ev = new (std::nothrow) cudaEvent_t[2 * kProfMax];
        if (!c->prof_ev) return set_err(c, FIL_ENOMEM, "fil_profile: host allocation");
        for (int i = 0; i < 2 * kProfMax; ++i) CK(cudaEventCreate(&c->prof_ev[i]));
    }
    c->prof_on = enable ? 1 : 0;
    return FIL_OK;
}

fil_status fil_profile_read(fil_ctx *c, int64_t *launches, double *total_ms) {
    if (!c) return FIL_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    double sum = 0.0;
    const int n = c->prof_n;
    c->prof_n = 0;   // the record is cleared whatever happens below
    for (int i = 0; i < n; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
        sum += ms;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = sum;
    return FIL_OK;
}

}  // extern "C"
