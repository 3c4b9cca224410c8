// Per-filament warm-start MLP (include/fil_mlp.h): inference and training on
// the tensor cores (tc_gemm.cuh), FP32 master weights with Adam.
//
// Layer l maps in_l -> out_l: (800 padded to 832) -> 256 -> 256 -> 256 -> 192.
// Forward (rows = batch b):
//   X^  = BF16((x - in_mean) / in_std)                 [B x 832] (+ transposed)
//   H_l = BF16(relu(H_{l-1} W_l^T + b_l)), l = 1..3     [B x 256] (+ transposed)
//   Y^  = H_3 W_4^T + b_4 (FP32)                        [B x 192]
// Backward of L = sum (Y^ - T^)^2 / (2B):
//   dY = (Y^ - T^) / B;  dH_3 = (dY W_4) * [H_3 > 0];  dH_{l-1} = (dH_l W_l) * [H_{l-1} > 0]
//   dW_l = dZ_l^T H_{l-1} (K = batch), db_l = column sums of dZ_l (FP32)
// Every product is C = A . B^T with both operands K-major: the weights are
// kept in BF16 both as [out x in] and transposed, and activations and
// gradients are stored both row-major and transposed by the GEMM epilogues.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/fil_mlp.h"
#include "tc_gemm.cuh"

using bf16 = __nv_bfloat16;

namespace fil {
namespace {

constexpr int kLayers = 4;
constexpr int kIn = FIL_MLP_IN, kInP = (FIL_MLP_IN + 63) / 64 * 64, kHid = FIL_MLP_HIDDEN, kOut = FIL_MLP_OUT;
constexpr int kDimIn[kLayers] = {kIn, kHid, kHid, kHid};
constexpr int kDimInP[kLayers] = {kInP, kHid, kHid, kHid};
constexpr int kDimOut[kLayers] = {kHid, kHid, kHid, kOut};

// offsets of W_l and b_l in the packed parameter vector
struct Offsets {
    int64_t w[kLayers], b[kLayers];
};
Offsets param_offsets() {
    Offsets o;
    int64_t p = 0;
    for (int l = 0; l < kLayers; ++l) {
        o.w[l] = p;
        p += (int64_t)kDimOut[l] * kDimIn[l];
        o.b[l] = p;
        p += kDimOut[l];
    }
    return o;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

cudaError_t gemm(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K,
                 const tc::Epilogue &ep, int *err, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(tc::gemm_bf16_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::kSmemBytes);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((M + tc::kTileM - 1) / tc::kTileM),
              (unsigned)((N + tc::kMaxTileN - 1) / tc::kMaxTileN));
    tc::gemm_bf16_kernel<<<grid, tc::kThreads, tc::kSmemBytes, st>>>(A, lda, B, ldb, M, N, K,
                                                                     ep, err);
    return cudaGetLastError();
}

tc::Epilogue epi() {
    tc::Epilogue e{};
    e.alpha = 1.f;
    e.n_valid = 1 << 30;
    return e;
}

// x^ = (x - mean) / std in BF16, row-major [B x kInP] (zero padding) and
// transposed [kInP x ldt] (columns >= B are zeroed by the caller).
__global__ void input_kernel(const float *__restrict__ x, int64_t B, const float *__restrict__ mean,
                             const float *__restrict__ stdv, bf16 *__restrict__ X,
                             bf16 *__restrict__ Xt, int64_t ldt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * kInP) return;
    const int64_t b = i / kInP;
    const int c = (int)(i - b * kInP);
    const float v = c < kIn ? (x[b * kIn + c] - mean[c]) / stdv[c] : 0.f;
    const bf16 h = __float2bfloat16_rn(v);
    X[i] = h;
    if (Xt) Xt[(int64_t)c * ldt + b] = h;
}

__global__ void output_kernel(const float *__restrict__ yhat, int64_t n, const float *__restrict__ mean,
                              const float *__restrict__ stdv, float *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % kOut);
    y[i] = mean[c] + stdv[c] * yhat[i];
}

// dY = (y^ - t^) / B (FP32 and BF16, row-major and transposed) and the loss,
// summed by one CTA in a fixed order.
constexpr int kLossThreads = 1024;
__global__ void __launch_bounds__(kLossThreads)
loss_kernel(const float *__restrict__ yhat, const float *__restrict__ t, int64_t B,
            const float *__restrict__ mean, const float *__restrict__ stdv, float *__restrict__ dYf,
            bf16 *__restrict__ dY, bf16 *__restrict__ dYt, int64_t ldt, float *__restrict__ loss) {
    __shared__ double red[kLossThreads];
    double acc = 0.0;
    const float inv = 1.f / (float)B;
    for (int64_t i = threadIdx.x; i < B * kOut; i += blockDim.x) {
        const int64_t b = i / kOut;
        const int c = (int)(i - b * kOut);
        const float d = yhat[i] - (t[i] - mean[c]) / stdv[c];
        acc += 0.5 * (double)d * (double)d;
        const float g = d * inv;
        dYf[i] = g;
        const bf16 h = __float2bfloat16_rn(g);
        dY[i] = h;
        dYt[(int64_t)c * ldt + b] = h;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kLossThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(red[0] / (double)B);
}

// db[c] = sum_b dZ[b][c], one CTA per column, fixed-order tree.
__global__ void bias_grad_kernel(const float *__restrict__ dZ, int64_t B, int N, float *__restrict__ db) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) acc += dZ[b * N + c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = red[0];
}

// BF16 copies of W_l: [out x inP] (zero-padded columns) and [inP x out].
__global__ void pack_weights_kernel(const float *__restrict__ w, int out, int in, int inP,
                                    bf16 *__restrict__ W, bf16 *__restrict__ Wt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)out * inP) return;
    const int o = (int)(i / inP), c = (int)(i - (int64_t)o * inP);
    const bf16 h = __float2bfloat16_rn(c < in ? w[(int64_t)o * in + c] : 0.f);
    W[i] = h;
    Wt[(int64_t)c * out + o] = h;
}

__global__ void adam_kernel(int64_t n, const float *__restrict__ g, float *__restrict__ p,
                            float *__restrict__ m, float *__restrict__ v, float lr, float c1,
                            float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void zero_cols_kernel(bf16 *__restrict__ a, int rows, int64_t ld, int64_t c0) {
    const int64_t w = ld - c0;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * w) return;
    const int64_t r = i / w;
    a[r * ld + c0 + (i - r * w)] = __float2bfloat16_rn(0.f);
}

__device__ int g_tc_err;   // wait-limit flag of the standalone GEMM entry point

bool dev_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace fil

using namespace fil;

struct fil_mlp {
    cudaStream_t stream;
    int64_t max_batch, ldt;          // ldt: padded batch (K of the weight gradients)
    Offsets off;
    float *params, *grad, *adam_m, *adam_v;
    int64_t adam_t;
    bf16 *W[kLayers], *Wt[kLayers];
    float *in_mean, *in_std, *out_mean, *out_std;
    bf16 *X, *Xt, *H[3], *Ht[3], *dY, *dYt, *dH[3], *dHt[3];
    float *Y, *dYf, *dHf, *loss;
    int *err;
    void *arena;
};

namespace {

struct Carver {
    char *base;
    size_t used = 0;
    template <typename T>
    T *take(size_t n) {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + n * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

void carve(fil_mlp *m, Carver &c) {
    const int64_t B = m->max_batch, T = m->ldt;
    m->params = c.take<float>(FIL_MLP_NPARAM);
    m->grad = c.take<float>(FIL_MLP_NPARAM);
    m->adam_m = c.take<float>(FIL_MLP_NPARAM);
    m->adam_v = c.take<float>(FIL_MLP_NPARAM);
    for (int l = 0; l < kLayers; ++l) {
        m->W[l] = c.take<bf16>((size_t)kDimOut[l] * kDimInP[l]);
        m->Wt[l] = c.take<bf16>((size_t)kDimOut[l] * kDimInP[l]);
    }
    m->in_mean = c.take<float>(kIn);
    m->in_std = c.take<float>(kIn);
    m->out_mean = c.take<float>(kOut);
    m->out_std = c.take<float>(kOut);
    m->X = c.take<bf16>((size_t)B * kInP);
    m->Xt = c.take<bf16>((size_t)kInP * T);
    for (int l = 0; l < 3; ++l) {
        m->H[l] = c.take<bf16>((size_t)B * kHid);
        m->Ht[l] = c.take<bf16>((size_t)kHid * T);
        m->dH[l] = c.take<bf16>((size_t)B * kHid);
        m->dHt[l] = c.take<bf16>((size_t)kHid * T);
    }
    m->dY = c.take<bf16>((size_t)B * kOut);
    m->dYt = c.take<bf16>((size_t)kOut * T);
    m->Y = c.take<float>((size_t)B * kOut);
    m->dYf = c.take<float>((size_t)B * kOut);
    m->dHf = c.take<float>((size_t)B * kHid);
    m->loss = c.take<float>(1);
    m->err = c.take<int>(1);
}

const float *to_device(fil_mlp *m, const float *p, size_t n, float *scratch, cudaError_t &e) {
    if (dev_ptr(p)) return p;
    e = cudaMemcpyAsync(scratch, p, n * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    return scratch;
}

cudaError_t refresh_weights(fil_mlp *m) {
    for (int l = 0; l < kLayers; ++l) {
        const int64_t n = (int64_t)kDimOut[l] * kDimInP[l];
        pack_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(
            m->params + m->off.w[l], kDimOut[l], kDimIn[l], kDimInP[l], m->W[l], m->Wt[l]);
    }
    return cudaGetLastError();
}

// Forward pass on normalised inputs; `train` also writes the transposed
// activations. Output: m->Y (normalised, FP32).
cudaError_t forward(fil_mlp *m, const float *x, int64_t B, bool train) {
    cudaError_t e = cudaSuccess;
    const int64_t n = B * kInP;
    input_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(
        x, B, m->in_mean, m->in_std, m->X, train ? m->Xt : nullptr, m->ldt);
    const bf16 *act = m->X;
    int ld = kInP;
    for (int l = 0; l < 3; ++l) {
        tc::Epilogue ep = epi();
        ep.c_bf16 = m->H[l];
        ep.ldh = kHid;
        if (train) {
            ep.c_bf16_t = m->Ht[l];
            ep.ldt = (int)m->ldt;
        }
        ep.bias = m->params + m->off.b[l];
        ep.relu = 1;
        e = gemm(act, ld, m->W[l], kDimInP[l], (int)B, kHid, kDimInP[l], ep, m->err, m->stream);
        if (e != cudaSuccess) return e;
        act = m->H[l];
        ld = kHid;
    }
    tc::Epilogue ep = epi();
    ep.c_f32 = m->Y;
    ep.ldc = kOut;
    ep.bias = m->params + m->off.b[3];
    return gemm(act, ld, m->W[3], kHid, (int)B, kOut, kHid, ep, m->err, m->stream);
}

cudaError_t zero_pad_columns(fil_mlp *m, int64_t B) {
    // transposed buffers: columns [B, ldt) are the zero padding of the K = batch dimension
    if (B == m->ldt) return cudaSuccess;
    struct {
        bf16 *p;
        int rows;
    } bufs[] = {{m->Xt, kInP}, {m->Ht[0], kHid}, {m->Ht[1], kHid}, {m->Ht[2], kHid},
                {m->dHt[0], kHid}, {m->dHt[1], kHid}, {m->dHt[2], kHid}, {m->dYt, kOut}};
    for (auto &b : bufs) {
        const int64_t n = (int64_t)b.rows * (m->ldt - B);
        zero_cols_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(b.p, b.rows, m->ldt, B);
    }
    return cudaGetLastError();
}

// Loss and gradient into m->grad; the loss (device) in m->loss.
cudaError_t gradients(fil_mlp *m, const float *x, const float *t, int64_t B) {
    const int64_t Kb = round_up(B, tc::kTileK);
    cudaError_t e = zero_pad_columns(m, B);
    if (e != cudaSuccess) return e;
    e = forward(m, x, B, true);
    if (e != cudaSuccess) return e;
    loss_kernel<<<1, kLossThreads, 0, m->stream>>>(m->Y, t, B, m->out_mean, m->out_std, m->dYf,
                                                    m->dY, m->dYt, m->ldt, m->loss);
    // layer 4: dW4 = dY^T H3, db4, dH3 = (dY W4) * [H3 > 0]
    const bf16 *dZ = m->dY, *dZt = m->dYt;
    const float *dZf = m->dYf;
    int ldz = kOut;
    for (int l = 3; l >= 0; --l) {
        const bf16 *Aprev_t = l > 0 ? m->Ht[l - 1] : m->Xt;
        tc::Epilogue eg = epi();
        eg.c_f32 = m->grad + m->off.w[l];
        eg.ldc = kDimIn[l];
        eg.n_valid = kDimIn[l];
        e = gemm(dZt, (int)m->ldt, Aprev_t, (int)m->ldt, kDimOut[l], kDimInP[l], (int)Kb, eg,
                 m->err, m->stream);
        if (e != cudaSuccess) return e;
        bias_grad_kernel<<<kDimOut[l], 256, 0, m->stream>>>(dZf, B, kDimOut[l],
                                                            m->grad + m->off.b[l]);
        if (l == 0) break;
        tc::Epilogue eb = epi();
        eb.c_f32 = m->dHf;
        eb.ldc = kHid;
        eb.c_bf16 = m->dH[l - 1];
        eb.ldh = kHid;
        eb.c_bf16_t = m->dHt[l - 1];
        eb.ldt = (int)m->ldt;
        eb.mask = m->H[l - 1];
        eb.ldm = kHid;
        e = gemm(dZ, ldz, m->Wt[l], kDimOut[l], (int)B, kHid, kDimOut[l], eb, m->err, m->stream);
        if (e != cudaSuccess) return e;
        dZ = m->dH[l - 1];
        dZt = m->dHt[l - 1];
        dZf = m->dHf;
        ldz = kHid;
    }
    return cudaGetLastError();
}

fil_status check_err(fil_mlp *m) {
    int h = 0;
    if (cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return FIL_ECUDA;
    return h ? FIL_ECUDA : FIL_OK;
}

}  // namespace

namespace fil {

cudaError_t mlp_forward_async(fil_mlp *m, const float *x, float *y, int64_t batch,
                              cudaStream_t st, int64_t *launches) {
    const cudaStream_t own = m->stream;
    m->stream = st;
    cudaError_t e = forward(m, x, batch, false);
    if (e == cudaSuccess) {
        const int64_t n = batch * kOut;
        output_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->Y, n, m->out_mean,
                                                                   m->out_std, y);
        e = cudaGetLastError();
    }
    m->stream = own;
    if (launches) *launches += 6;
    return e;
}

int64_t mlp_max_batch(const fil_mlp *m) { return m->max_batch; }

}  // namespace fil

extern "C" {

fil_status fil_mlp_create(int64_t max_batch, void *stream, fil_mlp **out) {
    if (!out || max_batch < 1 || max_batch > (1 << 24)) return FIL_EINVAL;
    *out = nullptr;
    fil_mlp *m = new fil_mlp();
    m->stream = (cudaStream_t)stream;
    m->max_batch = max_batch;
    m->ldt = round_up(max_batch, tc::kTileK);
    m->off = param_offsets();
    Carver sizing{nullptr};
    carve(m, sizing);
    if (cudaMalloc(&m->arena, sizing.used) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return FIL_ENOMEM;
    }
    Carver c{static_cast<char *>(m->arena)};
    carve(m, c);
    cudaError_t e = cudaMemsetAsync(m->arena, 0, sizing.used, m->stream);
    std::vector<float> ones(std::max(kIn, kOut), 1.f);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->in_std, ones.data(), kIn * sizeof(float), cudaMemcpyHostToDevice,
                            m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->out_std, ones.data(), kOut * sizeof(float), cudaMemcpyHostToDevice,
                            m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        cudaFree(m->arena);
        delete m;
        return FIL_ECUDA;
    }
    *out = m;
    return FIL_OK;
}

void fil_mlp_destroy(fil_mlp *m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->arena);
    delete m;
}

fil_status fil_mlp_set_params(fil_mlp *m, const float *params) {
    if (!m || !params) return FIL_EINVAL;
    cudaError_t e = cudaSuccess;
    const float *p = to_device(m, params, FIL_MLP_NPARAM, m->params, e);
    if (e == cudaSuccess && p != m->params)
        e = cudaMemcpyAsync(m->params, p, FIL_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice,
                            m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->adam_m, 0, FIL_MLP_NPARAM * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->adam_v, 0, FIL_MLP_NPARAM * sizeof(float), m->stream);
    m->adam_t = 0;
    if (e == cudaSuccess) e = refresh_weights(m);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? FIL_OK : FIL_ECUDA;
}

fil_status fil_mlp_get_params(fil_mlp *m, float *params) {
    if (!m || !params) return FIL_EINVAL;
    cudaError_t e = cudaMemcpyAsync(params, m->params, FIL_MLP_NPARAM * sizeof(float),
                                    cudaMemcpyDefault, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? FIL_OK : FIL_ECUDA;
}

fil_status fil_mlp_set_norm(fil_mlp *m, const float *in_mean, const float *in_std,
                            const float *out_mean, const float *out_std) {
    if (!m || !in_mean || !in_std || !out_mean || !out_std) return FIL_EINVAL;
    cudaError_t e = cudaMemcpyAsync(m->in_mean, in_mean, kIn * sizeof(float), cudaMemcpyDefault,
                                    m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->in_std, in_std, kIn * sizeof(float), cudaMemcpyDefault, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->out_mean, out_mean, kOut * sizeof(float), cudaMemcpyDefault,
                            m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->out_std, out_std, kOut * sizeof(float), cudaMemcpyDefault, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? FIL_OK : FIL_ECUDA;
}

fil_status fil_mlp_forward(fil_mlp *m, const float *x, float *y, int64_t batch) {
    if (!m || !x || !y || batch < 1 || batch > m->max_batch) return FIL_EINVAL;
    if (!dev_ptr(x) || !dev_ptr(y)) return FIL_EINVAL;
    cudaError_t e = forward(m, x, batch, false);
    const int64_t n = batch * kOut;
    if (e == cudaSuccess) {
        output_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->Y, n, m->out_mean,
                                                                          m->out_std, y);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return FIL_ECUDA;
    return check_err(m);
}

fil_status fil_mlp_gradients(fil_mlp *m, const float *x, const float *target, int64_t batch,
                             float *grad, float *loss) {
    if (!m || !x || !target || !grad || batch < 1 || batch > m->max_batch) return FIL_EINVAL;
    if (!dev_ptr(x) || !dev_ptr(target) || !dev_ptr(grad)) return FIL_EINVAL;
    cudaError_t e = gradients(m, x, target, batch);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grad, m->grad, FIL_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice,
                            m->stream);
    if (e == cudaSuccess && loss)
        e = cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return FIL_ECUDA;
    return check_err(m);
}

fil_status fil_mlp_train_step(fil_mlp *m, const float *x, const float *target, int64_t batch,
                              float lr, float *loss) {
    if (!m || !x || !target || batch < 1 || batch > m->max_batch || !(lr > 0.f)) return FIL_EINVAL;
    if (!dev_ptr(x) || !dev_ptr(target)) return FIL_EINVAL;
    cudaError_t e = gradients(m, x, target, batch);
    m->adam_t += 1;
    const float c1 = 1.f - std::pow(0.9f, (float)m->adam_t);
    const float c2 = 1.f - std::pow(0.999f, (float)m->adam_t);
    if (e == cudaSuccess) {
        adam_kernel<<<(FIL_MLP_NPARAM + 255) / 256, 256, 0, m->stream>>>(
            FIL_MLP_NPARAM, m->grad, m->params, m->adam_m, m->adam_v, lr, c1, c2);
        e = refresh_weights(m);
    }
    if (e == cudaSuccess && loss)
        e = cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return FIL_ECUDA;
    return loss ? check_err(m) : FIL_OK;
}

fil_status fil_tc_gemm_bf16(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb,
                            float *C, int64_t ldc, int64_t M, int64_t N, int64_t K, void *stream) {
    if (!A || !B || !C || M < 1 || N < 32 || N % 32 || K < 64 || K % 64 || lda % 8 || ldb % 8 ||
        ldc % 4 || lda < K || ldb < K || ldc < N || M > (1 << 24) || N > (1 << 16) ||
        K > (1 << 24))
        return FIL_EINVAL;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
         reinterpret_cast<uintptr_t>(C)) & 15)
        return FIL_EINVAL;
    if (!dev_ptr(A) || !dev_ptr(B) || !dev_ptr(C)) return FIL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int *err = nullptr;
    if (cudaGetSymbolAddress((void **)&err, g_tc_err) != cudaSuccess) return FIL_ECUDA;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return FIL_ECUDA;
    tc::Epilogue ep = epi();
    ep.c_f32 = C;
    ep.ldc = (int)ldc;
    if (gemm(reinterpret_cast<const bf16 *>(A), (int)lda, reinterpret_cast<const bf16 *>(B),
             (int)ldb, (int)M, (int)N, (int)K, ep, err, st) != cudaSuccess)
        return FIL_ECUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FIL_ECUDA;
    return h ? FIL_ECUDA : FIL_OK;
}

}  // extern "C"
