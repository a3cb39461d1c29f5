// ppm_mlp.cu -- the learned radius proposer: a 12 -> 64 -> 64 -> 2 MLP (ReLU
// hidden layers) with BF16 weights and FP32 biases, activations and
// accumulation.
//
// Inputs: the 12 window features the gather's epilogue writes per hit
// point (ppm_gather_impl.cuh).  Outputs: o0 = predicted log(r_final / r),
// o1 = logit of "this radius will be rejected within the next few tests".
// Training data comes from runs of the plain method; the loss is
// 0.5 (o0 - y0)^2 + BCE(o1, y1) with per-sample weights, minimized with Adam
// (Kingma & Ba 2015) on FP32 master weights whose BF16 copies drive the
// forward passes.  After the F-test update of every iteration the proposer
// shrinks the radius of a hit point the test did not just reject when the
// network calls it doomed: r <- max(r max(exp(o0), min_ratio), bound); the
// window is cleared as on a rejection.  The F-test still runs every
// iteration on whatever radius a hit point has: it stays the judge.
//
// The network is tiny (4,992 MACs per sample): one thread per sample on the
// FP32 pipes, weights broadcast from shared memory.  Gradients are reduced
// per 128-sample tile from shared-memory activations stored feature-major
// with a row stride of 129 words, so the lanes of a warp always hit
// distinct banks.
#include <cuda_bf16.h>

#include "ppm_internal.cuh"

namespace {

constexpr int kIn = PPM_MLP_IN, kH = PPM_MLP_HIDDEN, kOut = PPM_MLP_OUT;
constexpr int kW1 = kH * kIn, kW2 = kH * kH, kW3 = kOut * kH;
constexpr int kParams = kW1 + kW2 + kW3 + kH + kH + kOut;   // 5,122
// blob: W1, W2, W3 as bf16 (row-major [out][in]), then b1, b2, b3 as f32
constexpr int kOffB = (kW1 + kW2 + kW3) * 2;                 // 9,984 bytes

struct MlpSmem {
    float W1[kW1], W2[kW2], W3[kW3], b1[kH], b2[kH], b3[kOut];
};

__device__ __forceinline__ void load_weights(MlpSmem& w, const uint8_t* blob)
{
    const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(blob);
    const float* bb = reinterpret_cast<const float*>(blob + kOffB);
    for (int e = threadIdx.x; e < kW1 + kW2 + kW3; e += blockDim.x) {
        const float v = __bfloat162float(wb[e]);
        if (e < kW1) w.W1[e] = v;
        else if (e < kW1 + kW2) w.W2[e - kW1] = v;
        else w.W3[e - kW1 - kW2] = v;
    }
    for (int e = threadIdx.x; e < kH + kH + kOut; e += blockDim.x) {
        const float v = bb[e];
        if (e < kH) w.b1[e] = v;
        else if (e < 2 * kH) w.b2[e - kH] = v;
        else w.b3[e - 2 * kH] = v;
    }
    __syncthreads();
}

__device__ __forceinline__ void mlp_forward(const MlpSmem& w, const float (&x)[kIn], float& o0, float& o1)
{
    float h1[kH];
#pragma unroll
    for (int k = 0; k < kH; ++k) {
        float z = w.b1[k];
#pragma unroll
        for (int i = 0; i < kIn; ++i) z = fmaf(w.W1[k * kIn + i], x[i], z);
        h1[k] = fmaxf(z, 0.f);
    }
    o0 = w.b3[0];
    o1 = w.b3[1];
#pragma unroll 4
    for (int j = 0; j < kH; ++j) {
        float z = w.b2[j];
#pragma unroll
        for (int k = 0; k < kH; ++k) z = fmaf(w.W2[j * kH + k], h1[k], z);
        z = fmaxf(z, 0.f);
        o0 = fmaf(w.W3[j], z, o0);
        o1 = fmaf(w.W3[kH + j], z, o1);
    }
}

__global__ void __launch_bounds__(256)
k_mlp_forward(const uint8_t* __restrict__ blob, const float* __restrict__ X, int64_t n,
              float* __restrict__ Y)
{
    __shared__ MlpSmem w;
    load_weights(w, blob);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) x[i] = X[s * kIn + i];
    float o0, o1;
    mlp_forward(w, x, o0, o1);
    Y[2 * s] = o0;
    Y[2 * s + 1] = o1;
}

// ---- gradient of one 128-sample tile ----------------------------------------
constexpr int kTile = 128;
constexpr int kLd = kTile + 1;        // row stride: lanes hit distinct banks

struct GradSmem {
    MlpSmem w;
    float x[kIn][kLd];
    float h1[kH][kLd];
    float h2[kH][kLd];
    float d1[kH][kLd];
    float d2[kH][kLd];
    float dout[kOut][kLd];
    float loss[kTile / 32];
};

__global__ void __launch_bounds__(kTile)
k_mlp_grad(const uint8_t* __restrict__ blob, const float* __restrict__ X, const float* __restrict__ Y,
           const float* __restrict__ M, int64_t n, float scale, float* __restrict__ grad,
           float* __restrict__ loss)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    GradSmem& sm = *reinterpret_cast<GradSmem*>(smem_raw);
    load_weights(sm.w, blob);
    const int s = threadIdx.x;
    const int64_t gs = (int64_t)blockIdx.x * kTile + s;
    const bool live = gs < n;
    // forward, keeping the activations
    float x[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) { x[i] = live ? X[gs * kIn + i] : 0.f; sm.x[i][s] = x[i]; }
#pragma unroll 4
    for (int k = 0; k < kH; ++k) {
        float z = sm.w.b1[k];
#pragma unroll
        for (int i = 0; i < kIn; ++i) z = fmaf(sm.w.W1[k * kIn + i], x[i], z);
        sm.h1[k][s] = fmaxf(z, 0.f);
    }
    float o0 = sm.w.b3[0], o1 = sm.w.b3[1];
    for (int j = 0; j < kH; ++j) {
        float z = sm.w.b2[j];
#pragma unroll 8
        for (int k = 0; k < kH; ++k) z = fmaf(sm.w.W2[j * kH + k], sm.h1[k][s], z);
        z = fmaxf(z, 0.f);
        sm.h2[j][s] = z;
        o0 = fmaf(sm.w.W3[j], z, o0);
        o1 = fmaf(sm.w.W3[kH + j], z, o1);
    }
    // loss 0.5 m0 (o0 - y0)^2 + m1 BCE(o1, y1) and its derivatives
    float g0 = 0.f, g1 = 0.f, l = 0.f;
    if (live) {
        const float y0 = Y[2 * gs], y1 = Y[2 * gs + 1];
        const float m0 = M[2 * gs], m1 = M[2 * gs + 1];
        const float e = o0 - y0;
        const float sig = 1.f / (1.f + expf(-o1));
        g0 = m0 * e * scale;
        g1 = m1 * (sig - y1) * scale;
        l = (0.5f * m0 * e * e + m1 * (fmaxf(o1, 0.f) - o1 * y1 + log1pf(expf(-fabsf(o1))))) * scale;
    }
    sm.dout[0][s] = g0;
    sm.dout[1][s] = g1;
    // backward through the hidden layers
    for (int j = 0; j < kH; ++j) {
        const float d = fmaf(sm.w.W3[j], g0, sm.w.W3[kH + j] * g1);
        sm.d2[j][s] = sm.h2[j][s] > 0.f ? d : 0.f;
    }
    for (int k = 0; k < kH; ++k) {
        float d = 0.f;
#pragma unroll 8
        for (int j = 0; j < kH; ++j) d = fmaf(sm.w.W2[j * kH + k], sm.d2[j][s], d);
        sm.d1[k][s] = sm.h1[k][s] > 0.f ? d : 0.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((s & 31) == 0) sm.loss[s >> 5] = l;
    __syncthreads();
    if (s == 0) {
        float t = 0.f;
        for (int q = 0; q < kTile / 32; ++q) t += sm.loss[q];
        atomicAdd(loss, t);
    }
    // weight gradients: sums over the tile's samples, one atomic per entry
    for (int e = s; e < kParams; e += kTile) {
        float acc = 0.f;
        if (e < kW1) {
            const int k = e / kIn, i = e % kIn;
            for (int q = 0; q < kTile; ++q) acc = fmaf(sm.d1[k][q], sm.x[i][q], acc);
        } else if (e < kW1 + kW2) {
            const int j = (e - kW1) / kH, k = (e - kW1) % kH;
            for (int q = 0; q < kTile; ++q) acc = fmaf(sm.d2[j][q], sm.h1[k][q], acc);
        } else if (e < kW1 + kW2 + kW3) {
            const int o = (e - kW1 - kW2) / kH, j = (e - kW1 - kW2) % kH;
            for (int q = 0; q < kTile; ++q) acc = fmaf(sm.dout[o][q], sm.h2[j][q], acc);
        } else if (e < kW1 + kW2 + kW3 + kH) {
            const int k = e - kW1 - kW2 - kW3;
            for (int q = 0; q < kTile; ++q) acc += sm.d1[k][q];
        } else if (e < kW1 + kW2 + kW3 + 2 * kH) {
            const int j = e - kW1 - kW2 - kW3 - kH;
            for (int q = 0; q < kTile; ++q) acc += sm.d2[j][q];
        } else {
            const int o = e - kW1 - kW2 - kW3 - 2 * kH;
            for (int q = 0; q < kTile; ++q) acc += sm.dout[o][q];
        }
        atomicAdd(grad + e, acc);
    }
}

// Adam on the FP32 master parameters; writes the blob and clears the gradient
__global__ void k_mlp_adam(float* __restrict__ master, float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps,
                           float c1, float c2, uint8_t* __restrict__ blob)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kParams) return;
    const float g = grad[e];
    const float mm = b1 * m[e] + (1.f - b1) * g;
    const float vv = b2 * v[e] + (1.f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    const float p = master[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    master[e] = p;
    grad[e] = 0.f;
    if (e < kW1 + kW2 + kW3) reinterpret_cast<__nv_bfloat16*>(blob)[e] = __float2bfloat16_rn(p);
    else reinterpret_cast<float*>(blob + kOffB)[e - (kW1 + kW2 + kW3)] = p;
}

__global__ void k_mlp_pack(const float* __restrict__ master, uint8_t* __restrict__ blob)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kParams) return;
    if (e < kW1 + kW2 + kW3) reinterpret_cast<__nv_bfloat16*>(blob)[e] = __float2bfloat16_rn(master[e]);
    else reinterpret_cast<float*>(blob + kOffB)[e - (kW1 + kW2 + kW3)] = master[e];
}

// after the F-test update: shrink the doomed radii the test did not reject
__global__ void __launch_bounds__(256)
k_mlp_propose(int64_t nh, int ntc, const uint8_t* __restrict__ blob, const float* __restrict__ feat,
              float* __restrict__ r, int32_t* __restrict__ t, uint32_t* __restrict__ cnt,
              float* __restrict__ S, float* __restrict__ Q, float bound, float thr_logit,
              float min_ratio, unsigned long long* __restrict__ proposals)
{
    __shared__ MlpSmem w;
    load_weights(w, blob);
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long shrunk = 0;
    if (h < nh && t[h] > 0) {                       // t == 0: the test rejected it just now
        float x[kIn];
#pragma unroll
        for (int q = 0; q < kIn; ++q) x[q] = feat[(int64_t)q * nh + h];
        float o0, o1;
        mlp_forward(w, x, o0, o1);
        if (o1 > thr_logit && o0 < 0.f) {
            const float rr = r[h];
            const float rn = fmaxf(__fmul_rn(rr, fmaxf(expf(o0), min_ratio)), bound);
            if (rn < rr) {
                r[h] = rn;
                t[h] = 0;
#pragma unroll
                for (int g = 0; g < PPM_NG; ++g) cnt[g * nh + h] = 0u;
                for (int c = 0; c < ntc; ++c)
#pragma unroll
                    for (int g = 0; g < PPM_NG; ++g) {
                        S[((int64_t)c * PPM_NG + g) * nh + h] = 0.f;
                        Q[((int64_t)c * PPM_NG + g) * nh + h] = 0.f;
                    }
                shrunk = 1;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) shrunk += __shfl_xor_sync(0xffffffffu, shrunk, o);
    if ((threadIdx.x & 31) == 0 && shrunk) atomicAdd(proposals, shrunk);
}

__global__ void k_features_out(int64_t nh, const float* __restrict__ feat, const uint32_t* __restrict__ orig,
                               float* __restrict__ out)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    const int64_t o = orig[h];
#pragma unroll
    for (int q = 0; q < kIn; ++q) out[o * kIn + q] = feat[(int64_t)q * nh + h];
}

}  // namespace

int ppm_mlp_propose_launch(ppm_ctx* c, float bound)
{
    if (!c->mlp || c->nh == 0) return PPM_OK;
    const float thr = c->mlp_threshold;
    const float thr_logit = logf(thr / (1.f - thr));
    k_mlp_propose<<<(unsigned)((c->nh + 255) / 256), 256, 0, c->stream>>>(
        c->nh, c->ntc, (const uint8_t*)c->mlp, c->feat, c->r, c->t, c->cnt, c->S, c->Q, bound,
        thr_logit, c->mlp_max_shrink, c->counters + 4);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

extern "C" {

int ppm_set_features(ppm_ctx* c, int32_t enable)
{
    PPM_ENTRY();
    if (!c) return PPM_EINVAL;
    if (!enable) {
        if (c->mlp) return PPM_ESTATE;          // the proposer reads the features
        PPM_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(c->feat);
        c->feat = nullptr;
        return PPM_OK;
    }
    if (!c->feat && c->nh > 0) {
        if (cudaMalloc(&c->feat, (size_t)c->nh * kIn * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            c->feat = nullptr;
            return PPM_ENOMEM;
        }
        PPM_CUDA(cudaMemsetAsync(c->feat, 0, (size_t)c->nh * kIn * sizeof(float), c->stream));
    }
    return PPM_OK;
}

int ppm_get_features(ppm_ctx* c, float* out)
{
    PPM_ENTRY();
    if (!c || (!out && c->nh > 0)) return PPM_EINVAL;
    if (!c->feat) return PPM_ESTATE;
    if (c->nh > 0) {
        k_features_out<<<(unsigned)((c->nh + 255) / 256), 256, 0, c->stream>>>(c->nh, c->feat, c->hp_orig, out);
        PPM_LAUNCH_CHECK();
    }
    return PPM_OK;
}

int ppm_set_mlp(ppm_ctx* c, const void* blob, float doom_threshold, float min_ratio)
{
    PPM_ENTRY();
    if (!c) return PPM_EINVAL;
    if (!blob) { c->mlp = nullptr; return PPM_OK; }
    if (!(doom_threshold > 0.f && doom_threshold < 1.f) || !(min_ratio > 0.f && min_ratio <= 1.f))
        return PPM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(blob) & 15u) != 0) return PPM_EINVAL;
    const int rc = ppm_set_features(c, 1);
    if (rc) return rc;
    c->mlp = blob;
    c->mlp_threshold = doom_threshold;
    c->mlp_max_shrink = min_ratio;
    return PPM_OK;
}

int ppm_mlp_forward(const void* blob, const float* X, int64_t n, float* Y, void* stream)
{
    PPM_ENTRY();
    if (!blob || n < 0 || (n > 0 && (!X || !Y))) return PPM_EINVAL;
    if (n == 0) return PPM_OK;
    k_mlp_forward<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((const uint8_t*)blob, X, n, Y);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_mlp_grad(const void* blob, const float* X, const float* Y, const float* M, int64_t n,
                 float scale, float* grad, float* loss, void* stream)
{
    PPM_ENTRY();
    if (!blob || !grad || !loss || n < 0 || (n > 0 && (!X || !Y || !M))) return PPM_EINVAL;
    if (n == 0) return PPM_OK;
    static bool attr_set[256] = {};
    int dev = 0;
    PPM_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 256 && !attr_set[dev]) {
        PPM_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem)));
        attr_set[dev] = true;
    }
    k_mlp_grad<<<(unsigned)((n + kTile - 1) / kTile), kTile, sizeof(GradSmem), (cudaStream_t)stream>>>(
        (const uint8_t*)blob, X, Y, M, n, scale, grad, loss);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_mlp_adam(float* master, float* grad, float* m, float* v, int32_t step, float lr, void* blob,
                 void* stream)
{
    PPM_ENTRY();
    if (!master || !grad || !m || !v || !blob || step < 1 || !(lr > 0.f)) return PPM_EINVAL;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(master, grad, m, v, lr, b1, b2, 1e-8f,
                                                                         c1, c2, (uint8_t*)blob);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_mlp_pack(const float* master, void* blob, void* stream)
{
    PPM_ENTRY();
    if (!master || !blob) return PPM_EINVAL;
    k_mlp_pack<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(master, (uint8_t*)blob);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

}  // extern "C"
