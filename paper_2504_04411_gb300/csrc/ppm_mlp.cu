// ppm_mlp.cu -- the learned radius proposer: a 12 -> 64 -> 64 -> 2 MLP (ReLU
// hidden layers).  Arithmetic: BF16 weights, FP32 biases, every layer's
// input (features, h1, h2) rounded to BF16 (round to nearest even from the
// FP32 value), FP32 accumulation.
//
// Inputs: the 12 window features the gather's epilogue writes per hit
// point (ppm_gather_impl.cuh).  Outputs: o0 = predicted log(r_final / r),
// o1 = logit of "this radius will be rejected within the next few tests".
// Training data comes from runs of the plain method; the loss is
// 0.5 (o0 - y0)^2 + BCE(o1, y1) with per-sample weights, minimized with Adam
// (Kingma & Ba 2015) on FP32 master weights whose BF16 copies drive the
// forward passes (the BF16 rounding of the activations is differentiated
// as the identity).  After the F-test update of every iteration the proposer
// shrinks the radius of a hit point the test did not just reject when the
// network calls it doomed: r <- max(r max(exp(o0), min_ratio), bound); the
// window is cleared as on a rejection.  The F-test still runs every
// iteration on whatever radius a hit point has: it keeps the final say.
//
// Inference (k_mlp_forward, k_mlp_propose) runs on the tensor cores: a warp
// takes 16 samples through all three layers with mma.sync m16n8k16 BF16
// products (8 + 32 + 4 per tile).  The FP32 accumulator fragment of one
// layer, after bias, ReLU and BF16 packing, is exactly the A fragment of the
// next, so activations never leave registers; weights sit in shared memory
// with padded rows (B-fragment loads hit 32 distinct banks).  Training
// (k_mlp_grad) is one thread per sample on the FP32 pipes: it needs the
// activations of a 128-sample tile in shared memory for the weight
// gradients anyway, stored feature-major with a row stride of 129 words so
// the lanes of a warp always hit distinct banks.  Each tile's gradient goes
// to scratch and k_mlp_grad_reduce adds the tiles in order (no floating
// atomics), so a training run is bitwise reproducible.
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

// ---- tensor-core inference --------------------------------------------------
// B fragments of m16n8k16 (k x n, column-major) are pairs W[n][k], W[n][k+1]
// of the row-major [out][in] weights: one 32-bit shared load each.  Row
// strides of 12 words (W1: 12 inputs + 4 zero, + pad) and 36 words (W2, W3)
// put the 8 rows x 4 words a warp loads on 32 distinct banks.
constexpr int kLdW1 = 24;   // bf16 per W1 row
constexpr int kLdW2 = 72;   // bf16 per W2 / W3 row

struct __align__(16) TcSmem {
    __nv_bfloat16 W1[kH][kLdW1];     // k >= 12 zero
    __nv_bfloat16 W2[kH][kLdW2];
    __nv_bfloat16 W3[8][kLdW2];      // rows >= 2 zero (the output tile is 8 wide)
    float b1[kH], b2[kH], b3[kOut];
};

__device__ void load_tc_weights(TcSmem& w, const uint8_t* blob)
{
    const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(blob);
    const float* bb = reinterpret_cast<const float*>(blob + kOffB);
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int e = threadIdx.x; e < kH * kLdW1; e += blockDim.x) {
        const int n = e / kLdW1, k = e % kLdW1;
        w.W1[n][k] = k < kIn ? wb[n * kIn + k] : zero;
    }
    for (int e = threadIdx.x; e < kH * kLdW2; e += blockDim.x) {
        const int n = e / kLdW2, k = e % kLdW2;
        w.W2[n][k] = k < kH ? wb[kW1 + n * kH + k] : zero;
    }
    for (int e = threadIdx.x; e < 8 * kLdW2; e += blockDim.x) {
        const int n = e / kLdW2, k = e % kLdW2;
        w.W3[n][k] = (n < kOut && k < kH) ? wb[kW1 + kW2 + n * kH + k] : zero;
    }
    for (int e = threadIdx.x; e < kH + kH + kOut; e += blockDim.x) {
        const float v = bb[e];
        if (e < kH) w.b1[e] = v;
        else if (e < 2 * kH) w.b2[e - kH] = v;
        else w.b3[e - 2 * kH] = v;
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t lds_u32(const __nv_bfloat16* p)
{
    return *reinterpret_cast<const uint32_t*>(p);
}

// c += A (16 x 16, row-major BF16) * B (16 x 8, column-major BF16), FP32
__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One hidden layer's 8 output tiles (64 units) -> the next layer's A
// fragments: tile j holds units 8j..8j+7, i.e. half j % 2 of k-step j / 2.
// c[0], c[1]: row g, units 8j + 2t, +1; c[2], c[3]: row g + 8.
__device__ __forceinline__ void to_next_a(uint32_t (&A)[4][4], int j, const float (&c)[4], float bA, float bB)
{
    const uint32_t lo = pack_bf16x2(fmaxf(c[0] + bA, 0.f), fmaxf(c[1] + bB, 0.f));
    const uint32_t hi = pack_bf16x2(fmaxf(c[2] + bA, 0.f), fmaxf(c[3] + bB, 0.f));
    if (j % 2 == 0) { A[j / 2][0] = lo; A[j / 2][1] = hi; }
    else            { A[j / 2][2] = lo; A[j / 2][3] = hi; }
}

// 16 samples through the network.  xa: this lane's layer-1 A fragment
// (rows g = lane / 4 and g + 8 of the tile, features 2t, 2t+1 and 2t+8,
// 2t+9 with t = lane % 4, BF16).  On return, lanes with t == 0 hold
// o[0], o[1] = (o0, o1) of row g and o[2], o[3] of row g + 8.
__device__ __forceinline__ void mlp_tile(const TcSmem& w, const uint32_t (&xa)[4], float (&o)[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t A2[4][4], A3[4][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16_16816(c, xa, lds_u32(&w.W1[8 * j + g][2 * t]), lds_u32(&w.W1[8 * j + g][2 * t + 8]));
        to_next_a(A2, j, c, w.b1[8 * j + 2 * t], w.b1[8 * j + 2 * t + 1]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            mma_bf16_16816(c, A2[q], lds_u32(&w.W2[8 * j + g][16 * q + 2 * t]),
                           lds_u32(&w.W2[8 * j + g][16 * q + 2 * t + 8]));
        to_next_a(A3, j, c, w.b2[8 * j + 2 * t], w.b2[8 * j + 2 * t + 1]);
    }
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        mma_bf16_16816(c, A3[q], lds_u32(&w.W3[g][16 * q + 2 * t]), lds_u32(&w.W3[g][16 * q + 2 * t + 8]));
    o[0] = c[0] + w.b3[0];
    o[1] = c[1] + w.b3[1];
    o[2] = c[2] + w.b3[0];
    o[3] = c[3] + w.b3[1];
}

// layer-1 A fragment of the tile whose row g is sample s0 + g; feature f of
// sample s is x(s, f); samples >= n and features >= 12 are zero
template <typename XF>
__device__ __forceinline__ void load_x_fragment(uint32_t (&xa)[4], int64_t s0, int64_t n, XF x)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t sA = s0 + g, sB = s0 + g + 8;
    const int f0 = 2 * t, f1 = 2 * t + 8;
    auto val = [&](int64_t s, int f) { return (s < n && f < kIn) ? x(s, f) : 0.f; };
    xa[0] = pack_bf16x2(val(sA, f0), val(sA, f0 + 1));
    xa[1] = pack_bf16x2(val(sB, f0), val(sB, f0 + 1));
    xa[2] = pack_bf16x2(val(sA, f1), val(sA, f1 + 1));
    xa[3] = pack_bf16x2(val(sB, f1), val(sB, f1 + 1));
}

constexpr int kTcWarps = 4;

__global__ void __launch_bounds__(32 * kTcWarps)
k_mlp_forward(const uint8_t* __restrict__ blob, const float* __restrict__ X, int64_t n,
              float* __restrict__ Y)
{
    __shared__ TcSmem w;
    load_tc_weights(w, blob);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t tiles = (n + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * kTcWarps + (threadIdx.x >> 5); tile < tiles;
         tile += (int64_t)gridDim.x * kTcWarps) {
        const int64_t s0 = tile * 16;
        uint32_t xa[4];
        load_x_fragment(xa, s0, n, [&](int64_t s, int f) { return X[s * kIn + f]; });
        float o[4];
        mlp_tile(w, xa, o);
        if (t == 0) {
            if (s0 + g < n) { Y[2 * (s0 + g)] = o[0]; Y[2 * (s0 + g) + 1] = o[1]; }
            if (s0 + g + 8 < n) { Y[2 * (s0 + g + 8)] = o[2]; Y[2 * (s0 + g + 8) + 1] = o[3]; }
        }
    }
}

// ---- gradient of one 128-sample tile ----------------------------------------
__device__ __forceinline__ float bf16_round(float v)
{
    return __bfloat162float(__float2bfloat16_rn(v));
}

constexpr int kTile = 128;
constexpr int kGradChunk = 256;     // tiles of partial gradients held at once (5.2 MB)
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
           const float* __restrict__ M, int64_t n, int64_t tile0, float scale, float* __restrict__ part,
           float* __restrict__ lpart)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    GradSmem& sm = *reinterpret_cast<GradSmem*>(smem_raw);
    load_weights(sm.w, blob);
    const int s = threadIdx.x;
    const int64_t gs = (tile0 + blockIdx.x) * kTile + s;
    const bool live = gs < n;
    // forward, keeping the activations
    float x[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) { x[i] = bf16_round(live ? X[gs * kIn + i] : 0.f); sm.x[i][s] = x[i]; }
#pragma unroll 4
    for (int k = 0; k < kH; ++k) {
        float z = sm.w.b1[k];
#pragma unroll
        for (int i = 0; i < kIn; ++i) z = fmaf(sm.w.W1[k * kIn + i], x[i], z);
        sm.h1[k][s] = bf16_round(fmaxf(z, 0.f));
    }
    float o0 = sm.w.b3[0], o1 = sm.w.b3[1];
    for (int j = 0; j < kH; ++j) {
        float z = sm.w.b2[j];
#pragma unroll 8
        for (int k = 0; k < kH; ++k) z = fmaf(sm.w.W2[j * kH + k], sm.h1[k][s], z);
        z = bf16_round(fmaxf(z, 0.f));
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
        lpart[blockIdx.x] = t;
    }
    // weight gradients: sums over the tile's samples, this tile's row of part
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
        part[(int64_t)blockIdx.x * kParams + e] = acc;
    }
}

// the tiles' partial gradients and losses added to grad and loss in tile
// order: equal inputs give bitwise equal results
__global__ void k_mlp_grad_reduce(const float* __restrict__ part, const float* __restrict__ lpart, int ntiles,
                                  float* __restrict__ grad, float* __restrict__ loss)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kParams) {
        float acc = 0.f;
        for (int t = 0; t < ntiles; ++t) acc += part[(int64_t)t * kParams + e];
        grad[e] += acc;
    }
    if (e == 0) {
        float l = 0.f;
        for (int t = 0; t < ntiles; ++t) l += lpart[t];
        *loss += l;
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
__device__ __forceinline__ unsigned long long propose_one(int64_t h, int64_t nh, int ntc, float o0, float o1,
                                                          float* r, int32_t* t, uint32_t* cnt, float* S,
                                                          float* Q, float bound, float thr_logit,
                                                          float min_ratio)
{
    if (h >= nh || t[h] <= 0) return 0;            // t == 0: the test rejected it just now
    if (!(o1 > thr_logit && o0 < 0.f)) return 0;
    const float rr = r[h];
    const float rn = fmaxf(__fmul_rn(rr, fmaxf(expf(o0), min_ratio)), bound);
    if (!(rn < rr)) return 0;
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
    return 1;
}

__global__ void __launch_bounds__(32 * kTcWarps)
k_mlp_propose(int64_t nh, int ntc, const uint8_t* __restrict__ blob, const float* __restrict__ feat,
              float* __restrict__ r, int32_t* __restrict__ t, uint32_t* __restrict__ cnt,
              float* __restrict__ S, float* __restrict__ Q, float bound, float thr_logit,
              float min_ratio, unsigned long long* __restrict__ proposals)
{
    __shared__ TcSmem w;
    load_tc_weights(w, blob);
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int64_t tiles = (nh + 15) / 16;
    unsigned long long shrunk = 0;
    for (int64_t tile = (int64_t)blockIdx.x * kTcWarps + (threadIdx.x >> 5); tile < tiles;
         tile += (int64_t)gridDim.x * kTcWarps) {
        const int64_t s0 = tile * 16;
        uint32_t xa[4];
        load_x_fragment(xa, s0, nh, [&](int64_t s, int f) { return feat[(int64_t)f * nh + s]; });
        float o[4];
        mlp_tile(w, xa, o);
        if (tq == 0) {
            shrunk += propose_one(s0 + g, nh, ntc, o[0], o[1], r, t, cnt, S, Q, bound, thr_logit, min_ratio);
            shrunk += propose_one(s0 + g + 8, nh, ntc, o[2], o[3], r, t, cnt, S, Q, bound, thr_logit, min_ratio);
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

// blocks for n samples: one 16-sample tile per warp, at most 4096 blocks
// (the kernels loop over the tiles)
unsigned tc_grid(int64_t n)
{
    const int64_t tiles = (n + 15) / 16;
    const int64_t blocks = (tiles + kTcWarps - 1) / kTcWarps;
    return (unsigned)(blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks));
}

}  // namespace

int ppm_mlp_propose_launch(ppm_ctx* c, float bound)
{
    if (!c->mlp || c->nh == 0) return PPM_OK;
    const float thr = c->mlp_threshold;
    const float thr_logit = logf(thr / (1.f - thr));
    k_mlp_propose<<<tc_grid(c->nh), 32 * kTcWarps, 0, c->stream>>>(
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
    if (enable && c->prm.test) return PPM_EINVAL;   // features describe the F-test's window
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
    k_mlp_forward<<<tc_grid(n), 32 * kTcWarps, 0, (cudaStream_t)stream>>>((const uint8_t*)blob, X, n, Y);
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
    // per-tile partial sums in stream-ordered scratch, reduced in tile
    // order, at most kGradChunk tiles at a time
    const cudaStream_t st = (cudaStream_t)stream;
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int chunk = (int)(ntiles < kGradChunk ? ntiles : kGradChunk);
    float* part = nullptr;
    if (cudaMallocAsync((void**)&part, ((size_t)chunk * kParams + chunk) * sizeof(float), st) != cudaSuccess) {
        cudaGetLastError();
        return PPM_ENOMEM;
    }
    float* lpart = part + (size_t)chunk * kParams;
    int rc = PPM_OK;
    for (int64_t t0 = 0; t0 < ntiles && rc == PPM_OK; t0 += chunk) {
        const int nt = (int)(ntiles - t0 < chunk ? ntiles - t0 : chunk);
        k_mlp_grad<<<(unsigned)nt, kTile, sizeof(GradSmem), st>>>((const uint8_t*)blob, X, Y, M, n, t0, scale,
                                                                   part, lpart);
        k_mlp_grad_reduce<<<(kParams + 255) / 256, 256, 0, st>>>(part, lpart, nt, grad, loss);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            ppm_note_cuda_error(e, "launch", __FILE__, __LINE__);
            rc = PPM_ECUDA;
        }
    }
    cudaFreeAsync(part, st);
    return rc;
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
