// ppm_api.cu -- the C ABI of libppm (declared in include/ppm.h): argument
// checks, context lifecycle, the per-iteration sequence and state I/O.
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "ppm_internal.cuh"

void ppm_note_cuda_error(cudaError_t e, const char* what, const char* file, int line)
{
    if (getenv("PPM_DEBUG"))
        fprintf(stderr, "libppm: %s failed: %s (%s:%d)\n", what, cudaGetErrorString(e), file, line);
}

namespace {

// ---- hit-point preparation ---------------------------------------------
__device__ __forceinline__ uint32_t ord_bits(float f)
{   // float -> uint32 with the same order
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_float(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_bbox(int64_t n, const float* __restrict__ pos, uint32_t* __restrict__ bb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const uint32_t o = ord_bits(pos[3 * i + d]);
        atomicMin(bb + d, o);
        atomicMax(bb + 3 + d, o);
    }
}

__device__ __forceinline__ uint32_t spread3(uint32_t x)
{   // 10 bits -> every third bit of 30
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// Index of a point on the 3D Hilbert curve of order 10, from the
// "transpose" formulation of J. Skilling, "Programming the Hilbert curve"
// (AIP Conf. Proc. 707, 2004): undo the curve's excess rotations level by
// level, Gray-encode, then interleave the bits (X[0] most significant).
// Unlike Morton order the curve has no jumps, so any 32 consecutive hit
// points form one compact patch -- the unit a warp gathers over.
__device__ __forceinline__ uint32_t hilbert3(uint32_t x0, uint32_t x1, uint32_t x2)
{
    uint32_t X[3] = {x0, x1, x2};
    const uint32_t M = 1u << 9;
    for (uint32_t Q = M; Q > 1u; Q >>= 1) {
        const uint32_t P = Q - 1u;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1u; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1u;
    X[0] ^= t; X[1] ^= t; X[2] ^= t;
    return (spread3(X[0]) << 2) | (spread3(X[1]) << 1) | spread3(X[2]);
}

__global__ void k_morton(int64_t n, const float* __restrict__ pos, const uint32_t* __restrict__ bb,
                         uint32_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float lo = ord_float(bb[d]), hi = ord_float(bb[3 + d]);
        const float ext = hi - lo;
        float f = ext > 0.f ? (pos[3 * i + d] - lo) / ext : 0.f;
        f = fminf(fmaxf(f, 0.f), 1.f);
        q[d] = (uint32_t)(f * 1023.0f);
    }
    keys[i] = hilbert3(q[0], q[1], q[2]);
    vals[i] = (uint32_t)i;
}

__global__ void k_hp_permute(int64_t n, const uint32_t* __restrict__ vals,
                             const float* __restrict__ pos, const float* __restrict__ u,
                             const float* __restrict__ v, const uint32_t* __restrict__ nq,
                             const float* __restrict__ rho, uint32_t* __restrict__ orig,
                             float4* __restrict__ hp_pos, float4* __restrict__ hp_u,
                             float4* __restrict__ hp_v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = vals[i];
    if (orig) orig[i] = (uint32_t)j;   // NULL: the order is kept
    hp_pos[i] = make_float4(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2],
                            __uint_as_float(nq ? nq[j] : 0u));
    hp_u[i] = make_float4(u[3 * j], u[3 * j + 1], u[3 * j + 2], rho ? rho[2 * j] : 0.f);
    hp_v[i] = make_float4(v[3 * j], v[3 * j + 1], v[3 * j + 2], rho ? rho[2 * j + 1] : 0.f);
}

__global__ void k_fill_f32(int64_t n, float* __restrict__ p, float v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_rmax(int64_t n, const float* __restrict__ r, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float v = i < n ? r[i] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int*)out, __float_as_int(v));
}

// state: internal (sorted, [slot][nh]) <-> caller order ([n][slot])
template <bool OUT>
__global__ void k_state_io(int64_t nh, int ntc, int nch, const uint32_t* __restrict__ orig,
                           float* r, int32_t* t, float* F, double* tau, uint32_t* cnt,
                           float* S, float* Q, ppm_state_view v)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    const int64_t o = orig[h];
    if (v.r) { if (OUT) v.r[o] = r[h]; else r[h] = v.r[o]; }
    if (v.t) { if (OUT) v.t[o] = t[h]; else t[h] = v.t[o]; }
    if (v.F) { if (OUT) v.F[o] = F[h]; else F[h] = v.F[o]; }
    if (v.tau)
        for (int c = 0; c < nch; ++c) {
            if (OUT) v.tau[o * nch + c] = tau[h * nch + c]; else tau[h * nch + c] = v.tau[o * nch + c];
        }
    if (v.counts)
        for (int g = 0; g < PPM_NG; ++g) {
            if (OUT) v.counts[o * PPM_NG + g] = (int32_t)cnt[g * nh + h];
            else cnt[g * nh + h] = (uint32_t)v.counts[o * PPM_NG + g];
        }
    for (int c = 0; c < ntc; ++c)
        for (int g = 0; g < PPM_NG; ++g) {
            const int64_t in = ((int64_t)c * PPM_NG + g) * nh + h;
            const int64_t ex = (o * ntc + c) * PPM_NG + g;
            if (v.S) { if (OUT) v.S[ex] = S[in]; else S[in] = v.S[ex]; }
            if (v.Q) { if (OUT) v.Q[ex] = Q[in]; else Q[in] = v.Q[ex]; }
        }
}

template <typename T>
bool dalloc(T** p, int64_t n)
{
    if (n <= 0) n = 1;
    if (cudaMalloc(p, (size_t)n * sizeof(T)) != cudaSuccess) { cudaGetLastError(); *p = nullptr; return false; }
    return true;
}

bool finite_pos(float x) { return isfinite(x) && x > 0.f; }

int ensure_fc(ppm_ctx* c, int upto, int* launches)
{
    if (upto <= c->fc_upto) return PPM_OK;
    *launches += 2;
    if (upto >= c->fc_cap) {
        int cap = c->fc_cap > 0 ? c->fc_cap : 256;
        while (cap <= upto) cap *= 2;
        double* nt = nullptr;
        float2* nm = nullptr;
        if (!dalloc(&nt, cap + 1)) return PPM_ENOMEM;
        if (!dalloc(&nm, cap + 1)) { cudaFree(nt); return PPM_ENOMEM; }
        if (c->fc) {
            PPM_CUDA(cudaMemcpyAsync(nt, c->fc, (c->fc_upto + 1) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            PPM_CUDA(cudaMemcpyAsync(nm, c->fm, (c->fc_upto + 1) * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
            PPM_CUDA(cudaStreamSynchronize(c->stream));
            cudaFree(c->fc);
            cudaFree(c->fm);
        } else {
            PPM_CUDA(cudaMemsetAsync(nt, 0, sizeof(double), c->stream));
            PPM_CUDA(cudaMemsetAsync(nm, 0, sizeof(float2), c->stream));
        }
        c->fc = nt;
        c->fm = nm;
        c->fc_cap = cap;
    }
    // fill up to the capacity in one launch: later iterations hit the table
    const int to = c->fc_cap;
    int rc = c->prm.test ? ppm_chi2_fill(c->fc, c->fc_upto + 1, to, PPM_NG - 1, c->prm.alpha_f, c->stream)
                         : ppm_fcrit_fill(c->fc, c->fc_upto + 1, to, (double)c->J, c->prm.alpha_f, c->stream);
    if (rc) return rc;
    rc = ppm_window_m_fill(c->fm, c->fc_upto + 1, to, (double)c->J, c->stream);
    if (rc) return rc;
    c->fc_upto = to;
    return PPM_OK;
}

void free_ctx(ppm_ctx* c)
{
    if (!c) return;
    cudaFree(c->hp_orig); cudaFree(c->hp_pos); cudaFree(c->hp_u); cudaFree(c->hp_v);
    cudaFree(c->r); cudaFree(c->t); cudaFree(c->F); cudaFree(c->tau);
    cudaFree(c->cnt); cudaFree(c->S); cudaFree(c->Q);
    cudaFree(c->cell_start);
    cudaFree(c->rec0); cudaFree(c->rec1); cudaFree(c->aux);
    cudaFree(c->pack);
    ppm_sort_scratch_free(&c->sort);
    cudaFree(c->geom_dev); cudaFree(c->rmax); cudaFree(c->fc); cudaFree(c->fm);
    cudaFree(c->counters); cudaFree(c->err_dev); cudaFree(c->feat);
    if (c->copy_st) cudaStreamSynchronize(c->copy_st);
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->hbuf[k]);
        if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
        if (c->ev_used[k]) cudaEventDestroy(c->ev_used[k]);
        if (c->ev_stats[k]) cudaEventDestroy(c->ev_stats[k]);
    }
    if (c->hstats) cudaFreeHost(c->hstats);
    if (c->copy_st) cudaStreamDestroy(c->copy_st);
    delete c;
}

}  // namespace

int ppm_prepare_hitpoints(const ppm_hitpoints* hp, bool with_rho, uint32_t* orig, float4* pos,
                          float4* u, float4* v, cudaStream_t st)
{
    const int64_t n = hp->n;
    if (n <= 0) return PPM_OK;
    // spatial order: 30-bit Hilbert index of the position in the hit
    // points' bounding box, stable radix sort
    SortScratch hs;
    uint32_t* bb = nullptr;
    if (!dalloc(&bb, 6)) return PPM_ENOMEM;
    int rc = PPM_OK;
    const uint32_t init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    if (cudaMemcpyAsync(bb, init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = PPM_ECUDA;
    if (rc == PPM_OK) rc = ppm_sort_scratch_reserve(&hs, n);
    if (rc == PPM_OK) {
        const unsigned nb = (unsigned)((n + 255) / 256);
        k_bbox<<<nb, 256, 0, st>>>(n, hp->pos, bb);
        k_morton<<<nb, 256, 0, st>>>(n, hp->pos, bb, hs.keys, hs.vals);
        rc = ppm_radix_sort_pairs(&hs, n, 30, st);
        if (rc == PPM_OK) {
            k_hp_permute<<<nb, 256, 0, st>>>(n, hs.vals, hp->pos, hp->u, hp->v, hp->nq,
                                             with_rho ? hp->rho : nullptr, orig, pos, u, v);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                ppm_note_cuda_error(e, "hit-point preparation", __FILE__, __LINE__);
                rc = PPM_ECUDA;
            }
        }
    }
    cudaFree(bb);
    ppm_sort_scratch_free(&hs);
    return rc;
}

extern "C" {

void ppm_default_params(ppm_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->k = 0.7f;
    p->alpha_f = 0.01;
    p->rmin_ratio = 0.001f;
    p->cell_factor = 1.0f;
    p->channels = 1;
    p->rgb_test = 0;
    p->vcm = 0;
    p->n_vm = 0.f;
    p->mapping = 0;
}

const char* ppm_strerror(int code)
{
    switch (code) {
        case PPM_OK: return "ok";
        case PPM_EINVAL: return "invalid argument";
        case PPM_ENOMEM: return "device allocation failed";
        case PPM_ECUDA: return "CUDA runtime error";
        case PPM_ETIMEOUT: return "bounded device wait timed out";
        case PPM_ESTATE: return "call out of order";
        case PPM_EINCOMPLETE: return "a gather skipped cells (a sphere spanned more cells than a hash block)";
        default: return "unknown error";
    }
}

int ppm_create(const ppm_hitpoints* hp, float r0, float alpha, const ppm_params* params,
               void* stream, ppm_ctx** out)
{
    PPM_ENTRY();
    if (!out) return PPM_EINVAL;
    *out = nullptr;
    if (!hp || hp->n < 0 || hp->n > 0x7fffffffll) return PPM_EINVAL;
    if (hp->n > 0 && (!hp->pos || !hp->u || !hp->v)) return PPM_EINVAL;
    if (!finite_pos(r0) || !(alpha > 0.f && alpha < 1.f)) return PPM_EINVAL;
    ppm_params prm;
    if (params) prm = *params; else ppm_default_params(&prm);
    if (!(prm.k > 0.f && prm.k < 1.f) || !(prm.alpha_f > 0.0 && prm.alpha_f < 1.0)) return PPM_EINVAL;
    if (!(prm.rmin_ratio >= 0.f && prm.rmin_ratio < 1.f)) return PPM_EINVAL;
    if (!(prm.cell_factor >= 0.5f && prm.cell_factor <= 4.0f)) return PPM_EINVAL;
    if (prm.channels != 1 && prm.channels != 3) return PPM_EINVAL;
    if (prm.rgb_test && prm.channels != 3) return PPM_EINVAL;
    if (prm.vcm && hp->n > 0 && (!hp->rho || !hp->nq)) return PPM_EINVAL;
    if (prm.n_vm < 0.f) return PPM_EINVAL;
    if (prm.mapping < 0 || prm.mapping > 4) return PPM_EINVAL;
    // traversal 3 tests one channel, traversal 4 gathers one flux channel
    if ((prm.mapping == 3 && prm.rgb_test) || (prm.mapping == 4 && prm.channels == 3)) return PPM_EINVAL;
    if (prm.test != 0 && prm.test != 1) return PPM_EINVAL;
    if (prm.test && prm.rgb_test) return PPM_EINVAL;   // the count test has one statistic

    ppm_ctx* c = new (std::nothrow) ppm_ctx();
    if (!c) return PPM_ENOMEM;
    cudaGetDevice(&c->dev);
    c->stream = (cudaStream_t)stream;
    c->prm = prm;
    c->r0 = r0;
    c->alpha = alpha;
    c->r_min = prm.rmin_ratio * r0;
    c->nh = hp->n;
    c->nch = prm.channels;
    c->ntc = prm.rgb_test ? 3 : 1;
    c->normals = hp->nq != nullptr;
    const int64_t n = c->nh;
    bool ok = dalloc(&c->hp_orig, n) && dalloc(&c->hp_pos, n) && dalloc(&c->hp_u, n) &&
              dalloc(&c->hp_v, n) && dalloc(&c->r, n) && dalloc(&c->t, n) && dalloc(&c->F, n) &&
              dalloc(&c->tau, n * c->nch) && dalloc(&c->cnt, n * PPM_NG) &&
              dalloc(&c->S, n * PPM_NG * c->ntc) && dalloc(&c->Q, n * PPM_NG * c->ntc) &&
              dalloc(&c->geom_dev, 1) && dalloc(&c->rmax, 2) && dalloc(&c->counters, 8) &&
              dalloc(&c->err_dev, 1);
    if (!ok) { free_ctx(c); return PPM_ENOMEM; }
    cudaStream_t st = c->stream;
    int rc = PPM_OK;
    do {
        if (n > 0) {
            rc = ppm_prepare_hitpoints(hp, prm.vcm != 0, c->hp_orig, c->hp_pos, c->hp_u, c->hp_v, st);
            if (rc) break;
            const unsigned nb = (unsigned)((n + 255) / 256);
            k_fill_f32<<<nb, 256, 0, st>>>(n, c->r, r0);
        }
        if (cudaMemsetAsync(c->t, 0, n * sizeof(int32_t), st) != cudaSuccess ||
            cudaMemsetAsync(c->F, 0, n * sizeof(float), st) != cudaSuccess ||
            cudaMemsetAsync(c->tau, 0, n * c->nch * sizeof(double), st) != cudaSuccess ||
            cudaMemsetAsync(c->cnt, 0, n * PPM_NG * sizeof(uint32_t), st) != cudaSuccess ||
            cudaMemsetAsync(c->S, 0, n * PPM_NG * c->ntc * sizeof(float), st) != cudaSuccess ||
            cudaMemsetAsync(c->Q, 0, n * PPM_NG * c->ntc * sizeof(float), st) != cudaSuccess ||
            cudaMemsetAsync(c->counters, 0, 8 * sizeof(unsigned long long), st) != cudaSuccess ||
            cudaMemsetAsync(c->err_dev, 0, sizeof(int32_t), st) != cudaSuccess) { rc = PPM_ECUDA; break; }
        float rm[2] = {r0, 0.f};
        if (cudaMemcpyAsync(c->rmax, rm, sizeof(rm), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { rc = PPM_ECUDA; break; }
    } while (0);
    if (rc) { cudaGetLastError(); free_ctx(c); return rc; }
    *out = c;
    return PPM_OK;
}

int ppm_set_stream(ppm_ctx* c, void* stream)
{
    if (!c) return PPM_EINVAL;
    c->stream = (cudaStream_t)stream;
    return PPM_OK;
}

int ppm_build_grid(ppm_ctx* c, const ppm_photons* ph)
{
    PPM_ENTRY();
    if (!c || !ph || ph->n < 0 || ph->n > 0xfffffff0ll || ph->J < 2) return PPM_EINVAL;
    if (ph->channels != c->nch) return PPM_EINVAL;
    if (ph->n > 0 && (!ph->pos || !ph->flux)) return PPM_EINVAL;
    if (c->prm.vcm && ph->n > 0 && (!ph->rho || !ph->wq)) return PPM_EINVAL;
    if (c->J != 0 && ph->J != c->J) return PPM_EINVAL;
    c->J = ph->J;
    c->use_normals = c->normals && ph->nq != nullptr;
    c->ph_aux = c->use_normals || c->prm.vcm;
    c->grid_valid = false;
    int rc = ppm_grid_build(c, ph);
    if (rc) return rc;
    c->grid_valid = true;
    return PPM_OK;
}

int ppm_gather_test_update(ppm_ctx* c, int32_t iter)
{
    PPM_ENTRY();
    if (!c) return PPM_EINVAL;
    if (iter != c->iter + 1 || !c->grid_valid) return PPM_ESTATE;
    int launches = c->launches_build + (c->nh > 0 ? 1 : 0);
    int rc = ensure_fc(c, iter, &launches);
    if (rc) return rc;
    // Eq. (radiusupdate) lower bound r_min sqrt((i+1)^(alpha-1)) for i = iter
    const float bound = (float)((double)c->r_min * sqrt(pow((double)iter + 1.0, (double)c->alpha - 1.0)));
    PPM_CUDA(cudaMemsetAsync(c->rmax + (c->rmax_cur ^ 1), 0, sizeof(float), c->stream));
    PPM_CUDA(cudaMemsetAsync(c->counters, 0, 3 * sizeof(unsigned long long), c->stream));
    PPM_CUDA(cudaMemsetAsync(c->counters + 4, 0, sizeof(unsigned long long), c->stream));
    rc = ppm_gather_launch(c, bound);
    if (rc) return rc;
    if (c->mlp) {
        rc = ppm_mlp_propose_launch(c, bound);
        if (rc) return rc;
        ++launches;
    }
    c->iter = iter;
    c->rmax_cur ^= 1;
    c->grid_valid = false;
    c->launches_iter = launches;
    return PPM_OK;
}

int ppm_radiance(ppm_ctx* c, float* out)
{
    PPM_ENTRY();
    if (!c || (!out && c->nh > 0)) return PPM_EINVAL;
    return ppm_radiance_launch(c, out);
}

int ppm_get_state(ppm_ctx* c, const ppm_state_view* v)
{
    PPM_ENTRY();
    if (!c || !v) return PPM_EINVAL;
    if (c->nh > 0) {
        k_state_io<true><<<(unsigned)((c->nh + 255) / 256), 256, 0, c->stream>>>(
            c->nh, c->ntc, c->nch, c->hp_orig, c->r, c->t, c->F, c->tau, c->cnt, c->S, c->Q, *v);
        PPM_LAUNCH_CHECK();
    }
    PPM_CUDA(cudaStreamSynchronize(c->stream));
    int32_t err = 0;
    PPM_CUDA(cudaMemcpy(&err, c->err_dev, sizeof(err), cudaMemcpyDeviceToHost));
    return ppm_flags_status(err);
}

int ppm_set_state(ppm_ctx* c, const ppm_state_view* v)
{
    PPM_ENTRY();
    if (!c || !v) return PPM_EINVAL;
    if (c->nh > 0) {
        const unsigned nb = (unsigned)((c->nh + 255) / 256);
        k_state_io<false><<<nb, 256, 0, c->stream>>>(
            c->nh, c->ntc, c->nch, c->hp_orig, c->r, c->t, c->F, c->tau, c->cnt, c->S, c->Q, *v);
        PPM_LAUNCH_CHECK();
        // the next grid is sized for the largest radius now held
        PPM_CUDA(cudaMemsetAsync(c->rmax + c->rmax_cur, 0, sizeof(float), c->stream));
        k_rmax<<<nb, 256, 0, c->stream>>>(c->nh, c->r, c->rmax + c->rmax_cur);
        PPM_LAUNCH_CHECK();
    }
    c->grid_valid = false;
    PPM_CUDA(cudaStreamSynchronize(c->stream));
    return PPM_OK;
}

int ppm_set_iteration(ppm_ctx* c, int32_t iter)
{
    if (!c || iter < 0) return PPM_EINVAL;
    c->iter = iter;
    c->grid_valid = false;
    return PPM_OK;
}

int ppm_stats(ppm_ctx* c, ppm_iter_stats* out)
{
    PPM_ENTRY();
    if (!c || !out) return PPM_EINVAL;
    unsigned long long cnt[5];
    float rm;
    GridGeom g;
    int32_t err;
    PPM_CUDA(cudaStreamSynchronize(c->stream));
    PPM_CUDA(cudaMemcpy(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    PPM_CUDA(cudaMemcpy(&rm, c->rmax + c->rmax_cur, sizeof(float), cudaMemcpyDeviceToHost));
    PPM_CUDA(cudaMemcpy(&g, c->geom_dev, sizeof(g), cudaMemcpyDeviceToHost));
    PPM_CUDA(cudaMemcpy(&err, c->err_dev, sizeof(err), cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->iter = c->iter;
    out->flags = err;
    out->pairs = (int64_t)cnt[0];
    out->candidates = (int64_t)cnt[1];
    out->rejects = (int64_t)cnt[2];
    out->pairs_total = (int64_t)cnt[3];
    out->r_max = rm;
    out->cell = g.h;
    out->launches = c->launches_iter;
    out->gather_ms = -1.f;
    out->proposals = (int64_t)cnt[4];
    return ppm_flags_status(err);
}

}  // extern "C"

namespace {

// bytes of one slot's photon arrays for n photons, each array 256-aligned
struct HostLayout {
    size_t pos, flux, nq, rho, wq, total;
};

HostLayout host_layout(int64_t n, int nch)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    HostLayout L;
    L.pos = 0;
    L.flux = L.pos + up((size_t)n * 3 * sizeof(float));
    L.nq = L.flux + up((size_t)n * nch * sizeof(float));
    L.rho = L.nq + up((size_t)n * sizeof(uint32_t));
    L.wq = L.rho + up((size_t)n * 2 * sizeof(float));
    L.total = L.wq + up((size_t)n * sizeof(uint32_t));
    return L;
}

int host_feed_init(ppm_ctx* c)
{
    if (c->copy_st) return PPM_OK;
    PPM_CUDA(cudaStreamCreateWithFlags(&c->copy_st, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        PPM_CUDA(cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming));
        PPM_CUDA(cudaEventCreateWithFlags(&c->ev_used[k], cudaEventDisableTiming));
        PPM_CUDA(cudaEventCreateWithFlags(&c->ev_stats[k], cudaEventDisableTiming));
    }
    void* hs = nullptr;
    PPM_CUDA(cudaHostAlloc(&hs, 2 * sizeof(ppm_ctx::HostStats), cudaHostAllocDefault));
    c->hstats = static_cast<ppm_ctx::HostStats*>(hs);
    memset(c->hstats, 0, 2 * sizeof(ppm_ctx::HostStats));
    return PPM_OK;
}

}  // namespace

extern "C" {

int ppm_iterate_host(ppm_ctx* c, const ppm_photons* ph, int32_t iter)
{
    PPM_ENTRY();
    if (!c || !ph || ph->n < 0 || ph->n > 0xfffffff0ll || ph->J < 2) return PPM_EINVAL;
    if (ph->channels != c->nch) return PPM_EINVAL;
    if (ph->n > 0 && (!ph->pos || !ph->flux)) return PPM_EINVAL;
    if (c->prm.vcm && ph->n > 0 && (!ph->rho || !ph->wq)) return PPM_EINVAL;
    if (c->J != 0 && ph->J != c->J) return PPM_EINVAL;
    if (iter != c->iter + 1) return PPM_ESTATE;
    int rc = host_feed_init(c);
    if (rc) return rc;
    const int64_t n = ph->n;
    const int k = c->host_slot;
    if (n > c->hbuf_cap) {
        // grow both slots: wait until neither is in use
        PPM_CUDA(cudaStreamSynchronize(c->copy_st));
        PPM_CUDA(cudaStreamSynchronize(c->stream));
        const int64_t cap = n + n / 4 + 1024;
        const HostLayout L = host_layout(cap, c->nch);
        for (int s = 0; s < 2; ++s) {
            cudaFree(c->hbuf[s]);
            c->hbuf[s] = nullptr;
        }
        c->hbuf_cap = 0;
        for (int s = 0; s < 2; ++s)
            if (cudaMalloc(&c->hbuf[s], L.total) != cudaSuccess) { cudaGetLastError(); return PPM_ENOMEM; }
        c->hbuf_cap = cap;
    }
    const HostLayout L = host_layout(c->hbuf_cap, c->nch);
    unsigned char* base = c->hbuf[k];
    ppm_photons d = *ph;
    d.pos = reinterpret_cast<const float*>(base + L.pos);
    d.flux = reinterpret_cast<const float*>(base + L.flux);
    d.nq = ph->nq ? reinterpret_cast<const uint32_t*>(base + L.nq) : nullptr;
    d.rho = ph->rho ? reinterpret_cast<const float*>(base + L.rho) : nullptr;
    d.wq = ph->wq ? reinterpret_cast<const uint32_t*>(base + L.wq) : nullptr;
    // the slot's previous contents were read by the build two iterations ago
    PPM_CUDA(cudaStreamWaitEvent(c->copy_st, c->ev_used[k], 0));
    if (n > 0) {
        PPM_CUDA(cudaMemcpyAsync(base + L.pos, ph->pos, (size_t)n * 3 * sizeof(float),
                                 cudaMemcpyHostToDevice, c->copy_st));
        PPM_CUDA(cudaMemcpyAsync(base + L.flux, ph->flux, (size_t)n * c->nch * sizeof(float),
                                 cudaMemcpyHostToDevice, c->copy_st));
        if (ph->nq)
            PPM_CUDA(cudaMemcpyAsync(base + L.nq, ph->nq, (size_t)n * sizeof(uint32_t),
                                     cudaMemcpyHostToDevice, c->copy_st));
        if (ph->rho)
            PPM_CUDA(cudaMemcpyAsync(base + L.rho, ph->rho, (size_t)n * 2 * sizeof(float),
                                     cudaMemcpyHostToDevice, c->copy_st));
        if (ph->wq)
            PPM_CUDA(cudaMemcpyAsync(base + L.wq, ph->wq, (size_t)n * sizeof(uint32_t),
                                     cudaMemcpyHostToDevice, c->copy_st));
    }
    PPM_CUDA(cudaEventRecord(c->ev_copied[k], c->copy_st));
    PPM_CUDA(cudaStreamWaitEvent(c->stream, c->ev_copied[k], 0));
    rc = ppm_build_grid(c, &d);
    if (rc) return rc;
    PPM_CUDA(cudaEventRecord(c->ev_used[k], c->stream));
    rc = ppm_gather_test_update(c, iter);
    if (rc) return rc;
    // this iteration's counters to page-locked memory
    ppm_ctx::HostStats* hs = c->hstats + k;
    PPM_CUDA(cudaMemcpyAsync(hs->cnt, c->counters, sizeof(hs->cnt), cudaMemcpyDeviceToHost, c->stream));
    PPM_CUDA(cudaMemcpyAsync(&hs->r_max, c->rmax + c->rmax_cur, sizeof(float), cudaMemcpyDeviceToHost,
                             c->stream));
    PPM_CUDA(cudaMemcpyAsync(&hs->cell, reinterpret_cast<const char*>(c->geom_dev) + offsetof(GridGeom, h),
                             sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    PPM_CUDA(cudaMemcpyAsync(&hs->err, c->err_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    PPM_CUDA(cudaEventRecord(c->ev_stats[k], c->stream));
    c->host_iter[k] = iter;
    c->host_launches[k] = c->launches_iter;
    c->host_slot = k ^ 1;
    return PPM_OK;
}

int ppm_stats_host(ppm_ctx* c, int32_t iter, ppm_iter_stats* out)
{
    PPM_ENTRY();
    if (!c || !out) return PPM_EINVAL;
    int k = -1;
    for (int s = 0; s < 2; ++s)
        if (c->hstats && iter > 0 && c->host_iter[s] == iter) k = s;
    if (k < 0) return PPM_ESTATE;
    PPM_CUDA(cudaEventSynchronize(c->ev_stats[k]));
    const ppm_ctx::HostStats& hs = c->hstats[k];
    memset(out, 0, sizeof(*out));
    out->iter = iter;
    out->flags = hs.err;
    out->pairs = (int64_t)hs.cnt[0];
    out->candidates = (int64_t)hs.cnt[1];
    out->rejects = (int64_t)hs.cnt[2];
    out->pairs_total = (int64_t)hs.cnt[3];
    out->proposals = (int64_t)hs.cnt[4];
    out->r_max = hs.r_max;
    out->cell = hs.cell;
    out->launches = c->host_launches[k];
    out->gather_ms = -1.f;
    return ppm_flags_status(hs.err);
}

int ppm_f_critical(int64_t J, double alpha_f, int32_t t_max, double* out, void* stream)
{
    PPM_ENTRY();
    if (J < 2 || !(alpha_f > 0.0 && alpha_f < 1.0) || t_max < 1 || !out) return PPM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    PPM_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
    return ppm_fcrit_fill(out, 1, t_max, (double)J, alpha_f, st);
}

int ppm_set_hitpoints(ppm_ctx* c, const ppm_hitpoints* hp)
{
    PPM_ENTRY();
    if (!c || !hp || hp->n != c->nh) return PPM_EINVAL;
    if (c->nh == 0) return PPM_OK;
    if (!hp->pos || !hp->u || !hp->v) return PPM_EINVAL;
    if ((hp->nq != nullptr) != c->normals) return PPM_EINVAL;
    if (c->prm.vcm && !hp->rho) return PPM_EINVAL;
    // internal slot i holds caller entry hp_orig[i]: gather the new arrays
    // into the same slots
    const unsigned nb = (unsigned)((c->nh + 255) / 256);
    k_hp_permute<<<nb, 256, 0, c->stream>>>(c->nh, c->hp_orig, hp->pos, hp->u, hp->v, hp->nq,
                                           c->prm.vcm ? hp->rho : nullptr, nullptr, c->hp_pos, c->hp_u,
                                           c->hp_v);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_chi2_critical(int32_t dof, double alpha, double* out, void* stream)
{
    PPM_ENTRY();
    if (dof < 1 || dof > 1000 || !(alpha > 0.0 && alpha < 1.0) || !out) return PPM_EINVAL;
    return ppm_chi2_fill(out, 0, 0, (double)dof, alpha, (cudaStream_t)stream);
}

int ppm_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                   uint32_t* vals_out, int64_t n, int32_t bits, void* stream)
{
    PPM_ENTRY();
    if (n < 0 || n >= 0xffffffffll || bits < 1 || bits > 32) return PPM_EINVAL;
    if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out)) return PPM_EINVAL;
    if (n == 0) return PPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (keys_out != keys_in)
        PPM_CUDA(cudaMemcpyAsync(keys_out, keys_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    if (vals_out != vals_in)
        PPM_CUDA(cudaMemcpyAsync(vals_out, vals_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    if (n == 1) return PPM_OK;
    // scratch: alternate keys and values, the look-back words, the digit
    // counts and an error word (the single-pass form of the grid's sort)
    const int64_t ntiles = (n + 2047) / 2048;
    const int64_t status_words = 32 + 256 * ntiles;
    const size_t off_status = ((size_t)2 * n * sizeof(uint32_t) + 255) & ~(size_t)255;
    const size_t off_digit = off_status + (size_t)status_words * sizeof(unsigned long long);
    const size_t off_err = off_digit + 4 * 256 * sizeof(uint32_t);
    const size_t bytes = off_err + 256;
    unsigned char* scratch = nullptr;
    if (cudaMallocAsync((void**)&scratch, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return PPM_ENOMEM;
    }
    SortScratch s;
    s.keys = keys_out;
    s.vals = vals_out;
    s.keys_alt = reinterpret_cast<uint32_t*>(scratch);
    s.vals_alt = reinterpret_cast<uint32_t*>(scratch) + n;
    s.status = reinterpret_cast<unsigned long long*>(scratch + off_status);
    s.digit = reinterpret_cast<uint32_t*>(scratch + off_digit);
    s.cap = n;
    s.status_cap = status_words;
    int32_t* err = reinterpret_cast<int32_t*>(scratch + off_err);
    int rc = PPM_OK;
    if (cudaMemsetAsync(err, 0, sizeof(int32_t), st) != cudaSuccess) { cudaGetLastError(); rc = PPM_ECUDA; }
    if (rc == PPM_OK) rc = ppm_radix_sort_pairs_lookback(&s, n, bits, err, st);
    if (rc == PPM_OK && s.keys != keys_out) {   // odd number of passes
        if (cudaMemcpyAsync(keys_out, s.keys, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(vals_out, s.vals, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = PPM_ECUDA;
    }
    if (cudaFreeAsync(scratch, st) != cudaSuccess && rc == PPM_OK) rc = PPM_ECUDA;
    return rc;
}

void ppm_destroy(ppm_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

}  // extern "C"
