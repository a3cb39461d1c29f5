// ppm_gather.cu -- per-hit-point gather, ANOVA F-test and update (Sec. 5.1
// steps 2-4), one thread per hit point, hit points in spatial order so that
// a warp's hit points scan the same cells (their photons come from L1).
//
// Per hit point h with radius r (this iteration's r_i):
//   * visit the grid cells overlapping the sphere's bounding box, a run of
//     cells along x inside one block being one contiguous photon range;
//   * per photon p: closed-disk test d2 <= r^2 with dx = x_h - x_p, then the
//     same-surface test (snorm8 normal dot > 8064), then the map of Eq.
//     (map-function) y = (<x_h - x_p, u>, <x_h - x_p, v>), the equi-areal
//     annulus (2 |y|^2 < r^2 -> inner) and the 60-degree sector by exact
//     sign logic against sqrt(3); group = annulus * 6 + sector.  These
//     decisions use one fixed FP32 operation sequence (explicit fma / _rn
//     intrinsics, no contraction) so that they are reproducible bit for bit;
//   * per group: count, sum psi, sum psi^2 in shared memory, laid out
//     [slot][thread] so every access of a warp hits 32 distinct banks;
//   * epilogue: add the iteration's sums to the window sums, F of Eq.
//     (f-statistic) with m = t' J samples per group, compare with F_c(t')
//     (FP64 table), tau += Phi_i / (pi r_i^2) in FP64, and on rejection
//     Eq. (radiusupdate) with the window cleared (Sec. 5.1).
//   * VCM+: every pair's psi and flux carry the balance-heuristic merge
//     weight w = 1 / (1 + R_VM + R_VC / (n_VM pi r^2)) of Eq. (mis-weight).
#include "ppm_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kNormalDotMin = 8064;   // 127^2 / 2: cosine > ~0.5

struct GatherArgs {
    int64_t nh;
    const float4* hp_pos;
    const float4* hp_u;
    const float4* hp_v;
    float* r;
    int32_t* t;
    float* F;
    double* tau;
    uint32_t* cnt;
    float* S;
    float* Q;
    const uint32_t* cell_start;
    const float4* rec0;
    const float4* rec1;
    const uint4* aux;
    const GridGeom* geom;
    const double* fc;
    float* rmax_next;
    unsigned long long* counters;
    float J;
    float k;
    float bound;
    float n_vm;
    int32_t fc_max;     // last valid index of fc
    int32_t* err;
};

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// group of an in-disk pair (annulus * 6 + sector)
__device__ __forceinline__ int pair_group(float yu, float yv, float r2)
{
    const float rho2 = fmaf(yv, yv, __fmul_rn(yu, yu));
    const int ring = (__fadd_rn(rho2, rho2) < r2) ? 0 : 6;
    const float tx = __fmul_rn(1.7320508f, fabsf(yu));
    const bool up = (yv > 0.f) || (yv == 0.f && yu >= 0.f);
    int sector;
    if (fabsf(yv) >= tx) sector = up ? 1 : 4;
    else sector = up ? (yu > 0.f ? 0 : 2) : (yu < 0.f ? 3 : 5);
    return ring + sector;
}

template <int NCH, int NTC, bool NORMALS, bool VCM>
__global__ void __launch_bounds__(kThreads)
k_gather_update(GatherArgs a)
{
    __shared__ uint32_t s_c[PPM_NG][kThreads];
    __shared__ float s_S[NTC][PPM_NG][kThreads];
    __shared__ float s_Q[NTC][PPM_NG][kThreads];
    const int tid = threadIdx.x;
    const int64_t h = (int64_t)blockIdx.x * kThreads + tid;
    const bool live = h < a.nh;

#pragma unroll
    for (int g = 0; g < PPM_NG; ++g) {
        s_c[g][tid] = 0u;
#pragma unroll
        for (int c = 0; c < NTC; ++c) { s_S[c][g][tid] = 0.f; s_Q[c][g][tid] = 0.f; }
    }

    float r = 0.f;
    float phi[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) phi[c] = 0.f;
    unsigned long long cand = 0, pairs = 0;

    if (live) {
        const float4 P = a.hp_pos[h];
        const float4 U = a.hp_u[h];
        const float4 V = a.hp_v[h];
        r = a.r[h];
        const float r2 = __fmul_rn(r, r);
        const GridGeom G = *a.geom;
        const uint32_t nqh = __float_as_uint(P.w);
        // VCM+ constants of this hit point: w = 1 / (1 + R_VM + R_VC / eta)
        float inv_eta = 0.f;
        if (VCM) inv_eta = __frcp_rn(__fmul_rn(__fmul_rn(a.n_vm, 3.14159265358979f), r2));
        // cull radius: every photon whose FP32 disk test passes lies inside
        // [x - rc, x + rc] per axis (rounding of dx and of d2 included)
        const float rc = fmaf(r, 1.0009765625f,
                              (fabsf(P.x) + fabsf(P.y) + fabsf(P.z) + r) * 1.0e-6f);
        const int ix0 = ppm_cell_coord(__fsub_rn(P.x, rc), G.inv_h);
        int ix1 = ppm_cell_coord(__fadd_rn(P.x, rc), G.inv_h);
        const int iy0 = ppm_cell_coord(__fsub_rn(P.y, rc), G.inv_h);
        int iy1 = ppm_cell_coord(__fadd_rn(P.y, rc), G.inv_h);
        const int iz0 = ppm_cell_coord(__fsub_rn(P.z, rc), G.inv_h);
        int iz1 = ppm_cell_coord(__fadd_rn(P.z, rc), G.inv_h);
        const int B = 1 << G.lb;
        if (ix1 - ix0 >= B || iy1 - iy0 >= B || iz1 - iz0 >= B) {
            // the sphere spans more cells than a block: distinct cells could
            // share a bucket; never happens for r <= max radius and sane
            // coordinates -- flag it instead of double counting
            atomicOr(a.err, 1);
            ix1 = min(ix1, ix0 + B - 1); iy1 = min(iy1, iy0 + B - 1); iz1 = min(iz1, iz0 + B - 1);
        }
        for (int iz = iz0; iz <= iz1; ++iz) {
            for (int iy = iy0; iy <= iy1; ++iy) {
                int ix = ix0;
                while (ix <= ix1) {
                    const int ixe = min(ix1, ix | (B - 1));          // end of this block's run
                    const uint32_t b0 = ppm_bucket(ix, iy, iz, G);
                    const uint32_t s = __ldg(a.cell_start + b0);
                    const uint32_t e = __ldg(a.cell_start + b0 + (uint32_t)(ixe - ix) + 1u);
                    cand += e - s;
                    for (uint32_t p = s; p < e; ++p) {
                        const float4 X = __ldg(a.rec0 + p);
                        const float dx = __fsub_rn(P.x, X.x);
                        const float dy = __fsub_rn(P.y, X.y);
                        const float dz = __fsub_rn(P.z, X.z);
                        const float d2 = fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
                        if (!(d2 <= r2)) continue;
                        uint4 A = make_uint4(0u, 0u, 0u, 0u);
                        if constexpr (NORMALS || VCM) A = __ldg(a.aux + p);
                        if constexpr (NORMALS) {
                            if (__dp4a((int)A.x, (int)nqh, 0) <= kNormalDotMin) continue;
                        }
                        const float yu = fmaf(dz, U.z, fmaf(dy, U.y, __fmul_rn(dx, U.x)));
                        const float yv = fmaf(dz, V.z, fmaf(dy, V.y, __fmul_rn(dx, V.x)));
                        const int g = pair_group(yu, yv, r2);
                        float w = 1.f;
                        float4 X1 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if constexpr (NCH == 3 || VCM) X1 = __ldg(a.rec1 + p);
                        if constexpr (VCM) {
                            const int cd = __dp4a((int)A.y, (int)nqh, 0);
                            const float cosl = cd > 0 ? __fmul_rn((float)cd, 1.0f / 16129.0f) : 0.f;
                            const float r_vm = fmaf(U.w, __fmul_rn(cosl, 0.318309886f), X1.w);
                            const float r_vc = __fadd_rn(V.w, __uint_as_float(A.z));
                            w = __frcp_rn(1.f + r_vm + r_vc * inv_eta);
                        }
                        ++pairs;
                        s_c[g][tid] += 1u;
                        if constexpr (NTC == 1) {
                            const float psi = VCM ? __fmul_rn(w, X.w) : X.w;
                            s_S[0][g][tid] += psi;
                            s_Q[0][g][tid] = fmaf(psi, psi, s_Q[0][g][tid]);
                        } else {
                            const float pr = __fmul_rn(w, X1.x), pg = __fmul_rn(w, X1.y), pb = __fmul_rn(w, X1.z);
                            s_S[0][g][tid] += pr; s_Q[0][g][tid] = fmaf(pr, pr, s_Q[0][g][tid]);
                            s_S[NTC - 2][g][tid] += pg; s_Q[NTC - 2][g][tid] = fmaf(pg, pg, s_Q[NTC - 2][g][tid]);
                            s_S[NTC - 1][g][tid] += pb; s_Q[NTC - 1][g][tid] = fmaf(pb, pb, s_Q[NTC - 1][g][tid]);
                        }
                        if constexpr (NCH == 3) {
                            phi[0] = fmaf(w, X1.x, phi[0]);
                            phi[NCH - 2] = fmaf(w, X1.y, phi[NCH - 2]);
                            phi[NCH - 1] = fmaf(w, X1.z, phi[NCH - 1]);
                        } else {
                            phi[0] = fmaf(w, VCM ? X1.x : X.w, phi[0]);
                        }
                    }
                    ix = ixe + 1;
                }
            }
        }
    }

    // ---------------- epilogue: F-test, estimate, radius update ----------
    float r_new = 0.f;
    unsigned long long rej = 0;
    if (live) {
        const int32_t tp = a.t[h] + 1;
        // a window longer than the table can only come from ppm_set_state
        // with t >= the iteration count: clamp the lookup and flag it
        int32_t tpi = tp;
        if (tp < 1 || tp > a.fc_max) { atomicOr(a.err, 2); tpi = max(1, min(tp, a.fc_max)); }
        const float m = __fmul_rn((float)tp, a.J);
        const int64_t nh = a.nh;
        bool reject = false;
        float F0 = 0.f;
        float Sg[PPM_NG];
#pragma unroll
        for (int c = 0; c < NTC; ++c) {
            float Ssum = 0.f, Qsum = 0.f, S2 = 0.f;
#pragma unroll
            for (int g = 0; g < PPM_NG; ++g) {
                const int64_t o = ((int64_t)c * PPM_NG + g) * nh + h;
                Sg[g] = a.S[o] + s_S[c][g][tid];
                Qsum += a.Q[o] + s_Q[c][g][tid];
                Ssum += Sg[g];
                S2 = fmaf(Sg[g], Sg[g], S2);
            }
            const float Sbar = Ssum * (1.0f / PPM_NG);
            float dev2 = 0.f;
#pragma unroll
            for (int g = 0; g < PPM_NG; ++g) { const float d = Sg[g] - Sbar; dev2 = fmaf(d, d, dev2); }
            // SSB = dev2 / m, SSW = sum Q - sum S^2 / m,
            // F = (SSB / 11) / (SSW / (12 (m-1))) = (dev2 / SSW) * 12 (m-1) / (11 m)
            const float ssw = Qsum - S2 / m;
            float F = 0.f;
            if (ssw > 0.f) F = (dev2 / ssw) * (((float)PPM_NG * (m - 1.0f)) / ((float)(PPM_NG - 1) * m));
            if (c == 0) F0 = F;
            if (ssw > 0.f && (double)F > a.fc[tpi]) reject = true;
        }
        // Eq. (progressive-VCM-estimator): kernel estimate with this r_i
        const float inv_area = __frcp_rn(__fmul_rn(3.14159265358979f, __fmul_rn(r, r)));
#pragma unroll
        for (int c = 0; c < NCH; ++c) a.tau[h * NCH + c] += (double)__fmul_rn(phi[c], inv_area);
        a.F[h] = F0;
        if (reject) {
            r_new = fmaxf(__fmul_rn(a.k, r), a.bound);
            a.r[h] = r_new;
            a.t[h] = 0;
#pragma unroll
            for (int g = 0; g < PPM_NG; ++g) a.cnt[g * nh + h] = 0u;
#pragma unroll
            for (int c = 0; c < NTC; ++c)
#pragma unroll
                for (int g = 0; g < PPM_NG; ++g) {
                    const int64_t o = ((int64_t)c * PPM_NG + g) * nh + h;
                    a.S[o] = 0.f;
                    a.Q[o] = 0.f;
                }
            rej = 1;
        } else {
            r_new = r;
            a.t[h] = tp;
#pragma unroll
            for (int g = 0; g < PPM_NG; ++g) a.cnt[g * nh + h] += s_c[g][tid];
#pragma unroll
            for (int c = 0; c < NTC; ++c)
#pragma unroll
                for (int g = 0; g < PPM_NG; ++g) {
                    const int64_t o = ((int64_t)c * PPM_NG + g) * nh + h;
                    a.S[o] += s_S[c][g][tid];
                    a.Q[o] += s_Q[c][g][tid];
                }
        }
    }

    // block reductions: max radius for the next grid, counters
    __shared__ float s_rmax[kThreads / 32];
    __shared__ unsigned long long s_cnt3[3][kThreads / 32];
    const float wm = warp_max(r_new);
    const unsigned long long wp = warp_sum_u64(pairs), wc = warp_sum_u64(cand), wr = warp_sum_u64(rej);
    if ((tid & 31) == 0) {
        s_rmax[tid >> 5] = wm;
        s_cnt3[0][tid >> 5] = wp; s_cnt3[1][tid >> 5] = wc; s_cnt3[2][tid >> 5] = wr;
    }
    __syncthreads();
    if (tid == 0) {
        float m = 0.f;
        unsigned long long p = 0, c = 0, j = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            m = fmaxf(m, s_rmax[w]); p += s_cnt3[0][w]; c += s_cnt3[1][w]; j += s_cnt3[2][w];
        }
        atomicMax((int*)a.rmax_next, __float_as_int(m));
        atomicAdd(a.counters + 0, p);
        atomicAdd(a.counters + 1, c);
        atomicAdd(a.counters + 2, j);
        atomicAdd(a.counters + 3, p);
    }
}

__global__ void k_radiance(int64_t nh, int nch, const double* __restrict__ tau,
                           const uint32_t* __restrict__ orig, double inv_iter,
                           float* __restrict__ out)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    const int64_t o = orig[h];
    for (int c = 0; c < nch; ++c) out[o * nch + c] = (float)(tau[h * nch + c] * inv_iter);
}

template <int NCH, int NTC, bool NORMALS, bool VCM>
int launch_gather(ppm_ctx* c, const GatherArgs& a)
{
    const unsigned nb = (unsigned)((c->nh + kThreads - 1) / kThreads);
    k_gather_update<NCH, NTC, NORMALS, VCM><<<nb, kThreads, 0, c->stream>>>(a);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

}  // namespace

int ppm_gather_launch(ppm_ctx* c, float bound)
{
    if (c->nh == 0) return PPM_OK;
    GatherArgs a;
    a.nh = c->nh;
    a.hp_pos = c->hp_pos; a.hp_u = c->hp_u; a.hp_v = c->hp_v;
    a.r = c->r; a.t = c->t; a.F = c->F; a.tau = c->tau;
    a.cnt = c->cnt; a.S = c->S; a.Q = c->Q;
    a.cell_start = c->cell_start;
    a.rec0 = c->rec0; a.rec1 = c->rec1; a.aux = c->aux;
    a.geom = c->geom_dev;
    a.fc = c->fc;
    a.rmax_next = c->rmax + (c->rmax_cur ^ 1);
    a.counters = c->counters;
    a.J = (float)c->J;
    a.k = c->prm.k;
    a.bound = bound;
    a.n_vm = c->prm.n_vm > 0.f ? c->prm.n_vm : (float)c->J;
    a.fc_max = c->fc_upto;
    a.err = c->err_dev;
    const bool nrm = c->use_normals;
    const bool vcm = c->prm.vcm != 0;
    if (c->nch == 1) {
        if (vcm) return nrm ? launch_gather<1, 1, true, true>(c, a) : launch_gather<1, 1, false, true>(c, a);
        return nrm ? launch_gather<1, 1, true, false>(c, a) : launch_gather<1, 1, false, false>(c, a);
    }
    if (c->ntc == 3) {
        if (vcm) return nrm ? launch_gather<3, 3, true, true>(c, a) : launch_gather<3, 3, false, true>(c, a);
        return nrm ? launch_gather<3, 3, true, false>(c, a) : launch_gather<3, 3, false, false>(c, a);
    }
    if (vcm) return nrm ? launch_gather<3, 1, true, true>(c, a) : launch_gather<3, 1, false, true>(c, a);
    return nrm ? launch_gather<3, 1, true, false>(c, a) : launch_gather<3, 1, false, false>(c, a);
}

int ppm_radiance_launch(ppm_ctx* c, float* out)
{
    if (c->nh == 0) return PPM_OK;
    const double inv = c->iter > 0 ? 1.0 / c->iter : 0.0;
    k_radiance<<<(unsigned)((c->nh + 255) / 256), 256, 0, c->stream>>>(c->nh, c->nch, c->tau, c->hp_orig, inv, out);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}
