// ppm_gather.cu -- per-hit-point gather, ANOVA F-test and update (Sec. 5.1
// steps 2-4), hit points in spatial (Morton) order, 128 threads per block,
// one thread per hit point.
//
// Per hit point h with radius r (this iteration's r_i):
//   * the photons of the grid cells overlapping the sphere's bounding box
//     are candidates; per candidate: closed-disk test d2 <= r^2 with
//     dx = x_h - x_p, then the same-surface test (snorm8 normal dot > 8064),
//     then the map of Eq. (map-function) y = (<x_h - x_p, u>, <x_h - x_p, v>),
//     the equi-areal annulus (2 |y|^2 < r^2 -> inner) and the 60-degree
//     sector by exact sign logic against sqrt(3); group = annulus * 6 +
//     sector.  These decisions use one fixed FP32 operation sequence
//     (explicit fma / _rn intrinsics, no contraction): reproducible bit for
//     bit on any device and by the CPU oracle;
//   * per group: count and (sum psi, sum psi^2) in shared memory, laid
//     out [slot][thread] so a warp's accesses hit distinct banks; the
//     iteration's flux Phi_i and pair count are the sums over groups
//     (no per-pair flux accumulator unless RGB flux is tested on luminance);
//   * epilogue: window sums += this iteration's sums, F of Eq.
//     (f-statistic) with m = t' J samples per group, compared with F_c(t')
//     (FP64 table); tau += Phi_i / (pi r_i^2) in FP64; on rejection Eq.
//     (radiusupdate) and the window is cleared (Sec. 5.1);
//   * VCM+: every pair's psi and flux carry the balance-heuristic merge
//     weight w = 1 / (1 + R_VM + R_VC / (n_VM pi r^2)) of Eq. (mis-weight).
//
// Traversals (ppm_params.mapping):
//   0  thread-owned: each thread walks the cells of its own sphere;
//   1, 2  warp-union (queues of 32 / 64 entries per lane): the warp walks
//      the union of its 32 spheres' cells
//      (skipping rows no lane needs), loads 32 photons at a time into shared
//      memory with one coalesced load and every lane tests each one
//      (broadcast reads, no divergence in the test loop); in-disk hits are
//      queued per lane and processed in lockstep when a queue fills, so the
//      long in-disk path runs with most lanes active.  Warps whose union is
//      wider than a hash block fall back to traversal 0.
#include "ppm_internal.cuh"

#include <limits.h>

#include <type_traits>

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
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

template <int NTC>
struct Smem {
    uint32_t c[PPM_NG][kThreads];
    float2 SQ[NTC][PPM_NG][kThreads];   // (sum psi, sum psi^2)
};

template <int QCAP>
struct UnionSmem {
    float4 chunk[kWarps][32];
    uint32_t queue[kWarps][QCAP][32];   // per-lane in-disk queues
};

// this thread's hit point
struct Hit {
    float4 P, U, V;
    float r, r2, inv_eta;
    uint32_t nqh;
};

// RGB flux of this hit point when only its luminance is tested:
// Kahan-compensated FP32 sums (a disk can hold thousands of photons; plain
// FP32 summation would drift past 1e-5).  Otherwise Phi_i is the sum of the
// tested group sums.
template <int NCH>
struct Acc {
    float phi[NCH];
    float comp[NCH];
    unsigned long long cand = 0;
    __device__ __forceinline__ void add(int c, float v)
    {
        const float y = __fsub_rn(v, comp[c]);
        const float t = __fadd_rn(phi[c], y);
        comp[c] = __fsub_rn(__fsub_rn(t, phi[c]), y);
        phi[c] = t;
    }
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

// disk test; returns the offsets hit point minus photon
__device__ __forceinline__ bool in_disk(const Hit& H, const float4& X, float& dx, float& dy, float& dz)
{
    dx = __fsub_rn(H.P.x, X.x);
    dy = __fsub_rn(H.P.y, X.y);
    dz = __fsub_rn(H.P.z, X.z);
    const float d2 = fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
    return d2 <= H.r2;
}

// everything after the disk test for photon p (record X)
template <int NCH, int NTC, bool NORMALS, bool VCM>
__device__ __forceinline__ void gather_pair(const GatherArgs& a, const Hit& H, Smem<NTC>& sm, int tid,
                                            Acc<NCH>& acc, uint32_t p, const float4& X,
                                            float dx, float dy, float dz)
{
    uint4 A = make_uint4(0u, 0u, 0u, 0u);
    if constexpr (NORMALS || VCM) A = __ldg(a.aux + p);
    if constexpr (NORMALS) {
        if (__dp4a((int)A.x, (int)H.nqh, 0) <= kNormalDotMin) return;
    }
    const float yu = fmaf(dz, H.U.z, fmaf(dy, H.U.y, __fmul_rn(dx, H.U.x)));
    const float yv = fmaf(dz, H.V.z, fmaf(dy, H.V.y, __fmul_rn(dx, H.V.x)));
    const int g = pair_group(yu, yv, H.r2);
    float w = 1.f;
    float4 X1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (NCH == 3 || VCM) X1 = __ldg(a.rec1 + p);
    if constexpr (VCM) {
        const int cd = __dp4a((int)A.y, (int)H.nqh, 0);
        const float cosl = cd > 0 ? __fmul_rn((float)cd, 1.0f / 16129.0f) : 0.f;
        const float r_vm = fmaf(H.U.w, __fmul_rn(cosl, 0.318309886f), X1.w);
        const float r_vc = __fadd_rn(H.V.w, __uint_as_float(A.z));
        w = __frcp_rn(1.f + r_vm + r_vc * H.inv_eta);
    }
    sm.c[g][tid] += 1u;
    if constexpr (NTC == 1) {
        const float psi = VCM ? __fmul_rn(w, X.w) : X.w;
        float2 v = sm.SQ[0][g][tid];
        v.x += psi;
        v.y = fmaf(psi, psi, v.y);
        sm.SQ[0][g][tid] = v;
    } else {
        const float pc[3] = {__fmul_rn(w, X1.x), __fmul_rn(w, X1.y), __fmul_rn(w, X1.z)};
#pragma unroll
        for (int c = 0; c < NTC; ++c) {
            float2 v = sm.SQ[c][g][tid];
            v.x += pc[c];
            v.y = fmaf(pc[c], pc[c], v.y);
            sm.SQ[c][g][tid] = v;
        }
    }
    if constexpr (NCH == 3 && NTC == 1) {
        acc.add(0, VCM ? __fmul_rn(w, X1.x) : X1.x);
        acc.add(1, VCM ? __fmul_rn(w, X1.y) : X1.y);
        acc.add(2, VCM ? __fmul_rn(w, X1.z) : X1.z);
    }
}

struct CellBox { int ix0, ix1, iy0, iy1, iz0, iz1; };

// cells that can hold a photon passing this hit point's FP32 disk test:
// the cull radius covers the rounding of dx and of d2
__device__ __forceinline__ CellBox cell_box(const Hit& H, const GridGeom& G)
{
    const float rc = fmaf(H.r, 1.0009765625f,
                          (fabsf(H.P.x) + fabsf(H.P.y) + fabsf(H.P.z) + H.r) * 1.0e-6f);
    CellBox b;
    b.ix0 = ppm_cell_coord(__fsub_rn(H.P.x, rc), G.inv_h);
    b.ix1 = ppm_cell_coord(__fadd_rn(H.P.x, rc), G.inv_h);
    b.iy0 = ppm_cell_coord(__fsub_rn(H.P.y, rc), G.inv_h);
    b.iy1 = ppm_cell_coord(__fadd_rn(H.P.y, rc), G.inv_h);
    b.iz0 = ppm_cell_coord(__fsub_rn(H.P.z, rc), G.inv_h);
    b.iz1 = ppm_cell_coord(__fadd_rn(H.P.z, rc), G.inv_h);
    return b;
}

// traversal 0: the thread walks its own cells
template <int NCH, int NTC, bool NORMALS, bool VCM>
__device__ void gather_own(const GatherArgs& a, const Hit& H, const GridGeom& G, CellBox b,
                           Smem<NTC>& sm, int tid, Acc<NCH>& acc)
{
    const int B = 1 << G.lb;
    if (b.ix1 - b.ix0 >= B || b.iy1 - b.iy0 >= B || b.iz1 - b.iz0 >= B) {
        // the sphere spans more cells than a block: distinct cells could
        // share a bucket; never happens for r <= max radius and sane
        // coordinates -- flag it instead of double counting
        atomicOr(a.err, 1);
        b.ix1 = min(b.ix1, b.ix0 + B - 1); b.iy1 = min(b.iy1, b.iy0 + B - 1); b.iz1 = min(b.iz1, b.iz0 + B - 1);
    }
    for (int iz = b.iz0; iz <= b.iz1; ++iz) {
        for (int iy = b.iy0; iy <= b.iy1; ++iy) {
            int ix = b.ix0;
            while (ix <= b.ix1) {
                const int ixe = min(b.ix1, ix | (B - 1));          // end of this block's run
                const uint32_t b0 = ppm_bucket(ix, iy, iz, G);
                const uint32_t s = __ldg(a.cell_start + b0);
                const uint32_t e = __ldg(a.cell_start + b0 + (uint32_t)(ixe - ix) + 1u);
                acc.cand += e - s;
                // software pipeline: the next record is in flight while the
                // current one is classified
                float4 Xn = s < e ? __ldg(a.rec0 + s) : make_float4(0.f, 0.f, 0.f, 0.f);
                for (uint32_t p = s; p < e; ++p) {
                    const float4 X = Xn;
                    if (p + 1u < e) Xn = __ldg(a.rec0 + p + 1u);
                    float dx, dy, dz;
                    if (in_disk(H, X, dx, dy, dz))
                        gather_pair<NCH, NTC, NORMALS, VCM>(a, H, sm, tid, acc, p, X, dx, dy, dz);
                }
                ix = ixe + 1;
            }
        }
    }
}

// traversal 1, drain: each lane processes its queued in-disk photons in
// queue (= traversal) order; the warp loops to the longest queue
template <int NCH, int NTC, bool NORMALS, bool VCM, typename US>
__device__ __forceinline__ void drain_queue(const GatherArgs& a, const Hit& H, Smem<NTC>& sm,
                                            US& us, int w, int lane, int tid,
                                            Acc<NCH>& acc, int& qlen)
{
    const int qmax = __reduce_max_sync(0xffffffffu, qlen);
    for (int q = 0; q < qmax; ++q) {
        if (q < qlen) {
            const uint32_t p = us.queue[w][q][lane];
            const float4 X = __ldg(a.rec0 + p);
            float dx, dy, dz;
            in_disk(H, X, dx, dy, dz);
            gather_pair<NCH, NTC, NORMALS, VCM>(a, H, sm, tid, acc, p, X, dx, dy, dz);
        }
    }
    qlen = 0;
    __syncwarp();
}

template <int NCH, int NTC, bool NORMALS, bool VCM, int MAPPING>
__global__ void __launch_bounds__(kThreads, MAPPING == 0 ? 8 : (MAPPING == 1 ? 6 : 4))
k_gather_update(GatherArgs a)
{
    constexpr int kQueue = MAPPING == 2 ? 64 : 32;
    using US = UnionSmem<kQueue>;
    __shared__ Smem<NTC> sm;
    __shared__ typename std::conditional<MAPPING != 0, US, int>::type us_raw;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t h = (int64_t)blockIdx.x * kThreads + tid;
    const bool live = h < a.nh;

#pragma unroll
    for (int g = 0; g < PPM_NG; ++g) {
        sm.c[g][tid] = 0u;
#pragma unroll
        for (int c = 0; c < NTC; ++c) sm.SQ[c][g][tid] = make_float2(0.f, 0.f);
    }

    Acc<NCH> acc;
#pragma unroll
    for (int c = 0; c < NCH; ++c) { acc.phi[c] = 0.f; acc.comp[c] = 0.f; }
    Hit H;
    H.r = 0.f; H.r2 = 0.f;
    const GridGeom G = *a.geom;
    CellBox b{INT_MAX, INT_MIN, INT_MAX, INT_MIN, INT_MAX, INT_MIN};
    if (live) {
        H.P = a.hp_pos[h];
        H.U = a.hp_u[h];
        H.V = a.hp_v[h];
        H.r = a.r[h];
        H.r2 = __fmul_rn(H.r, H.r);
        H.nqh = __float_as_uint(H.P.w);
        H.inv_eta = 0.f;
        if constexpr (VCM) H.inv_eta = __frcp_rn(__fmul_rn(__fmul_rn(a.n_vm, 3.14159265358979f), H.r2));
        b = cell_box(H, G);
    } else {
        H.P = make_float4(0.f, 0.f, 0.f, 0.f);
        H.U = H.V = H.P;
        H.nqh = 0u;
        H.inv_eta = 0.f;
        H.r2 = -1.f;                      // no photon passes d2 <= -1
    }

    if constexpr (MAPPING == 0) {
        if (live) gather_own<NCH, NTC, NORMALS, VCM>(a, H, G, b, sm, tid, acc);
    } else {
        US& us = *reinterpret_cast<US*>(&us_raw);
        const unsigned full = 0xffffffffu;
        const int X0 = __reduce_min_sync(full, b.ix0), X1 = __reduce_max_sync(full, b.ix1);
        const int Y0 = __reduce_min_sync(full, b.iy0), Y1 = __reduce_max_sync(full, b.iy1);
        const int Z0 = __reduce_min_sync(full, b.iz0), Z1 = __reduce_max_sync(full, b.iz1);
        const int B = 1 << G.lb;
        const bool any_live = __any_sync(full, live);
        if (any_live && (X1 - X0 >= B || Y1 - Y0 >= B || Z1 - Z0 >= B)) {
            // union wider than a hash block: walk per lane instead
            if (live) gather_own<NCH, NTC, NORMALS, VCM>(a, H, G, b, sm, tid, acc);
        } else if (any_live) {
            int qlen = 0;
            for (int iz = Z0; iz <= Z1; ++iz) {
                for (int iy = Y0; iy <= Y1; ++iy) {
                    const bool need = live && b.iy0 <= iy && iy <= b.iy1 && b.iz0 <= iz && iz <= b.iz1;
                    if (!__any_sync(full, need)) continue;
                    const int rx0 = __reduce_min_sync(full, need ? b.ix0 : INT_MAX);
                    const int rx1 = __reduce_max_sync(full, need ? b.ix1 : INT_MIN);
                    int ix = rx0;
                    while (ix <= rx1) {
                        const int ixe = min(rx1, ix | (B - 1));
                        const uint32_t b0 = ppm_bucket(ix, iy, iz, G);
                        const uint32_t s = __ldg(a.cell_start + b0);
                        const uint32_t e = __ldg(a.cell_start + b0 + (uint32_t)(ixe - ix) + 1u);
                        if (need) acc.cand += e - s;
                        for (uint32_t base = s; base < e; base += 32u) {
                            const int n = (int)min(32u, e - base);
                            if (lane < n) us.chunk[w][lane] = __ldg(a.rec0 + base + lane);
                            __syncwarp();
                            // test the chunk 8 photons at a time; drain the
                            // queues whenever one could overflow
                            for (int j0 = 0; j0 < n; j0 += 8) {
#pragma unroll
                                for (int jj = 0; jj < 8; ++jj) {
                                    const int j = j0 + jj;
                                    if (j < n) {
                                        const float4 X = us.chunk[w][j];
                                        float dx, dy, dz;
                                        if (in_disk(H, X, dx, dy, dz)) {
                                            us.queue[w][qlen][lane] = base + (uint32_t)j;
                                            ++qlen;
                                        }
                                    }
                                }
                                if (__any_sync(full, qlen > kQueue - 8))
                                    drain_queue<NCH, NTC, NORMALS, VCM>(a, H, sm, us, w, lane, tid, acc, qlen);
                            }
                            __syncwarp();
                        }
                        ix = ixe + 1;
                    }
                }
            }
            drain_queue<NCH, NTC, NORMALS, VCM>(a, H, sm, us, w, lane, tid, acc, qlen);
        }
    }

    // ---------------- epilogue: F-test, estimate, radius update ----------
    float r_new = 0.f;
    unsigned long long rej = 0, pairs = 0;
    if (live) {
        const float r = H.r;
        const int32_t tp = a.t[h] + 1;
        // a window longer than the table can only come from ppm_set_state
        // with t >= the iteration count: clamp the lookup and flag it
        int32_t tpi = tp;
        if (tp < 1 || tp > a.fc_max) { atomicOr(a.err, 2); tpi = max(1, min(tp, a.fc_max)); }
        const float m = __fmul_rn((float)tp, a.J);
        const int64_t nh = a.nh;
        bool reject = false;
        float F0 = 0.f;
#pragma unroll
        for (int c = 0; c < NTC; ++c) {
            float Sg[PPM_NG];
            float Ssum = 0.f, Qsum = 0.f, S2 = 0.f;
#pragma unroll
            for (int g = 0; g < PPM_NG; ++g) {
                const int64_t o = ((int64_t)c * PPM_NG + g) * nh + h;
                const float2 v = sm.SQ[c][g][tid];
                Sg[g] = a.S[o] + v.x;
                Qsum += a.Q[o] + v.y;
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
        // Eq. (progressive-VCM-estimator): kernel estimate with this r_i;
        // Phi_i = sum over groups of this iteration's psi sums unless RGB
        // flux is tested on its luminance
        if constexpr (!(NCH == 3 && NTC == 1)) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                float f = 0.f;
#pragma unroll
                for (int g = 0; g < PPM_NG; ++g) f += sm.SQ[c][g][tid].x;
                acc.phi[c] = f;
            }
        }
        const float inv_area = __frcp_rn(__fmul_rn(3.14159265358979f, __fmul_rn(r, r)));
#pragma unroll
        for (int c = 0; c < NCH; ++c) a.tau[h * NCH + c] += (double)__fmul_rn(acc.phi[c], inv_area);
#pragma unroll
        for (int g = 0; g < PPM_NG; ++g) pairs += sm.c[g][tid];
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
            for (int g = 0; g < PPM_NG; ++g) a.cnt[g * nh + h] += sm.c[g][tid];
#pragma unroll
            for (int c = 0; c < NTC; ++c)
#pragma unroll
                for (int g = 0; g < PPM_NG; ++g) {
                    const int64_t o = ((int64_t)c * PPM_NG + g) * nh + h;
                    const float2 v = sm.SQ[c][g][tid];
                    a.S[o] += v.x;
                    a.Q[o] += v.y;
                }
        }
    }

    // block reductions: max radius for the next grid, counters
    __shared__ float s_rmax[kWarps];
    __shared__ unsigned long long s_cnt3[3][kWarps];
    const float wm = warp_max(r_new);
    const unsigned long long wp = warp_sum_u64(pairs), wc = warp_sum_u64(acc.cand),
                             wr = warp_sum_u64(rej);
    if (lane == 0) {
        s_rmax[w] = wm;
        s_cnt3[0][w] = wp; s_cnt3[1][w] = wc; s_cnt3[2][w] = wr;
    }
    __syncthreads();
    if (tid == 0) {
        float m = 0.f;
        unsigned long long p = 0, c = 0, j = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            m = fmaxf(m, s_rmax[ww]); p += s_cnt3[0][ww]; c += s_cnt3[1][ww]; j += s_cnt3[2][ww];
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
    if (c->prm.mapping == 0)
        k_gather_update<NCH, NTC, NORMALS, VCM, 0><<<nb, kThreads, 0, c->stream>>>(a);
    else if (c->prm.mapping == 1)
        k_gather_update<NCH, NTC, NORMALS, VCM, 1><<<nb, kThreads, 0, c->stream>>>(a);
    else
        k_gather_update<NCH, NTC, NORMALS, VCM, 2><<<nb, kThreads, 0, c->stream>>>(a);
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
