// ppm_gather_impl.cuh -- device code of the gather / F-test / update,
// shared by the single-problem kernel (ppm_gather.cu) and the batched
// persistent kernel (ppm_batch.cu).  See ppm_gather.cu for the method.
#pragma once

#include <limits.h>

#include <type_traits>

#include "ppm_internal.cuh"

namespace {

constexpr int kThreads = 64;
constexpr int kWarps = kThreads / 32;
// resident blocks per SM that traversals 0-4 are register-budgeted for
// (64 / 85 / 128 / 102 / 85 registers a thread), scaled with the block size;
// halved for three tested channels, whose 3x larger shared accumulators
// cap the resident blocks anyway (and whose sums need the registers)
template <int MAPPING, int NTC = 1>
constexpr int kMinBlocks =
    (MAPPING == 0 ? 8 : (MAPPING == 1 || MAPPING == 4 ? 6 : (MAPPING == 2 ? 4 : 5))) * (128 / kThreads) /
    (NTC == 3 ? 2 : 1);
constexpr int kNormalDotMin = 8064;   // 127^2 / 2: cosine > ~0.5

// rec1 and aux of an in-disk photon: side by side (aux = rec1 + 1, a stride
// of 2 float4) when a launch uses both, else each in its own array
template <int NCH, bool NORMALS, bool VCM, bool BATCH>
constexpr int kSideStride = ((NCH == 3 || VCM) && (NORMALS || VCM || BATCH)) ? 2 : 1;

// 1 / x for the merge weight's denominator x >= 1: the hardware's
// approximate reciprocal (relative error below 2^-22); the weight scales a
// sum that the tests hold to 2e-5, and no decision depends on it alone
__device__ __forceinline__ float rcp_weight(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// arrays shared by all hit points of a launch (state is [slot][nh])
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
    float* feat;        // [12][nh] features of the learned proposer, or NULL
    const uint32_t* cell_start;
    const float4* rec0;
    const float4* rec1;
    const uint4* aux;
    int32_t* err;
};

// one problem: a context, or one problem of a batch
struct Prob {
    const GridGeom* geom;
    const double* fc;               // F_c by window length
    const float2* fm;               // (1/m, 12 (m-1) / (11 m)) by window length, m = t J (from FP64)
    float* rmax_next;               // max radius after the update
    unsigned long long* counters;   // pairs, candidates, rejects, pairs total
    float k, bound, n_vm;
    int32_t fc_max;                 // last valid index of fc
    uint32_t pid;                   // problem id carried by its photons (batch)
    float inv_r0;                   // features: 1 / initial radius
    float log_iter;                 // features: log of the iteration index
};

// The 12 features of the learned radius proposer, from the window the test
// just used (channel 0): log(1+C), log(1+t'), log i, r/r0, log(r/r0),
// log(1+F), F/F_c, max_g S_g/S, min_g S_g/S, fraction of empty groups,
// coefficient of variation of the group sums, max_g c_g/C.
constexpr int kFeatures = 12;

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
    uint32_t nqh, pid;
};

// RGB flux of this hit point when only its luminance is tested: the terms
// of one run of photons (one hash-block run of a row, or one drained queue)
// are added in plain FP32, and each run's sum is added to the total with
// Kahan compensation (a disk can hold thousands of photons: one plain FP32
// sum over all of them would drift towards 1e-5).  Otherwise Phi_i is the
// sum of the tested group sums.
template <int NCH>
struct Acc {
    float phi[NCH];
    float comp[NCH];
    float part[NCH];
    unsigned long long cand = 0;
    __device__ __forceinline__ void add(int c, float v) { part[c] = __fadd_rn(part[c], v); }
    __device__ __forceinline__ void flush()
    {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const float y = __fsub_rn(part[c], comp[c]);
            const float t = __fadd_rn(phi[c], y);
            comp[c] = __fsub_rn(__fsub_rn(t, phi[c]), y);
            phi[c] = t;
            part[c] = 0.f;
        }
    }
};

// flush a run's RGB sums where they are kept (luminance test of RGB flux)
template <int NCH, int NTC>
__device__ __forceinline__ void flush_run(Acc<NCH>& acc)
{
    if constexpr (NCH == 3 && NTC == 1) acc.flush();
}

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
    // selects, not branches: the sector of the 60-degree wedge around +-v,
    // else of the side wedges
    const int s_mid = up ? 1 : 4;
    const int s_side = up ? (yu > 0.f ? 0 : 2) : (yu < 0.f ? 3 : 5);
    return ring + (fabsf(yv) >= tx ? s_mid : s_side);
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
template <int NCH, int NTC, bool NORMALS, bool VCM, bool BATCH, typename SM>
__device__ __forceinline__ void gather_pair(const GatherArgs& a, const Hit& H, SM& sm, int tid,
                                            Acc<NCH>& acc, uint32_t p, const float4& X,
                                            float dx, float dy, float dz)
{
    uint4 A = make_uint4(0u, 0u, 0u, 0u);
    constexpr int SIDE = kSideStride<NCH, NORMALS, VCM, BATCH>;
    if constexpr (NORMALS || VCM || BATCH) A = __ldg(a.aux + (size_t)p * SIDE);
    if constexpr (BATCH) {
        if (A.w != H.pid) return;      // a photon of another problem sharing the bucket
    }
    if constexpr (NORMALS) {
        if (__dp4a((int)A.x, (int)H.nqh, 0) <= kNormalDotMin) return;
    }
    const float yu = fmaf(dz, H.U.z, fmaf(dy, H.U.y, __fmul_rn(dx, H.U.x)));
    const float yv = fmaf(dz, H.V.z, fmaf(dy, H.V.y, __fmul_rn(dx, H.V.x)));
    const int g = pair_group(yu, yv, H.r2);
    float w = 1.f;
    float4 X1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (NCH == 3 || VCM) X1 = __ldg(a.rec1 + (size_t)p * SIDE);
    if constexpr (VCM) {
        const int cd = __dp4a((int)A.y, (int)H.nqh, 0);
        const float cosl = cd > 0 ? __fmul_rn((float)cd, 1.0f / 16129.0f) : 0.f;
        const float r_vm = fmaf(H.U.w, __fmul_rn(cosl, 0.318309886f), X1.w);
        const float r_vc = __fadd_rn(H.V.w, __uint_as_float(A.z));
        w = rcp_weight(1.f + r_vm + r_vc * H.inv_eta);
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

struct CellBox { int ix0, ix1, iy0, iy1, iz0, iz1; float rc; };

// cells that can hold a photon passing this hit point's FP32 disk test:
// the cull radius rc covers the rounding of dx and of d2
__device__ __forceinline__ CellBox cell_box(const Hit& H, const GridGeom& G)
{
    const float rc = fmaf(H.r, 1.0009765625f,
                          (fabsf(H.P.x) + fabsf(H.P.y) + fabsf(H.P.z) + H.r) * 1.0e-6f);
    CellBox b;
    b.ix0 = ppm_cell_coord(__fsub_rn(H.P.x, rc), G.inv_hx);
    b.ix1 = ppm_cell_coord(__fadd_rn(H.P.x, rc), G.inv_hx);
    b.iy0 = ppm_cell_coord(__fsub_rn(H.P.y, rc), G.inv_h);
    b.iy1 = ppm_cell_coord(__fadd_rn(H.P.y, rc), G.inv_h);
    b.iz0 = ppm_cell_coord(__fsub_rn(H.P.z, rc), G.inv_h);
    b.iz1 = ppm_cell_coord(__fadd_rn(H.P.z, rc), G.inv_h);
    b.rc = rc;
    return b;
}

// Row trimming: a photon passing the disk test lies within rc of P, so in
// the row of cells (iy, iz) it lies within the chord of that sphere at the
// row's nearest point.  RowCull holds what every row needs:
//   eps    bounds how far a photon of cell i can lie outside [i h, (i+1) h]
//          (the FP32 products behind the cell coordinates and i h itself),
//          and the rounding of P.x -+ half;
//   slack  keeps the squared chord from going negative through rounding
//          near a tangent row (rc^2 / 65536 >> the few ulps of rc^2 lost).
// Only photons that fail the test are skipped: the in-disk pairs and their
// order are those of the full box.
struct RowCull { float rc2, slack, eps; };

__device__ __forceinline__ RowCull row_cull(const Hit& H, const GridGeom& G, const CellBox& b)
{
    RowCull c;
    c.rc2 = __fmul_rn(b.rc, b.rc);
    c.slack = __fmul_rn(c.rc2, 1.0f / 65536.0f);
    c.eps = fmaf(fabsf(H.P.x) + fabsf(H.P.y) + fabsf(H.P.z) + b.rc + G.h, 2.0e-6f,
                 __fmul_rn(G.h, 1.0f / 1024.0f));
    return c;
}

// lower bound of the distance from coordinate p to the slab of cell i
__device__ __forceinline__ float slab_gap(float p, int i, const GridGeom& G, float eps)
{
    const float lo = __fmul_rn((float)i, G.h);
    const float hi = __fadd_rn(lo, G.h);
    return fmaxf(fmaxf(lo - p, p - hi) - eps, 0.f);
}

// this hit point's trimmed x-range of row (iy, iz) (the computation of
// traversal 0's walk); empty (x0 > x1) for a row outside its cell box or
// missing its sphere, and for a lane without a hit point
__device__ __forceinline__ void row_xrange(const Hit& H, const GridGeom& G, const CellBox& b, const RowCull& rcu,
                                           bool live, int iy, int iz, int& x0, int& x1)
{
    x0 = INT_MAX;
    x1 = INT_MIN;
    if (!live || iy < b.iy0 || iy > b.iy1 || iz < b.iz0 || iz > b.iz1) return;
    const float gz = slab_gap(H.P.z, iz, G, rcu.eps);
    const float rz2 = rcu.rc2 - gz * gz;
    const float gy = slab_gap(H.P.y, iy, G, rcu.eps);
    const float ryz2 = rz2 - gy * gy;
    if (rz2 + rcu.slack < 0.f || ryz2 + rcu.slack < 0.f) return;
    const float half = sqrtf(fmaxf(ryz2, 0.f) + rcu.slack) + rcu.eps;
    x0 = max(b.ix0, ppm_cell_coord(__fsub_rn(H.P.x, half), G.inv_hx));
    x1 = min(b.ix1, ppm_cell_coord(__fadd_rn(H.P.x, half), G.inv_hx));
}

// traversal 0: the thread walks its own cells
template <int NCH, int NTC, bool NORMALS, bool VCM, bool BATCH, typename SM>
__device__ void gather_own(const GatherArgs& a, const Hit& H, const GridGeom& G, CellBox b,
                           SM& sm, int tid, Acc<NCH>& acc)
{
    const int B = 1 << G.lb, BX = ppm_block_x(G);
    if (b.ix1 - b.ix0 >= BX || b.iy1 - b.iy0 >= B || b.iz1 - b.iz0 >= B) {
        // the sphere spans more cells than a block: distinct cells could
        // share a bucket; never happens for r <= max radius and sane
        // coordinates -- flag it instead of double counting
        atomicOr(a.err, 1);
        b.ix1 = min(b.ix1, b.ix0 + BX - 1); b.iy1 = min(b.iy1, b.iy0 + B - 1); b.iz1 = min(b.iz1, b.iz0 + B - 1);
    }
    const RowCull rcu = row_cull(H, G, b);
    for (int iz = b.iz0; iz <= b.iz1; ++iz) {
        const float gz = slab_gap(H.P.z, iz, G, rcu.eps);
        const float rz2 = rcu.rc2 - gz * gz;
        if (rz2 + rcu.slack < 0.f) continue;
        for (int iy = b.iy0; iy <= b.iy1; ++iy) {
            const float gy = slab_gap(H.P.y, iy, G, rcu.eps);
            const float ryz2 = rz2 - gy * gy;
            if (ryz2 + rcu.slack < 0.f) continue;
            const float half = sqrtf(fmaxf(ryz2, 0.f) + rcu.slack) + rcu.eps;
            const int xa = max(b.ix0, ppm_cell_coord(__fsub_rn(H.P.x, half), G.inv_hx));
            const int xb = min(b.ix1, ppm_cell_coord(__fadd_rn(H.P.x, half), G.inv_hx));
            int ix = xa;
            while (ix <= xb) {
                const int ixe = min(xb, ix | (BX - 1));         // end of this block's run
                const uint32_t b0 = ppm_bucket(ix, iy, iz, G);
                const uint32_t s = __ldg(a.cell_start + b0);
                const uint32_t e = __ldg(a.cell_start + b0 + (uint32_t)(ixe - ix) + 1u);
                acc.cand += e - s;
                // software pipeline: the next record is in flight while the
                // current one is classified (an unrolled two-register
                // variant measured 12% slower)
                float4 Xn = s < e ? __ldg(a.rec0 + s) : make_float4(0.f, 0.f, 0.f, 0.f);
                for (uint32_t p = s; p < e; ++p) {
                    const float4 X = Xn;
                    if (p + 1u < e) Xn = __ldg(a.rec0 + p + 1u);
                    float dx, dy, dz;
                    if (in_disk(H, X, dx, dy, dz))
                        gather_pair<NCH, NTC, NORMALS, VCM, BATCH>(a, H, sm, tid, acc, p, X, dx, dy, dz);
                }
                if (e > s) flush_run<NCH, NTC>(acc);
                ix = ixe + 1;
            }
        }
    }
}

// traversal 1, drain: each lane processes its queued in-disk photons in
// queue (= traversal) order; the warp loops to the longest queue
template <int NCH, int NTC, bool NORMALS, bool VCM, bool BATCH, typename US>
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
            gather_pair<NCH, NTC, NORMALS, VCM, BATCH>(a, H, sm, tid, acc, p, X, dx, dy, dz);
        }
    }
    flush_run<NCH, NTC>(acc);
    qlen = 0;
    __syncwarp();
}

struct Empty {};

// traversal 3: warp-level queue of in-disk pairs, classified by any lane
constexpr int kPairQ = 160;

struct PairSmem {
    float4 chunk[kWarps][32];        // staged photon records
    uint32_t qp[kWarps][kPairQ];     // queued pair: photon index
    uint8_t qo[kWarps][kPairQ];      //              owning lane
    float4 hP[kWarps][32];           // the warp's hit points: x, y, z, normal
    float4 hU[kWarps][32];           //   u, rho_vm
    float4 hV[kWarps][32];           //   v, rho_vc
    float2 hR[kWarps][32];           //   r^2, 1/eta
};

// Group sums as 64-bit fixed point (psi * 2^40 / psi_max): integer adds are
// exact and order-independent, so lanes of a warp can add into any hit
// point's sums with shared-memory atomics and the result stays bit-for-bit
// deterministic (and is a correctly rounded sum, unlike sequential FP32).
template <int NCH>
struct FixSmem {
    unsigned long long S[PPM_NG][kThreads];
    unsigned long long Q[PPM_NG][kThreads];
    uint32_t c[PPM_NG][kThreads];
    unsigned long long F[NCH == 3 ? 3 : 1][kThreads];   // RGB flux (luminance test)
};

template <int NCH, int NTC, int MAPPING>
struct BlockShared {
    typename std::conditional<MAPPING == 3, Empty, Smem<NTC>>::type sm;
    typename std::conditional<MAPPING == 1 || MAPPING == 2, UnionSmem<MAPPING == 2 ? 64 : 32>, Empty>::type us;
    typename std::conditional<MAPPING == 3, PairSmem, Empty>::type ps;
    typename std::conditional<MAPPING == 3, FixSmem<NCH>, Empty>::type fx;
    typename std::conditional<MAPPING == 4, Smem<NTC>, Empty>::type lp;   // lanes' partial sums
};

// this iteration's sums of one hit point, read where they are kept
template <int NCH, int NTC, int MAPPING>
struct GroupSums;

struct FixScale {
    float s1;    // psi -> fixed point: psi * 2^40 / psi_max
    float t;     // psi -> q with q^2 the fixed point of psi^2: psi * 2^20 / psi_max
    float dS;    // fixed point -> sum of psi:    psi_max * 2^-40
    float dQ;    // fixed point -> sum of psi^2: (psi_max * 2^-20)^2
};

template <int NCH, int NTC, int MAPPING>
struct GroupSums {
    const BlockShared<NCH, NTC, MAPPING>& b;
    int tid;
    FixScale fs;
    __device__ __forceinline__ float S(int c, int g) const
    {
        if constexpr (MAPPING == 3) return __fmul_rn(__ull2float_rn(b.fx.S[g][tid]), fs.dS);
        else return b.sm.SQ[c][g][tid].x;
    }
    __device__ __forceinline__ float Q(int c, int g) const
    {
        if constexpr (MAPPING == 3) return __fmul_rn(__ull2float_rn(b.fx.Q[g][tid]), fs.dQ);
        else return b.sm.SQ[c][g][tid].y;
    }
    __device__ __forceinline__ uint32_t C(int g) const
    {
        if constexpr (MAPPING == 3) return b.fx.c[g][tid];
        else return b.sm.c[g][tid];
    }
};

__device__ __forceinline__ FixScale fix_scale(float psimax)
{
    const float pm = fmaxf(psimax, 1e-25f);
    FixScale f;
    f.s1 = 1099511627776.0f / pm;
    f.t = 1048576.0f / pm;
    f.dS = pm * (1.0f / 1099511627776.0f);
    const float r = pm * (1.0f / 1048576.0f);
    f.dQ = r * r;
    return f;
}

// traversal 3: everything after the disk test, accumulated into hit point
// `slot` of the block with integer atomics
template <int NCH, bool NORMALS, bool VCM, bool BATCH>
__device__ __forceinline__ void gather_pair_fix(const GatherArgs& a, const Hit& H, FixSmem<NCH>& fx, int slot,
                                                const FixScale& fs, uint32_t p, const float4& X,
                                                float dx, float dy, float dz)
{
    uint4 A = make_uint4(0u, 0u, 0u, 0u);
    constexpr int SIDE = kSideStride<NCH, NORMALS, VCM, BATCH>;
    if constexpr (NORMALS || VCM || BATCH) A = __ldg(a.aux + (size_t)p * SIDE);
    if constexpr (BATCH) {
        if (A.w != H.pid) return;
    }
    if constexpr (NORMALS) {
        if (__dp4a((int)A.x, (int)H.nqh, 0) <= kNormalDotMin) return;
    }
    const float yu = fmaf(dz, H.U.z, fmaf(dy, H.U.y, __fmul_rn(dx, H.U.x)));
    const float yv = fmaf(dz, H.V.z, fmaf(dy, H.V.y, __fmul_rn(dx, H.V.x)));
    const int g = pair_group(yu, yv, H.r2);
    float w = 1.f;
    float4 X1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (NCH == 3 || VCM) X1 = __ldg(a.rec1 + (size_t)p * SIDE);
    if constexpr (VCM) {
        const int cd = __dp4a((int)A.y, (int)H.nqh, 0);
        const float cosl = cd > 0 ? __fmul_rn((float)cd, 1.0f / 16129.0f) : 0.f;
        const float r_vm = fmaf(H.U.w, __fmul_rn(cosl, 0.318309886f), X1.w);
        const float r_vc = __fadd_rn(H.V.w, __uint_as_float(A.z));
        w = rcp_weight(1.f + r_vm + r_vc * H.inv_eta);
    }
    const float psi = VCM ? __fmul_rn(w, X.w) : X.w;
    const float q = psi * fs.t;
    atomicAdd(&fx.c[g][slot], 1u);
    atomicAdd(&fx.S[g][slot], (unsigned long long)__float2ull_rn(psi * fs.s1));
    atomicAdd(&fx.Q[g][slot], (unsigned long long)__float2ull_rn(q * q));
    if constexpr (NCH == 3) {
        atomicAdd(&fx.F[0][slot], (unsigned long long)__float2ull_rn((VCM ? __fmul_rn(w, X1.x) : X1.x) * fs.s1));
        atomicAdd(&fx.F[1][slot], (unsigned long long)__float2ull_rn((VCM ? __fmul_rn(w, X1.y) : X1.y) * fs.s1));
        atomicAdd(&fx.F[2][slot], (unsigned long long)__float2ull_rn((VCM ? __fmul_rn(w, X1.z) : X1.z) * fs.s1));
    }
}

// traversal 3: classify the warp's queued pairs, 32 at a time, any lane
template <int NCH, bool NORMALS, bool VCM, bool BATCH>
__device__ __forceinline__ void drain_pairs(const GatherArgs& a, PairSmem& ps, FixSmem<NCH>& fx,
                                            const FixScale& fs, uint32_t pid, int w, int lane, int qn)
{
    for (int e0 = 0; e0 < qn; e0 += 32) {
        const int e = e0 + lane;
        if (e < qn) {
            const uint32_t p = ps.qp[w][e];
            const int o = ps.qo[w][e];
            Hit Ho;
            Ho.P = ps.hP[w][o];
            Ho.U = ps.hU[w][o];
            Ho.V = ps.hV[w][o];
            const float2 R = ps.hR[w][o];
            Ho.r2 = R.x;
            Ho.inv_eta = R.y;
            Ho.nqh = __float_as_uint(Ho.P.w);
            Ho.pid = pid;
            const float4 X = __ldg(a.rec0 + p);
            float dx, dy, dz;
            in_disk(Ho, X, dx, dy, dz);
            gather_pair_fix<NCH, NORMALS, VCM, BATCH>(a, Ho, fx, w * 32 + o, fs, p, X, dx, dy, dz);
        }
    }
    __syncwarp();
}

// the 12 features of the learned proposer for hit point h (out of line:
// only contexts with features enabled pay for its registers)
template <int NCH, int NTC, typename GS>
__device__ __noinline__ void write_features(const GatherArgs& a, const Prob& pr,
                                            const GS& gs, int64_t h,
                                            const float* Sg, float Ssum, float dev2, float F, float fc,
                                            float r, int32_t tp)
{
    const int64_t nh = a.nh;
    uint32_t C = 0, cmax = 0, empty = 0;
    float smax = 0.f, smin = Sg[0];
#pragma unroll
    for (int g = 0; g < PPM_NG; ++g) {
        const uint32_t cg = a.cnt[g * nh + h] + gs.C(g);
        C += cg;
        cmax = max(cmax, cg);
        empty += cg == 0u;
        smax = fmaxf(smax, Sg[g]);
        smin = fminf(smin, Sg[g]);
    }
    const float f[kFeatures] = {
        log1pf((float)C), log1pf((float)tp), pr.log_iter, r * pr.inv_r0,
        logf(fmaxf(r * pr.inv_r0, 1e-30f)), log1pf(F), F / fc,
        Ssum > 0.f ? smax / Ssum : 0.f, Ssum > 0.f ? smin / Ssum : 0.f,
        (float)empty * (1.0f / PPM_NG),
        Ssum > 0.f ? sqrtf(dev2 * (1.0f / PPM_NG)) / (Ssum * (1.0f / PPM_NG)) : 0.f,
        C > 0u ? (float)cmax / (float)C : 0.f};
#pragma unroll
    for (int q = 0; q < kFeatures; ++q) a.feat[(int64_t)q * nh + h] = f[q];
}

// Eq. f-statistic, the test, Eq. radiusupdate and the estimate of
// Eq. progressive-VCM-estimator for hit point h (radius r) from this
// iteration's sums gs (S(c, g), Q(c, g), C(g)) and the stored window; the
// new radius, the rejection and the pair count are returned for the
// block's reductions
template <int NCH, int NTC, bool FEAT, bool CHI2, typename GS>
__device__ __forceinline__ void update_hit(const GatherArgs& a, const Prob& pr, const GS& gs, int64_t h, float r,
                                           Acc<NCH>& acc, float& r_new, unsigned long long& rej,
                                           unsigned long long& pairs)
{
    const int32_t tp = a.t[h] + 1;
    // a window longer than the table can only come from ppm_set_state
    // with t >= the iteration count: clamp the lookup and flag it
    int32_t tpi = tp;
    if (tp < 1 || tp > pr.fc_max) { atomicOr(a.err, 2); tpi = max(1, min(tp, pr.fc_max)); }
    // m = t' J samples per group never exists in FP32: the table holds
    // 1/m and 12 (m-1) / (11 m), each computed in FP64 and rounded once
    const float2 mf = pr.fm[tpi];
    const int64_t nh = a.nh;
    bool reject = false;
    float F0 = 0.f;
    // CPPM (Sec. 3.2.3): Pearson's X^2 of the window's in-disk counts
    // against an even spread, from exact integers:
    // X^2 = (12 sum_g c_g^2 - C^2) / C, C = sum_g c_g (0 without photons)
    double x2 = 0.0;
    if constexpr (CHI2) {
        unsigned long long C = 0ull, C2 = 0ull;
#pragma unroll
        for (int g = 0; g < PPM_NG; ++g) {
            const unsigned long long cg = (unsigned long long)a.cnt[g * nh + h] + gs.C(g);
            C += cg;
            C2 += cg * cg;
        }
        if (C > 0ull) x2 = (double)(PPM_NG * C2 - C * C) / (double)C;
        reject = x2 > pr.fc[tpi];
    }
#pragma unroll
    for (int c = 0; c < NTC; ++c) {
        float Sg[PPM_NG];
        float Ssum = 0.f, Qsum = 0.f, S2 = 0.f;
#pragma unroll
        for (int g = 0; g < PPM_NG; ++g) {
            const int64_t o = ((int64_t)c * PPM_NG + g) * nh + h;
            Sg[g] = a.S[o] + gs.S(c, g);
            Qsum += a.Q[o] + gs.Q(c, g);
            Ssum += Sg[g];
            S2 = fmaf(Sg[g], Sg[g], S2);
        }
        const float Sbar = Ssum * (1.0f / PPM_NG);
        float dev2 = 0.f;
#pragma unroll
        for (int g = 0; g < PPM_NG; ++g) { const float d = Sg[g] - Sbar; dev2 = fmaf(d, d, dev2); }
        // SSB = dev2 / m, SSW = sum Q - sum S^2 / m,
        // F = (SSB / 11) / (SSW / (12 (m-1))) = (dev2 / SSW) * 12 (m-1) / (11 m)
        const float ssw = Qsum - S2 * mf.x;
        float F = 0.f;
        if (ssw > 0.f) F = (dev2 / ssw) * mf.y;
        if (c == 0) F0 = CHI2 ? (float)x2 : F;
        if (!CHI2 && ssw > 0.f && (double)F > pr.fc[tpi]) reject = true;
        if constexpr (FEAT)
            if (c == 0) write_features<NCH, NTC>(a, pr, gs, h, Sg, Ssum, dev2, F, (float)pr.fc[tpi], r, tp);
    }
    // Eq. (progressive-VCM-estimator): kernel estimate with this r_i;
    // Phi_i = sum over groups of this iteration's psi sums unless RGB
    // flux is tested on its luminance
    if constexpr (!(NCH == 3 && NTC == 1)) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            float f = 0.f;
#pragma unroll
            for (int g = 0; g < PPM_NG; ++g) f += gs.S(c, g);
            acc.phi[c] = f;
        }
    }
    const float inv_area = __frcp_rn(__fmul_rn(3.14159265358979f, __fmul_rn(r, r)));
#pragma unroll
    for (int c = 0; c < NCH; ++c) a.tau[h * NCH + c] += (double)__fmul_rn(acc.phi[c], inv_area);
#pragma unroll
    for (int g = 0; g < PPM_NG; ++g) pairs += gs.C(g);
    a.F[h] = F0;
    if (reject) {
        r_new = fmaxf(__fmul_rn(pr.k, r), pr.bound);
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
        for (int g = 0; g < PPM_NG; ++g) a.cnt[g * nh + h] += gs.C(g);
#pragma unroll
        for (int c = 0; c < NTC; ++c)
#pragma unroll
            for (int g = 0; g < PPM_NG; ++g) {
                const int64_t o = ((int64_t)c * PPM_NG + g) * nh + h;
                a.S[o] += gs.S(c, g);
                a.Q[o] += gs.Q(c, g);
            }
    }
}

// Reduce-scatter of N values (N a power of two, <= 32) over the warp by
// recursive halving: at each step a lane keeps half of its values, adds its
// partner's copy of that half and passes on the other half.  Returns, on
// lane l, the warp sum of value l / (32 / N).  N - 1 shuffles for N values
// (plus log2(32 / N) for the lanes that end up sharing a value).
template <int N, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[N], int lane)
{
    static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "N: a power of two up to 32");
#pragma unroll
    for (int half = N / 2, off = 16; half >= 1; half >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const T send = upper ? v[i] : v[i + half];
            const T keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    T t = v[0];
#pragma unroll
    for (int off = 16 / N; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    return t;
}

__device__ __forceinline__ float4 shfl_f4(float4 v, int src)
{
    v.x = __shfl_sync(0xffffffffu, v.x, src);
    v.y = __shfl_sync(0xffffffffu, v.y, src);
    v.z = __shfl_sync(0xffffffffu, v.z, src);
    v.w = __shfl_sync(0xffffffffu, v.w, src);
    return v;
}

// Traversal 4: hit point Hj (lane j's, owner thread `owner`) by the whole
// warp.  The warp walks its trimmed rows; the lanes split each segment's
// photons and accumulate into their own column of lp; then the 36 group
// sums are reduced across the warp with shuffles into the owner's slots of
// sm.  One flux channel.
template <int NTC, bool NORMALS, bool VCM, bool BATCH>
__device__ __forceinline__ void gather_warp_hit(const GatherArgs& a, const Hit& Hj, const GridGeom& G, CellBox b,
                                                Smem<NTC>& lp, Smem<NTC>& sm, int tid, int lane, int owner,
                                                Acc<1>& acc)
{
    static_assert(NTC == 1, "traversal 4 tests one channel");
    const int B = 1 << G.lb, BX = ppm_block_x(G);
    if (b.ix1 - b.ix0 >= BX || b.iy1 - b.iy0 >= B || b.iz1 - b.iz0 >= B) {
        if (lane == 0) atomicOr(a.err, 1);
        b.ix1 = min(b.ix1, b.ix0 + BX - 1); b.iy1 = min(b.iy1, b.iy0 + B - 1); b.iz1 = min(b.iz1, b.iz0 + B - 1);
    }
    const RowCull rcu = row_cull(Hj, G, b);
    for (int iz = b.iz0; iz <= b.iz1; ++iz) {
        const float gz = slab_gap(Hj.P.z, iz, G, rcu.eps);
        const float rz2 = rcu.rc2 - gz * gz;
        if (rz2 + rcu.slack < 0.f) continue;
        for (int iy = b.iy0; iy <= b.iy1; ++iy) {
            const float gy = slab_gap(Hj.P.y, iy, G, rcu.eps);
            const float ryz2 = rz2 - gy * gy;
            if (ryz2 + rcu.slack < 0.f) continue;
            const float half = sqrtf(fmaxf(ryz2, 0.f) + rcu.slack) + rcu.eps;
            const int xa = max(b.ix0, ppm_cell_coord(__fsub_rn(Hj.P.x, half), G.inv_hx));
            const int xb = min(b.ix1, ppm_cell_coord(__fadd_rn(Hj.P.x, half), G.inv_hx));
            int ix = xa;
            while (ix <= xb) {
                const int ixe = min(xb, ix | (BX - 1));
                const uint32_t b0 = ppm_bucket(ix, iy, iz, G);
                const uint32_t s = __ldg(a.cell_start + b0);
                const uint32_t e = __ldg(a.cell_start + b0 + (uint32_t)(ixe - ix) + 1u);
                if (lane == 0) acc.cand += e - s;
                for (uint32_t p = s + (uint32_t)lane; p < e; p += 32u) {
                    const float4 X = __ldg(a.rec0 + p);
                    float dx, dy, dz;
                    if (in_disk(Hj, X, dx, dy, dz))
                        gather_pair<1, NTC, NORMALS, VCM, BATCH>(a, Hj, lp, tid, acc, p, X, dx, dy, dz);
                }
                ix = ixe + 1;
            }
        }
    }
    // this lane's column -> registers (cleared for the next hit point)
    float v[32];
    uint32_t c[16];
#pragma unroll
    for (int g = 0; g < PPM_NG; ++g) {
        const float2 q = lp.SQ[0][g][tid];
        v[g] = q.x;
        v[PPM_NG + g] = q.y;
        c[g] = lp.c[g][tid];
        lp.SQ[0][g][tid] = make_float2(0.f, 0.f);
        lp.c[g][tid] = 0u;
    }
#pragma unroll
    for (int i = 2 * PPM_NG; i < 32; ++i) v[i] = 0.f;
#pragma unroll
    for (int i = PPM_NG; i < 16; ++i) c[i] = 0u;
    const float t = warp_reduce_scatter<32>(v, lane);        // lane l: value l
    const uint32_t ct = warp_reduce_scatter<16>(c, lane);    // lane l: count l / 2
    if (lane < PPM_NG) sm.SQ[0][lane][owner].x = t;
    else if (lane < 2 * PPM_NG) sm.SQ[0][lane - PPM_NG][owner].y = t;
    if ((lane & 1) == 0 && (lane >> 1) < PPM_NG) sm.c[lane >> 1][owner] = ct;
}

// The hit points [h0, h_end) (at most one block's worth, h0 + tid for this
// thread) of problem pr: gather, test, update; block-wide reductions into
// pr's counters.  Ends with a block barrier, so it can be called in a loop.
// FEAT: also write the proposer's features (a separate instantiation: the
// call alone costs the feature-free kernel about 10% through register
// allocation in the cell walk).  CHI2: CPPM's count test decides instead of
// the F-test (its own instantiation too).
template <int NCH, int NTC, bool NORMALS, bool VCM, int MAPPING, bool BATCH, bool FEAT = false,
          bool CHI2 = false>
__device__ __forceinline__ void gather_block(const GatherArgs& a, const Prob& pr, int64_t h0,
                                             int64_t h_end, BlockShared<NCH, NTC, MAPPING>& bsh)
{
    static_assert(MAPPING != 3 || NTC == 1, "traversal 3 tests one channel");
    static_assert(MAPPING != 4 || NCH == 1, "traversal 4 gathers one flux channel");
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t h = h0 + tid;
    const bool live = h < h_end;
    constexpr int kQueue = MAPPING == 2 ? 64 : 32;
    auto& sm = bsh.sm;
    if constexpr (MAPPING != 3) {
#pragma unroll
        for (int g = 0; g < PPM_NG; ++g) {
            sm.c[g][tid] = 0u;
#pragma unroll
            for (int c = 0; c < NTC; ++c) sm.SQ[c][g][tid] = make_float2(0.f, 0.f);
        }
        if constexpr (MAPPING == 4) {
#pragma unroll
            for (int g = 0; g < PPM_NG; ++g) {
                bsh.lp.c[g][tid] = 0u;
#pragma unroll
                for (int c = 0; c < NTC; ++c) bsh.lp.SQ[c][g][tid] = make_float2(0.f, 0.f);
            }
        }
    } else {
#pragma unroll
        for (int g = 0; g < PPM_NG; ++g) {
            bsh.fx.S[g][tid] = 0ull;
            bsh.fx.Q[g][tid] = 0ull;
            bsh.fx.c[g][tid] = 0u;
        }
#pragma unroll
        for (int c = 0; c < (NCH == 3 ? 3 : 1); ++c) bsh.fx.F[c][tid] = 0ull;
    }

    Acc<NCH> acc;
#pragma unroll
    for (int c = 0; c < NCH; ++c) { acc.phi[c] = 0.f; acc.comp[c] = 0.f; acc.part[c] = 0.f; }
    Hit H;
    H.r = 0.f; H.r2 = 0.f;
    GridGeom G = *pr.geom;
    // one problem: problem id 0 as a constant, so the bucket hash keeps no
    // register for it through the cell walk
    if constexpr (!BATCH) G.pid = 0u;
    H.pid = BATCH ? pr.pid : 0u;
    CellBox b{INT_MAX, INT_MIN, INT_MAX, INT_MIN, INT_MAX, INT_MIN, 0.f};
    if (live) {
        H.P = a.hp_pos[h];
        H.U = a.hp_u[h];
        H.V = a.hp_v[h];
        H.r = a.r[h];
        H.r2 = __fmul_rn(H.r, H.r);
        H.nqh = __float_as_uint(H.P.w);
        H.inv_eta = 0.f;
        if constexpr (VCM) H.inv_eta = __frcp_rn(__fmul_rn(__fmul_rn(pr.n_vm, 3.14159265358979f), H.r2));
        b = cell_box(H, G);
    } else {
        H.P = make_float4(0.f, 0.f, 0.f, 0.f);
        H.U = H.V = H.P;
        H.nqh = 0u;
        H.inv_eta = 0.f;
        H.r2 = -1.f;                      // no photon passes d2 <= -1
    }

    const FixScale fs = fix_scale(MAPPING == 3 ? G.psimax : 1.f);
    if constexpr (MAPPING == 0) {
        if (live) gather_own<NCH, NTC, NORMALS, VCM, BATCH>(a, H, G, b, sm, tid, acc);
    } else if constexpr (MAPPING == 4) {
        __syncwarp();
        for (int j = 0; j < 32; ++j) {
            if (!__shfl_sync(0xffffffffu, (int)live, j)) continue;   // warp-uniform
            Hit Hj;
            Hj.P = shfl_f4(H.P, j);
            Hj.U = shfl_f4(H.U, j);
            Hj.V = shfl_f4(H.V, j);
            Hj.r = __shfl_sync(0xffffffffu, H.r, j);
            Hj.r2 = __shfl_sync(0xffffffffu, H.r2, j);
            Hj.inv_eta = __shfl_sync(0xffffffffu, H.inv_eta, j);
            Hj.nqh = __shfl_sync(0xffffffffu, H.nqh, j);
            Hj.pid = H.pid;
            CellBox bj;
            bj.ix0 = __shfl_sync(0xffffffffu, b.ix0, j); bj.ix1 = __shfl_sync(0xffffffffu, b.ix1, j);
            bj.iy0 = __shfl_sync(0xffffffffu, b.iy0, j); bj.iy1 = __shfl_sync(0xffffffffu, b.iy1, j);
            bj.iz0 = __shfl_sync(0xffffffffu, b.iz0, j); bj.iz1 = __shfl_sync(0xffffffffu, b.iz1, j);
            bj.rc = __shfl_sync(0xffffffffu, b.rc, j);
            gather_warp_hit<NTC, NORMALS, VCM, BATCH>(a, Hj, G, bj, bsh.lp, sm, tid, lane, w * 32 + j, acc);
        }
        __syncwarp();
    } else if constexpr (MAPPING == 3) {
        const RowCull rcu = row_cull(H, G, b);     // row trimming of the union walk
        PairSmem& ps = bsh.ps;
        auto& fx = bsh.fx;
        const unsigned full = 0xffffffffu;
        const unsigned lt = (1u << lane) - 1u;
        ps.hP[w][lane] = H.P;
        ps.hU[w][lane] = H.U;
        ps.hV[w][lane] = H.V;
        ps.hR[w][lane] = make_float2(H.r2, H.inv_eta);
        __syncwarp();
        const int X0 = __reduce_min_sync(full, b.ix0), X1 = __reduce_max_sync(full, b.ix1);
        const int Y0 = __reduce_min_sync(full, b.iy0), Y1 = __reduce_max_sync(full, b.iy1);
        const int Z0 = __reduce_min_sync(full, b.iz0), Z1 = __reduce_max_sync(full, b.iz1);
        const int B = 1 << G.lb, BX = ppm_block_x(G);
        const bool any_live = __any_sync(full, live);
        if (any_live && (X1 - X0 >= BX || Y1 - Y0 >= B || Z1 - Z0 >= B)) {
            // union wider than a hash block: every lane walks its own cells
            // and queues only its own pairs (its own slots: no conflicts)
            if (live) {
                int bx1 = b.ix1, by1 = b.iy1, bz1 = b.iz1;
                if (b.ix1 - b.ix0 >= BX || b.iy1 - b.iy0 >= B || b.iz1 - b.iz0 >= B) {
                    atomicOr(a.err, 1);
                    bx1 = min(bx1, b.ix0 + BX - 1); by1 = min(by1, b.iy0 + B - 1); bz1 = min(bz1, b.iz0 + B - 1);
                }
                for (int iz = b.iz0; iz <= bz1; ++iz)
                    for (int iy = b.iy0; iy <= by1; ++iy) {
                        int ix = b.ix0;
                        while (ix <= bx1) {
                            const int ixe = min(bx1, ix | (BX - 1));
                            const uint32_t b0 = ppm_bucket(ix, iy, iz, G);
                            const uint32_t s = __ldg(a.cell_start + b0);
                            const uint32_t e = __ldg(a.cell_start + b0 + (uint32_t)(ixe - ix) + 1u);
                            acc.cand += e - s;
                            for (uint32_t p = s; p < e; ++p) {
                                const float4 X = __ldg(a.rec0 + p);
                                float dx, dy, dz;
                                if (in_disk(H, X, dx, dy, dz))
                                    gather_pair_fix<NCH, NORMALS, VCM, BATCH>(a, H, fx, tid, fs, p, X, dx, dy, dz);
                            }
                            ix = ixe + 1;
                        }
                    }
            }
        } else if (any_live) {
            int qn = 0;                     // warp-uniform queue length
            for (int iz = Z0; iz <= Z1; ++iz) {
                for (int iy = Y0; iy <= Y1; ++iy) {
                    // the union of the lanes' trimmed ranges of this row
                    int tx0, tx1;
                    row_xrange(H, G, b, rcu, live, iy, iz, tx0, tx1);
                    const bool need = tx0 <= tx1;
                    if (!__any_sync(full, need)) continue;
                    const int rx0 = __reduce_min_sync(full, need ? tx0 : INT_MAX);
                    const int rx1 = __reduce_max_sync(full, need ? tx1 : INT_MIN);
                    int ix = rx0;
                    while (ix <= rx1) {
                        const int ixe = min(rx1, ix | (BX - 1));
                        const uint32_t b0 = ppm_bucket(ix, iy, iz, G);
                        const uint32_t s = __ldg(a.cell_start + b0);
                        const uint32_t e = __ldg(a.cell_start + b0 + (uint32_t)(ixe - ix) + 1u);
                        if (need) acc.cand += e - s;
                        for (uint32_t base = s; base < e; base += 32u) {
                            const int n = (int)min(32u, e - base);
                            if (lane < n) ps.chunk[w][lane] = __ldg(a.rec0 + base + lane);
                            __syncwarp();
                            for (int j = 0; j < n; ++j) {
                                const float4 X = ps.chunk[w][j];
                                float dx, dy, dz;
                                const bool in = in_disk(H, X, dx, dy, dz);
                                const unsigned bal = __ballot_sync(full, in);
                                if (in) {
                                    const int pos = qn + __popc(bal & lt);
                                    ps.qp[w][pos] = base + (uint32_t)j;
                                    ps.qo[w][pos] = (uint8_t)lane;
                                }
                                qn += __popc(bal);
                                if (qn > kPairQ - 32) {
                                    __syncwarp();
                                    drain_pairs<NCH, NORMALS, VCM, BATCH>(a, ps, fx, fs, pr.pid, w, lane, qn);
                                    qn = 0;
                                }
                            }
                            __syncwarp();
                        }
                        ix = ixe + 1;
                    }
                }
            }
            __syncwarp();
            drain_pairs<NCH, NORMALS, VCM, BATCH>(a, ps, fx, fs, pr.pid, w, lane, qn);
        }
    } else {
        const RowCull rcu = row_cull(H, G, b);     // row trimming of the union walk
        using US = UnionSmem<kQueue>;
        US& us = bsh.us;
        const unsigned full = 0xffffffffu;
        const int X0 = __reduce_min_sync(full, b.ix0), X1 = __reduce_max_sync(full, b.ix1);
        const int Y0 = __reduce_min_sync(full, b.iy0), Y1 = __reduce_max_sync(full, b.iy1);
        const int Z0 = __reduce_min_sync(full, b.iz0), Z1 = __reduce_max_sync(full, b.iz1);
        const int B = 1 << G.lb, BX = ppm_block_x(G);
        const bool any_live = __any_sync(full, live);
        if (any_live && (X1 - X0 >= BX || Y1 - Y0 >= B || Z1 - Z0 >= B)) {
            // union wider than a hash block: walk per lane instead
            if (live) gather_own<NCH, NTC, NORMALS, VCM, BATCH>(a, H, G, b, sm, tid, acc);
        } else if (any_live) {
            int qlen = 0;
            for (int iz = Z0; iz <= Z1; ++iz) {
                for (int iy = Y0; iy <= Y1; ++iy) {
                    // the union of the lanes' trimmed ranges of this row
                    int tx0, tx1;
                    row_xrange(H, G, b, rcu, live, iy, iz, tx0, tx1);
                    const bool need = tx0 <= tx1;
                    if (!__any_sync(full, need)) continue;
                    const int rx0 = __reduce_min_sync(full, need ? tx0 : INT_MAX);
                    const int rx1 = __reduce_max_sync(full, need ? tx1 : INT_MIN);
                    int ix = rx0;
                    while (ix <= rx1) {
                        const int ixe = min(rx1, ix | (BX - 1));
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
                                    drain_queue<NCH, NTC, NORMALS, VCM, BATCH>(a, H, sm, us, w, lane, tid, acc, qlen);
                            }
                            __syncwarp();
                        }
                        ix = ixe + 1;
                    }
                }
            }
            drain_queue<NCH, NTC, NORMALS, VCM, BATCH>(a, H, sm, us, w, lane, tid, acc, qlen);
        }
    }

    flush_run<NCH, NTC>(acc);       // a run's sums not yet flushed (fallback walks)
    // this iteration's sums of this thread's hit point
    const GroupSums<NCH, NTC, MAPPING> gs{bsh, tid, fs};
    if constexpr (MAPPING == 3) {
        __syncwarp();
        if constexpr (NCH == 3) {
#pragma unroll
            for (int c = 0; c < 3; ++c) acc.phi[c] = __fmul_rn(__ull2float_rn(bsh.fx.F[c][tid]), fs.dS);
        }
    }

    // ---------------- epilogue: F-test, estimate, radius update ----------
    float r_new = 0.f;
    unsigned long long rej = 0, pairs = 0;
    if (live) update_hit<NCH, NTC, FEAT, CHI2>(a, pr, gs, h, H.r, acc, r_new, rej, pairs);

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
        atomicMax((int*)pr.rmax_next, __float_as_int(m));
        atomicAdd(pr.counters + 0, p);
        atomicAdd(pr.counters + 1, c);
        atomicAdd(pr.counters + 2, j);
        atomicAdd(pr.counters + 3, p);
    }
    __syncthreads();
}

// one context: one block per kThreads hit points
template <int NCH, int NTC, bool NORMALS, bool VCM, int MAPPING, bool FEAT = false, bool CHI2 = false>
__global__ void __launch_bounds__(kThreads, kMinBlocks<MAPPING, NTC>)
k_gather_update(GatherArgs a, Prob pr)
{
    __shared__ BlockShared<NCH, NTC, MAPPING> bsh;
    if (*a.err & 4) return;          // the grid's sort gave up: no usable grid
    const int64_t h0 = (int64_t)blockIdx.x * kThreads;
    gather_block<NCH, NTC, NORMALS, VCM, MAPPING, false, FEAT, CHI2>(a, pr, h0, a.nh, bsh);
}

}  // namespace
