// ppm_batch.cu -- many independent problems in one iteration: every
// problem has its own hit points, radii, photons (J_p per iteration), grid
// cell size and F_c table, and an iteration of all of them is
//   one pack pass over all photons (the problem id is mixed into the bucket
//   hash and carried in every record), one stable radix sort, one cell-range
//   pass, one permute, and ONE persistent gather launch: resident blocks pull
//   tiles of one problem (params.tile hit points, run as blocks of kThreads in
//   turn; the autotuner picks the size) from an atomic queue, heaviest
//   problems first, and run the same gather / F-test / update as a single
//   context (bit-identical results for the same mapping and cell factor).
// From the second iteration on the whole sequence is replayed as a CUDA
// graph on a private stream; per-iteration inputs (photon pointers, the
// radius-bound factor) reach it through pinned host staging copied by the
// graph's first node.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ppm_gather_impl.cuh"

namespace {

struct PhotonPtrs {
    const float* pos;
    const float* flux;
    const uint32_t* nq;
    const float* rho;
    const uint32_t* wq;
    int64_t pad;
};

struct IterScalars {
    double bound_scale;      // sqrt((i+1)^(alpha-1)) of Eq. (radiusupdate)
    double pad;
};

constexpr int kFcCap0 = 1024;    // window lengths with a precomputed F_c at create (grows)

}  // namespace

struct ppm_batch {
    int dev = 0;
    cudaStream_t user = nullptr;     // caller's stream
    cudaStream_t st = nullptr;       // private stream (graph capture)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_staged = nullptr;
    cudaEvent_t ev_g0 = nullptr, ev_g1 = nullptr;   // around the gather (timing)
    ppm_params prm{};
    float alpha = 0.75f;
    int P = 0;
    int nch = 1, ntc = 1;
    bool normals = false;
    std::vector<int64_t> hp_n, hp_off, J, ph_off;
    std::vector<float> r0, rmin, cf;
    int64_t nh_total = 0, np_total = 0;
    // hit points and state ([slot][nh_total])
    uint32_t* hp_orig = nullptr;
    float4 *hp_pos = nullptr, *hp_u = nullptr, *hp_v = nullptr;
    float* r = nullptr;
    int32_t* t = nullptr;
    float* F = nullptr;
    double* tau = nullptr;
    uint32_t* cnt = nullptr;
    float *S = nullptr, *Q = nullptr;
    // per problem
    GridGeom* geom = nullptr;
    float *rmax = nullptr, *rmax_next = nullptr, *cf_dev = nullptr, *rmin_dev = nullptr;
    float *nvm = nullptr, *bound = nullptr;
    double* fc = nullptr;            // [P][fc_cap + 1] F_c by window length
    float2* fm = nullptr;            // [P][fc_cap + 1] (1/m, 12 (m-1) / (11 m)), m = t J
    int fc_cap = 0;
    unsigned long long* counters = nullptr;   // 4 per problem
    unsigned long long* pairs_total = nullptr;
    // work lists
    int4* tiles = nullptr;
    int ntiles = 0;
    int4* pack_blocks = nullptr;
    int npack = 0;
    unsigned* head = nullptr;
    int gather_grid = 0;
    // per-iteration staging
    PhotonPtrs *ptab_h = nullptr, *ptab_d = nullptr;
    IterScalars *sc_h = nullptr, *sc_d = nullptr;
    // grid
    SortScratch sort;
    int tbits = 0, lb = 4;      // hash blocks 16 cells wide along y and z
    uint32_t* cell_start = nullptr;
    float4 *pack = nullptr, *rec0 = nullptr, *rec1 = nullptr;   // pack: a photon's records side by side
    uint4* aux = nullptr;
    int32_t* err = nullptr;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int iter = 0;
    int launches = 0;
};

namespace {

template <typename T>
bool dal(T** p, int64_t n)
{
    if (n <= 0) n = 1;
    const cudaError_t e = cudaMalloc(p, (size_t)n * sizeof(T));
    if (e != cudaSuccess) {
        ppm_note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

// event record that the host can wait on / time: while the stream is being
// captured it must become an external event node (a plain record there is
// only a capture-internal dependency); outside capture a plain record
cudaError_t record_host_event(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, st);
}

// true if ok; notes the failing call under PPM_DEBUG
bool ok_call(cudaError_t e, const char* what, int line)
{
    if (e == cudaSuccess) return true;
    ppm_note_cuda_error(e, what, __FILE__, line);
    cudaGetLastError();
    return false;
}
#define OKC(call) ok_call((call), #call, __LINE__)

void free_batch(ppm_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->hp_orig); cudaFree(b->hp_pos); cudaFree(b->hp_u); cudaFree(b->hp_v);
    cudaFree(b->r); cudaFree(b->t); cudaFree(b->F); cudaFree(b->tau); cudaFree(b->cnt);
    cudaFree(b->S); cudaFree(b->Q);
    cudaFree(b->geom); cudaFree(b->rmax); cudaFree(b->rmax_next); cudaFree(b->cf_dev);
    cudaFree(b->rmin_dev); cudaFree(b->nvm); cudaFree(b->bound); cudaFree(b->fc); cudaFree(b->fm);
    cudaFree(b->counters); cudaFree(b->pairs_total);
    cudaFree(b->tiles); cudaFree(b->pack_blocks); cudaFree(b->head);
    cudaFree(b->ptab_d); cudaFree(b->sc_d);
    if (b->ptab_h) cudaFreeHost(b->ptab_h);
    if (b->sc_h) cudaFreeHost(b->sc_h);
    ppm_sort_scratch_free(&b->sort);
    cudaFree(b->cell_start); cudaFree(b->pack); cudaFree(b->rec0);
    cudaFree(b->rec1); cudaFree(b->aux); cudaFree(b->err);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_staged) cudaEventDestroy(b->ev_staged);
    if (b->ev_g0) cudaEventDestroy(b->ev_g0);
    if (b->ev_g1) cudaEventDestroy(b->ev_g1);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

// ---- kernels ---------------------------------------------------------------
__global__ void k_batch_geom(int P, const float* __restrict__ rmax, const float* __restrict__ cf,
                             const float* __restrict__ rmin, const IterScalars* __restrict__ sc,
                             uint32_t tmask, int lb, GridGeom* __restrict__ geom,
                             float* __restrict__ bound, float* __restrict__ rmax_next,
                             unsigned long long* __restrict__ counters, unsigned* __restrict__ head)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) *head = 0u;
    if (p >= P) return;
    float r = rmax[p];
    if (!(r > 0.f)) r = 1e-30f;
    geom[p] = ppm_make_geom(__fmul_rn(cf[p], r), tmask, lb, (uint32_t)p);
    // Eq. (radiusupdate) bound r_min sqrt((i+1)^(alpha-1)), FP64 then FP32
    bound[p] = (float)((double)rmin[p] * sc->bound_scale);
    rmax_next[p] = 0.f;
    counters[4 * p + 0] = 0ull;
    counters[4 * p + 1] = 0ull;
    counters[4 * p + 2] = 0ull;
}

// PSIMAX: also record each problem's largest tested value (traversal 3 only)
template <int NCH, bool VCM, bool PSIMAX>
__global__ void __launch_bounds__(256)
k_batch_pack(const int4* __restrict__ blocks, const PhotonPtrs* __restrict__ ptab,
             GridGeom* __restrict__ geom, uint32_t* __restrict__ keys,
             uint32_t* __restrict__ vals, float4* __restrict__ pack)
{
    // a photon's records side by side: x y z psi | (R G B rho_vm) | aux
    constexpr bool REC1 = NCH == 3 || VCM;
    constexpr int S = 2 + (REC1 ? 1 : 0);
    const int4 B = blocks[blockIdx.x];          // (problem, first local index, count, offset)
    const int i = B.y + threadIdx.x;
    const int p = B.x;
    __shared__ float s_w[8];
    float vmax = 0.f;
    if (i < B.z) {
    const PhotonPtrs pt = ptab[p];
    const GridGeom g = geom[p];
    const int64_t o = (int64_t)B.w + i;
    const float x = pt.pos[3ll * i], y = pt.pos[3ll * i + 1], z = pt.pos[3ll * i + 2];
    float R, G = 0.f, Bc = 0.f, psi;
    if (NCH == 3) {
        R = pt.flux[3ll * i]; G = pt.flux[3ll * i + 1]; Bc = pt.flux[3ll * i + 2];
        psi = fmaf(0.0722f, Bc, fmaf(0.7152f, G, __fmul_rn(0.2126f, R)));
    } else {
        R = pt.flux[i];
        psi = R;
    }
    float4* rec = pack + o * S;
    rec[0] = make_float4(x, y, z, psi);
    if constexpr (REC1) rec[1] = make_float4(R, G, Bc, VCM ? pt.rho[2ll * i] : 0.f);
    reinterpret_cast<uint4*>(rec)[S - 1] = make_uint4(pt.nq ? pt.nq[i] : 0u, VCM ? pt.wq[i] : 0u,
                                                      VCM ? __float_as_uint(pt.rho[2ll * i + 1]) : 0u,
                                                      (uint32_t)p);
    keys[o] = ppm_bucket(ppm_cell_coord(x, g.inv_hx), ppm_cell_coord(y, g.inv_h),
                         ppm_cell_coord(z, g.inv_h), g);
    vals[o] = (uint32_t)o;
    vmax = NCH == 3 ? fmaxf(fmaxf(psi, R), fmaxf(G, Bc)) : psi;
    }
    // every block holds photons of one problem: fold its max into that
    // problem's geometry (scale of the fixed-point group sums)
    if constexpr (PSIMAX) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = vmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_w[w]);
            atomicMax((int*)&geom[p].psimax, __float_as_int(fmaxf(m, 0.f)));
        }
    }
}

struct BatchArgs {
    const int4* tiles;         // (problem, h0, h_end, 0), heaviest first
    int ntiles;
    unsigned* head;
    const GridGeom* geom;
    const double* fc;
    const float2* fm;
    int fc_cap;
    float* rmax_next;
    unsigned long long* counters;
    const float* nvm;
    const float* bound;
    float k;
};

template <int NCH, int NTC, bool NORMALS, bool VCM, int MAPPING>
__global__ void __launch_bounds__(kThreads, kMinBlocks<MAPPING, NTC>)
k_batch_gather(GatherArgs a, BatchArgs bt)
{
    __shared__ BlockShared<NCH, NTC, MAPPING> bsh;
    __shared__ int s_tile;
    if (*a.err & 4) return;          // the grid's sort gave up: no usable grid
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(bt.head, 1u);
        __syncthreads();
        const int ti = s_tile;
        __syncthreads();
        if (ti >= bt.ntiles) break;
        const int4 T = bt.tiles[ti];
        const int p = T.x;
        Prob pr;
        pr.geom = bt.geom + p;
        pr.fc = bt.fc + (int64_t)p * (bt.fc_cap + 1);
        pr.fm = bt.fm + (int64_t)p * (bt.fc_cap + 1);
        pr.rmax_next = bt.rmax_next + p;
        pr.counters = bt.counters + 4 * p;
        pr.k = bt.k;
        pr.bound = bt.bound[p];
        pr.n_vm = bt.nvm[p];
        pr.fc_max = bt.fc_cap;
        pr.pid = (uint32_t)p;
        pr.inv_r0 = 0.f;
        pr.log_iter = 0.f;
        // a tile is one or more blocks' worth of hit points, done in turn
        for (int64_t h0 = T.y; h0 < T.z; h0 += kThreads)
            gather_block<NCH, NTC, NORMALS, VCM, MAPPING, true>(a, pr, h0, T.z, bsh);
    }
}

__global__ void k_batch_finish(int P, float* __restrict__ rmax, const float* __restrict__ rmax_next,
                               const unsigned long long* __restrict__ counters,
                               unsigned long long* __restrict__ pairs_total)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    rmax[p] = rmax_next[p];
    pairs_total[p] += counters[4 * p];
}

template <bool OUT>
__global__ void k_batch_state_io(int64_t n, int64_t off, int64_t nh, int ntc, int nch,
                                 const uint32_t* __restrict__ orig, float* r, int32_t* t, float* F,
                                 double* tau, uint32_t* cnt, float* S, float* Q, ppm_state_view v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t h = off + i;
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

__global__ void k_batch_radiance(int64_t n, int64_t off, int nch, const double* __restrict__ tau,
                                 const uint32_t* __restrict__ orig, double inv_iter, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t h = off + i;
    const int64_t o = orig[h];
    for (int c = 0; c < nch; ++c) out[o * nch + c] = (float)(tau[h * nch + c] * inv_iter);
}

// ---- the iteration ---------------------------------------------------------
// traversal 4 exists for one flux channel only
template <int NCH, int NTC, bool NORMALS, bool VCM>
void launch_batch_warp_per_hit(ppm_batch* b, const GatherArgs& a, const BatchArgs& bt)
{
    if constexpr (NCH == 1) k_batch_gather<1, NTC, NORMALS, VCM, 4><<<b->gather_grid, kThreads, 0, b->st>>>(a, bt);
}

template <int NCH, int NTC, bool NORMALS, bool VCM>
cudaError_t batch_warp_per_hit_occupancy(int* per_sm)
{
    if constexpr (NCH == 1)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_gather<1, NTC, NORMALS, VCM, 4>, kThreads, 0);
    return cudaErrorInvalidValue;
}

template <int NCH, int NTC, bool NORMALS, bool VCM>
int launch_batch_gather(ppm_batch* b, const GatherArgs& a, const BatchArgs& bt)
{
    const int m = b->prm.mapping;
    if (m == 1) k_batch_gather<NCH, NTC, NORMALS, VCM, 1><<<b->gather_grid, kThreads, 0, b->st>>>(a, bt);
    else if (m == 2) k_batch_gather<NCH, NTC, NORMALS, VCM, 2><<<b->gather_grid, kThreads, 0, b->st>>>(a, bt);
    else if (m == 3 && NTC == 1) k_batch_gather<NCH, 1, NORMALS, VCM, 3><<<b->gather_grid, kThreads, 0, b->st>>>(a, bt);
    else if (m == 4 && NCH == 1) launch_batch_warp_per_hit<NCH, NTC, NORMALS, VCM>(b, a, bt);
    else k_batch_gather<NCH, NTC, NORMALS, VCM, 0><<<b->gather_grid, kThreads, 0, b->st>>>(a, bt);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

template <int NCH, int NTC, bool NORMALS, bool VCM>
int gather_occupancy(ppm_batch* b)
{
    int per_sm = 0;
    const int m = b->prm.mapping;
    cudaError_t e;
    if (m == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_gather<NCH, NTC, NORMALS, VCM, 1>, kThreads, 0);
    else if (m == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_gather<NCH, NTC, NORMALS, VCM, 2>, kThreads, 0);
    else if (m == 3 && NTC == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_gather<NCH, 1, NORMALS, VCM, 3>, kThreads, 0);
    else if (m == 4 && NCH == 1) e = batch_warp_per_hit_occupancy<NCH, NTC, NORMALS, VCM>(&per_sm);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_gather<NCH, NTC, NORMALS, VCM, 0>, kThreads, 0);
    if (e != cudaSuccess) { cudaGetLastError(); return 1; }
    return per_sm > 0 ? per_sm : 1;
}

int run_gather(ppm_batch* b)
{
    GatherArgs a;
    a.nh = b->nh_total;
    a.hp_pos = b->hp_pos; a.hp_u = b->hp_u; a.hp_v = b->hp_v;
    a.r = b->r; a.t = b->t; a.F = b->F; a.tau = b->tau;
    a.cnt = b->cnt; a.S = b->S; a.Q = b->Q;
    a.cell_start = b->cell_start;
    // batches always carry the aux record: with rec1 the two sit side by side
    a.rec0 = b->rec0; a.rec1 = b->rec1;
    a.aux = (b->nch == 3 || b->prm.vcm) ? reinterpret_cast<const uint4*>(b->rec1 + 1) : b->aux;
    a.err = b->err;
    a.feat = nullptr;
    BatchArgs bt;
    bt.tiles = b->tiles; bt.ntiles = b->ntiles; bt.head = b->head;
    bt.geom = b->geom; bt.fc = b->fc; bt.fm = b->fm; bt.fc_cap = b->fc_cap;
    bt.rmax_next = b->rmax_next; bt.counters = b->counters;
    bt.nvm = b->nvm; bt.bound = b->bound; bt.k = b->prm.k;
    const bool nrm = b->normals, vcm = b->prm.vcm != 0;
    if (b->nch == 1) {
        if (vcm) return nrm ? launch_batch_gather<1, 1, true, true>(b, a, bt) : launch_batch_gather<1, 1, false, true>(b, a, bt);
        return nrm ? launch_batch_gather<1, 1, true, false>(b, a, bt) : launch_batch_gather<1, 1, false, false>(b, a, bt);
    }
    if (b->ntc == 3) {
        if (vcm) return nrm ? launch_batch_gather<3, 3, true, true>(b, a, bt) : launch_batch_gather<3, 3, false, true>(b, a, bt);
        return nrm ? launch_batch_gather<3, 3, true, false>(b, a, bt) : launch_batch_gather<3, 3, false, false>(b, a, bt);
    }
    if (vcm) return nrm ? launch_batch_gather<3, 1, true, true>(b, a, bt) : launch_batch_gather<3, 1, false, true>(b, a, bt);
    return nrm ? launch_batch_gather<3, 1, true, false>(b, a, bt) : launch_batch_gather<3, 1, false, false>(b, a, bt);
}

int occupancy(ppm_batch* b)
{
    const bool nrm = b->normals, vcm = b->prm.vcm != 0;
    if (b->nch == 1) {
        if (vcm) return nrm ? gather_occupancy<1, 1, true, true>(b) : gather_occupancy<1, 1, false, true>(b);
        return nrm ? gather_occupancy<1, 1, true, false>(b) : gather_occupancy<1, 1, false, false>(b);
    }
    if (b->ntc == 3) {
        if (vcm) return nrm ? gather_occupancy<3, 3, true, true>(b) : gather_occupancy<3, 3, false, true>(b);
        return nrm ? gather_occupancy<3, 3, true, false>(b) : gather_occupancy<3, 3, false, false>(b);
    }
    if (vcm) return nrm ? gather_occupancy<3, 1, true, true>(b) : gather_occupancy<3, 1, false, true>(b);
    return nrm ? gather_occupancy<3, 1, true, false>(b) : gather_occupancy<3, 1, false, false>(b);
}

// F_c and window-m tables of every problem for window lengths up to at
// least `upto` (doubling the capacity): new arrays, the old rows copied, the
// new entries computed; the captured graph holds the old pointers, so it is
// dropped and captured again by the next iteration
int grow_fc(ppm_batch* b, int upto)
{
    if (upto <= b->fc_cap) return PPM_OK;
    int cap = b->fc_cap > 0 ? b->fc_cap : kFcCap0;
    while (cap < upto) cap *= 2;
    const int P = b->P;
    double* nfc = nullptr;
    float2* nfm = nullptr;
    if (!dal(&nfc, (int64_t)P * (cap + 1))) return PPM_ENOMEM;
    if (!dal(&nfm, (int64_t)P * (cap + 1))) { cudaFree(nfc); return PPM_ENOMEM; }
    cudaStream_t st = b->st;
    int rc = PPM_OK;
    const int from = b->fc_cap + 1;
    if (b->fc) {
        if (!OKC(cudaMemcpy2DAsync(nfc, (cap + 1) * sizeof(double), b->fc, (b->fc_cap + 1) * sizeof(double),
                                   (b->fc_cap + 1) * sizeof(double), P, cudaMemcpyDeviceToDevice, st)) ||
            !OKC(cudaMemcpy2DAsync(nfm, (cap + 1) * sizeof(float2), b->fm, (b->fc_cap + 1) * sizeof(float2),
                                   (b->fc_cap + 1) * sizeof(float2), P, cudaMemcpyDeviceToDevice, st)))
            rc = PPM_ECUDA;
    } else {
        if (!OKC(cudaMemsetAsync(nfc, 0, (size_t)P * (cap + 1) * sizeof(double), st)) ||
            !OKC(cudaMemsetAsync(nfm, 0, (size_t)P * (cap + 1) * sizeof(float2), st)))
            rc = PPM_ECUDA;
    }
    for (int p = 0; p < P && rc == PPM_OK; ++p) {
        rc = ppm_fcrit_fill(nfc + (int64_t)p * (cap + 1), from, cap, (double)b->J[p], b->prm.alpha_f, st);
        if (rc == PPM_OK) rc = ppm_window_m_fill(nfm + (int64_t)p * (cap + 1), from, cap, (double)b->J[p], st);
    }
    if (rc == PPM_OK && !OKC(cudaStreamSynchronize(st))) rc = PPM_ECUDA;
    if (rc) { cudaFree(nfc); cudaFree(nfm); return rc; }
    cudaFree(b->fc);
    cudaFree(b->fm);
    b->fc = nfc;
    b->fm = nfm;
    b->fc_cap = cap;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    return PPM_OK;
}

// enqueue one whole iteration on b->st (captured into the graph)
int enqueue_iteration(ppm_batch* b)
{
    cudaStream_t st = b->st;
    int launches = 0;
    PPM_CUDA(cudaMemcpyAsync(b->ptab_d, b->ptab_h, b->P * sizeof(PhotonPtrs), cudaMemcpyHostToDevice, st));
    PPM_CUDA(cudaMemcpyAsync(b->sc_d, b->sc_h, sizeof(IterScalars), cudaMemcpyHostToDevice, st));
    // external event nodes (a plain record inside a capture would only be a
    // capture-internal dependency): the host waits on / times these
    PPM_CUDA(record_host_event(b->ev_staged, st));      // staging consumed
    const uint32_t T = 1u << b->tbits;
    k_batch_geom<<<(b->P + 127) / 128, 128, 0, st>>>(b->P, b->rmax, b->cf_dev, b->rmin_dev, b->sc_d,
                                                    T - 1, b->lb, b->geom, b->bound, b->rmax_next,
                                                    b->counters, b->head);
    PPM_LAUNCH_CHECK();
    ++launches;
    const int64_t n = b->np_total;
    if (n > 0) {
        const bool vcm = b->prm.vcm != 0;
        const bool pm = b->prm.mapping == 3;
        auto pack = [&](auto kern) {
            kern<<<b->npack, 256, 0, st>>>(b->pack_blocks, b->ptab_d, b->geom, b->sort.keys, b->sort.vals,
                                           b->pack);
        };
        if (b->nch == 3) {
            if (vcm) pm ? pack(k_batch_pack<3, true, true>) : pack(k_batch_pack<3, true, false>);
            else pm ? pack(k_batch_pack<3, false, true>) : pack(k_batch_pack<3, false, false>);
        } else {
            if (vcm) pm ? pack(k_batch_pack<1, true, true>) : pack(k_batch_pack<1, true, false>);
            else pm ? pack(k_batch_pack<1, false, true>) : pack(k_batch_pack<1, false, false>);
        }
        PPM_LAUNCH_CHECK();
        ++launches;
        // the ping-pong pointer sequence of the sort is recorded into the
        // graph as it is at capture time, so every replay is consistent
        int rc = ppm_radix_sort_pairs_lookback(&b->sort, n, b->tbits, b->err, st, b->prm.wait_limit);
        if (rc) return rc;
        launches += 2 + (b->tbits + 7) / 8;
    }
    int rc = ppm_cell_start_launch(b->sort.keys, n, T, b->cell_start, b->err, st);
    if (rc) return rc;
    ++launches;
    if (n > 0) {
        const bool rec1 = b->nch == 3 || b->prm.vcm;
        rc = ppm_permute_launch(n, b->sort.vals, b->pack, b->rec0, rec1 ? b->rec1 : nullptr, b->aux, b->err, st);
        if (rc) return rc;
        ++launches;
    }
    PPM_CUDA(record_host_event(b->ev_g0, st));
    if (b->nh_total > 0) {
        rc = run_gather(b);
        if (rc) return rc;
        ++launches;
    }
    PPM_CUDA(record_host_event(b->ev_g1, st));
    k_batch_finish<<<(b->P + 127) / 128, 128, 0, st>>>(b->P, b->rmax, b->rmax_next, b->counters, b->pairs_total);
    PPM_LAUNCH_CHECK();
    ++launches;
    b->launches = launches;
    return PPM_OK;
}

}  // namespace

extern "C" {

int ppm_batch_create(int32_t n_problems, const ppm_hitpoints* hp, const float* r0, const int64_t* J,
                     float alpha, const ppm_params* params, const float* cell_factor, void* stream,
                     ppm_batch** out)
{
    PPM_ENTRY();
    if (!out) return PPM_EINVAL;
    *out = nullptr;
    if (n_problems < 1 || n_problems > (1 << 20) || !hp || !r0 || !J) return PPM_EINVAL;
    if (!(alpha > 0.f && alpha < 1.f)) return PPM_EINVAL;
    ppm_params prm;
    if (params) prm = *params; else ppm_default_params(&prm);
    if (!(prm.k > 0.f && prm.k < 1.f) || !(prm.alpha_f > 0.0 && prm.alpha_f < 1.0)) return PPM_EINVAL;
    if (!(prm.rmin_ratio >= 0.f && prm.rmin_ratio < 1.f)) return PPM_EINVAL;
    if (prm.channels != 1 && prm.channels != 3) return PPM_EINVAL;
    if (prm.rgb_test && prm.channels != 3) return PPM_EINVAL;
    if (prm.mapping < 0 || prm.mapping > 4 || prm.n_vm < 0.f) return PPM_EINVAL;
    if ((prm.mapping == 3 && prm.rgb_test) || (prm.mapping == 4 && prm.channels == 3)) return PPM_EINVAL;
    if (prm.test != 0) return PPM_EINVAL;   // the count test runs in contexts only
    if (prm.tile < 0 || prm.tile > 1024 || prm.tile % kThreads != 0) return PPM_EINVAL;
    const int64_t tile_hits = prm.tile > 0 ? prm.tile : kThreads;
    const int P = n_problems;
    bool any_nq = false, all_nq = true;
    for (int p = 0; p < P; ++p) {
        if (hp[p].n < 0 || hp[p].n > 0x7fffffffll) return PPM_EINVAL;
        if (hp[p].n > 0 && (!hp[p].pos || !hp[p].u || !hp[p].v)) return PPM_EINVAL;
        if (prm.vcm && hp[p].n > 0 && (!hp[p].rho || !hp[p].nq)) return PPM_EINVAL;
        if (!(isfinite(r0[p]) && r0[p] > 0.f) || J[p] < 2) return PPM_EINVAL;
        const float cf = cell_factor ? cell_factor[p] : prm.cell_factor;
        if (!(cf >= 0.5f && cf <= 4.0f)) return PPM_EINVAL;
        if (hp[p].n > 0) { any_nq |= hp[p].nq != nullptr; all_nq &= hp[p].nq != nullptr; }
    }
    if (any_nq && !all_nq) return PPM_EINVAL;   // normals for every problem or none

    ppm_batch* b = new (std::nothrow) ppm_batch();
    if (!b) return PPM_ENOMEM;
    cudaGetDevice(&b->dev);
    b->user = (cudaStream_t)stream;
    b->prm = prm;
    b->alpha = alpha;
    b->P = P;
    b->nch = prm.channels;
    b->ntc = prm.rgb_test ? 3 : 1;
    b->normals = any_nq;
    b->hp_n.resize(P); b->hp_off.resize(P + 1); b->J.resize(P); b->ph_off.resize(P + 1);
    b->r0.resize(P); b->rmin.resize(P); b->cf.resize(P);
    int64_t off = 0, poff = 0;
    for (int p = 0; p < P; ++p) {
        b->hp_n[p] = hp[p].n;
        b->hp_off[p] = off;
        off += (hp[p].n + kThreads - 1) / kThreads * kThreads;   // problems start on a tile
        b->J[p] = J[p];
        b->ph_off[p] = poff;
        poff += J[p];
        b->r0[p] = r0[p];
        b->rmin[p] = prm.rmin_ratio * r0[p];
        b->cf[p] = cell_factor ? cell_factor[p] : prm.cell_factor;
    }
    b->hp_off[P] = off;
    b->ph_off[P] = poff;
    b->nh_total = off;
    b->np_total = poff;
    // tile and pack-block offsets are 32-bit
    if (poff > 0x7fffffffll || off > 0x7fffffffll) { free_batch(b); return PPM_EINVAL; }
    const int64_t nh = b->nh_total, np = b->np_total;
    int rc = PPM_OK;
    bool ok = dal(&b->hp_orig, nh) && dal(&b->hp_pos, nh) && dal(&b->hp_u, nh) && dal(&b->hp_v, nh) &&
              dal(&b->r, nh) && dal(&b->t, nh) && dal(&b->F, nh) && dal(&b->tau, nh * b->nch) &&
              dal(&b->cnt, nh * PPM_NG) && dal(&b->S, nh * PPM_NG * b->ntc) && dal(&b->Q, nh * PPM_NG * b->ntc) &&
              dal(&b->geom, P) && dal(&b->rmax, P) && dal(&b->rmax_next, P) && dal(&b->cf_dev, P) &&
              dal(&b->rmin_dev, P) && dal(&b->nvm, P) && dal(&b->bound, P) &&
              dal(&b->counters, 4ll * P) &&
              dal(&b->pairs_total, P) && dal(&b->head, 1) && dal(&b->ptab_d, P) && dal(&b->sc_d, 1) &&
              dal(&b->err, 1) && dal(&b->rec0, np) && dal(&b->aux, np) &&
              dal(&b->pack, np * ((b->nch == 3 || prm.vcm) ? 3 : 2));
    if (ok && (b->nch == 3 || prm.vcm)) ok = dal(&b->rec1, 2 * np);   // rec1 | aux side by side
    if (ok) ok = cudaMallocHost(&b->ptab_h, P * sizeof(PhotonPtrs)) == cudaSuccess &&
                 cudaMallocHost(&b->sc_h, sizeof(IterScalars)) == cudaSuccess;
    if (ok) ok = ppm_sort_scratch_reserve(&b->sort, np > 0 ? np : 1) == PPM_OK;
    b->tbits = ppm_table_bits(np, b->lb);
    if (ok) ok = dal(&b->cell_start, (int64_t)(1u << b->tbits) + 1);
    if (!ok) { cudaGetLastError(); free_batch(b); return PPM_ENOMEM; }
    if (!OKC(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking)) ||
        !OKC(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) ||
        !OKC(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) ||
        !OKC(cudaEventCreateWithFlags(&b->ev_staged, cudaEventDisableTiming)) ||
        !OKC(cudaEventCreate(&b->ev_g0)) || !OKC(cudaEventCreate(&b->ev_g1))) {
        cudaGetLastError(); free_batch(b); return PPM_ECUDA;
    }
    cudaStream_t st = b->st;
    do {
        // hit points of every problem into its slice, Hilbert-sorted
        for (int p = 0; p < P && rc == PPM_OK; ++p) {
            if (hp[p].n == 0) continue;
            const int64_t o = b->hp_off[p];
            rc = ppm_prepare_hitpoints(&hp[p], prm.vcm != 0, b->hp_orig + o, b->hp_pos + o,
                                       b->hp_u + o, b->hp_v + o, st);
        }
        if (rc) break;
        std::vector<float> rfill(nh, 0.f), nv(P);
        for (int p = 0; p < P; ++p) {
            for (int64_t i = 0; i < b->hp_n[p]; ++i) rfill[b->hp_off[p] + i] = r0[p];
            nv[p] = prm.n_vm > 0.f ? prm.n_vm : (float)J[p];
        }
        if (!OKC(cudaMemcpyAsync(b->r, rfill.data(), nh * sizeof(float), cudaMemcpyHostToDevice, st)) ||
            !OKC(cudaMemcpyAsync(b->rmax, b->r0.data(), P * sizeof(float), cudaMemcpyHostToDevice, st)) ||
            !OKC(cudaMemcpyAsync(b->cf_dev, b->cf.data(), P * sizeof(float), cudaMemcpyHostToDevice, st)) ||
            !OKC(cudaMemcpyAsync(b->rmin_dev, b->rmin.data(), P * sizeof(float), cudaMemcpyHostToDevice, st)) ||
            !OKC(cudaMemcpyAsync(b->nvm, nv.data(), P * sizeof(float), cudaMemcpyHostToDevice, st)) ||
            !OKC(cudaMemsetAsync(b->t, 0, nh * sizeof(int32_t), st)) ||
            !OKC(cudaMemsetAsync(b->F, 0, nh * sizeof(float), st)) ||
            !OKC(cudaMemsetAsync(b->tau, 0, nh * b->nch * sizeof(double), st)) ||
            !OKC(cudaMemsetAsync(b->cnt, 0, nh * PPM_NG * sizeof(uint32_t), st)) ||
            !OKC(cudaMemsetAsync(b->S, 0, nh * PPM_NG * b->ntc * sizeof(float), st)) ||
            !OKC(cudaMemsetAsync(b->Q, 0, nh * PPM_NG * b->ntc * sizeof(float), st)) ||
            !OKC(cudaMemsetAsync(b->pairs_total, 0, P * sizeof(unsigned long long), st)) ||
            !OKC(cudaMemsetAsync(b->err, 0, sizeof(int32_t), st)) ||
            !OKC(cudaStreamSynchronize(st))) { rc = PPM_ECUDA; break; }
        // F_c tables, one per problem (J differs)
        rc = grow_fc(b, kFcCap0);
        if (rc) break;
        // tiles of tile_hits hit points, problems with the most photons per disk
        // (J r0^2) first so the long tiles start early
        std::vector<int> order(P);
        for (int p = 0; p < P; ++p) order[p] = p;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return (double)J[x] * r0[x] * r0[x] > (double)J[y] * r0[y] * r0[y];
        });
        std::vector<int4> tiles;
        for (int p : order)
            for (int64_t h = 0; h < b->hp_n[p]; h += tile_hits) {
                const int64_t h0 = b->hp_off[p] + h;
                const int64_t he = b->hp_off[p] + std::min<int64_t>(b->hp_n[p], h + tile_hits);
                tiles.push_back(make_int4(p, (int)h0, (int)he, 0));
            }
        b->ntiles = (int)tiles.size();
        std::vector<int4> pblocks;
        for (int p = 0; p < P; ++p)
            for (int64_t i = 0; i < J[p]; i += 256)
                pblocks.push_back(make_int4(p, (int)i, (int)J[p], (int)b->ph_off[p]));
        b->npack = (int)pblocks.size();
        if (!dal(&b->tiles, b->ntiles) || !dal(&b->pack_blocks, b->npack)) { rc = PPM_ENOMEM; break; }
        if ((b->ntiles && !OKC(cudaMemcpyAsync(b->tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st))) ||
            (b->npack && !OKC(cudaMemcpyAsync(b->pack_blocks, pblocks.data(), pblocks.size() * sizeof(int4), cudaMemcpyHostToDevice, st))) ||
            !OKC(cudaStreamSynchronize(st))) { rc = PPM_ECUDA; break; }
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
        b->gather_grid = std::max(1, std::min(b->ntiles, sms * occupancy(b)));
    } while (0);
    if (rc) { cudaGetLastError(); free_batch(b); return rc; }
    *out = b;
    return PPM_OK;
}

int ppm_batch_iterate(ppm_batch* b, const ppm_photons* ph, int32_t iter)
{
    PPM_ENTRY();
    if (!b || !ph) return PPM_EINVAL;
    if (iter != b->iter + 1) return PPM_ESTATE;
    for (int p = 0; p < b->P; ++p) {
        const ppm_photons& q = ph[p];
        if (q.n != b->J[p] || q.J != b->J[p] || q.channels != b->nch) return PPM_EINVAL;
        if (q.n > 0 && (!q.pos || !q.flux)) return PPM_EINVAL;
        if (b->prm.vcm && q.n > 0 && (!q.rho || !q.wq)) return PPM_EINVAL;
        if (b->normals && q.n > 0 && !q.nq) return PPM_EINVAL;
    }
    // a window can reach length iter: keep the tables ahead of it (the last
    // launch must be done with the old tables first)
    if (iter > b->fc_cap) {
        PPM_CUDA(cudaStreamSynchronize(b->st));
        int rc = grow_fc(b, iter);
        if (rc) return rc;
    }
    // staging for this launch: wait until the previous launch has copied it
    PPM_CUDA(cudaEventSynchronize(b->ev_staged));
    for (int p = 0; p < b->P; ++p)
        b->ptab_h[p] = PhotonPtrs{ph[p].pos, ph[p].flux, b->normals ? ph[p].nq : nullptr,
                                  ph[p].rho, ph[p].wq, 0};
    b->sc_h->bound_scale = sqrt(pow((double)iter + 1.0, (double)b->alpha - 1.0));
    PPM_CUDA(cudaEventRecord(b->ev_in, b->user));
    PPM_CUDA(cudaStreamWaitEvent(b->st, b->ev_in, 0));
    if (b->iter == 0) {
        // first iteration eagerly (loads every module), then capture
        int rc = enqueue_iteration(b);
        if (rc) return rc;
    } else {
        if (!b->exec) {
            PPM_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_iteration(b);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(b->st, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) { ppm_note_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__); return PPM_ECUDA; }
            b->graph = g;
            PPM_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
        }
        PPM_CUDA(cudaGraphLaunch(b->exec, b->st));
    }
    PPM_CUDA(cudaEventRecord(b->ev_out, b->st));
    PPM_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    b->iter = iter;
    return PPM_OK;
}

int ppm_batch_radiance(ppm_batch* b, int32_t problem, float* out)
{
    PPM_ENTRY();
    if (!b || problem < 0 || problem >= b->P) return PPM_EINVAL;
    const int64_t n = b->hp_n[problem];
    if (n == 0) return PPM_OK;
    if (!out) return PPM_EINVAL;
    const double inv = b->iter > 0 ? 1.0 / b->iter : 0.0;
    PPM_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    k_batch_radiance<<<(unsigned)((n + 255) / 256), 256, 0, b->user>>>(n, b->hp_off[problem], b->nch, b->tau,
                                                                      b->hp_orig, inv, out);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_batch_get_state(ppm_batch* b, int32_t problem, const ppm_state_view* v)
{
    PPM_ENTRY();
    if (!b || !v || problem < 0 || problem >= b->P) return PPM_EINVAL;
    const int64_t n = b->hp_n[problem];
    PPM_CUDA(cudaStreamSynchronize(b->st));
    if (n > 0) {
        k_batch_state_io<true><<<(unsigned)((n + 255) / 256), 256, 0, b->st>>>(
            n, b->hp_off[problem], b->nh_total, b->ntc, b->nch, b->hp_orig, b->r, b->t, b->F, b->tau,
            b->cnt, b->S, b->Q, *v);
        PPM_LAUNCH_CHECK();
    }
    PPM_CUDA(cudaStreamSynchronize(b->st));
    int32_t err = 0;
    PPM_CUDA(cudaMemcpy(&err, b->err, sizeof(err), cudaMemcpyDeviceToHost));
    return ppm_flags_status(err);
}

int ppm_batch_stats(ppm_batch* b, ppm_iter_stats* out)
{
    PPM_ENTRY();
    if (!b || !out) return PPM_EINVAL;
    PPM_CUDA(cudaStreamSynchronize(b->st));
    std::vector<unsigned long long> cnt(4 * b->P), tot(b->P);
    std::vector<float> rm(b->P);
    std::vector<GridGeom> g(b->P);
    int32_t err = 0;
    float gms = -1.f;
    if (b->iter > 0 && cudaEventElapsedTime(&gms, b->ev_g0, b->ev_g1) != cudaSuccess) {
        cudaGetLastError();
        gms = -1.f;
    }
    PPM_CUDA(cudaMemcpy(cnt.data(), b->counters, cnt.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    PPM_CUDA(cudaMemcpy(tot.data(), b->pairs_total, tot.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    PPM_CUDA(cudaMemcpy(rm.data(), b->rmax, rm.size() * sizeof(float), cudaMemcpyDeviceToHost));
    PPM_CUDA(cudaMemcpy(g.data(), b->geom, g.size() * sizeof(GridGeom), cudaMemcpyDeviceToHost));
    PPM_CUDA(cudaMemcpy(&err, b->err, sizeof(err), cudaMemcpyDeviceToHost));
    for (int p = 0; p < b->P; ++p) {
        ppm_iter_stats& s = out[p];
        memset(&s, 0, sizeof(s));
        s.iter = b->iter;
        s.flags = err;
        s.pairs = (int64_t)cnt[4 * p];
        s.candidates = (int64_t)cnt[4 * p + 1];
        s.rejects = (int64_t)cnt[4 * p + 2];
        s.pairs_total = (int64_t)tot[p];
        s.r_max = rm[p];
        s.cell = g[p].h;
        s.launches = b->launches;
        s.gather_ms = gms;
    }
    return ppm_flags_status(err);
}

int ppm_batch_graph_ready(ppm_batch* b)
{
    return b && b->exec ? 1 : 0;
}

void ppm_batch_destroy(ppm_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->st);
    free_batch(b);
}

}  // extern "C"
