// ppm_internal.cuh -- shared declarations of the libppm CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ppm.h"

#define PPM_NG 12

// Return PPM_ECUDA from the enclosing function if a runtime call fails
// (the thread's last-error slot is cleared so later checks are not fooled).
#define PPM_CUDA(call)                                                       \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) { ppm_note_cuda_error(e_, #call, __FILE__, __LINE__); cudaGetLastError(); return PPM_ECUDA; } \
    } while (0)

// Launch checks read the thread's last-error slot, which other code in the
// process may have left set: every entry point clears it first.
#define PPM_ENTRY() ((void)cudaGetLastError())

#define PPM_LAUNCH_CHECK()                                                   \
    do {                                                                     \
        cudaError_t e_ = cudaGetLastError();                                 \
        if (e_ != cudaSuccess) { ppm_note_cuda_error(e_, "launch", __FILE__, __LINE__); return PPM_ECUDA; } \
    } while (0)

void ppm_note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// The return code that a call reporting the device error flags gives:
// bit 2 (a bounded device wait gave up) before bit 0 (a gather skipped
// cells); bit 1 (a window clamped to the F_c table) is only reported.
inline int ppm_flags_status(int32_t flags)
{
    return (flags & 4) ? PPM_ETIMEOUT : ((flags & 1) ? PPM_EINCOMPLETE : PPM_OK);
}

// ---------------------------------------------------------------------------
// Grid: a uniform grid of cell edge h along y and z and h / 2^sx along x
// (kXSplit = sx), hashed into T = 2^tbits buckets.  A row of cells along x
// is what the gather walks and trims to the sphere's chord, so the finer x
// edge cuts the photons tested at the row ends without adding rows.  Cells
// are grouped in blocks of Bx x B x B (B = 2^lb, Bx = 2^(lb + sx), the same
// extent B h along every axis); the low bits of a bucket are the cell's
// coordinates inside its block, the high bits a hash of the block
// coordinates.  Two consequences the gather relies on:
//   * distinct cells less than a block apart along every axis never share
//     a bucket, so a hit point whose sphere spans <= Bx cells along x and
//     <= B along y and z visits each bucket at most once (no duplicate
//     gathering);
//   * cells consecutive along x inside one block have consecutive buckets,
//     so a run of them is one contiguous range of the sorted photons.
// ---------------------------------------------------------------------------
constexpr int kXSplit = 1;

struct GridGeom {
    float inv_h;       // 1 / cell edge along y and z
    float h;           // cell edge along y and z
    uint32_t tmask;    // T - 1
    int32_t lb;        // log2 of the block edge in cells along y and z (2 to 4)
    uint32_t pid;      // problem id mixed into the hash (0 for one problem)
    float psimax;      // largest tested value psi of the grid's photons (>= 0)
    float inv_hx;      // 1 / cell edge along x (2^sx / h)
    int32_t sx;        // log2 of the x split
};

// cells a block spans along x
__device__ __forceinline__ int ppm_block_x(const GridGeom& g) { return 1 << (g.lb + g.sx); }

// the geometry of a cell edge h (both grid builders fill it the same way)
__device__ __forceinline__ GridGeom ppm_make_geom(float h, uint32_t tmask, int lb, uint32_t pid)
{
    GridGeom o;
    o.h = h;
    o.inv_h = __frcp_rn(h);
    o.tmask = tmask;
    o.lb = lb;
    o.pid = pid;
    o.psimax = 0.f;
    o.sx = kXSplit;
    o.inv_hx = __frcp_rn(__fmul_rn(h, 1.0f / (float)(1 << kXSplit)));
    return o;
}

__device__ __forceinline__ uint32_t ppm_fmix32(uint32_t x)
{
    // 32-bit finalizer of MurmurHash3 (Appleby): a bijective avalanche mix.
    x ^= x >> 16; x *= 0x85ebca6bu;
    x ^= x >> 13; x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ int ppm_cell_coord(float p, float inv_h)
{
    float c = floorf(__fmul_rn(p, inv_h));
    c = fminf(fmaxf(c, -1073741824.0f), 1073741824.0f);
    return (int)c;
}

__device__ __forceinline__ uint32_t ppm_bucket(int ix, int iy, int iz, const GridGeom& g)
{
    const int lb = g.lb, lx = g.lb + g.sx;
    const uint32_t m = (1u << lb) - 1u, mx = (1u << lx) - 1u;
    uint32_t local = ((uint32_t)ix & mx) | (((uint32_t)iy & m) << lx) | (((uint32_t)iz & m) << (lx + lb));
    uint32_t bx = (uint32_t)(ix >> lx), by = (uint32_t)(iy >> lb), bz = (uint32_t)(iz >> lb);
    uint32_t hb = ppm_fmix32(bx * 0x9E3779B1u ^ ppm_fmix32(by * 0x85EBCA77u ^
                              ppm_fmix32(bz + 0x27D4EB2Fu + g.pid * 0x632BE59Bu)));
    return ((hb << (lx + 2 * lb)) | local) & g.tmask;
}

// Photon records in cell order.  rec0 = (x, y, z, psi) where psi is the
// tested value of the photon before any VCM+ weight: the flux (1 channel)
// or its luminance (3 channels).  rec1 = (R, G, B, rho_vm_l) for 3-channel
// or VCM+ photons.  aux = (nq, wq, rho_vc_l bits, 0) when normals or VCM+.

// ---------------------------------------------------------------------------
// Device-wide primitives (ppm_sort.cu)
// ---------------------------------------------------------------------------
// Owner of the (key, value) arrays being sorted and of the sort's scratch:
// both ping-pong pairs share one capacity, so swapping them is always safe.
struct SortScratch {
    uint32_t* keys = nullptr;
    uint32_t* vals = nullptr;
    uint32_t* keys_alt = nullptr;
    uint32_t* vals_alt = nullptr;
    uint32_t* hist = nullptr;       // 256 * ntiles
    uint32_t* partials = nullptr;   // scan block partials
    unsigned long long* status = nullptr;   // look-back words (single-pass form)
    uint32_t* digit = nullptr;      // 4 x 256 digit counts / offsets (single-pass form)
    int64_t cap = 0;                // elements of each key/value array
    int64_t hist_cap = 0;
    int64_t part_cap = 0;
    int64_t status_cap = 0;
};

// Stable LSD radix sort of (s->keys, s->vals)[0, n) on the low `bits` bits
// of the keys; the sorted pairs end up in (s->keys, s->vals) again (the
// pointers are swapped with the alternates after each 8-bit pass).
// Requires ppm_sort_scratch_reserve(s, >= n) first.
int ppm_radix_sort_pairs(SortScratch* s, int64_t n, int bits, cudaStream_t st);
// The same sort in one kernel per pass (decoupled look-back between the
// blocks of a pass; the counts of every pass first).  A look-back wait that
// gives up after spin_limit polls (0: the default 2^22; it should never
// happen) sets bit 2 of *err (device); every write stays inside [0, n), but
// the keys and values are then no permutation of the input.  Launches 2 +
// ceil(bits / 8) kernels.
int ppm_radix_sort_pairs_lookback(SortScratch* s, int64_t n, int bits, int32_t* err, cudaStream_t st,
                                  int spin_limit = 0);
int ppm_sort_scratch_reserve(SortScratch* s, int64_t n);
void ppm_sort_scratch_free(SortScratch* s);

// Exclusive prefix sum of n uint32 in place (partials: >= ceil(n/4096)+1).
int ppm_exclusive_scan_u32(uint32_t* data, int64_t n, uint32_t* partials,
                           cudaStream_t st);

// ---------------------------------------------------------------------------
// F critical values (ppm_fcrit.cu)
// ---------------------------------------------------------------------------
int ppm_fcrit_fill(double* table, int t_from, int t_to, double J, double alpha,
                   cudaStream_t st);
// every entry t_from .. t_to = the (1 - alpha) quantile of chi^2(k)
int ppm_chi2_fill(double* table, int t_from, int t_to, double k, double alpha, cudaStream_t st);
// mtab[t] = (1/m, 12 (m-1) / (11 m)) with m = t J samples per group, from FP64
int ppm_window_m_fill(float2* mtab, int t_from, int t_to, double J, cudaStream_t st);

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct ppm_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    ppm_params prm{};
    float r0 = 0.f, alpha = 0.75f, r_min = 0.f;
    int64_t nh = 0;
    int ntc = 1;          // tested channels
    int nch = 1;          // flux channels
    bool normals = false; // hit points carry normals
    // hit points, spatially sorted
    uint32_t* hp_orig = nullptr;  // sorted index -> caller index
    float4* hp_pos = nullptr;     // x, y, z, nq bits
    float4* hp_u = nullptr;       // ux, uy, uz, rho_vm_h
    float4* hp_v = nullptr;       // vx, vy, vz, rho_vc_h
    // state
    float* r = nullptr;
    int32_t* t = nullptr;
    float* F = nullptr;
    double* tau = nullptr;        // nh * nch
    uint32_t* cnt = nullptr;      // [12][nh]
    float* S = nullptr;           // [ntc][12][nh]
    float* Q = nullptr;           // [ntc][12][nh]
    // grid
    int64_t ph_cap = 0;
    int64_t n_ph = 0;             // photons in the current grid
    int64_t J = 0;                // light paths per iteration (fixed)
    int tbits = 0;
    uint32_t* cell_start = nullptr;   // T + 1
    int64_t cs_cap = 0;
    float4* rec0 = nullptr;
    float4* rec1 = nullptr;
    uint4* aux = nullptr;
    float4* pack = nullptr;       // unsorted records, a photon's side by side
    SortScratch sort;
    GridGeom* geom_dev = nullptr;     // written on the device by the build
    int lb = 2;
    bool grid_valid = false;
    bool ph_aux = false;              // photon records carry the aux word
    bool use_normals = false;         // same-surface filter this iteration
    // radius bookkeeping: rmax[cur] is the max radius the current grid was
    // built for; the update writes rmax[cur ^ 1]
    float* rmax = nullptr;        // 2 floats
    int rmax_cur = 0;
    // F_c table, indexed by window length t' (1-based), and the F statistic's
    // factors of m = t' J for the same t' (ppm_window_m_fill)
    double* fc = nullptr;
    float2* fm = nullptr;
    int fc_cap = 0;
    int fc_upto = 0;
    // counters: [0] pairs, [1] candidates, [2] rejects, [3] pairs_total
    unsigned long long* counters = nullptr;
    int32_t* err_dev = nullptr;       // device error flags (bit 0: span > block)
    int32_t iter = 0;
    int32_t launches_build = 0;       // kernels launched by the last build
    int32_t launches_iter = 0;        // ... by the last build + gather
    // learned radius proposer (ppm_mlp.cu)
    float* feat = nullptr;            // [12][nh] features of the last test
    const void* mlp = nullptr;        // caller-owned weight blob (device) or NULL
    float mlp_threshold = 0.5f;
    float mlp_max_shrink = 0.1f;
    // host-fed iterations (ppm_iterate_host): two device photon buffers used
    // in turn, filled on a private copy stream; counters land in pinned memory
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};   // slot filled (copy stream)
    cudaEvent_t ev_used[2] = {nullptr, nullptr};     // slot read by its build
    cudaEvent_t ev_stats[2] = {nullptr, nullptr};    // counters copied out
    unsigned char* hbuf[2] = {nullptr, nullptr};     // pos | flux | nq | rho | wq
    int64_t hbuf_cap = 0;                            // photons per slot
    struct HostStats {
        unsigned long long cnt[5];
        float r_max;
        float cell;
        int32_t err;
        int32_t pad;
    }* hstats = nullptr;                             // [2], page-locked
    int32_t host_iter[2] = {0, 0};
    int32_t host_launches[2] = {0, 0};
    int host_slot = 0;
};

// ppm_grid.cu / ppm_gather.cu
int ppm_grid_build(ppm_ctx* c, const ppm_photons* ph);
// bucket-table size for n photons and hash blocks of 2^lb cells per axis
int ppm_table_bits(int64_t n, int lb);
// cell_start[b] = first sorted photon with bucket >= b, b in [0, T]; no
// writes when *err (device) has bit 2 (the sort's look-back gave up)
int ppm_cell_start_launch(const uint32_t* keys, int64_t n, uint32_t T, uint32_t* cell_start,
                          const int32_t* err, cudaStream_t st);
// packed records gathered into sorted order (rec1 / aux when non-NULL);
// nothing when *err has bit 2
int ppm_permute_launch(int64_t n, const uint32_t* vals, const float4* pack, float4* rec0, float4* rec1,
                       uint4* aux, const int32_t* err, cudaStream_t st);
// ppm_api.cu: hit points -> Hilbert-sorted internal layout (synchronizes st)
int ppm_prepare_hitpoints(const ppm_hitpoints* hp, bool with_rho, uint32_t* orig, float4* pos,
                          float4* u, float4* v, cudaStream_t st);
int ppm_gather_launch(ppm_ctx* c, float bound);
int ppm_radiance_launch(ppm_ctx* c, float* out);
// learned proposer after the F-test update of iteration c->iter
int ppm_mlp_propose_launch(ppm_ctx* c, float bound);
