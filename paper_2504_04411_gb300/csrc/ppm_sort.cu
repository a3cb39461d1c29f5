// ppm_sort.cu -- stable LSD radix sort of (uint32 key, uint32 value) pairs
// and a device-wide exclusive scan, used to build the photon grid (cell key
// + stable radix sort) and to sort hit points spatially.
//
// One pass per 8-bit digit, three kernels per pass:
//   hist    : per 2048-key tile, the digit histogram, stored digit-major
//             (hist[d * ntiles + tile]) so that ...
//   scan    : ... one flat exclusive scan gives every (digit, tile) its
//             global output offset;
//   scatter : each warp ranks its 256 keys with __match_any_sync (peers with
//             the same digit) in input order, warps are combined per digit in
//             warp order, so equal digits keep their input order (stable).
#include "ppm_internal.cuh"

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kTile = kSortThreads * kSortItems;   // 2048 keys per tile
constexpr int kWarps = kSortThreads / 32;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
             uint32_t mask, uint32_t* __restrict__ hist, int ntiles)
{
    __shared__ uint32_t s_h[kWarps][256];
    const int tid = threadIdx.x, w = tid >> 5;
    for (int i = tid; i < kWarps * 256; i += kSortThreads) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        int64_t idx = base + (int64_t)j * kSortThreads + tid;
        if (idx < n) atomicAdd(&s_h[w][(keys[idx] >> shift) & mask], 1u);
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) tot += s_h[ww][tid];
    hist[(int64_t)tid * ntiles + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                int64_t n, int shift, uint32_t mask,
                const uint32_t* __restrict__ offs, int ntiles)
{
    __shared__ uint32_t s_cnt[kWarps][256];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = lane; i < 256; i += 32) s_cnt[w][i] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)w * (32 * kSortItems);
    uint32_t k[kSortItems], v[kSortItems], d[kSortItems], rank[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t idx = base + j * 32 + lane;
        const bool valid = idx < n;
        k[j] = valid ? kin[idx] : 0u;
        v[j] = valid ? vin[idx] : 0u;
        d[j] = valid ? ((k[j] >> shift) & mask) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d[j]);
        const uint32_t before = __popc(peers & lt);
        const uint32_t c = valid ? s_cnt[w][d[j]] : 0u;
        rank[j] = c + before;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) s_cnt[w][d[j]] = c + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // per digit: global offset of this tile + counts of earlier warps
        const int dg = tid;
        uint32_t run = offs[(int64_t)dg * ntiles + blockIdx.x];
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t c = s_cnt[ww][dg];
            s_cnt[ww][dg] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        if (d[j] < 256u) {
            const uint32_t pos = s_cnt[w][d[j]] + rank[j];
            kout[pos] = k[j];
            vout[pos] = v[j];
        }
    }
}

// ---- scan ------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of one tile held as kScanItems consecutive values per
// thread; returns the tile total.  Writes results back into `vals`.
__device__ uint32_t block_excl_scan_tile(uint32_t (&vals)[kScanItems], uint32_t carry)
{
    __shared__ uint32_t s_w[kScanThreads / 32];
    __shared__ uint32_t s_tot;
    uint32_t loc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) { uint32_t x = vals[i]; vals[i] = loc; loc += x; }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(loc);
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = lane < kScanThreads / 32 ? s_w[lane] : 0u;
        uint32_t y = warp_incl_scan(x);
        if (lane < kScanThreads / 32) s_w[lane] = y - x;
        if (lane == kScanThreads / 32 - 1) s_tot = y;
    }
    __syncthreads();
    const uint32_t off = carry + s_w[w] + (inc - loc);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) vals[i] += off;
    const uint32_t tot = s_tot;
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t* __restrict__ data, int64_t n, uint32_t* __restrict__ partials)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t idx = base + i;
        if (idx < n) s += data[idx];
    }
    __shared__ uint32_t s_w[kScanThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kScanThreads / 32; ++i) t += s_w[i];
        partials[blockIdx.x] = t;
    }
}

// Single block: exclusive scan of the block partials, any count.
__global__ void __launch_bounds__(kScanThreads)
k_scan_partials(uint32_t* __restrict__ partials, int64_t nb)
{
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanTile) {
        uint32_t v[kScanItems];
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
            v[i] = idx < nb ? partials[idx] : 0u;
        }
        uint32_t tot = block_excl_scan_tile(v, carry);
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
            if (idx < nb) partials[idx] = v[i];
        }
        carry += tot;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(uint32_t* __restrict__ data, int64_t n, const uint32_t* __restrict__ partials)
{
    __shared__ uint32_t s_d[kScanTile];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t idx = base + i;
        s_d[i] = idx < n ? data[idx] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] = s_d[threadIdx.x * kScanItems + i];
    block_excl_scan_tile(v, partials[blockIdx.x]);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) s_d[threadIdx.x * kScanItems + i] = v[i];
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t idx = base + i;
        if (idx < n) data[idx] = s_d[i];
    }
}

}  // namespace

int ppm_exclusive_scan_u32(uint32_t* data, int64_t n, uint32_t* partials, cudaStream_t st)
{
    if (n <= 0) return PPM_OK;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, partials);
    PPM_LAUNCH_CHECK();
    k_scan_partials<<<1, kScanThreads, 0, st>>>(partials, nb);
    PPM_LAUNCH_CHECK();
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, partials);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_sort_scratch_reserve(SortScratch* s, int64_t n)
{
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int64_t hist = 256 * (ntiles > 0 ? ntiles : 1);
    const int64_t part = hist / kScanTile + 2;
    if (n > s->cap) {
        cudaFree(s->keys); cudaFree(s->vals); cudaFree(s->keys_alt); cudaFree(s->vals_alt);
        s->keys = s->vals = s->keys_alt = s->vals_alt = nullptr;
        s->cap = 0;
        const int64_t cap = n + n / 4 + 1024;
        if (cudaMalloc(&s->keys, cap * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&s->vals, cap * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&s->keys_alt, cap * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&s->vals_alt, cap * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return PPM_ENOMEM;
        }
        s->cap = cap;
    }
    if (hist > s->hist_cap) {
        cudaFree(s->hist); s->hist = nullptr; s->hist_cap = 0;
        const int64_t cap = hist + hist / 4 + 256;
        if (cudaMalloc(&s->hist, cap * sizeof(uint32_t)) != cudaSuccess) { cudaGetLastError(); return PPM_ENOMEM; }
        s->hist_cap = cap;
    }
    if (part > s->part_cap) {
        cudaFree(s->partials); s->partials = nullptr; s->part_cap = 0;
        const int64_t cap = part + 64;
        if (cudaMalloc(&s->partials, cap * sizeof(uint32_t)) != cudaSuccess) { cudaGetLastError(); return PPM_ENOMEM; }
        s->part_cap = cap;
    }
    return PPM_OK;
}

void ppm_sort_scratch_free(SortScratch* s)
{
    cudaFree(s->keys); cudaFree(s->vals); cudaFree(s->keys_alt); cudaFree(s->vals_alt);
    cudaFree(s->hist); cudaFree(s->partials);
    *s = SortScratch{};
}

int ppm_radix_sort_pairs(SortScratch* s, int64_t n, int bits, cudaStream_t st)
{
    if (n <= 1 || bits <= 0) return PPM_OK;
    if (n > 0xFFFFFFFFll || bits > 32 || n > s->cap) return PPM_EINVAL;
    const int ntiles = (int)((n + kTile - 1) / kTile);
    for (int shift = 0; shift < bits; shift += 8) {
        const int nb = bits - shift < 8 ? bits - shift : 8;
        const uint32_t mask = (1u << nb) - 1u;
        k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(s->keys, n, shift, mask, s->hist, ntiles);
        PPM_LAUNCH_CHECK();
        int rc = ppm_exclusive_scan_u32(s->hist, 256ll * ntiles, s->partials, st);
        if (rc) return rc;
        k_radix_scatter<<<ntiles, kSortThreads, 0, st>>>(s->keys, s->vals, s->keys_alt, s->vals_alt,
                                                          n, shift, mask, s->hist, ntiles);
        PPM_LAUNCH_CHECK();
        uint32_t* t;
        t = s->keys; s->keys = s->keys_alt; s->keys_alt = t;
        t = s->vals; s->vals = s->vals_alt; s->vals_alt = t;
    }
    return PPM_OK;
}
