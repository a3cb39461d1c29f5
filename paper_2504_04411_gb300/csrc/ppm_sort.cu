// ppm_sort.cu -- stable LSD radix sort of (uint32 key, uint32 value) pairs
// and a device-wide exclusive scan, used to build the photon grid (cell key
// + stable radix sort) and to sort hit points spatially.
//
// Two forms of the same sort (same output: both are stable).
//
// Three kernels per 8-bit pass (ppm_radix_sort_pairs; no block waits for
// another):
//   hist    : per 2048-key tile, the digit histogram, stored digit-major
//             (hist[d * ntiles + tile]) so that ...
//   scan    : ... one flat exclusive scan gives every (digit, tile) its
//             global output offset;
//   scatter : each warp ranks its 256 keys with __match_any_sync (peers with
//             the same digit) in input order, warps are combined per digit in
//             warp order, so equal digits keep their input order (stable).
//
// One kernel per pass after one counting pass for all of them
// (ppm_radix_sort_pairs_lookback, used by the grid builds):
//   counts  : every pass's global digit counts in one read of the keys, and
//             their exclusive scans (one block);
//   onesweep: each block takes the next tile number from a counter, ranks
//             its tile as the scatter above does, and finds, per digit, how
//             many keys of that digit earlier tiles hold by decoupled
//             look-back: it publishes its own count at once (flag
//             AGGREGATE), then walks back over earlier tiles' words adding
//             counts until one carries an INCLUSIVE prefix, and publishes
//             its own inclusive prefix.  A tile only waits for tiles with
//             lower numbers, which took theirs earlier and are running, so
//             every wait ends; each is still capped (kSpinLimit polls),
//             after which bit 2 of *err is set and the order is unspecified.
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

// ---- single-pass form ------------------------------------------------------
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagInclusive = 2ull << 62;
constexpr unsigned long long kCountMask = (1ull << 62) - 1ull;
constexpr int kSpinLimit = 1 << 22;
constexpr int kStatusHead = 32;          // words before the per-tile words: [0] tile counter
constexpr int kSweepItems = 8;           // keys a thread in the single-pass kernel
constexpr int kSweepTile = kSortThreads * kSweepItems;
constexpr int kLookBack = 4;             // earlier tiles' words a look-back round trip reads

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// every pass's digit counts (counts[p * 256 + d], zeroed by the caller)
__global__ void __launch_bounds__(kSortThreads)
k_digit_counts(const uint32_t* __restrict__ keys, int64_t n, int bits, uint32_t* __restrict__ counts)
{
    __shared__ uint32_t s_c[4][256];
    const int npass = (bits + 7) / 8;
    for (int i = threadIdx.x; i < 4 * 256; i += kSortThreads) (&s_c[0][0])[i] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kSortThreads) {
        const uint32_t k = keys[i];
        for (int p = 0; p < npass; ++p) {
            const int nb = bits - 8 * p < 8 ? bits - 8 * p : 8;
            atomicAdd(&s_c[p][(k >> (8 * p)) & ((1u << nb) - 1u)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += kSortThreads) {
        const uint32_t v = (&s_c[0][0])[i];
        if (v) atomicAdd(counts + i, v);
    }
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x);

// counts[p][d] -> exclusive prefix over d, per pass (one block of 256)
__global__ void __launch_bounds__(256)
k_digit_offsets(uint32_t* __restrict__ counts, int npass)
{
    __shared__ uint32_t s_w[8];
    const int d = threadIdx.x, lane = d & 31, w = d >> 5;
    for (int p = 0; p < npass; ++p) {
        const uint32_t x = counts[p * 256 + d];
        const uint32_t inc = warp_incl_scan(x);
        if (lane == 31) s_w[w] = inc;
        __syncthreads();
        uint32_t before = 0;
        for (int ww = 0; ww < w; ++ww) before += s_w[ww];
        counts[p * 256 + d] = before + inc - x;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_onesweep(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                 uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                 uint32_t mask, const uint32_t* __restrict__ goff, unsigned long long* status,
                 int32_t* err, int spin_limit)
{
    __shared__ uint32_t s_cnt[kWarps][256];
    __shared__ uint32_t s_base[256];
    __shared__ int s_t;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (tid == 0) s_t = (int)atomicAdd(reinterpret_cast<unsigned*>(status), 1u);
    for (int i = lane; i < 256; i += 32) s_cnt[w][i] = 0;
    __syncthreads();
    const int t = s_t;
    // rank the tile's keys in input order (as k_radix_scatter)
    const int64_t base = (int64_t)t * kSweepTile + (int64_t)w * (32 * kSweepItems);
    uint32_t k[kSweepItems], v[kSweepItems], d[kSweepItems], rank[kSweepItems];
#pragma unroll
    for (int j = 0; j < kSweepItems; ++j) {
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
    {   // digit dg: the tile's count, per-warp prefixes, then earlier tiles by look-back
        const int dg = tid;
        uint32_t local = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t c = s_cnt[ww][dg];
            s_cnt[ww][dg] = local;
            local += c;
        }
        unsigned long long* word = status + kStatusHead;
        unsigned long long excl = 0;
        if (t == 0) {
            st_relaxed_u64(word + dg, kFlagInclusive | local);
        } else {
            st_relaxed_u64(word + (int64_t)t * 256 + dg, kFlagAggregate | local);
            // kLookBack earlier tiles' words per round trip, consumed from
            // the nearest one back to the first INCLUSIVE one or the first
            // one not yet published (waited for, then read again)
            int q = t - 1, spins = 0;
            bool found = false;
            while (!found) {
                unsigned long long x[kLookBack];
#pragma unroll
                for (int i = 0; i < kLookBack; ++i)
                    x[i] = q - i >= 0 ? ld_relaxed_u64(word + (int64_t)(q - i) * 256 + dg) : kFlagInclusive;
                int used = 0;
                bool stop = false;
#pragma unroll
                for (int i = 0; i < kLookBack; ++i) {
                    if (!stop) {
                        const unsigned long long f = x[i] & ~kCountMask;
                        if (f == 0ull) {
                            stop = true;
                        } else {
                            excl += x[i] & kCountMask;
                            ++used;
                            if (f == kFlagInclusive) stop = found = true;
                        }
                    }
                }
                q -= used;
                if (!found && used < kLookBack) {
                    if (++spins > spin_limit) { atomicOr(err, 4); break; }
                    __nanosleep(32);
                }
            }
            st_relaxed_u64(word + (int64_t)t * 256 + dg, kFlagInclusive | (excl + local));
        }
        s_base[dg] = goff[dg] + (uint32_t)excl;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSweepItems; ++j) {
        if (d[j] < 256u) {
            // positions are in [0, n) unless a look-back wait gave up
            const uint32_t pos = s_base[d[j]] + s_cnt[w][d[j]] + rank[j];
            if ((int64_t)pos < n) {
                kout[pos] = k[j];
                vout[pos] = v[j];
            }
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
    const int64_t words = kStatusHead + 256 * (ntiles > 0 ? ntiles : 1);
    if (words > s->status_cap) {
        cudaFree(s->status); s->status = nullptr; s->status_cap = 0;
        const int64_t cap = words + words / 4 + 256;
        if (cudaMalloc(&s->status, cap * sizeof(unsigned long long)) != cudaSuccess) { cudaGetLastError(); return PPM_ENOMEM; }
        s->status_cap = cap;
    }
    if (!s->digit) {
        if (cudaMalloc(&s->digit, 4 * 256 * sizeof(uint32_t)) != cudaSuccess) { cudaGetLastError(); return PPM_ENOMEM; }
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
    cudaFree(s->hist); cudaFree(s->partials); cudaFree(s->status); cudaFree(s->digit);
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

int ppm_radix_sort_pairs_lookback(SortScratch* s, int64_t n, int bits, int32_t* err, cudaStream_t st,
                                  int spin_limit)
{
    if (spin_limit <= 0) spin_limit = kSpinLimit;
    if (n <= 1 || bits <= 0) return PPM_OK;
    if (n > 0xFFFFFFFFll || bits > 32 || n > s->cap || !s->status || !s->digit || !err) return PPM_EINVAL;
    const int ntiles = (int)((n + kSweepTile - 1) / kSweepTile);
    if (kStatusHead + 256ll * ntiles > s->status_cap) return PPM_EINVAL;
    const int npass = (bits + 7) / 8;
    PPM_CUDA(cudaMemsetAsync(s->digit, 0, (size_t)npass * 256 * sizeof(uint32_t), st));
    const int cblocks = ntiles < 1024 ? ntiles : 1024;
    k_digit_counts<<<cblocks, kSortThreads, 0, st>>>(s->keys, n, bits, s->digit);
    PPM_LAUNCH_CHECK();
    k_digit_offsets<<<1, 256, 0, st>>>(s->digit, npass);
    PPM_LAUNCH_CHECK();
    for (int p = 0; p < npass; ++p) {
        const int shift = 8 * p;
        const int nb = bits - shift < 8 ? bits - shift : 8;
        const uint32_t mask = (1u << nb) - 1u;
        PPM_CUDA(cudaMemsetAsync(s->status, 0, (size_t)(kStatusHead + 256ll * ntiles) * sizeof(unsigned long long), st));
        k_radix_onesweep<<<ntiles, kSortThreads, 0, st>>>(s->keys, s->vals, s->keys_alt, s->vals_alt, n, shift,
                                                         mask, s->digit + p * 256, s->status, err,
                                                         spin_limit);
        PPM_LAUNCH_CHECK();
        uint32_t* t;
        t = s->keys; s->keys = s->keys_alt; s->keys_alt = t;
        t = s->vals; s->vals = s->vals_alt; s->vals_alt = t;
    }
    return PPM_OK;
}
