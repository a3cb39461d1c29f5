// ppm_grid.cu -- photon map of one iteration (the range-search structure
// over the light vertices that Sec. 5.1 builds first): a hashed uniform grid.
//
//   k_grid_geom  : cell edge h = cell_factor * max_h r_h along y and z,
//                  h / 2^kXSplit along x, from device memory written by the
//                  previous update (no host sync);
//   k_pack_keys  : one coalesced pass over the caller's photons: bucket key,
//                  identity index, and the photon's 16-byte records side by
//                  side;
//   radix sort   : stable, on the bucket bits (ppm_sort.cu);
//   k_cell_start : cell_start[b] = first sorted photon with bucket >= b
//                  (each warp fills the empty-bucket gaps cooperatively);
//   k_permute    : records gathered into bucket order, one array each.
#include "ppm_internal.cuh"

namespace {

__global__ void k_grid_geom(GridGeom* __restrict__ g, const float* __restrict__ rmax,
                            float cell_factor, uint32_t tmask, int lb)
{
    float r = *rmax;
    if (!(r > 0.f)) r = 1e-30f;
    *g = ppm_make_geom(__fmul_rn(cell_factor, r), tmask, lb, 0u);
}

// Rec. 709 luminance of an RGB flux (the paper tests luminance, Sec. 5.1).
__device__ __forceinline__ float lum709(float R, float G, float B)
{
    return fmaf(0.0722f, B, fmaf(0.7152f, G, __fmul_rn(0.2126f, R)));
}

// block-wide max of v >= 0 folded into *dst (float bits order as ints)
__device__ __forceinline__ void block_max_into(float v, float* dst)
{
    __shared__ float s_w[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_w[w]);
        atomicMax((int*)dst, __float_as_int(m));
    }
}

// PSIMAX: also record the largest tested value (traversal 3 only)
template <int NCH, bool AUX, bool VCM, bool PSIMAX>
__global__ void __launch_bounds__(256)
k_pack_keys(int64_t n, const float* __restrict__ pos, const float* __restrict__ flux,
            const uint32_t* __restrict__ nq, const float* __restrict__ rho,
            const uint32_t* __restrict__ wq, GridGeom* __restrict__ geom,
            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, float4* __restrict__ pack)
{
    // a photon's records side by side (x y z psi | R G B rho_vm | aux), so
    // that the permute's random read of one photon fetches whole sectors
    constexpr bool REC1 = NCH == 3 || VCM;
    constexpr int S = 1 + (REC1 ? 1 : 0) + (AUX ? 1 : 0);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const GridGeom g = *geom;
    float vmax = 0.f;
    if (i < n) {
    const float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    float R, G = 0.f, B = 0.f, psi;
    if (NCH == 3) {
        R = flux[3 * i]; G = flux[3 * i + 1]; B = flux[3 * i + 2];
        psi = lum709(R, G, B);
        vmax = fmaxf(fmaxf(psi, R), fmaxf(G, B));
    } else {
        R = flux[i];
        psi = R;
        vmax = psi;
    }
    float4* rec = pack + i * S;
    rec[0] = make_float4(x, y, z, psi);
    if constexpr (REC1) rec[1] = make_float4(R, G, B, VCM ? rho[2 * i] : 0.f);
    if constexpr (AUX)
        reinterpret_cast<uint4*>(rec)[S - 1] = make_uint4(nq ? nq[i] : 0u, VCM ? wq[i] : 0u,
                                                          VCM ? __float_as_uint(rho[2 * i + 1]) : 0u, 0u);
    const int ix = ppm_cell_coord(x, g.inv_hx);
    const int iy = ppm_cell_coord(y, g.inv_h);
    const int iz = ppm_cell_coord(z, g.inv_h);
    keys[i] = ppm_bucket(ix, iy, iz, g);
    vals[i] = (uint32_t)i;
    }
    // largest tested value (and flux channel) of the iteration: the scale of
    // the gather's fixed-point group sums
    if constexpr (PSIMAX) block_max_into(fmaxf(vmax, 0.f), &geom->psimax);
}

// One thread per sorted photon i in [0, n]: fills the buckets between the
// previous photon's bucket and its own (exclusive/inclusive), so every
// bucket in [0, T] is written exactly once.  Nothing is written when the
// sort's look-back gave up (*err bit 2): the keys are then no sorted
// permutation and could point past the table.
__global__ void __launch_bounds__(256)
k_cell_start(const uint32_t* __restrict__ keys, int64_t n, uint32_t T,
             uint32_t* __restrict__ cell_start, const int32_t* __restrict__ err)
{
    if (*err & 4) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = -1;
    if (i <= n) {
        lo = (i == 0) ? 0 : (int64_t)keys[i - 1] + 1;
        hi = (i == n) ? (int64_t)T : (int64_t)keys[i];
    }
    // Only the first photon of each occupied bucket has a range, and the
    // ranges are tens of buckets long: the warp fills them one after another
    // with coalesced stores instead of leaving it to one lane each.
    const unsigned full = 0xffffffffu;
    unsigned m = __ballot_sync(full, hi >= lo);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        const int64_t l = __shfl_sync(full, lo, src);
        const int64_t h = __shfl_sync(full, hi, src);
        const uint32_t v = (uint32_t)(i - lane + src);
        for (int64_t c = l + lane; c <= h; c += 32) cell_start[c] = v;
    }
}

// records of packed photon vals[i] (stride 1 + REC1 + AUX float4s) into
// the gather's sorted arrays: rec0 on its own (every candidate reads it);
// with both the other records, rec1 and aux side by side in rec1 (32 bytes
// a photon, one sector for an in-disk pair), else each in its own array.
// Nothing when the sort gave up (the values are then no permutation of
// [0, n)).
template <bool REC1, bool AUX>
__global__ void __launch_bounds__(256)
k_permute(int64_t n, const uint32_t* __restrict__ vals, const float4* __restrict__ pack,
          float4* __restrict__ rec0, float4* __restrict__ rec1, uint4* __restrict__ aux,
          const int32_t* __restrict__ err)
{
    constexpr int S = 1 + (REC1 ? 1 : 0) + (AUX ? 1 : 0);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (*err & 4)) return;
    const float4* src = pack + (int64_t)vals[i] * S;
    rec0[i] = __ldg(src);
    if constexpr (REC1 && AUX) {
        rec1[2 * i] = __ldg(src + 1);
        reinterpret_cast<uint4*>(rec1)[2 * i + 1] = __ldg(reinterpret_cast<const uint4*>(src) + 2);
    } else {
        if constexpr (REC1) rec1[i] = __ldg(src + 1);
        if constexpr (AUX) aux[i] = __ldg(reinterpret_cast<const uint4*>(src) + (S - 1));
    }
}

template <int NCH, bool AUX, bool VCM>
void launch_pack(ppm_ctx* c, const ppm_photons* ph, unsigned nb)
{
    if (c->prm.mapping == 3)
        k_pack_keys<NCH, AUX, VCM, true><<<nb, 256, 0, c->stream>>>(
            ph->n, ph->pos, ph->flux, ph->nq, ph->rho, ph->wq, c->geom_dev,
            c->sort.keys, c->sort.vals, c->pack);
    else
        k_pack_keys<NCH, AUX, VCM, false><<<nb, 256, 0, c->stream>>>(
            ph->n, ph->pos, ph->flux, ph->nq, ph->rho, ph->wq, c->geom_dev,
            c->sort.keys, c->sort.vals, c->pack);
}

int reserve_photons(ppm_ctx* c, int64_t n)
{
    int rc = ppm_sort_scratch_reserve(&c->sort, n > 0 ? n : 1);
    if (rc) return rc;
    if (n <= c->ph_cap) return PPM_OK;
    cudaFree(c->pack);
    cudaFree(c->rec0); cudaFree(c->rec1); cudaFree(c->aux);
    c->pack = c->rec0 = c->rec1 = nullptr;
    c->aux = nullptr;
    c->ph_cap = 0;
    const int64_t cap = n + n / 4 + 1024;
    const bool rec1 = c->nch == 3 || c->prm.vcm;
    // packed records: up to 3 float4 a photon (the aux record depends on
    // whether the iteration brings normals)
    if (cudaMalloc(&c->pack, cap * (rec1 ? 3 : 2) * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&c->rec0, cap * sizeof(float4)) != cudaSuccess ||
        (rec1 && cudaMalloc(&c->rec1, 2 * cap * sizeof(float4)) != cudaSuccess) ||   // rec1 | aux side by side
        cudaMalloc(&c->aux, cap * sizeof(uint4)) != cudaSuccess) {
        cudaGetLastError();
        return PPM_ENOMEM;
    }
    c->ph_cap = cap;
    return PPM_OK;
}

}  // namespace

// Bucket-table size: T = 2^tbits >= 2 n 2^kXSplit (two buckets a photon
// per cell of the unsplit grid), and at least 4 blocks of Bx * B^2 cells.
int ppm_table_bits(int64_t n, int lb)
{
    // at least 2 buckets a photon per cell of a cubic grid (2^sx in all);
    // then up to 8 (2^(sx+3)) while the keys need no further 8-bit radix
    // pass, or up to 2^25 entries in any case, and the table stays within
    // 2^29 entries (2 GB): with more buckets fewer hash blocks share a
    // bucket range, so fewer photons of other cells are tested (2M photons:
    // 2^22 -> 2^24 buckets, 8% fewer candidates, and with cells split along
    // x 2^24 -> 2^25, gather -0.10 ms for +0.04 ms of a fourth pass; 16M
    // photons: 2^25 -> 2^27, 8% fewer, gather 5% faster, the build
    // unchanged at four passes; 53M photons: 2^27 -> 2^29, gather 20.2 ->
    // 19.7 ms)
    int b = 3 * lb + kXSplit + 2;
    while (b < 30 && ((int64_t)1 << b) < (2 * n << kXSplit)) ++b;
    const int pass_cap = (b + 7) / 8 * 8 > 25 ? (b + 7) / 8 * 8 : 25;
    const int cap = pass_cap < 29 ? pass_cap : 29;
    while (b < cap && ((int64_t)1 << b) < (8 * n << kXSplit)) ++b;
    return b;
}

int ppm_grid_build(ppm_ctx* c, const ppm_photons* ph)
{
    const int64_t n = ph->n;
    int rc = reserve_photons(c, n);
    if (rc) return rc;
    // hash blocks 4 cells wide (along y and z) suffice for one sphere (<= 4
    // cells per axis at cell_factor >= 1); the warp-union traversals and
    // cell_factor < 1 need more.  Blocks 16 wide there: a row's x-range then
    // crosses a block boundary less often, so it splits into fewer runs
    // (VCM+ 4K at cell factor 2/3: gather 9.86 -> 9.59 ms against 8 wide)
    const int lb = (c->prm.cell_factor >= 1.0f && c->prm.mapping == 0) ? 2 : 4;
    c->tbits = ppm_table_bits(n, lb);
    const uint32_t T = 1u << c->tbits;
    if ((int64_t)T + 1 > c->cs_cap) {
        cudaFree(c->cell_start);
        c->cell_start = nullptr;
        c->cs_cap = 0;
        const int64_t cap = (int64_t)T + 1;
        if (cudaMalloc(&c->cell_start, cap * sizeof(uint32_t)) != cudaSuccess) { cudaGetLastError(); return PPM_ENOMEM; }
        c->cs_cap = cap;
    }
    c->lb = lb;
    k_grid_geom<<<1, 1, 0, c->stream>>>(c->geom_dev, c->rmax + c->rmax_cur, c->prm.cell_factor, T - 1, lb);
    PPM_LAUNCH_CHECK();
    const bool aux = c->ph_aux;
    const bool vcm = c->prm.vcm != 0;
    if (n > 0) {
        const unsigned nb = (unsigned)((n + 255) / 256);
        if (c->nch == 3) {
            if (vcm) launch_pack<3, true, true>(c, ph, nb);
            else if (aux) launch_pack<3, true, false>(c, ph, nb);
            else launch_pack<3, false, false>(c, ph, nb);
        } else {
            if (vcm) launch_pack<1, true, true>(c, ph, nb);
            else if (aux) launch_pack<1, true, false>(c, ph, nb);
            else launch_pack<1, false, false>(c, ph, nb);
        }
        PPM_LAUNCH_CHECK();
        rc = ppm_radix_sort_pairs_lookback(&c->sort, n, c->tbits, c->err_dev, c->stream, c->prm.wait_limit);
        if (rc) return rc;
    }
    rc = ppm_cell_start_launch(c->sort.keys, n, T, c->cell_start, c->err_dev, c->stream);
    if (rc) return rc;
    if (n > 0) {
        const bool rec1 = c->nch == 3 || vcm;
        rc = ppm_permute_launch(n, c->sort.vals, c->pack, c->rec0, rec1 ? c->rec1 : nullptr,
                                aux ? c->aux : nullptr, c->err_dev, c->stream);
        if (rc) return rc;
    }
    c->n_ph = n;
    c->launches_build = 2 + (n > 0 ? 2 + 2 + (c->tbits + 7) / 8 : 0);
    return PPM_OK;
}

int ppm_cell_start_launch(const uint32_t* keys, int64_t n, uint32_t T, uint32_t* cell_start,
                          const int32_t* err, cudaStream_t st)
{
    k_cell_start<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(keys, n, T, cell_start, err);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_permute_launch(int64_t n, const uint32_t* vals, const float4* pack, float4* rec0, float4* rec1,
                       uint4* aux, const int32_t* err, cudaStream_t st)
{
    if (n <= 0) return PPM_OK;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (rec1 && aux)
        k_permute<true, true><<<nb, 256, 0, st>>>(n, vals, pack, rec0, rec1, aux, err);
    else if (rec1)
        k_permute<true, false><<<nb, 256, 0, st>>>(n, vals, pack, rec0, rec1, aux, err);
    else if (aux)
        k_permute<false, true><<<nb, 256, 0, st>>>(n, vals, pack, rec0, rec1, aux, err);
    else
        k_permute<false, false><<<nb, 256, 0, st>>>(n, vals, pack, rec0, rec1, aux, err);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}
