// ppm_noalloc.cu -- ppm_sort_pairs_noalloc: the stable radix sort of
// ppm_sort_pairs (in its three-kernel-per-pass form, same results) with its
// scratch in a fixed device array instead of memory allocated per call.
//
// For callers that cannot call cudaMalloc while they run: real-time loops
// that cannot pay for an allocator call or the synchronization it may
// bring, and hosts whose device memory is entirely owned by another
// allocator.  The scratch (both ping-pong arrays, the per-tile digit
// histograms and the scan partials for up to PPM_NOALLOC_MAX_PAIRS = n
// pairs: 2n + n/8 + 34 words, 8.9 MB) is a file-scope __device__ array:
// every GPU that loads this library holds it until the process exits.
//
// In host code the array's name only stands for the symbol; its device
// address is obtained once per device with cudaGetSymbolAddress while that
// device is current (the first call on a device does this set-up, so that
// first call should come before any stream capture).  The address is cached
// for the life of the process, so cudaDeviceReset after the first call is
// not supported (the cached address would be stale).
// All calls share the array: calls whose work overlaps on the GPU
// (different streams, or different host threads on one device) race on
// it.  Every word of the scratch that a call reads is written earlier in
// the same call, so nothing needs clearing between calls.
#include <mutex>

#include "ppm_internal.cuh"

namespace {

constexpr int64_t kMaxPairs = PPM_NOALLOC_MAX_PAIRS;
constexpr int64_t kTiles = (kMaxPairs + 2047) / 2048;     // radix-sort tiles of 2048 keys
constexpr int64_t kHist = 256 * kTiles;                     // digit histograms
constexpr int64_t kPart = kHist / 4096 + 2;                 // scan block partials
constexpr int64_t kWords = 2 * kMaxPairs + kHist + kPart;

static __device__ __align__(256) uint32_t g_sort_scratch[kWords];

constexpr int kMaxDevices = 256;
std::mutex g_setup_mu;
uint32_t* g_scratch_addr[kMaxDevices] = {};

// device address of g_sort_scratch on the current device
int scratch_address(uint32_t** out)
{
    int dev = -1;
    PPM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return PPM_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || !p) {
            ppm_note_cuda_error(e, "cudaGetSymbolAddress(g_sort_scratch)", __FILE__, __LINE__);
            cudaGetLastError();
            return PPM_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return PPM_OK;
}

}  // namespace

extern "C" int ppm_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in,
                                      uint32_t* keys_out, uint32_t* vals_out, int64_t n,
                                      int32_t bits, void* stream)
{
    PPM_ENTRY();
    if (n < 0 || n > kMaxPairs || bits < 1 || bits > 32) return PPM_EINVAL;
    if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out)) return PPM_EINVAL;
    uint32_t* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    if (n == 0) return PPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (keys_out != keys_in)
        PPM_CUDA(cudaMemcpyAsync(keys_out, keys_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    if (vals_out != vals_in)
        PPM_CUDA(cudaMemcpyAsync(vals_out, vals_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    if (n == 1) return PPM_OK;
    const int64_t hist = 256 * ((n + 2047) / 2048);
    SortScratch s;
    s.keys = keys_out;
    s.vals = vals_out;
    s.keys_alt = scratch;
    s.vals_alt = scratch + kMaxPairs;
    s.hist = scratch + 2 * kMaxPairs;
    s.partials = scratch + 2 * kMaxPairs + kHist;
    s.cap = n;
    s.hist_cap = hist;
    s.part_cap = kPart;
    rc = ppm_radix_sort_pairs(&s, n, bits, st);
    if (rc) return rc;
    if (s.keys != keys_out) {   // odd number of passes: result is in the scratch
        PPM_CUDA(cudaMemcpyAsync(keys_out, s.keys, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        PPM_CUDA(cudaMemcpyAsync(vals_out, s.vals, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    return PPM_OK;
}
