// hgs_bin_static: the binning step (scan, key emission, radix sort, ranges) with
// its scratch workspace in a fixed device array owned by this library, for
// callers that must not allocate device memory themselves.
//
// Who cannot allocate: a plug-in running inside a host application that owns
// the whole device-memory budget and forbids its plug-ins to call the CUDA
// allocator; a real-time loop that cannot afford a driver allocation, which may
// synchronise the device; code that enqueues work while a stream is being
// captured, where allocation calls are not allowed.  Such callers still provide
// the inputs and the outputs (keys, ids, ranges, pair count, status); only the
// scratch moves into the library.
//
// The array is kHgsStaticScratchBytes (HGS_BIN_STATIC_SCRATCH_BYTES) bytes.  Every
// GPU that loads this code holds it until the process exits.  Its device address
// is looked up once per device, on the first call made with that device current,
// with cudaGetSymbolAddress; that first call should therefore come before any
// stream capture.  All calls share the one array and it keeps the previous
// call's contents: the binning kernels clear everything that must start at zero
// (the control block with the digit totals) at the start of each
// call, and overwrite the rest before reading it.  Calls whose work overlaps on
// the GPU (other streams, other threads) race on the array; calls in order on
// one stream do not.
#include <mutex>

#include "hgs_internal.cuh"

namespace {

constexpr size_t kHgsStaticScratchBytes = HGS_BIN_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_bin_scratch[kHgsStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_bin_scratch for the current device (looked up once).
cudaError_t scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" hgs_status hgs_bin_static(const hgs_proj *proj, int n, const hgs_camera *cams_host, int n_views,
                                     const hgs_config *cfg, size_t pair_capacity, uint64_t *keys_out,
                                     uint32_t *ids_out, uint32_t *ranges, uint64_t *dev_num_pairs, int *dev_status,
                                     void *stream) {
    // Size check first: the scratch this call needs must fit the fixed array.
    if (n < 0 || n_views < 1 || n_views > HGS_MAX_VIEWS || pair_capacity > HGS_MAX_PAIRS) return HGS_ERR_INVALID;
    const size_t need = hgs::bin_workspace_bytes(n, n_views, pair_capacity);
    if (need > kHgsStaticScratchBytes) return HGS_ERR_CAPACITY;
    // The remaining argument checks are those of hgs_bin; run them before the
    // one-time address lookup so that a bad call touches no CUDA state.
    int total_tiles = 0;
    hgs_status st = hgs_layout(cams_host, n_views, cfg, &total_tiles, nullptr);
    if (st != HGS_OK) return st;
    void *ws = nullptr;
    if (scratch_for_current_device(&ws) != cudaSuccess || !ws) return HGS_ERR_CUDA;
    return hgs_bin(proj, n, cams_host, n_views, cfg, ws, kHgsStaticScratchBytes, pair_capacity, keys_out, ids_out,
                   ranges, dev_num_pairs, dev_status, stream);
}
