// hgs_bin_static: the binning step (scan, key emission, radix sort, ranges) with
// its scratch workspace in a fixed device array owned by this library, for
// callers that must not allocate device memory themselves.
//
// Who cannot allocate: a plug-in running inside a host application that owns
// the whole device-memory budget and forbids its plug-ins to call the CUDA
// allocator; a real-time loop that cannot afford a driver allocation, which may
// synchronise the device.  Such callers still provide the inputs and the
// outputs (keys, ids, ranges, pair count, status); only the scratch moves into
// the library.
//
// The array is kHgsStaticScratchBytes (HGS_BIN_STATIC_SCRATCH_BYTES) bytes.  Every
// GPU that loads this code holds it until the process exits.  Its device address
// is looked up with cudaGetSymbolAddress on the first call made with a device
// current, and again whenever that device's context has changed since (after a
// cudaDeviceReset the old address is dead); that first call should therefore
// come before any stream capture.  All calls share the one array and it keeps the
// previous call's contents: the binning kernels clear everything that must start
// at zero (the control block with the digit totals) at the start of each call,
// and overwrite the rest before reading it.  Calls whose work overlaps on the GPU
// (other streams, other threads) race on the array; calls in order on one stream
// do not.
#include <cuda.h>   // driver types only (CUcontext, CUresult); no link against libcuda

#include <mutex>

#include "hgs_internal.cuh"

namespace {

constexpr size_t kHgsStaticScratchBytes = HGS_BIN_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_bin_scratch[kHgsStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
struct Cached {
    unsigned long long ctx_id;   // driver context the address belongs to (0: none yet)
    void *ptr;
};
Cached g_scratch[kMaxDevices] = {};

// The unique id of the calling thread's current driver context (0 if there is none
// or the driver does not provide the query).  The two driver entry points are
// resolved at run time through the runtime, so the library needs no link against
// the driver library and still loads on a machine without a GPU.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_bin_scratch for the current device, looked up on the first
// call and again when the device's context is no longer the one of the cached
// address.
cudaError_t scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    Cached &c = g_scratch[dev];
    const unsigned long long id = current_context_id();
    if (!c.ptr || id == 0 || id != c.ctx_id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);   // also makes the primary context current
        if (e != cudaSuccess) return e;
        c.ptr = p;
        c.ctx_id = current_context_id();
    }
    *out = c.ptr;
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
