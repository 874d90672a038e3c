// Internal declarations shared by the CUDA sources of libhgs (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hgs.h"

namespace hgs {

constexpr int kMaxViews = HGS_MAX_VIEWS;

// Host-computed per-view offsets, passed to kernels by value (4 KB; kernels may
// take up to 32 KB of parameters on sm_70 and later).
struct ViewTable {
    int n_views;
    int total_tiles;
    int tile_off[kMaxViews + 1];       // global tile id offset of each view
    int tiles_x[kMaxViews];            // tiles per row of each view
    long long pix_off[kMaxViews + 1];  // pixel offset of each view
};

// Which view a global tile id belongs to (binary search over tile_off).
__device__ __forceinline__ int view_of_tile(const ViewTable &vt, int gtile) {
    int lo = 0, hi = vt.n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (vt.tile_off[mid] <= gtile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__host__ __device__ __forceinline__ int div_up(int a, int b) { return (a + b - 1) / b; }

__device__ __forceinline__ void set_status(int *st, int bit) {
    if (st) atomicOr(st, bit);
}

// Host-side launchers (one per kernel family), defined in the .cu files.
struct ProjLaunch {
    hgs_gaussians g;
    const hgs_camera *cams;
    int n_views;
    hgs_config cfg;
    hgs_proj out;
    ViewTable vt;
    int *status;
};
cudaError_t launch_project(const ProjLaunch &p, cudaStream_t s);

struct ProjBwdLaunch {
    hgs_gaussians g;
    const hgs_camera *cams;
    int n_views;
    hgs_config cfg;
    const float *grad2d;
    hgs_gaussian_grads out;
    uint32_t *fp64_list;
    int *status;
};
cudaError_t launch_project_bwd(const ProjBwdLaunch &p, cudaStream_t s);

// Binning workspace carve-up (see binning.cu).
struct BinLaunch {
    const hgs_proj *proj;
    int n, n_views;
    ViewTable vt;
    hgs_config cfg;
    void *ws;
    size_t ws_bytes;
    size_t capacity;
    uint64_t *keys_out;
    uint32_t *ids_out;
    uint32_t *ranges;
    uint64_t *num_pairs;
    int *status;
};
size_t bin_workspace_bytes(int n, int n_views, size_t capacity);
cudaError_t launch_bin(const BinLaunch &p, cudaStream_t s);

// Visibility mask, written by the forward compositing and read by the backward.  For
// each global tile t (sorted list [beg_t, end_t)) and each 32-entry chunk c of that list
// there is one 32-bit word per 8x4 warp block w of the tile, at
//   (vis_row(beg_t, t) + c) * (warps per tile) + w;
// bit j says that list entry beg_t + 32c + j was composited at some pixel of block w.
// Tile t's rows never reach tile t+1's: ceil(len/32) <= (end >> 5) - (beg >> 5) + 1.
__host__ __device__ __forceinline__ size_t vis_row(uint32_t beg, int gtile) {
    return (size_t)(beg >> 5) + (size_t)gtile;
}
inline size_t vis_words_for(size_t pair_capacity, int total_tiles, int tile_w, int tile_h) {
    return (pair_capacity / 32 + (size_t)total_tiles + 1) * (size_t)(tile_w * tile_h / 32);
}

struct RenderLaunch {
    hgs_proj proj;
    int n;
    const uint32_t *ids;
    const uint32_t *ranges;
    const hgs_camera *cams;
    ViewTable vt;
    hgs_config cfg;
    void *ws;
    size_t ws_bytes;
    // forward outputs / backward inputs
    float *image;
    float *final_T;
    uint32_t *n_contrib;
    uint32_t *vis;                  // visibility mask (forward output, backward input)
    size_t vis_words;
    float4 *clear;                  // forward: zeroed by the kernel (the backward's grad2d), or null
    size_t clear_n4;                // its length in float4
    bool from_forward;              // backward: follows its forward (grad2d cleared, queue built)
    // backward
    const float *dL_dimage;
    float *grad2d;
    int *status;
    unsigned long long *counters;   // non-null: counting launch (see hgs_render_stats)
};
size_t render_workspace_bytes(const ViewTable &vt, const hgs_config &cfg);
cudaError_t launch_render_fwd(const RenderLaunch &p, cudaStream_t s);
cudaError_t launch_render_bwd(const RenderLaunch &p, cudaStream_t s);
cudaError_t launch_wait_selftest(int *status, cudaStream_t s);

int num_sms();

}  // namespace hgs
