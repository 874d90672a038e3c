// C ABI entry points (include/hgs.h): argument validation, per-view tables and
// kernel launches.  No entry point allocates memory or synchronises the host.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "hgs_internal.cuh"

namespace hgs {

// SM count of the current device, looked up once per device (atomic: threads making
// their first calls at the same time store the same value).
int num_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    std::atomic<int> &slot = cache[dev & 63];
    int v = slot.load(std::memory_order_relaxed);
    if (!v) {
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        v = v > 0 ? v : 1;
        slot.store(v, std::memory_order_relaxed);
    }
    return v;
}

}  // namespace hgs

using namespace hgs;

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool cfg_ok(const hgs_config *c) {
    if (!c) return false;
    const bool shape = (c->tile_w == 16 && c->tile_h == 16) || (c->tile_w == 8 && c->tile_h == 8) ||
                       (c->tile_w == 32 && c->tile_h == 8);
    const bool batch = c->batch == 0 || c->batch == 32 || c->batch == 64 || c->batch == 128 || c->batch == 224 ||
                       c->batch == 256 || c->batch == 512;
    const bool rect = c->rect_mode == 0 || c->rect_mode == 1 || c->rect_mode == 2;
    const bool mip = c->mip == 0 || c->mip == 1;
    return shape && batch && rect && mip && isfinite(c->lowpass) && c->lowpass >= 0.0f;
}

hgs_status build_views(const hgs_camera *cams, int nv, const hgs_config *cfg, ViewTable *vt) {
    if (!cams || nv < 1 || nv > HGS_MAX_VIEWS || !cfg_ok(cfg)) return HGS_ERR_INVALID;
    memset(vt, 0, sizeof(*vt));
    vt->n_views = nv;
    long long tiles = 0, pix = 0;
    for (int v = 0; v < nv; ++v) {
        const hgs_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || !(c.fx > 0.0f) || !(c.fy > 0.0f) || !isfinite(c.fx) ||
            !isfinite(c.fy) || !isfinite(c.cx) || !isfinite(c.cy) || !isfinite(c.near_plane))
            return HGS_ERR_INVALID;
        for (int k = 0; k < 12; ++k)
            if (!isfinite(c.viewmat[k])) return HGS_ERR_INVALID;
        const int tx = div_up(c.width, cfg->tile_w), ty = div_up(c.height, cfg->tile_h);
        vt->tile_off[v] = (int)tiles;
        vt->tiles_x[v] = tx;
        vt->pix_off[v] = pix;
        tiles += (long long)tx * ty;
        pix += (long long)c.width * c.height;
        if (tiles > (1ll << 30) || pix > (1ll << 31) / 3) return HGS_ERR_INVALID;
    }
    vt->tile_off[nv] = (int)tiles;
    vt->pix_off[nv] = pix;
    vt->total_tiles = (int)tiles;
    return HGS_OK;
}

bool gaussians_ok(const hgs_gaussians *g) {
    if (!g || g->n < 0 || g->sh_degree < 0 || g->sh_degree > HGS_MAX_SH_DEGREE) return false;
    if (g->n == 0) return true;
    if (!g->means || !g->scales || !g->quats || !g->normals || !g->opac1 || !g->opac2 || !g->sh) return false;
    return aligned16(g->means) && aligned16(g->scales) && aligned16(g->quats) && aligned16(g->normals) &&
           aligned16(g->opac1) && aligned16(g->opac2) && aligned16(g->sh);
}

bool proj_ok(const hgs_proj *p, long long vn, bool need_list = false) {
    if (!p) return false;
    if (vn == 0) return true;
    return p->rec && p->depth && p->rect && p->tiles && (p->fp64_list || !need_list) && aligned16(p->rec) &&
           aligned16(p->depth) && aligned16(p->rect) && aligned16(p->tiles);
}

hgs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HGS_OK : HGS_ERR_CUDA; }

}  // namespace

extern "C" {

int hgs_version(void) { return HGS_VERSION; }

const char *hgs_status_string(hgs_status s) {
    switch (s) {
        case HGS_OK: return "ok";
        case HGS_ERR_INVALID: return "invalid argument";
        case HGS_ERR_CAPACITY: return "buffer too small";
        case HGS_ERR_CUDA: return "CUDA error";
        case HGS_ERR_TIMEOUT: return "timeout";
        case HGS_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

hgs_status hgs_layout(const hgs_camera *cams_host, int n_views, const hgs_config *cfg, int *total_tiles,
                      int64_t *total_pixels) {
    ViewTable vt;
    hgs_status st = build_views(cams_host, n_views, cfg, &vt);
    if (st != HGS_OK) return st;
    if (total_tiles) *total_tiles = vt.total_tiles;
    if (total_pixels) *total_pixels = vt.pix_off[n_views];
    return HGS_OK;
}

size_t hgs_bin_workspace_size(int n, int n_views, size_t pair_capacity) {
    if (n < 0 || n_views < 1) return 0;
    return bin_workspace_bytes(n, n_views, pair_capacity);
}

size_t hgs_render_workspace_size(const hgs_camera *cams_host, int n_views, const hgs_config *cfg, int n) {
    (void)n;
    ViewTable vt;
    if (build_views(cams_host, n_views, cfg, &vt) != HGS_OK) return 0;
    return render_workspace_bytes(vt, *cfg);
}

size_t hgs_vis_words(const hgs_camera *cams_host, int n_views, const hgs_config *cfg, size_t pair_capacity) {
    ViewTable vt;
    if (build_views(cams_host, n_views, cfg, &vt) != HGS_OK || pair_capacity > HGS_MAX_PAIRS) return 0;
    return vis_words_for(pair_capacity, vt.total_tiles, cfg->tile_w, cfg->tile_h);
}

hgs_status hgs_project(const hgs_gaussians *g, const hgs_camera *cams_host, const hgs_camera *cams_dev,
                       int n_views, const hgs_config *cfg, const hgs_proj *out, int *dev_status, void *stream) {
    ViewTable vt;
    hgs_status st = build_views(cams_host, n_views, cfg, &vt);
    if (st != HGS_OK) return st;
    if (!gaussians_ok(g) || !cams_dev || !proj_ok(out, (long long)g->n * n_views, true)) return HGS_ERR_INVALID;
    ProjLaunch p;
    p.g = *g;
    p.cams = cams_dev;
    p.n_views = n_views;
    p.cfg = *cfg;
    p.out = *out;
    p.vt = vt;
    p.status = dev_status;
    return cuda_status(launch_project(p, static_cast<cudaStream_t>(stream)));
}

hgs_status hgs_bin(const hgs_proj *proj, int n, const hgs_camera *cams_host, int n_views, const hgs_config *cfg,
                   void *ws, size_t ws_bytes, size_t pair_capacity, uint64_t *keys_out, uint32_t *ids_out,
                   uint32_t *ranges, uint64_t *dev_num_pairs, int *dev_status, void *stream) {
    ViewTable vt;
    hgs_status st = build_views(cams_host, n_views, cfg, &vt);
    if (st != HGS_OK) return st;
    if (n < 0 || !proj_ok(proj, (long long)n * n_views) || !dev_num_pairs || !ranges) return HGS_ERR_INVALID;
    if (pair_capacity > HGS_MAX_PAIRS) return HGS_ERR_INVALID;
    if (pair_capacity > 0 && !ids_out) return HGS_ERR_INVALID;
    if ((long long)n * n_views > 0xffffffffll) return HGS_ERR_INVALID;
    if (!ws || ws_bytes < bin_workspace_bytes(n, n_views, pair_capacity)) return HGS_ERR_CAPACITY;
    BinLaunch p;
    p.proj = proj;
    p.n = n;
    p.n_views = n_views;
    p.vt = vt;
    p.cfg = *cfg;
    p.ws = ws;
    p.ws_bytes = ws_bytes;
    p.capacity = pair_capacity;
    p.keys_out = keys_out;
    p.ids_out = ids_out;
    p.ranges = ranges;
    p.num_pairs = dev_num_pairs;
    p.status = dev_status;
    return cuda_status(launch_bin(p, static_cast<cudaStream_t>(stream)));
}

hgs_status hgs_selftest_wait(int *dev_status, void *stream) {
    if (!dev_status) return HGS_ERR_INVALID;
    return cuda_status(launch_wait_selftest(dev_status, static_cast<cudaStream_t>(stream)));
}

static hgs_status render_common(const hgs_proj *proj, int n, const uint32_t *ids, const uint32_t *ranges,
                                const hgs_camera *cams_host, const hgs_camera *cams_dev, int n_views,
                                const hgs_config *cfg, void *ws, size_t ws_bytes, RenderLaunch *p) {
    hgs_status st = build_views(cams_host, n_views, cfg, &p->vt);
    if (st != HGS_OK) return st;
    if (n < 0 || !cams_dev || !ranges || !proj_ok(proj, (long long)n * n_views)) return HGS_ERR_INVALID;
    if (n > 0 && !ids) return HGS_ERR_INVALID;
    if (cfg->persistent && (!ws || ws_bytes < render_workspace_bytes(p->vt, *cfg))) return HGS_ERR_CAPACITY;
    p->proj = *proj;
    p->n = n;
    p->ids = ids;
    p->ranges = ranges;
    p->cams = cams_dev;
    p->cfg = *cfg;
    p->ws = ws;
    p->ws_bytes = ws_bytes;
    p->image = nullptr;
    p->final_T = nullptr;
    p->n_contrib = nullptr;
    p->vis = nullptr;
    p->vis_words = 0;
    p->clear = nullptr;
    p->clear_n4 = 0;
    p->from_forward = false;
    p->dL_dimage = nullptr;
    p->grad2d = nullptr;
    p->status = nullptr;
    p->counters = nullptr;
    return HGS_OK;
}

hgs_status hgs_render_fwd(const hgs_proj *proj, int n, const uint32_t *ids, const uint32_t *ranges,
                          const hgs_camera *cams_host, const hgs_camera *cams_dev, int n_views,
                          const hgs_config *cfg, void *ws, size_t ws_bytes, float *image, float *final_T,
                          uint32_t *n_contrib, uint32_t *vis, size_t vis_words, float *grad2d_clear,
                          int *dev_status, void *stream) {
    RenderLaunch p;
    hgs_status st = render_common(proj, n, ids, ranges, cams_host, cams_dev, n_views, cfg, ws, ws_bytes, &p);
    if (st != HGS_OK) return st;
    if (!image || !final_T || !n_contrib || !vis || (grad2d_clear && !aligned16(grad2d_clear)))
        return HGS_ERR_INVALID;
    if (grad2d_clear) {
        p.clear = reinterpret_cast<float4 *>(grad2d_clear);
        p.clear_n4 = 3 * (size_t)n * (size_t)n_views;      // 12 floats per (view, splat)
    }
    p.image = image;
    p.final_T = final_T;
    p.n_contrib = n_contrib;
    p.vis = vis;
    p.vis_words = vis_words;
    p.status = dev_status;
    return cuda_status(launch_render_fwd(p, static_cast<cudaStream_t>(stream)));
}

hgs_status hgs_rasterize_bwd(const hgs_proj *proj, int n, const uint32_t *ids, const uint32_t *ranges,
                             const hgs_camera *cams_host, const hgs_camera *cams_dev, int n_views,
                             const hgs_config *cfg, void *ws, size_t ws_bytes, const float *final_T,
                             const uint32_t *n_contrib, const uint32_t *vis, size_t vis_words,
                             const float *dL_dimage, float *grad2d, int from_forward, int *dev_status,
                             void *stream) {
    RenderLaunch p;
    hgs_status st = render_common(proj, n, ids, ranges, cams_host, cams_dev, n_views, cfg, ws, ws_bytes, &p);
    if (st != HGS_OK) return st;
    if (!final_T || !n_contrib || !vis || !dL_dimage || (n > 0 && (!grad2d || !aligned16(grad2d))))
        return HGS_ERR_INVALID;
    p.final_T = const_cast<float *>(final_T);
    p.n_contrib = const_cast<uint32_t *>(n_contrib);
    p.vis = const_cast<uint32_t *>(vis);
    p.vis_words = vis_words;
    p.dL_dimage = dL_dimage;
    p.grad2d = grad2d;
    p.from_forward = from_forward != 0;
    p.status = dev_status;
    return cuda_status(launch_render_bwd(p, static_cast<cudaStream_t>(stream)));
}

hgs_status hgs_render_stats(const hgs_proj *proj, int n, const uint32_t *ids, const uint32_t *ranges,
                            const hgs_camera *cams_host, const hgs_camera *cams_dev, int n_views,
                            const hgs_config *cfg, void *ws, size_t ws_bytes, float *image, float *final_T,
                            uint32_t *n_contrib, uint32_t *vis, size_t vis_words, const float *dL_dimage,
                            float *grad2d, unsigned long long *counters, int *dev_status, void *stream) {
    RenderLaunch p;
    hgs_status st = render_common(proj, n, ids, ranges, cams_host, cams_dev, n_views, cfg, ws, ws_bytes, &p);
    if (st != HGS_OK) return st;
    if (!image || !final_T || !n_contrib || !vis || !dL_dimage || !counters ||
        (n > 0 && (!grad2d || !aligned16(grad2d))))
        return HGS_ERR_INVALID;
    p.image = image;
    p.final_T = final_T;
    p.n_contrib = n_contrib;
    p.vis = vis;
    p.vis_words = vis_words;
    p.dL_dimage = dL_dimage;
    p.grad2d = grad2d;
    p.status = dev_status;
    p.counters = counters;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(counters, 0, 8 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_render_fwd(p, s);
    if (e == cudaSuccess) e = launch_render_bwd(p, s);
    return cuda_status(e);
}

hgs_status hgs_project_bwd(const hgs_gaussians *g, const hgs_camera *cams_host, const hgs_camera *cams_dev,
                           int n_views, const hgs_config *cfg, const float *grad2d, const hgs_gaussian_grads *out,
                           uint32_t *fp64_list, int *dev_status, void *stream) {
    ViewTable vt;
    hgs_status st = build_views(cams_host, n_views, cfg, &vt);
    if (st != HGS_OK) return st;
    if (!gaussians_ok(g) || !cams_dev || !out) return HGS_ERR_INVALID;
    if (g->n > 0 && (!grad2d || !aligned16(grad2d) || !out->means || !out->scales || !out->quats ||
                     !out->normals || !out->opac1 || !out->opac2 || !out->sh || !aligned16(out->quats) ||
                     !fp64_list))
        return HGS_ERR_INVALID;
    ProjBwdLaunch p;
    p.g = *g;
    p.cams = cams_dev;
    p.n_views = n_views;
    p.cfg = *cfg;
    p.grad2d = grad2d;
    p.out = *out;
    p.fp64_list = fp64_list;
    p.status = dev_status;
    return cuda_status(launch_project_bwd(p, static_cast<cudaStream_t>(stream)));
}

hgs_status hgs_render_bwd(const hgs_gaussians *g, const hgs_proj *proj, const uint32_t *ids, const uint32_t *ranges,
                          const hgs_camera *cams_host, const hgs_camera *cams_dev, int n_views, const hgs_config *cfg,
                          void *ws, size_t ws_bytes, const float *final_T, const uint32_t *n_contrib,
                          const uint32_t *vis, size_t vis_words, const float *dL_dimage, float *grad2d,
                          const hgs_gaussian_grads *out, int *dev_status, void *stream) {
    if (!g) return HGS_ERR_INVALID;
    hgs_status st = hgs_rasterize_bwd(proj, g->n, ids, ranges, cams_host, cams_dev, n_views, cfg, ws, ws_bytes,
                                      final_T, n_contrib, vis, vis_words, dL_dimage, grad2d, 0, dev_status, stream);
    if (st != HGS_OK) return st;
    return hgs_project_bwd(g, cams_host, cams_dev, n_views, cfg, grad2d, out, proj->fp64_list, dev_status, stream);
}

}  // extern "C"
