/*
 * hgs.h -- C ABI of the B300 (sm_103a) half-Gaussian splatting rasterizer.
 *
 * The library implements the differentiable tile rasterizer of 3D Half-Gaussian
 * Splatting (3D-HGS, CVPR 2025): projection of each half-Gaussian pair to a 2D
 * splat with SH colour, tile binning with a 64-bit (tile | depth) key radix
 * sort, per-pixel front-to-back compositing of the pair weight of Eq. 10, and
 * the matching backward pass.
 *
 * Conventions shared by every call
 *  - Ownership: the caller allocates every buffer.  No call allocates or frees
 *    memory (device or host), and none synchronises the host with the device.
 *  - Pointers: unless a parameter says "host", it is a device pointer.  Float
 *    arrays are FP32; any pointer read with vector loads (marked "16-B aligned")
 *    must be 16-byte aligned.
 *  - Streams: every call only enqueues work on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  The calls are stateless and thread-safe and
 *    can be captured in a CUDA graph, provided the host arrays they read
 *    (cams_host, cfg) keep the sizes used at capture time.
 *  - Errors, two levels.  (1) The return value reports argument validation
 *    (null pointers, sizes, unsupported options) and launch errors.  Nothing is
 *    enqueued when it is not HGS_OK.  (2) `dev_status` is a device int that
 *    kernels OR error bits into (HGS_DEV_*): pair capacity exceeded (the needed
 *    count is still written to dev_num_pairs), a bounded spin-wait that timed
 *    out, an index outside its array (the access is skipped).  The caller
 *    zeroes it, reads it after the stream completes, and discards the outputs
 *    of a step that set it.  A wait that times out never hangs the device.
 *  - Layout of multi-view outputs: views are packed one after another.  View v
 *    starts at pixel offset pix_off[v] = sum_{u<v} W_u H_u.  Images are
 *    [3, H_v, W_v] planes at float offset 3*pix_off[v].  Per-pixel arrays are
 *    [H_v, W_v] at offset pix_off[v].  Per-(view, splat) arrays are [n_views, n].
 *    Global tile ids are tile_off[v] + ty*tiles_x(v) + tx, where
 *    tile_off[v] = sum_{u<v} tiles_x(u) tiles_y(u).
 */
#ifndef HGS_H
#define HGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HGS_VERSION 2
#define HGS_MAX_VIEWS 256                 /* views per call                                     */
#define HGS_MAX_PAIRS ((1u << 30) - 1u)   /* (tile, splat) pairs per call: 30-bit sort counters */
#define HGS_MAX_SH_DEGREE 3

typedef enum {
    HGS_OK = 0,
    HGS_ERR_INVALID = 1,      /* bad argument (null pointer, size, option)  */
    HGS_ERR_CAPACITY = 2,     /* a caller buffer is too small               */
    HGS_ERR_CUDA = 3,         /* a CUDA launch or runtime call failed       */
    HGS_ERR_TIMEOUT = 4,      /* reserved for host-side waits (none today)  */
    HGS_ERR_UNSUPPORTED = 5   /* option valid in principle but not built    */
} hgs_status;

/* bits OR-ed into *dev_status by kernels */
#define HGS_DEV_CAPACITY 0x1  /* more (tile, splat) pairs than pair_capacity, or
                                 a visibility mask too small for them           */
#define HGS_DEV_TIMEOUT 0x2   /* a bounded wait between the warps of one block
                                 (the forward and backward compositing
                                 pipelines) ran past its limit (1 s); the
                                 outputs are not meaningful                     */
#define HGS_DEV_BOUNDS 0x4    /* an index was outside its array; access skipped  */

/* Half-Gaussian parameters (Sec. 3.2), activated values, [n] rows; every array
 * 16-B aligned (blocks of rows are staged with 16-byte asynchronous copies):
 *   means   [n,3]  world position mu
 *   scales  [n,3]  standard deviations (> 0), the diagonal of S in Eq. 2
 *   quats   [n,4]  rotation quaternion (w,x,y,z), any nonzero length
 *   normals [n,3]  splitting-plane normal n, any length (0 => both halves weigh 1/2)
 *   opac1   [n]    alpha_1, opacity of the half n.(x - mu) >= 0, in [0,1]
 *   opac2   [n]    alpha_2, opacity of the other half, in [0,1]
 *   sh      [n,(sh_degree+1)^2,3] real SH colour coefficients (16-B aligned)
 * The real SH basis is sqrt2 Im Y_l^|m| (m<0), Y_l^0, sqrt2 Re Y_l^m (m>0) of the
 * complex harmonics with the Condon-Shortley phase, index l*l + l + m; the
 * colour is max(0, sum_lm c_lm Y_lm(dir) + 1/2), dir = unit(mu - camera centre). */
typedef struct {
    const float *means, *scales, *quats, *normals, *opac1, *opac2, *sh;
    int n;
    int sh_degree;
} hgs_gaussians;

/* Gradients, same shapes as hgs_gaussians (written, or added into when
 * hgs_config.accumulate is set). */
typedef struct {
    float *means, *scales, *quats, *normals, *opac1, *opac2, *sh;
} hgs_gaussian_grads;

/* Pinhole camera.  viewmat is world -> camera, row-major 3x4 [R | t]; pixel
 * coordinates are u = fx x/z + cx, v = fy y/z + cy, and pixel (i, j) has its
 * centre at (i + 1/2, j + 1/2).  Splats with camera z <= near_plane are culled.
 * bg is the background colour composited behind the splats. */
typedef struct {
    float viewmat[12];
    float fx, fy, cx, cy;
    int width, height;
    float near_plane;
    float bg[3];
} hgs_camera;

/* Options.
 *   tile_w, tile_h : 8x8, 16x16 or 32x8.  The tile shape changes the image
 *                    (tiles are culled by the 3-sigma square, not per pixel).
 *   batch          : splats staged in shared memory per round: 32, 64, 128,
 *                    224, 256 or 512 (0 = tile_w*tile_h); the backward's three
 *                    ring buffers hold min(batch, 224) splats each (0 = 224, 64
 *                    for 8x8 tiles)
 *   lowpass        : l added to the diagonal of hat Sigma (3D-GS uses 0.3)
 *   fov_clamp      : 1 = clamp x/z, y/z to +-1.3 tan(fov/2) inside J (3D-GS)
 *   plain          : 1 = plain 3D-GS weight alpha1 * hat G (no half split)
 *   persistent     : 1 = one persistent launch over a (view, tile) work queue,
 *                    0 = one thread block per tile
 *   accumulate     : 1 = hgs_project_bwd / hgs_render_bwd add into the
 *                    gradient buffers instead of overwriting them (to sum
 *                    gradients over several calls, e.g. one call per view)
 *   rect_mode      : tiles a splat is binned into.  0 = the square of half-side
 *                    ceil(3 sqrt(lambda_max)) (3D-GS).  1 = the valid region of
 *                    each half (Sec. 3.4): the bounding box, under the projection,
 *                    of the 3-sigma half-ellipsoid of every half whose opacity
 *                    reaches 1/255 (the whole ellipse's tangent edges where the
 *                    half's outer surface faces that way, the splitting plane's
 *                    cut ellipse elsewhere; low-pass added in quadrature); a splat
 *                    with both halves below 1/255 is culled.  Mode 1 changes the
 *                    image where a splat reached beyond its 3-sigma ellipse.
 *                    2 = as 1, with the splitting edge taken from Algorithm 1
 *                    (Suppl. B.1): the projection of the flattened covariance
 *                    whose in-plane part is the Gaussian's covariance given the
 *                    normal coordinate and whose variance along n is a hundredth
 *                    of the smaller in-plane one (a little wider than mode 1). 
 *   mip            : 1 = Mip-Splatting-HGS: the low-pass is Mip-Splatting's 2D
 *                    filter, a normalised convolution with N(0, lowpass I) rather
 *                    than a dilation, so both opacities are scaled by
 *                    sqrt(det hat Sigma_0 / det hat Sigma) per (view, splat) (hat
 *                    Sigma_0: before the low-pass).  The records then hold the
 *                    scaled opacities and grad2d[7..8] is taken w.r.t. them;
 *                    hgs_project_bwd carries the factor into the parameters.
 *                    Mip-Splatting's 3D filter needs no kernel: it is the scales
 *                    sqrt(s^2 + s_f^2) and opacities scaled by prod s / prod
 *                    sqrt(s^2 + s_f^2), applied by the caller.  The rect_mode 1
 *                    and 2 opacity test uses the unscaled opacities (a superset). */
typedef struct {
    int tile_w, tile_h;
    int batch;
    float lowpass;
    int fov_clamp;
    int plain;
    int persistent;
    int accumulate;
    int rect_mode;
    int mip;
} hgs_config;

/* Per-(view, splat) projected records written by hgs_project, [n_views*n] rows.
 *   rec    [.,16] (16-B aligned): mu_x = ax + fx, mu_y = ay + fy with (ax, ay)
 *                  integers and (fx, fy) the remainders (so the centre keeps
 *                  ~1e-7 px accuracy anywhere in the image), then u11, u12, u22,
 *                  w'_x, w'_y, alpha1, alpha2, r, g, b, 0, 0.  Layout:
 *                  [ax, ay, fx, fy, u11, u12, u22, w'x, w'y, a1, a2, r, g, b, 0, 0].
 *                  U = [[u11, u12], [0, u22]] is the Cholesky factor of the conic
 *                  hat Sigma^-1 = U^T U; w' = hat Sigma^-1 k / sqrt(2 v), so that
 *                  the half-plane fraction is P(d) = 1/2 erfc(-w'.d) (Eq. 8).
 *   depth  [.]     (16-B aligned) camera-space z of the mean (the sort key's low
 *                  32 bits)
 *   rect   [.,4]   (16-B aligned) covered tiles [x0,x1) x [y0,y1) of the view
 *   tiles  [.]     (16-B aligned) number of covered tiles, 0 if culled
 *   fp64_list [1 + n_views*n] uint32 scratch: hgs_project gathers here the
 *                  (view, splat) records whose splitting plane nearly contains
 *                  the ray (v < 1e-3 var_s) and recomputes their half-plane terms
 *                  in FP64 in a second kernel.  Contents are not meaningful to
 *                  the caller; hgs_render_bwd reuses it for the same purpose.     */
typedef struct {
    float *rec;
    float *depth;
    int32_t *rect;
    uint32_t *tiles;
    uint32_t *fp64_list;
} hgs_proj;

/* ---- sizes ------------------------------------------------------------- */

/* Tiles and pixels of all views (host arrays).  Returns HGS_ERR_INVALID on a
 * bad camera or option.  Any output pointer may be NULL. */
hgs_status hgs_layout(const hgs_camera *cams_host, int n_views, const hgs_config *cfg,
                      int *total_tiles, int64_t *total_pixels);

/* Workspace bytes needed by hgs_bin for n splats, n_views views and room for
 * pair_capacity (tile, splat) pairs. */
size_t hgs_bin_workspace_size(int n, int n_views, size_t pair_capacity);

/* Workspace bytes needed by hgs_render_fwd / hgs_rasterize_bwd / hgs_render_bwd. */
size_t hgs_render_workspace_size(const hgs_camera *cams_host, int n_views, const hgs_config *cfg,
                                 int n);

/* uint32 words of the visibility mask that hgs_render_fwd writes and the backward
 * compositing reads, for up to pair_capacity (tile, splat) pairs:
 * (pair_capacity / 32 + total_tiles + 1) * tile_w * tile_h / 32.  0 on a bad
 * camera or option. */
size_t hgs_vis_words(const hgs_camera *cams_host, int n_views, const hgs_config *cfg,
                     size_t pair_capacity);

/* ---- A1-A2: projection and SH colour ------------------------------------ */

/* Projects every splat into every view: Sigma^w = R S S^T R^T (Eq. 2),
 * hat Sigma = top-left 2x2 of J W Sigma^w W^T J^T (Eq. 3-5) plus the low-pass,
 * its inverse (the conic), mu-hat, the 3-sigma tile rect and the half-plane
 * terms of Eq. 7-8 (w'), and the SH colour.  Binning fields follow a fixed FP32
 * operation order without fused multiply-adds.  Splats whose splitting plane
 * nearly contains the ray (v < 1e-3 var_s, where the half-plane variance v
 * loses most of its FP32 digits) have their half-plane terms recomputed in FP64
 * by a second kernel over the list gathered in proj->fp64_list.
 * cams_host: host copy (sizes); cams_dev: the same cameras in device memory. */
hgs_status hgs_project(const hgs_gaussians *g, const hgs_camera *cams_host,
                       const hgs_camera *cams_dev, int n_views, const hgs_config *cfg,
                       const hgs_proj *out, int *dev_status, void *stream);

/* ---- A3-A5: binning ------------------------------------------------------ */

/* The (tile, splat) pairs sorted by the 64-bit key (global tile id << 32) |
 * bits of depth, one pair per covered tile of every (view, splat), ties in
 * ascending value order (value = view*n + splat), and per-tile [start, end)
 * ranges (ranges[2*t], ranges[2*t+1]; [0,0) for an empty tile).  This is the
 * stable LSD radix sort (8-bit digits) of the keys over the bits in use; its
 * passes over the depth half (as many 8-bit passes as the drawn splats' depth
 * range needs, at most four) run on the n_views*n per-splat depths before
 * the splats are expanded into their tiles, which gives the same order.
 *   keys_out [pair_capacity] uint64, optional (NULL: not written),
 *   ids_out  [pair_capacity] uint32, ranges [2*total_tiles] uint32,
 *   dev_num_pairs: uint64, the pair count.
 * If the count exceeds pair_capacity, HGS_DEV_CAPACITY is set, the count is
 * still written, and keys/ids/ranges are not meaningful. */
hgs_status hgs_bin(const hgs_proj *proj, int n, const hgs_camera *cams_host, int n_views,
                   const hgs_config *cfg, void *ws, size_t ws_bytes, size_t pair_capacity,
                   uint64_t *keys_out, uint32_t *ids_out, uint32_t *ranges,
                   uint64_t *dev_num_pairs, int *dev_status, void *stream);

/* Same as hgs_bin, but its scratch workspace is a fixed device array inside this
 * library instead of caller memory; the paper has no counterpart (it is an
 * interface for callers, not part of the method).  It is for callers that must
 * not allocate device memory: plug-ins inside a host application that owns the
 * device-memory budget, and real-time loops that cannot afford a driver
 * allocation (which may synchronise the device).  The caller still provides
 * every input and output; this call allocates nothing.
 * Limit: hgs_bin_workspace_size(n, n_views, pair_capacity) must not exceed
 * HGS_BIN_STATIC_SCRATCH_BYTES (32 MiB, held on every GPU that loads the library
 * until the process exits), else HGS_ERR_CAPACITY and nothing is enqueued.
 * The first call on a device (with that device current) looks up the array's
 * device address, and a call looks it up again when the device's context has
 * changed since (e.g. after cudaDeviceReset); make that first call before any
 * stream capture.  All calls share the array, which keeps the previous call's
 * contents (the call clears what must start at zero): calls that overlap on the
 * GPU (different streams or threads) race; calls in order on one stream are
 * safe.  Errors otherwise as hgs_bin. */
#define HGS_BIN_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
hgs_status hgs_bin_static(const hgs_proj *proj, int n, const hgs_camera *cams_host, int n_views,
                          const hgs_config *cfg, size_t pair_capacity, uint64_t *keys_out,
                          uint32_t *ids_out, uint32_t *ranges, uint64_t *dev_num_pairs,
                          int *dev_status, void *stream);

/* ---- A6: forward compositing ----------------------------------------------- */

/* Per pixel, front to back over its tile's sorted list (Sec. 3.3 blending with
 * the pair weight of Eq. 10):
 *   a = min(0.99, (alpha2 + (alpha1 - alpha2) P(d)) exp(-d^T conic d / 2)),
 * skip a < 1/255, stop before a splat that would take T below 1e-4.
 *   image     [3*total_pixels] : C + T_final * bg, per view [3,H,W]
 *   final_T   [total_pixels]   : T after the last composited splat
 *   n_contrib [total_pixels]   : 1 + position (in the tile's list) of the last
 *                                composited splat, 0 if none
 *   vis       [vis_words]      : visibility mask, hgs_vis_words() words for the
 *                                pair capacity.  Per tile t with sorted list
 *                                [beg, end), per 32-entry chunk c of that list
 *                                and per 8x4 pixel block w of the tile (row-major
 *                                blocks), the word at
 *                                ((beg >> 5) + t + c) * (tile_w*tile_h/32) + w
 *                                has bit j set iff entry beg + 32c + j was
 *                                composited at some pixel of block w.  Words of
 *                                chunks past every pixel's last composited entry
 *                                are left as they were.  A word beyond vis_words
 *                                is not written and sets HGS_DEV_CAPACITY.
 * Within a block, one warp stages each tile's list in batches and the others walk
 * them, synchronised by bounded waits: HGS_DEV_TIMEOUT if one runs out.
 * grad2d_clear (optional, [n_views*n, 12] floats, 16-B aligned; NULL: none): a
 * buffer the kernel sets to zero while it composites (its memory traffic is
 * light, so the stores cost it little), for a following hgs_rasterize_bwd given
 * from_forward = 1, which then skips clearing grad2d itself. */
hgs_status hgs_render_fwd(const hgs_proj *proj, int n, const uint32_t *ids,
                          const uint32_t *ranges, const hgs_camera *cams_host,
                          const hgs_camera *cams_dev, int n_views, const hgs_config *cfg,
                          void *ws, size_t ws_bytes, float *image, float *final_T,
                          uint32_t *n_contrib, uint32_t *vis, size_t vis_words,
                          float *grad2d_clear, int *dev_status, void *stream);

/* ---- A7: backward compositing ---------------------------------------------- */

/* Adjoint of hgs_render_fwd for the upstream gradient dL_dimage (layout of
 * image).  Per pixel, back to front from n_contrib, the transmittance is
 * rebuilt by division (T_i = T_{i+1} / (1 - a_i)).  It writes the screen-space
 * gradient of every (view, splat):
 *   grad2d [n_views*n, 12] (16-B aligned): d mu_x, d mu_y, d A, d B, d C,
 *          d w'_x, d w'_y, d alpha1, d alpha2, d r, d g, d b.
 * The call zeroes grad2d first and builds its tile queue in ws, unless
 * from_forward is non-zero: the caller then vouches that this call follows, on
 * the same stream, the hgs_render_fwd it differentiates, called with the same
 * proj, ranges, cameras, config and ws and with grad2d as its grad2d_clear, and
 * that nothing has used ws or written grad2d in between (a second backward of
 * the same forward passes 0).  grad2d is then already zero and the forward's
 * tile queue is reused.  Gradients through the 0.99 clamp, through
 * skipped or terminated splats and through P of a degenerate plane are 0.
 * final_T, n_contrib and vis are the outputs of the hgs_render_fwd being
 * differentiated (same inputs, tile shape and batch): each 8x4 pixel block visits
 * only the entries its vis words mark, and every pixel re-evaluates those with
 * the forward's arithmetic, so its decisions are the forward's.  A word beyond
 * vis_words counts as all ones (every entry visited; same result, slower).
 * Within a block, one warp stages each tile's list in batches and the others walk
 * them, synchronised by bounded waits: HGS_DEV_TIMEOUT if one runs out. */
hgs_status hgs_rasterize_bwd(const hgs_proj *proj, int n, const uint32_t *ids,
                             const uint32_t *ranges, const hgs_camera *cams_host,
                             const hgs_camera *cams_dev, int n_views, const hgs_config *cfg,
                             void *ws, size_t ws_bytes, const float *final_T,
                             const uint32_t *n_contrib, const uint32_t *vis, size_t vis_words,
                             const float *dL_dimage, float *grad2d, int from_forward,
                             int *dev_status, void *stream);

/* ---- A8: projection backward ------------------------------------------------ */

/* Chain rule from grad2d through Eq. 8, Eq. 3-5, Eq. 2 and the SH colour to
 * every parameter, summed over views.  Writes every entry of `out` (adds into
 * it when cfg->accumulate is set).  Near-degenerate (view, splat) pairs (as in
 * hgs_project) take the FP64 adjoint in a second kernel; fp64_list is their
 * [1 + n_views*n] uint32 scratch list. */
hgs_status hgs_project_bwd(const hgs_gaussians *g, const hgs_camera *cams_host,
                           const hgs_camera *cams_dev, int n_views, const hgs_config *cfg,
                           const float *grad2d, const hgs_gaussian_grads *out,
                           uint32_t *fp64_list, int *dev_status, void *stream);

/* hgs_rasterize_bwd followed by hgs_project_bwd; grad2d is caller scratch. */
hgs_status hgs_render_bwd(const hgs_gaussians *g, const hgs_proj *proj, const uint32_t *ids,
                          const uint32_t *ranges, const hgs_camera *cams_host,
                          const hgs_camera *cams_dev, int n_views, const hgs_config *cfg,
                          void *ws, size_t ws_bytes, const float *final_T,
                          const uint32_t *n_contrib, const uint32_t *vis, size_t vis_words,
                          const float *dL_dimage, float *grad2d,
                          const hgs_gaussian_grads *out, int *dev_status, void *stream);

/* ---- measurement ------------------------------------------------------------------- */

/* Work counters for the roofline: runs hgs_render_fwd and hgs_rasterize_bwd (same
 * outputs, same arithmetic) in variants that also count, into counters[8]
 * (uint64, zeroed by the call):
 *   [0] forward (pixel, splat) iterations  [1] forward full evaluations (past the
 *   3-sigma/opacity cut-off)  [2] splats composited  [3] backward iterations
 *   [4] backward full evaluations  [5] backward contributing pairs
 *   [6] backward (warp, splat) visits with more than 12 contributing lanes (folded
 *   by shuffles before the atomics: lane l + 16 into lane l, and above 16 lanes
 *   also l + 8 into l)  [7] backward gradient atomics: lanes that added their 12
 *   gradients to grad2d (three 16-byte vector reductions each), at most [5]. */
hgs_status hgs_render_stats(const hgs_proj *proj, int n, const uint32_t *ids, const uint32_t *ranges,
                            const hgs_camera *cams_host, const hgs_camera *cams_dev, int n_views,
                            const hgs_config *cfg, void *ws, size_t ws_bytes, float *image, float *final_T,
                            uint32_t *n_contrib, uint32_t *vis, size_t vis_words, const float *dL_dimage,
                            float *grad2d, unsigned long long *counters, int *dev_status, void *stream);

/* Issue-rate probe for the compositing kernels' roofline (the paper has no
 * counterpart: it measures this GPU, not the method).  kind 0 runs independent
 * chains of FP32 fused multiply-adds, kind 1 independent chains of the MUFU
 * ex2.approx instruction, on blocks_per_sm (1-4) blocks of 512 threads per SM,
 * each thread doing iters x 16 x 8 operations.  *lane_ops (host, optional)
 * receives the number of lane-operations enqueued, so that a caller timing the
 * launch with events on `stream` gets lane-operations per second.  sink is a
 * device float the kernel may write (never in practice); it exists only so
 * that the arithmetic is not optimised away.  HGS_ERR_INVALID on a bad
 * argument (nothing enqueued). */
hgs_status hgs_probe_peak(int kind, int blocks_per_sm, int iters, float *sink, double *lane_ops,
                          void *stream);

/* Self-test of the bounded wait of the compositing pipelines (hgs_render_fwd,
 * hgs_rasterize_bwd; the paper has no counterpart).  One warp waits on a shared-memory mbarrier that nothing completes;
 * the wait ends at its bound (about 1 s), HGS_DEV_TIMEOUT is OR-ed into
 * *dev_status and the kernel returns, so the device stays usable.  HGS_ERR_INVALID
 * if dev_status is NULL (nothing enqueued). */
hgs_status hgs_selftest_wait(int *dev_status, void *stream);

/* ---- misc ------------------------------------------------------------------- */
const char *hgs_status_string(hgs_status s);
int hgs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HGS_H */
