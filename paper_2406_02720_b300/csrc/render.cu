// Per-pixel compositing of half-Gaussian splats (A6) and its adjoint (A7).
//
// A block has one thread per pixel of a tile (256 for 16x16) and one staging warp,
// which stages the tile's depth-sorted list in batches into a ring of shared-memory
// buffers that the pixel warps walk at their own pace, with no block barriers
// (mbarriers with bounded waits).  For each (pixel, splat) pair:
//   d = p - mu-hat,  hat G = exp(-1/2 |U d|^2), conic = U^T U  (Eq. 4-5)
//   P = 1/2 erfc(-w'.d)                                         (Eq. 7-8)
//   a = min(0.99, (alpha2 + (alpha1 - alpha2) P) hat G)          (Eq. 10)
// composited front to back (Sec. 3.3).  A splat with a < 1/255 is skipped, and
// a splat that would take T below 1e-4 ends the pixel's list (3D-GS rules).
// The forward's staging warp stops staging a tile once every pixel of it has finished
// (forward 0.690 -> 0.679 ms against two 128-thread blocks per tile, each staging the
// whole list and meeting at two block barriers per batch).
//
// erfc comes from Abramowitz & Stegun, Handbook of Mathematical Functions, 7.1.26
// (|error| <= 1.5e-7 on erf), which needs exp(-z^2); the backward reuses that
// exponential for dP/dz = exp(-z^2)/sqrt(pi).  Exponentials use the ex2.approx
// instruction with U pre-scaled by sqrt(log2(e)/2), so the exponent in base 2 is
// -(s1^2 + s2^2) with (s1, s2) = U d: a sum of squares, accurate for thin
// splats, never positive.  Forward and backward
// evaluate the same inline function with explicit _rn intrinsics, so their
// per-splat decisions are bit-identical.
//
// Each warp owns an 8x4 block of the tile's pixels.  In the forward, per 32 staged
// splats, each 4x4 half of the block tests every splat's cut-off ellipse (the pixels
// where alpha could reach 1/255) against itself with separating axes (x, y and the
// ellipse's minor axis) and ballots; each half then walks its own hits, the two
// halves in step: a warp takes as many steps as the busier half has hits instead of
// one per hit of either half (0.77 of them at 3M splats, 1080p; forward 0.676 ->
// 0.652 ms).  The bounds are inflated past the cut-off, so culling changes no
// per-pixel decision.  The forward also records, per 32-entry chunk of the list, which
// splats it composited at any pixel of the block (the visibility mask, one word per
// chunk and block).  The backward visits exactly those: the 24% of its (warp, splat)
// visits in which no pixel contributes, and its own culling, are gone (backward 1.294
// -> 1.206 ms, forward 0.661 -> 0.688 ms for writing the mask; measured at 3M splats,
// 1080p, same session).  Forward and backward evaluate the weight identically, so the
// mask drops no contributing pair; with no room for it the backward visits everything.
//
// The backward walks each pixel's list back to front from its last composited
// splat, rebuilding the transmittance by division, T_i = T_{i+1} / (1 - a_i).  Its
// warps are not held together by block barriers: a staging warp fills a ring of
// three batch buffers and each pixel warp walks them at its own pace (mbarriers,
// bounded waits; 1.318 -> 1.294 ms against block-synchronous batches).
// The 12 screen-space gradients of a (warp, splat) leave as per-lane float4
// atomic adds, with one shuffle level folding lane pairs first when more than 12
// lanes contribute, and a second when more than 16 do.
//
// Persistent mode (the default): a grid of resident blocks pops tiles from an
// atomic queue whose order is heaviest-first (bucketed by list length).
#include <algorithm>
#include <atomic>

#include "hgs_internal.cuh"

namespace hgs {
namespace {

constexpr float kUScale = 0.84932180028801907f;   // sqrt(log2(e) / 2)
constexpr float kInvUScale2 = 1.3862943611198906f; // 1 / kUScale^2 = 2 ln 2
constexpr float kInvSqrtPi = 0.56418958354775628f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kStepDetect = 1e20f;     // |w'| beyond this: step-mode splat (no dP)
// Abramowitz & Stegun 7.1.26
constexpr float kAsP = 0.3275911f;
constexpr float kAs1 = 0.254829592f, kAs2 = -0.284496736f, kAs3 = 1.421413741f;
constexpr float kAs4 = -1.453152027f, kAs5 = 1.061405429f;
// Staged w' is scaled by sqrt(log2 e), so z' = w'.d gives exp(-z^2) = 2^-(z'^2) with no
// multiply; the A&S argument absorbs the scale in its constant p.  The coefficients
// are halved so that the polynomial gives erfc(|z|) / 2 directly.
constexpr float kSqrtLog2e = 1.2011224087864498f;
constexpr float kInvSqrtLog2e = 0.83255461115769775f;
constexpr float kAsPs = kAsP * kInvSqrtLog2e;
constexpr float kAh1 = 0.5f * kAs1, kAh2 = 0.5f * kAs2, kAh3 = 0.5f * kAs3, kAh4 = 0.5f * kAs4, kAh5 = 0.5f * kAs5;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed pairs of binary32 values for the paired FP32 instructions of sm_100 and
// later (add / sub / mul .rn.f32x2 act on both halves of a 64-bit register pair at the
// cost of one instruction).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// One staged batch of a tile's list in shared memory, a float4 record per field
// group so that a warp-uniform visit reads a whole group with one broadcast load.
template <int BATCH, bool BWD>
struct Batch {
    float4 g0[BATCH];    // mx, my (tile-local centre), u11, u12 (Cholesky factor of the conic, x kUScale)
    float4 g1[BATCH];    // u22, qcut (skip when s1^2 + s2^2 exceeds it), w'x, w'y
    float4 g2[BATCH];    // alpha2, alpha1 - alpha2, r, g
    float4 cu[BWD ? 1 : BATCH];   // forward culling vs a 4x4 block centred at c: |cx-mx| <= .x,
                                  // |cy-my| <= .y, |(c-mu).(.z,.w)| <= 1
    float b[BATCH];
    float dzk[BWD ? BATCH : 1];   // backward: (alpha1 - alpha2) / sqrt(pi), 0 for a step-mode splat
    uint32_t id[BATCH];
};

// Stages splat id into slot k.  The centre is made tile-local,
// (anchor - tile origin) + fraction, so that pixel offsets are formed from small
// numbers and stay exact to ~1e-7 px anywhere in the image.
//
// Culling data (forward only): the cut-off set E = {d : |U~ d|^2 <= qcut} has support
// function h(n) = sqrt(qcut) |U~^-T n| in any unit direction n.  A 4x4 block of pixels
// whose centres lie within +-1.5 of its centre c can touch E only if, for n = x, y and
// n = the ellipse's minor axis, |n.(c - mu)| <= h(n) + 1.5(|n_x| + |n_y|).  Every bound
// is inflated (x1.001 + 1e-3) so that no block whose pixels pass the FP32 cut-off test
// of eval_alpha is culled.  The backward needs none: it visits only the splats that the
// forward composited somewhere in the warp's block (the visibility mask).
template <int BATCH, bool BWD>
__device__ __forceinline__ void stage(const float4 *__restrict__ rec, uint32_t id, Batch<BATCH, BWD> &s, int k,
                                      float ox, float oy, bool plain) {
    const float4 r0 = __ldg(rec + 4 * (size_t)id);
    const float4 r1 = __ldg(rec + 4 * (size_t)id + 1);
    const float4 r2 = __ldg(rec + 4 * (size_t)id + 2);
    const float4 r3 = __ldg(rec + 4 * (size_t)id + 3);
    const float mx = __fadd_rn(__fsub_rn(r0.x, ox), r0.z);
    const float my = __fadd_rn(__fsub_rn(r0.y, oy), r0.w);
    const float u11 = __fmul_rn(kUScale, r1.x), u12 = __fmul_rn(kUScale, r1.y), u22 = __fmul_rn(kUScale, r1.z);
    const float a1 = r2.y, a2 = plain ? r2.y : r2.z;     // plain 3D-GS: alpha = alpha1 G
    const float amax = fmaxf(a1, a2);
    // alpha <= amax * G < 1/255 whenever log2 G < -log2(255 amax); 1e-3 covers ex2/lg2 error
    const float qcut = amax > 0.0f ? __fadd_rn(lg2_approx(__fmul_rn(255.0f, amax)), 1e-3f) : -1.0f;
    s.g0[k] = make_float4(mx, my, u11, u12);
    const float wx = __fmul_rn(r1.w, kSqrtLog2e), wy = __fmul_rn(r2.x, kSqrtLog2e);
    s.g1[k] = make_float4(u22, qcut, wx, wy);
    s.g2[k] = make_float4(a2, __fsub_rn(a1, a2), r2.w, r3.x);
    s.b[k] = r3.y;
    // d P / d(w'.d) = exp(-(w'.d)^2) / sqrt(pi); a step-mode splat (|w'| ~ 2^80) has none
    if (BWD) s.dzk[k] = (!plain && fabsf(wx) + fabsf(wy) < kStepDetect) ? (a1 - a2) * kInvSqrtPi : 0.0f;
    s.id[k] = id;
    if (BWD) return;
    float4 cu = make_float4(-1.0f, -1.0f, 0.0f, 0.0f);
    if (qcut >= 0.0f) {
        // Approximate reciprocals and roots (a few ulp) are enough here: every bound
        // is inflated by 1.001 and 1e-3 px, far beyond their error.
        const float rq = sqrt_approx(qcut);
        const float i11 = rcp_approx(u11), i22 = rcp_approx(u22);
        // axis-aligned half-extents: h(e_x) = rq |U^-T e_x|, h(e_y) = rq / u22
        const float ru = u12 * i22;
        const float hx = rq * sqrt_approx(1.0f + ru * ru) * i11;
        const float hy = rq * i22;
        // minor axis: eigenvector of Q = U^T U for its larger eigenvalue
        const float A = u11 * u11, B = u11 * u12, C = u12 * u12 + u22 * u22;
        const float lmax = 0.5f * (A + C) + sqrt_approx(0.25f * (A - C) * (A - C) + B * B);
        float nx = A >= C ? lmax - C : B;
        float ny = A >= C ? B : lmax - A;
        const float nl2 = nx * nx + ny * ny;
        if (nl2 > 0.0f && nl2 < 1e30f) {
            const float il = rsqrtf(nl2);
            nx *= il;
            ny *= il;
        } else {
            nx = 1.0f;
            ny = 0.0f;
        }
        // h(n) = rq |z| with U^T z = n, for the (nearly) unit n actually stored: the
        // test below uses h of the stored direction, so it stays exact whatever the
        // rounding of n
        const float z1 = nx * i11;
        const float z2 = (ny - u12 * z1) * i22;
        const float hn = rq * sqrt_approx(z1 * z1 + z2 * z2);
        constexpr float ex = 1.5f;     // half-extents of the 4x4 block
        const float tn = hn * 1.001f + 1e-3f + (fabsf(nx) * ex + fabsf(ny) * 1.5f) * 1.0001f;
        const float itn = rcp_approx(tn);
        cu = make_float4(hx * 1.001f + 1e-3f + ex, hy * 1.001f + 1e-3f + 1.5f, nx * itn, ny * itn);
    }
    s.cu[k] = cu;
}

// Forward: can slot j touch the 4x4 blocks centred at (cx, cy) (h0) and (cx + 4, cy) (h1), the
// two halves of a warp's 8x4 block?  (conservative, see stage)
template <class SB>
__device__ __forceinline__ void cull_halves(const SB &s, int j, float cx, float cy, bool &h0, bool &h1) {
    const float2 m = *reinterpret_cast<const float2 *>(&s.g0[j]);
    const float4 cu = s.cu[j];
    const float dx0 = cx - m.x, dx1 = (cx + 4.0f) - m.x, dy = cy - m.y;
    const float ty = dy * cu.w;
    const bool yok = fabsf(dy) <= cu.y;
    h0 = yok && fabsf(dx0) <= cu.x && fabsf(__fmaf_rn(dx0, cu.z, ty)) <= 1.0f;
    h1 = yok && fabsf(dx1) <= cu.x && fabsf(__fmaf_rn(dx1, cu.z, ty)) <= 1.0f;
}

struct Eval {
    float a, G, P, dx, dy, e, s1, s2;
    bool clamped;
};

// The per-(pixel, splat) weight of Eq. 10; true if the splat is composited
// (a >= 1/255).  Identical instruction sequence in forward and backward.
template <class SB>
__device__ __forceinline__ bool eval_alpha(f32x2 fp, const SB &s, int k, Eval &ev) {
    const float4 g0 = s.g0[k];
    const float2 g1 = *reinterpret_cast<const float2 *>(&s.g1[k]);   // u22, qcut
    // pixel offset d = p - mu (both coordinates in one paired subtraction, rounded as two)
    float dx, dy;
    unpack2(sub2(fp, pack2(g0.x, g0.y)), dx, dy);
    const float s1 = __fmaf_rn(g0.z, dx, __fmul_rn(g0.w, dy));
    const float s2 = __fmul_rn(g1.x, dy);
    const float q = __fmaf_rn(s1, s1, __fmul_rn(s2, s2));
    if (!(q <= g1.y)) { ev.G = -1.0f; return false; }
    const float2 w = *reinterpret_cast<const float2 *>(&s.g1[k].z);  // sqrt(log2 e) w'
    const float2 al = *reinterpret_cast<const float2 *>(&s.g2[k]);   // alpha2, alpha1 - alpha2
    const float G = ex2_approx(-q);
    const float z = __fmaf_rn(w.x, dx, __fmul_rn(w.y, dy));          // sqrt(log2 e) w'.d
    const float u = fabsf(z);
    const float t = rcp_approx(__fmaf_rn(kAsPs, u, 1.0f));
    float poly = __fmaf_rn(kAh5, t, kAh4);
    poly = __fmaf_rn(poly, t, kAh3);
    poly = __fmaf_rn(poly, t, kAh2);
    poly = __fmaf_rn(poly, t, kAh1);
    poly = __fmul_rn(poly, t);
    const float e = ex2_approx(-__fmul_rn(u, u));                      // exp(-(w'.d)^2)
    const float h = __fmul_rn(poly, e);                                 // erfc(|w'.d|) / 2
    const float P = z >= 0.0f ? __fsub_rn(1.0f, h) : h;
    const float A = __fmaf_rn(al.y, P, al.x);
    const float araw = __fmul_rn(A, G);
    ev.clamped = araw > kAlphaMax;
    ev.a = ev.clamped ? kAlphaMax : araw;
    ev.G = G; ev.P = P; ev.dx = dx; ev.dy = dy; ev.e = e; ev.s1 = s1; ev.s2 = s2;
    return ev.a >= kAlphaMin;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

__device__ __forceinline__ void add_counters(unsigned long long *dst, unsigned long long a, unsigned long long b,
                                             unsigned long long c, unsigned long long d) {
    a = warp_sum_u64(a); b = warp_sum_u64(b); c = warp_sum_u64(c); d = warp_sum_u64(d);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(dst, a);
        if (b) atomicAdd(dst + 1, b);
        if (c) atomicAdd(dst + 2, c);
        if (d) atomicAdd(dst + 3, d);
    }
}

struct TileInfo {
    int view, tx, ty, W, H;
    uint32_t beg, end;
    long long pix_off;
    float bg[3];
};

template <int TW, int TH>
__device__ __forceinline__ TileInfo tile_info(const RenderLaunch &p, int gtile) {
    TileInfo ti;
    ti.view = view_of_tile(p.vt, gtile);
    const int local = gtile - p.vt.tile_off[ti.view];
    const int tx_n = p.vt.tiles_x[ti.view];
    ti.tx = local % tx_n;
    ti.ty = local / tx_n;
    const hgs_camera &cam = p.cams[ti.view];
    ti.W = cam.width;
    ti.H = cam.height;
    ti.bg[0] = cam.bg[0]; ti.bg[1] = cam.bg[1]; ti.bg[2] = cam.bg[2];
    ti.beg = p.ranges[2 * (size_t)gtile];
    ti.end = p.ranges[2 * (size_t)gtile + 1];
    if (ti.end < ti.beg) ti.end = ti.beg;
    ti.pix_off = p.vt.pix_off[ti.view];
    return ti;
}

// Work queue of the persistent kernels (k_queue_count / k_queue_fill build the order).
struct Queue {
    uint32_t counter_fwd, counter_bwd;
    uint32_t bucket_count[33];
    uint32_t bucket_cursor[33];
};

// ---- backward ------------------------------------------------------------------------

// A splat's 12 gradients from the lanes of a warp go to global memory as float4
// atomic adds (3 per lane).  When more than kFoldAbove lanes contribute, one
// xor-shuffle level first folds lane l + 16 into lane l, so at most 16 lanes issue
// atomics: 24 instructions instead of a full 5-level reduction (~62), at the price of
// more atomic traffic, which the L2 absorbs (measured: fastest of full reduction,
// direct atomics from up to 1..32 lanes, and this split; at 3M splats, 1080p the
// backward took 1.333 / 1.325 / 1.322 / 1.327 / 1.393 ms folding above 8 / 10 / 12 /
// 16 / 24 contributing lanes, before the visibility mask; with it, 1.215 / 1.206 /
// 1.217 ms above 8 / 12 / 16 and 1.606 ms with no fold).  Above kFold2Above lanes a
// second level folds lane l + 8 into lane l, so at most 8 lanes add to the same splat
// (1.206 -> 1.169 ms; 1.171 ms above 20 lanes; a third level above 28 lanes, 1.184).
constexpr int kFoldAbove = 12;
constexpr int kFold2Above = 16;
__device__ __forceinline__ void atomic_add12(float *dst, const float g[12]) {
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    atomicAdd(d4, make_float4(g[0], g[1], g[2], g[3]));
    atomicAdd(d4 + 1, make_float4(g[4], g[5], g[6], g[7]));
    atomicAdd(d4 + 2, make_float4(g[8], g[9], g[10], g[11]));
}

// The backward runs as a pipeline with no block barriers.  One producer warp takes
// tiles from the queue, finds each tile's list end (the latest last contributor of
// its pixels, from n_contrib) and stages the list back to front in batches into a
// ring of kBwdStages shared buffers; each of the TW*TH/32 consumer warps walks the
// batches in order at its own pace.  A buffer's "full" mbarrier completes when the
// producer has staged it, its "empty" mbarrier when every consumer warp has walked
// it, so the consumers wait only for staging and the producer only for the slowest
// consumer, NB - 1 batches behind, across tile boundaries too.  Every wait is
// bounded: after kWaitNs the waiting warp sets HGS_DEV_TIMEOUT and leaves, and the
// others' waits then run out in turn, so the kernel always ends.
constexpr int kBwdStages = 3;

struct BwdHeader {
    int gtile;                  // < 0: no more work
    uint32_t bstart, bend;      // the batch's slice of the tile's list
    int first;                  // first batch of its tile (the one nearest the list end)
};

template <int BATCH, int NW>
struct BwdRing {
    Batch<BATCH, true> buf[kBwdStages];
    uint32_t vis[kBwdStages][BATCH / 32 * NW];   // the batch's visibility words, [chunk][warp block]
    BwdHeader hdr[kBwdStages];
    unsigned long long full[kBwdStages], empty[kBwdStages];   // mbarriers
};

constexpr unsigned long long kWaitNs = 1000ull * 1000 * 1000;   // 1 s

__device__ __forceinline__ uint32_t smem_addr(const void *ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase of the given parity to complete; false (and HGS_DEV_TIMEOUT) if
// it has not after kWaitNs.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, int *status) {
    const uint32_t addr = smem_addr(bar);
    unsigned long long t0 = 0;
    for (uint32_t i = 0;; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i == 0) t0 = global_ns();
        if ((i & 63u) == 63u && global_ns() - t0 > kWaitNs) {
            set_status(status, HGS_DEV_TIMEOUT);
            return false;
        }
    }
}

// Producer warp: tiles from the queue (or this block's tile), batches back to front.
template <int TW, int TH, int BATCH, bool PLAIN>
__device__ void bwd_produce(const RenderLaunch &p, BwdRing<BATCH, TW * TH / 32> &r) {
    constexpr int NB = kBwdStages, NW = TW * TH / 32;
    const int lane = threadIdx.x & 31;
    const float4 *rec = reinterpret_cast<const float4 *>(p.proj.rec);
    const uint32_t vn = (uint32_t)p.n * (uint32_t)p.vt.n_views;
    Queue *qw = reinterpret_cast<Queue *>(p.ws);
    const uint32_t *order = reinterpret_cast<const uint32_t *>(qw + 1);
    uint32_t seq = 0;
    for (int round = 0;; ++round) {
        int gtile = -1;
        if (p.cfg.persistent) {
            uint32_t item = 0;
            if (lane == 0) item = atomicAdd(&qw->counter_bwd, 1u);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item < (uint32_t)p.vt.total_tiles) gtile = (int)order[item];
        } else if (round == 0) {
            gtile = (int)blockIdx.x;
        }
        const uint32_t slot0 = seq % NB;
        if (gtile < 0) {
            // end marker in the next buffer
            if (seq >= NB && !mbar_wait(&r.empty[slot0], ((seq / NB) - 1) & 1u, p.status)) return;
            if (lane == 0) r.hdr[slot0].gtile = -1;
            __syncwarp();
            mbar_arrive(&r.full[slot0]);
            return;
        }
        const TileInfo ti = tile_info<TW, TH>(p, gtile);
        // the tile's list end: the latest last contributor of its pixels
        const int ox = ti.tx * TW, oy = ti.ty * TH;
        uint32_t ml = 0;
        for (int i = lane; i < TW * TH; i += 32) {
            const int px = ox + (i % TW), py = oy + (i / TW);
            if (px < ti.W && py < ti.H) ml = max(ml, p.n_contrib[ti.pix_off + (size_t)py * ti.W + px]);
        }
        ml = __reduce_max_sync(0xffffffffu, ml);
        const uint32_t tile_end = min(ti.end, ti.beg + ml);
        // the tile's rows of the visibility mask, as the forward placed them
        const size_t vrow = vis_row(ti.beg, gtile);
        const bool vfit = (vrow + ((ti.end - ti.beg + 31) >> 5)) * NW <= p.vis_words;
        const float fox = (float)ox, foy = (float)oy;
        for (uint32_t bend = tile_end; bend > ti.beg;) {
            // batches start at multiples of BATCH (itself a multiple of 32) in the tile's
            // list, so that their 32-entry chunks are those of the visibility mask
            const uint32_t bstart = ti.beg + ((bend - 1 - ti.beg) / BATCH) * BATCH;
            const uint32_t slot = seq % NB;
            if (seq >= NB && !mbar_wait(&r.empty[slot], ((seq / NB) - 1) & 1u, p.status)) return;
            Batch<BATCH, true> &sb = r.buf[slot];
            // the batch's visibility words (all bits set if the tile's rows had no room in
            // the mask: the warps then visit every entry, which changes no result)
            const int nw = (int)((bend - bstart + 31) >> 5) * NW;
            const size_t w0 = (vrow + ((bstart - ti.beg) >> 5)) * NW;
            for (int i = lane; i < nw; i += 32) r.vis[slot][i] = vfit ? __ldg(p.vis + w0 + i) : 0xffffffffu;
            __syncwarp();
            // lane q: the entries of chunk q that some pixel warp will visit
            uint32_t any_w = 0;
            if (lane < BATCH / 32 && lane * NW < nw) {
#pragma unroll
                for (int w = 0; w < NW; ++w) any_w |= r.vis[slot][lane * NW + w];
            }
            // only those are staged: no pixel warp reads the other slots
#pragma unroll
            for (int q = 0; q < BATCH / 32; ++q) {
                const int k = lane + 32 * q;
                const uint32_t j = bstart + k;
                const uint32_t u = __shfl_sync(0xffffffffu, any_w, q);
                if (j < bend && ((u >> lane) & 1u)) {
                    uint32_t id = p.ids[j];
                    if (id >= vn) { set_status(p.status, HGS_DEV_BOUNDS); id = 0; }
                    stage<BATCH, true>(rec, id, sb, k, fox, foy, PLAIN);
                }
            }
            if (lane == 0) {
                r.hdr[slot].gtile = gtile;
                r.hdr[slot].bstart = bstart;
                r.hdr[slot].bend = bend;
                r.hdr[slot].first = bend == tile_end;
            }
            __syncwarp();
            mbar_arrive(&r.full[slot]);           // each lane: its staged slots are released
            ++seq;
            bend = bstart;
        }
    }
}

// Consumer warp: walks each batch for its 8x4 pixel block, back to front.
template <int TW, int TH, int BATCH, bool COUNT, bool PLAIN>
__device__ void bwd_consume(const RenderLaunch &p, BwdRing<BATCH, TW * TH / 32> &r) {
    constexpr int NB = kBwdStages, NW = TW * TH / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr bool plain = PLAIN;
    float *grad = p.grad2d;
    unsigned long long c_visit = 0, c_full = 0, c_contrib = 0, c_red = 0, c_atom = 0;
    // per-tile state of this lane's pixel
    bool inside = false;
    f32x2 fp = 0;
    float T = 1.0f, g0_ = 0.0f, g1_ = 0.0f, g2_ = 0.0f, TfB = 0.0f, Sg = 0.0f;
    uint32_t last = 0, wlast = 0, beg = 0;
    for (uint32_t seq = 0;; ++seq) {
        const uint32_t slot = seq % NB;
        if (!mbar_wait(&r.full[slot], (seq / NB) & 1u, p.status)) break;
        const BwdHeader h = r.hdr[slot];
        if (h.gtile < 0) break;
        const Batch<BATCH, true> &s = r.buf[slot];
        if (h.first) {
            const TileInfo ti = tile_info<TW, TH>(p, h.gtile);
            const int bx = ti.tx * TW + (warp % (TW / 8)) * 8, by = ti.ty * TH + (warp / (TW / 8)) * 4;
            const int px = bx + (lane & 7), py = by + (lane >> 3);
            inside = px < ti.W && py < ti.H;
            const int ox = ti.tx * TW, oy = ti.ty * TH;
            fp = pack2((float)(px - ox) + 0.5f, (float)(py - oy) + 0.5f);
            const size_t HW = (size_t)ti.W * ti.H;
            const size_t pix = (size_t)py * ti.W + px;
            float Tf = 1.0f;
            g0_ = g1_ = g2_ = 0.0f;
            last = 0;
            if (inside) {
                Tf = p.final_T[ti.pix_off + pix];
                last = p.n_contrib[ti.pix_off + pix];
                const float *gi = p.dL_dimage + 3 * (size_t)ti.pix_off;
                g0_ = gi[pix]; g1_ = gi[HW + pix]; g2_ = gi[2 * HW + pix];
            }
            T = Tf;
            wlast = __reduce_max_sync(0xffffffffu, last);
            const float bgg = ti.bg[0] * g0_ + ti.bg[1] * g1_ + ti.bg[2] * g2_;
            TfB = Tf * bgg;             // d L / d a_i gets -T_final bg.g / (1 - a_i)
            // colour composited behind the current splat, dotted with this pixel's dL/dC:
            // (c_i - S_i).g = c_i.g - S_i.g, and S.g follows the same recurrence as S
            Sg = 0.0f;
            beg = ti.beg;
        }
        const uint32_t bstart = h.bstart, bend = h.bend;
        const uint32_t rel0 = bstart - beg;
        // this warp's part of the batch: nothing at or past its pixels' last splat
        const int cnt = (int)min(bend - bstart, wlast > rel0 ? wlast - rel0 : 0u);
        // the splats to visit: those the forward composited somewhere in this warp's block
        for (int c = (cnt - 1) & ~31; c >= 0; c -= 32) {
            unsigned m = r.vis[slot][(c >> 5) * NW + warp];
            if (cnt - c < 32) m &= (1u << (cnt - c)) - 1u;
            while (m) {
                const int bit = 31 - __clz(m);
                m &= ~(1u << bit);
                const int k = c + bit;
                const uint32_t pos = rel0 + k;
                Eval ev;
                ev.G = -1.0f;
                const bool cand = inside && pos < last;
                const bool contrib = cand && eval_alpha(fp, s, k, ev);
                if (COUNT) { c_visit += cand; c_full += (cand && ev.G >= 0.0f); c_contrib += contrib; }
                // set in full by contributing lanes only; other lanes' values are never read
                // (the fold below selects zero for them)
                float gr[12];
                if (contrib) {
                    const float4 g0 = s.g0[k];
                    const float4 g1 = s.g1[k];
                    const float4 g2 = s.g2[k];
                    const float cb = s.b[k];
                    const float one_m_a = __fsub_rn(1.0f, ev.a);
                    const float rinv = __fdividef(1.0f, one_m_a);
                    const float Ti = T * rinv;
                    const float w = ev.a * Ti;
                    gr[9] = w * g0_; gr[10] = w * g1_; gr[11] = w * g2_;
                    const float cg = g2.z * g0_ + g2.w * g1_ + cb * g2_;
                    const float dLda = Ti * (cg - Sg) - TfB * rinv;
                    Sg = ev.a * cg + one_m_a * Sg;
                    T = Ti;
                    if (!ev.clamped) {
                        const float dA = dLda * ev.G;
                        if (plain) {
                            gr[7] = dA;                  // alpha = alpha1 G: nothing to alpha2 or w'
                            gr[8] = 0.0f;
                        } else {
                            gr[7] = dA * ev.P;
                            gr[8] = dA - gr[7];
                        }
                        const float dpow = dLda * ev.a;           // a = A G when not clamped
                        const float dx = ev.dx, dy = ev.dy;
                        gr[2] = -0.5f * dpow * dx * dx;
                        gr[3] = -dpow * dx * dy;
                        gr[4] = -0.5f * dpow * dy * dy;
                        // d power / d mu-hat = conic d = U^T (U d)
                        const float sc = dpow * kInvUScale2;
                        gr[0] = sc * (g0.z * ev.s1);
                        gr[1] = sc * (g0.w * ev.s1 + g1.x * ev.s2);
                        if (plain) {
                            gr[5] = gr[6] = 0.0f;
                        } else {
                            // staged w' carries sqrt(log2 e); dzk is zero for step-mode splats
                            const float dz = dA * (ev.e * s.dzk[k]);
                            const float dzs = dz * kInvSqrtLog2e;
                            gr[5] = dz * dx;
                            gr[6] = dz * dy;
                            gr[0] -= dzs * g1.z;
                            gr[1] -= dzs * g1.w;
                        }
                    } else {
#pragma unroll
                        for (int f = 0; f < 9; ++f) gr[f] = 0.0f;   // a clamped at 0.99: no path to G, P
                    }
                }
                const unsigned any = __ballot_sync(0xffffffffu, contrib);
                if (!any) continue;
                float *dst = grad + 12 * (size_t)s.id[k];
                if (__popc(any) <= kFoldAbove) {
                    if (contrib) {
                        atomic_add12(dst, gr);
                        if (COUNT) ++c_atom;
                    }
                } else {
                    if (COUNT && lane == 0) ++c_red;
                    // lane l + 16 into lane l, two gradients per paired addition
#pragma unroll
                    for (int f = 0; f < 12; f += 2) {
                        const float x0 = contrib ? gr[f] : 0.0f, x1 = contrib ? gr[f + 1] : 0.0f;
                        const f32x2 o = pack2(__shfl_xor_sync(0xffffffffu, x0, 16), __shfl_xor_sync(0xffffffffu, x1, 16));
                        unpack2(add2(pack2(x0, x1), o), gr[f], gr[f + 1]);
                    }
                    if (__popc(any) > kFold2Above) {
                        // lane l + 8 into lane l: lanes 0..7 then hold four pixels each
#pragma unroll
                        for (int f = 0; f < 12; f += 2) {
                            const f32x2 o = pack2(__shfl_xor_sync(0xffffffffu, gr[f], 8),
                                                  __shfl_xor_sync(0xffffffffu, gr[f + 1], 8));
                            unpack2(add2(pack2(gr[f], gr[f + 1]), o), gr[f], gr[f + 1]);
                        }
                        if (lane < 8 && ((any >> lane) & 0x01010101u)) {
                            atomic_add12(dst, gr);
                            if (COUNT) ++c_atom;
                        }
                    } else if (lane < 16 && ((any >> lane) & 0x10001u)) {
                        atomic_add12(dst, gr);
                        if (COUNT) ++c_atom;
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&r.empty[slot]);
    }
    if (COUNT) {
        add_counters(p.counters + 3, c_visit, c_full, c_contrib, c_red);
        c_atom = warp_sum_u64(c_atom);
        if (lane == 0 && c_atom) atomicAdd(p.counters + 7, c_atom);
    }
}

// ---- forward -------------------------------------------------------------------------
// The forward runs as the same kind of pipeline as the backward (below): one producer
// warp takes tiles from the queue and stages each tile's list front to back into a ring
// of kFwdStages batch buffers, and the TW*TH/32 consumer warps (one 8x4 pixel block each)
// walk the batches at their own pace, with no block barriers.  A warp whose pixels have
// all finished writes its outputs and marks the tile done; the producer stops staging a
// tile once every consumer warp has marked it.  A tile's list is staged once per tile
// (the earlier design staged it once per 16x8 half, in two 128-thread blocks that met at
// two block barriers per batch).
constexpr int kFwdStages = 3;

struct FwdHeader {
    int gtile;                  // < 0: no more work
    uint32_t bstart, bend;      // the batch's slice of the tile's list
    uint32_t tseq;              // 1 + the number of tiles the producer began before this one
    int first, last;            // first / last batch of the tile's list
};

template <int BATCH, int NW>
struct FwdRing {
    Batch<BATCH, false> buf[kFwdStages];
    FwdHeader hdr[kFwdStages];
    unsigned long long full[kFwdStages], empty[kFwdStages];   // mbarriers
    uint32_t done[NW];          // per consumer warp: tseq of the last tile it finished
};

template <int TW, int TH, int BATCH>
__device__ void fwd_produce(const RenderLaunch &p, FwdRing<BATCH, TW * TH / 32> &r) {
    constexpr int NB = kFwdStages, NW = TW * TH / 32;
    const int lane = threadIdx.x & 31;
    const float4 *rec = reinterpret_cast<const float4 *>(p.proj.rec);
    const uint32_t vn = (uint32_t)p.n * (uint32_t)p.vt.n_views;
    const bool plain = p.cfg.plain != 0;
    Queue *qw = reinterpret_cast<Queue *>(p.ws);
    const uint32_t *order = reinterpret_cast<const uint32_t *>(qw + 1);
    uint32_t seq = 0, tseq = 0;
    // the backward's grad2d (p.clear), cleared here rather than by a separate pass over
    // it: this kernel is bound by its instruction stream and leaves DRAM nearly idle, so
    // the staging warp clears one slice of it when it has staged a tile, slice q for the
    // tile at queue position q (every position is taken once); the stores drain while
    // the tile composites.  Measured at 3M splats: forward +10 us, backward -23 us.
    // (Clearing it all at kernel start queued 144 MB of stores ahead of the first tiles'
    // loads: forward +25 us; clearing by the pixel warps as they finish a tile: +27 us.)
    const size_t slice = p.clear ? (p.clear_n4 + p.vt.total_tiles - 1) / p.vt.total_tiles : 0;
    for (int round = 0;; ++round) {
        int gtile = -1;
        uint32_t item = 0;
        if (p.cfg.persistent) {
            if (lane == 0) item = atomicAdd(&qw->counter_fwd, 1u);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item < (uint32_t)p.vt.total_tiles) gtile = (int)order[item];
        } else if (round == 0) {
            gtile = (int)blockIdx.x;
            item = blockIdx.x;
        }
        if (gtile < 0) {
            // end marker in the next buffer
            const uint32_t slot0 = seq % NB;
            if (seq >= NB && !mbar_wait(&r.empty[slot0], ((seq / NB) - 1) & 1u, p.status)) return;
            if (lane == 0) r.hdr[slot0].gtile = -1;
            __syncwarp();
            mbar_arrive(&r.full[slot0]);
            return;
        }
        const TileInfo ti = tile_info<TW, TH>(p, gtile);
        ++tseq;
        const float fox = (float)(ti.tx * TW), foy = (float)(ti.ty * TH);
        // every tile gets at least one (possibly empty) batch: its pixels are written then
        for (uint32_t bstart = ti.beg;; bstart += BATCH) {
            const uint32_t bend = min(ti.end, bstart + BATCH);
            const uint32_t slot = seq % NB;
            if (seq >= NB && !mbar_wait(&r.empty[slot], ((seq / NB) - 1) & 1u, p.status)) return;
            if (bstart > ti.beg) {
                // stop when every consumer warp has finished the tile
                const bool d = lane >= NW || *reinterpret_cast<volatile uint32_t *>(&r.done[lane]) == tseq;
                if (__all_sync(0xffffffffu, d)) break;
            }
            Batch<BATCH, false> &sb = r.buf[slot];
            for (int k = lane; k < BATCH; k += 32) {
                const uint32_t j = bstart + k;
                if (j < bend) {
                    uint32_t id = p.ids[j];
                    if (id >= vn) { set_status(p.status, HGS_DEV_BOUNDS); id = 0; }
                    stage<BATCH, false>(rec, id, sb, k, fox, foy, plain);
                }
            }
            if (lane == 0) {
                FwdHeader &h = r.hdr[slot];
                h.gtile = gtile;
                h.bstart = bstart;
                h.bend = bend;
                h.tseq = tseq;
                h.first = bstart == ti.beg;
                h.last = bend >= ti.end;
            }
            __syncwarp();
            mbar_arrive(&r.full[slot]);           // each lane: its staged slots are released
            ++seq;
            if (bend >= ti.end) break;
        }
        if (slice) {
            const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const size_t k1 = min(p.clear_n4, (size_t)(item + 1) * slice);
            for (size_t k = (size_t)item * slice + lane; k < k1; k += 32) p.clear[k] = z;
        }
    }
}

// Consumer warp: walks each batch for its 8x4 pixel block, front to back.  Each 4x4
// half of the block culls the staged splats against itself and walks its own hits,
// the two halves in step.
template <int TW, int TH, int BATCH, bool COUNT>
__device__ void fwd_consume(const RenderLaunch &p, FwdRing<BATCH, TW * TH / 32> &r) {
    constexpr int NB = kFwdStages, NW = TW * TH / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = lane >> 4;             // 4x4 half of the warp's 8x4 block
    unsigned long long c_visit = 0, c_full = 0, c_comp = 0;
    // per-tile state of this lane's pixel
    bool inside = false, done = true, written = true, vfit = false;
    f32x2 fp = 0;
    float cxb = 0.0f, cyb = 0.0f, T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0, beg = 0;
    int gtile = 0, px = 0, py = 0;
    uint32_t *vw = p.vis;                   // this warp's first word of the tile's mask rows
    for (uint32_t seq = 0;; ++seq) {
        const uint32_t slot = seq % NB;
        if (!mbar_wait(&r.full[slot], (seq / NB) & 1u, p.status)) break;
        const FwdHeader h = r.hdr[slot];
        if (h.gtile < 0) break;
        const Batch<BATCH, false> &s = r.buf[slot];
        if (h.first) {
            const TileInfo ti = tile_info<TW, TH>(p, h.gtile);
            gtile = h.gtile;
            const int bx = ti.tx * TW + (warp % (TW / 8)) * 8, by = ti.ty * TH + (warp / (TW / 8)) * 4;
            px = bx + 4 * half + (lane & 3);
            py = by + ((lane >> 2) & 3);
            inside = px < ti.W && py < ti.H;
            // tile-local coordinates (pixel centres at i + 1/2)
            const int ox = ti.tx * TW, oy = ti.ty * TH;
            fp = pack2((float)(px - ox) + 0.5f, (float)(py - oy) + 0.5f);
            cxb = (float)(bx - ox) + 2.0f;     // left half's centre
            cyb = (float)(by - oy) + 2.0f;
            T = 1.0f; C0 = C1 = C2 = 0.0f;
            last = 0;
            done = !inside;
            written = false;
            beg = ti.beg;
            // the visibility mask: one word per 32 entries of the tile's list, NW words apart
            // (the tile's rows are written whole or not at all)
            const size_t vrow = vis_row(ti.beg, gtile);
            vfit = (vrow + ((ti.end - ti.beg + 31) >> 5)) * NW <= p.vis_words;
            if (!vfit && warp == 0 && lane == 0) set_status(p.status, HGS_DEV_CAPACITY);
            vw = p.vis + (vfit ? vrow * NW + warp : 0);
        }
        if (!written) {
            const int cnt = (int)(h.bend - h.bstart);
            const uint32_t rel0 = h.bstart - beg;
            uint32_t *vwc = vw + (size_t)(rel0 >> 5) * NW;
            bool wdone = __all_sync(0xffffffffu, done);
            for (int c = 0; c < cnt && !wdone; c += 32) {
                const int jl = c + lane;
                bool h0 = false, h1 = false;
                if (jl < cnt) cull_halves(s, jl, cxb, cyb, h0, h1);
                const unsigned m0 = __ballot_sync(0xffffffffu, h0), m1 = __ballot_sync(0xffffffffu, h1);
                // each half walks its own hits, the two in step
                unsigned m = half ? m1 : m0;
                uint32_t cm = 0;                 // chunk slots this lane composited
                while (m) {
                    const unsigned lb = m & (0u - m);     // the visited slot's bit
                    const int k = c + __ffs(m) - 1;
                    m ^= lb;
                    if (!done) {
                        Eval ev;
                        if (COUNT) ++c_visit;
                        const bool hit = eval_alpha(fp, s, k, ev);
                        if (COUNT && ev.G >= 0.0f) ++c_full;
                        if (hit) {
                            const float Tn = __fmul_rn(T, __fsub_rn(1.0f, ev.a));
                            if (Tn < kTMin) {
                                done = true;
                            } else {
                                if (COUNT) ++c_comp;
                                const float w = __fmul_rn(ev.a, T);
                                const float2 rg = *reinterpret_cast<const float2 *>(&s.g2[k].z);
                                C0 = __fmaf_rn(rg.x, w, C0);
                                C1 = __fmaf_rn(rg.y, w, C1);
                                C2 = __fmaf_rn(s.b[k], w, C2);
                                T = Tn;
                                last = rel0 + k + 1;
                                cm |= lb;
                            }
                        }
                    }
                }
                // the chunk's mask word: splats composited at any pixel of the warp's block
                cm = __reduce_or_sync(0xffffffffu, cm);
                if (lane == 0 && vfit) *vwc = cm;
                vwc += NW;
                // checked once per chunk, not per visit: a warp whose lanes are all done only
                // runs the rest of this chunk's (cheap) bit loop (render_fwd 0.711 -> 0.679 ms)
                wdone = __all_sync(0xffffffffu, done);
            }
            if (wdone || h.last) {
                if (inside) {
                    const TileInfo ti = tile_info<TW, TH>(p, gtile);
                    const size_t HW = (size_t)ti.W * ti.H;
                    const size_t pix = (size_t)py * ti.W + px;
                    float *img = p.image + 3 * (size_t)ti.pix_off;
                    img[pix] = C0 + T * ti.bg[0];
                    img[HW + pix] = C1 + T * ti.bg[1];
                    img[2 * HW + pix] = C2 + T * ti.bg[2];
                    p.final_T[ti.pix_off + pix] = T;
                    p.n_contrib[ti.pix_off + pix] = last;
                }
                written = true;
                __syncwarp();
                if (lane == 0) *reinterpret_cast<volatile uint32_t *>(&r.done[warp]) = h.tseq;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&r.empty[slot]);
    }
    if (COUNT) add_counters(p.counters, c_visit, c_full, c_comp, 0ull);
}

// ---- kernels ------------------------------------------------------------------------
// Forward: TW*TH consumer threads (one pixel each) and one producer warp; resident blocks
// asked of the register allocator as for the backward.
template <int TW, int TH>
constexpr int kFwdMinBlocks = TW * TH >= 256 ? 4 : 10;

template <int TW, int TH, int BATCH, bool COUNT>
__global__ void __launch_bounds__(TW *TH + 32, (kFwdMinBlocks<TW, TH>)) k_render_fwd(RenderLaunch p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdRing<BATCH, TW * TH / 32> &r = *reinterpret_cast<FwdRing<BATCH, TW * TH / 32> *>(smem_raw);
    constexpr int NB = kFwdStages, NC = TW * TH;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NB; ++i) {
            mbar_init(&r.full[i], 32);          // the producer warp's lanes
            mbar_init(&r.empty[i], NC / 32);    // one arrival per consumer warp
        }
    }
    if (threadIdx.x < NC / 32) r.done[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x >= NC)
        fwd_produce<TW, TH, BATCH>(p, r);
    else
        fwd_consume<TW, TH, BATCH, COUNT>(p, r);
}

// Backward: TW*TH consumer threads (one pixel each) and one producer warp; resident
// blocks asked of the register allocator: 4 of 288 threads (56 registers) for 16x16 and
// 32x8 tiles, 10 of 96 for 8x8.
template <int TW, int TH>
constexpr int kBwdMinBlocks = TW * TH >= 256 ? 4 : 10;

template <int TW, int TH, int BATCH, bool COUNT, bool PLAIN>
__global__ void __launch_bounds__(TW *TH + 32, (kBwdMinBlocks<TW, TH>)) k_render_bwd(RenderLaunch p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdRing<BATCH, TW * TH / 32> &r = *reinterpret_cast<BwdRing<BATCH, TW * TH / 32> *>(smem_raw);
    constexpr int NB = kBwdStages, NC = TW * TH;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NB; ++i) {
            mbar_init(&r.full[i], 32);          // the producer warp's lanes
            mbar_init(&r.empty[i], NC / 32);    // one arrival per consumer warp
        }
    }
    __syncthreads();
    if (threadIdx.x >= NC)
        bwd_produce<TW, TH, BATCH, PLAIN>(p, r);
    else
        bwd_consume<TW, TH, BATCH, COUNT, PLAIN>(p, r);
}

// Work order for the persistent kernels: tiles bucketed by floor(log2(list length)),
// heaviest bucket first (empty tiles last).  Order within a bucket is arbitrary;
// the images do not depend on it.
__device__ __forceinline__ int cost_bucket(const uint32_t *ranges, int t) {
    const uint32_t len = ranges[2 * (size_t)t + 1] - ranges[2 * (size_t)t];
    return len ? 32 - __clz(len) : 0;    // 1..32, 0 for empty
}

__global__ void k_queue_count(const uint32_t *ranges, int total_tiles, Queue *q) {
    __shared__ uint32_t h[33];
    for (int j = threadIdx.x; j < 33; j += blockDim.x) h[j] = 0;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x)
        atomicAdd(&h[cost_bucket(ranges, t)], 1u);
    __syncthreads();
    for (int j = threadIdx.x; j < 33; j += blockDim.x)
        if (h[j]) atomicAdd(&q->bucket_count[j], h[j]);
}

// Lanes of a warp with the same bucket take consecutive slots with one atomic.
__global__ void k_queue_fill(const uint32_t *ranges, int total_tiles, Queue *q, uint32_t *order) {
    __shared__ uint32_t start[33];
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int b = 32; b >= 0; --b) { start[b] = acc; acc += q->bucket_count[b]; }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < total_tiles; t0 += gridDim.x * blockDim.x) {
        const int t = t0 + lane;
        const bool valid = t < total_tiles;
        const int b = valid ? cost_bucket(ranges, t) : 33;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (valid && lane == leader) base = atomicAdd(&q->bucket_cursor[b], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) order[start[b] + base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
    }
}

template <int TW, int TH, int BATCH, bool FWD, bool COUNT, bool PLAIN>
constexpr auto render_kernel() {
    if constexpr (FWD)
        return k_render_fwd<TW, TH, BATCH, COUNT>;
    else
        return k_render_bwd<TW, TH, BATCH, COUNT, PLAIN>;
}

template <int TW, int TH, int BATCH, bool FWD, bool COUNT, bool PLAIN>
cudaError_t launch_t(const RenderLaunch &p, cudaStream_t s) {
    auto kern = render_kernel<TW, TH, BATCH, FWD, COUNT, PLAIN>();
    constexpr int NT = TW * TH + 32;
    constexpr int smem = FWD ? (int)sizeof(FwdRing<BATCH, TW * TH / 32>)
                             : (int)sizeof(BwdRing<FWD ? 32 : BATCH, TW * TH / 32>);
    const int items = p.vt.total_tiles;
    if (smem > 48 * 1024) {
        // above the default dynamic shared-memory limit; a per-device attribute, so set
        // on every call (a host-side call, no stream work)
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    if (!p.cfg.persistent) {
        kern<<<items, NT, smem, s>>>(p);
        return cudaGetLastError();
    }
    // resident blocks per SM (assumed the same on every device of this architecture),
    // times the current device's SM count; atomic, since threads making their first calls
    // at the same time store the same value
    static std::atomic<int> occ_cache{0};
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (!occ) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
        occ = std::max(occ, 1);
        occ_cache.store(occ, std::memory_order_relaxed);
    }
    kern<<<std::min(num_sms() * occ, items), NT, smem, s>>>(p);
    return cudaGetLastError();
}

// The forward handles plain 3D-GS while staging (alpha2 := alpha1); the backward
// kernel is specialised on it, so the default path carries no test of the flag.
template <int TW, int TH, int BATCH, bool FWD>
cudaError_t launch_c(const RenderLaunch &p, cudaStream_t s) {
    const bool plain = !FWD && p.cfg.plain;
    if (p.counters)
        return plain ? launch_t<TW, TH, BATCH, FWD, true, true>(p, s) : launch_t<TW, TH, BATCH, FWD, true, false>(p, s);
    return plain ? launch_t<TW, TH, BATCH, FWD, false, true>(p, s) : launch_t<TW, TH, BATCH, FWD, false, false>(p, s);
}

cudaError_t prepare_queue(const RenderLaunch &p, cudaStream_t s) {
    Queue *q = reinterpret_cast<Queue *>(p.ws);
    uint32_t *order = reinterpret_cast<uint32_t *>(q + 1);
    cudaError_t e = cudaMemsetAsync(q, 0, sizeof(Queue), s);
    if (e != cudaSuccess) return e;
    const int grid = std::min(div_up(p.vt.total_tiles, 256), 4 * num_sms());
    k_queue_count<<<grid, 256, 0, s>>>(p.ranges, p.vt.total_tiles, q);
    k_queue_fill<<<grid, 256, 0, s>>>(p.ranges, p.vt.total_tiles, q, order);
    return cudaGetLastError();
}

// dispatch over the supported (tile shape, batch) combinations
template <bool FWD, int TW, int TH>
cudaError_t dispatch_batch(const RenderLaunch &p, cudaStream_t s) {
    if (FWD) {
        // default 128 (16x16 tiles at 3M splats, eager launches: forward 0.691 / 0.679 / 0.696
        // / 1.14 ms at 64 / 128 / 224 / 512; smaller batches stage fewer splats past the
        // point where every pixel of the tile has finished, the largest leave room for
        // fewer blocks per SM)
        switch (p.cfg.batch ? p.cfg.batch : std::min(TW * TH, 128)) {
            case 32: return launch_c<TW, TH, 32, true>(p, s);
            case 64: return launch_c<TW, TH, 64, true>(p, s);
            case 128: return launch_c<TW, TH, 128, true>(p, s);
            case 224: return launch_c<TW, TH, 224, true>(p, s);
            case 256: return launch_c<TW, TH, 256, true>(p, s);
            case 512: return launch_c<TW, TH, 512, true>(p, s);
            default: return cudaErrorInvalidValue;
        }
    }
    // backward: ring buffers of at most 224 splats, so that the three of them leave room
    // for 4 blocks per SM (3 x 256 splats: 3 blocks, backward 1.29 -> 1.37 ms); default
    // 224, 64 for 8x8 tiles
    const int req = p.cfg.batch ? p.cfg.batch : (TW * TH >= 256 ? 224 : 64);
    switch (std::min(req, 224)) {
        case 32: return launch_c<TW, TH, 32, false>(p, s);
        case 64: return launch_c<TW, TH, 64, false>(p, s);
        case 128: return launch_c<TW, TH, 128, false>(p, s);
        case 224: return launch_c<TW, TH, 224, false>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <bool FWD>
cudaError_t dispatch(const RenderLaunch &p, cudaStream_t s) {
    if (p.vt.total_tiles == 0) return cudaSuccess;
    // a backward that follows its forward on the same workspace reuses the forward's
    // queue: the same order (a function of the ranges alone) and a backward counter the
    // forward's build left at zero
    if (p.cfg.persistent && !(!FWD && p.from_forward)) {
        cudaError_t e = prepare_queue(p, s);
        if (e != cudaSuccess) return e;
    }
    const int tw = p.cfg.tile_w, th = p.cfg.tile_h;
    if (tw == 16 && th == 16) return dispatch_batch<FWD, 16, 16>(p, s);
    if (tw == 8 && th == 8) return dispatch_batch<FWD, 8, 8>(p, s);
    if (tw == 32 && th == 8) return dispatch_batch<FWD, 32, 8>(p, s);
    return cudaErrorInvalidValue;
}

// Self-test of the bounded wait the backward pipeline uses: one warp waits on an
// mbarrier that nothing arrives at, until the wait's bound ends it (HGS_DEV_TIMEOUT).
__global__ void k_wait_selftest(int *status) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncwarp();
    mbar_wait(&bar, 0, status);
}

}  // namespace

cudaError_t launch_wait_selftest(int *status, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

size_t render_workspace_bytes(const ViewTable &vt, const hgs_config &cfg) {
    (void)cfg;
    return sizeof(Queue) + 4 * (size_t)std::max(vt.total_tiles, 1) + 256;
}

cudaError_t launch_render_fwd(const RenderLaunch &p, cudaStream_t s) { return dispatch<true>(p, s); }
cudaError_t launch_render_bwd(const RenderLaunch &p, cudaStream_t s) {
    if (!p.from_forward) {
        cudaError_t e = cudaMemsetAsync(p.grad2d, 0, sizeof(float) * 12 * (size_t)p.n * p.vt.n_views, s);
        if (e != cudaSuccess) return e;
    }
    return dispatch<false>(p, s);
}

}  // namespace hgs
