// Tile binning (A3-A5): the sorted (tile | depth) pairs and per-tile ranges.
//
// The result is the stable LSD radix sort of the 64-bit keys
// (global tile id << 32) | bits(depth), one per covered tile of every
// (view, splat), emitted in (view, splat) order, i.e. the order of the keys with
// ties broken by the splat index.  It is computed in two stages:
//   1. the 8-bit passes over the depth half (up to four, as many as the drawn splats'
//      key range needs) run on the n_views*n per-splat
//      depth keys (culled splats get key 0xFFFFFFFF and sort last) -- duplicating
//      a splat into its tiles commutes with a stable sort on depth, so these
//      passes need not touch the much longer pair list;
//   2. tiles touched are gathered into that depth order and scanned (chunk sums,
//      a scan of the chunk sums, and the scan inside each chunk while emitting), each
//      splat emits its pairs (32-bit tile key, splat index) there, and the
//      ceil(tile_bits/8) passes over the tile half sort the pairs; the last pass
//      writes the 64-bit keys.
// Each radix pass is reduce-then-scan, with no inter-block waiting: an upsweep
// counts the digits of every 4096-element partition, one warp per digit scans
// those counts over the partitions, and a downsweep ranks each partition in
// shared memory (warp-level multisplit from per-bit ballots, stable by
// construction) and
// scatters it through shared memory so that global writes are runs of
// consecutive addresses.
#include <algorithm>

#include <mutex>

#include "hgs_internal.cuh"

namespace hgs {
namespace {

constexpr int kBlock = 256;                  // threads per block (8 warps)
constexpr int kItems = 16;                   // items per thread
constexpr int kPart = kBlock * kItems;       // 4096 elements per partition
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;      // 256 digits
constexpr int kDepthPasses = 4;              // 32 depth bits
constexpr int kGroup = kBlock / 32;          // chunks of kBlock splats per scan group (one k_scan_reduce block)

struct Ctrl {                                // zeroed at the start of every call
    uint32_t totals[kRadix];                 // per-digit totals of the current pass
    uint32_t kmin_inv, kmax;                 // ~(smallest) and largest valid depth key
    uint32_t pad[62];
};

// Depth passes actually needed: the valid depth keys (bits of positive floats, so
// ordered as integers) are sorted as key - kmin and the culled ones as R = kmax - kmin
// + 1, after every valid key; the order is the same as that of the raw keys, and
// ceil(bits(R) / 8) passes of 8 bits cover it (3 instead of 4 when every depth lies
// within a factor of about 2-4 of the nearest, as in a scene seen from outside).
// The first pass reads raw keys and writes shifted ones; passes past the count return
// at once, and the sorted order ends in the A buffers after an even count, else in B.
struct DepthPlan {
    int passes;
    uint32_t kmin, culled;
};
__device__ __forceinline__ DepthPlan depth_plan(const Ctrl *c) {
    DepthPlan d;
    d.kmin = ~c->kmin_inv;
    const uint32_t kmax = c->kmax;
    if (d.kmin > kmax) {                     // no valid key: the identity order
        d.passes = 0;
        d.kmin = 0;
        d.culled = 0;
        return d;
    }
    d.culled = kmax - d.kmin + 1u;
    d.passes = (32 - __clz(d.culled) + kRadixBits - 1) / kRadixBits;
    return d;
}
__device__ __forceinline__ uint32_t depth_key(const DepthPlan &d, uint32_t raw) {
    return raw == 0xffffffffu ? d.culled : raw - d.kmin;
}

struct Ws {
    Ctrl *ctrl;
    unsigned long long *chunk_sum;           // [chunks of kBlock splats] pair counts
    unsigned long long *group_pre;           // [groups of 8 chunks] pair counts, then exclusive prefixes
    uint32_t *dkA, *dvA, *dkB, *dvB;         // [VN] depth keys / splat indices, ping-pong
    uint32_t *tiles_sorted;                  // [VN] tiles touched, in depth order
    uint32_t *tkA, *tvA, *tkB, *tvB;         // [capacity] tile keys / splat indices, ping-pong
    uint32_t *counts;                        // [256][parts] digit counts, then offsets
    size_t depth_parts, pair_parts, parts_stride;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

Ws carve(void *base, size_t vn, size_t cap, size_t *total) {
    Ws w{};
    w.depth_parts = std::max<size_t>((vn + kPart - 1) / kPart, 1);
    w.pair_parts = std::max<size_t>((cap + kPart - 1) / kPart, 1);
    w.parts_stride = (std::max(w.depth_parts, w.pair_parts) + 3) & ~(size_t)3;   // rows 16-B aligned
    size_t off = 0;
    char *b = static_cast<char *>(base);
    auto take = [&](size_t bytes) { char *p = b ? b + off : nullptr; off += align_up(bytes); return p; };
    const size_t vn1 = std::max<size_t>(vn, 1), cap1 = std::max<size_t>(cap, 1);
    w.ctrl = reinterpret_cast<Ctrl *>(take(sizeof(Ctrl)));
    const size_t n_chunks = (vn1 + kBlock - 1) / kBlock;
    w.chunk_sum = reinterpret_cast<unsigned long long *>(take(8 * n_chunks));
    w.group_pre = reinterpret_cast<unsigned long long *>(take(8 * ((n_chunks + kGroup - 1) / kGroup)));
    w.dkA = reinterpret_cast<uint32_t *>(take(4 * vn1));
    w.dvA = reinterpret_cast<uint32_t *>(take(4 * vn1));
    w.dkB = reinterpret_cast<uint32_t *>(take(4 * vn1));
    w.dvB = reinterpret_cast<uint32_t *>(take(4 * vn1));
    w.tiles_sorted = reinterpret_cast<uint32_t *>(take(4 * vn1));
    w.tkA = reinterpret_cast<uint32_t *>(take(4 * cap1));
    w.tvA = reinterpret_cast<uint32_t *>(take(4 * cap1));
    w.tkB = reinterpret_cast<uint32_t *>(take(4 * cap1));
    w.tvB = reinterpret_cast<uint32_t *>(take(4 * cap1));
    w.counts = reinterpret_cast<uint32_t *>(take(4 * (size_t)kRadix * w.parts_stride));
    if (total) *total = off;
    return w;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Lanes of the warp holding the same 8-bit digit v: the AND over the bits of v of
// the ballot of that bit or of its complement.  Eight ballots, whatever the number
// of distinct digits.  (Measured faster here than __match_any_sync: 0.48 vs 0.57 ms
// for the whole binning.)
__device__ __forceinline__ unsigned peer_mask(uint32_t v) {
    unsigned m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
        const bool bit = (v >> b) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return m;
}

// Element count of a pass: a host count, or a device count clamped to capacity.
struct Count {
    unsigned long long host;
    const uint64_t *dev;
    size_t capacity;
    __device__ __forceinline__ uint32_t get() const {
        return (uint32_t)(dev ? min((size_t)*dev, capacity) : (size_t)host);
    }
};

// ---- stage 1: depth keys ------------------------------------------------------------------
// Four (view, splat) entries a thread, with 128-bit loads and stores (vn % 4 tail
// handled element by element).
// The block's smallest and largest valid key go to ctrl (one atomic each per block).
__global__ void __launch_bounds__(kBlock) k_depth_keys(const uint32_t *__restrict__ tiles,
                                                       const float *__restrict__ depth, long long vn,
                                                       uint32_t *__restrict__ dk, uint32_t *__restrict__ dv,
                                                       Ctrl *ctrl) {
    __shared__ uint32_t s_min[kBlock / 32], s_max[kBlock / 32];
    const long long i0 = 4 * ((long long)blockIdx.x * kBlock + threadIdx.x);
    uint32_t kmin_inv = 0, kmax = 0;      // ~min and max of this thread's valid keys
    if (i0 + 4 <= vn) {
        const uint4 t = *reinterpret_cast<const uint4 *>(tiles + i0);
        const float4 d = *reinterpret_cast<const float4 *>(depth + i0);
        const uint4 k = make_uint4(t.x ? __float_as_uint(d.x) : 0xffffffffu, t.y ? __float_as_uint(d.y) : 0xffffffffu,
                                   t.z ? __float_as_uint(d.z) : 0xffffffffu, t.w ? __float_as_uint(d.w) : 0xffffffffu);
        *reinterpret_cast<uint4 *>(dk + i0) = k;
        const uint32_t b = (uint32_t)i0;
        *reinterpret_cast<uint4 *>(dv + i0) = make_uint4(b, b + 1, b + 2, b + 3);
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (kk[j] != 0xffffffffu) { kmin_inv = max(kmin_inv, ~kk[j]); kmax = max(kmax, kk[j]); }
    } else {
        for (long long i = i0; i < vn; ++i) {
            const uint32_t k = tiles[i] ? __float_as_uint(depth[i]) : 0xffffffffu;
            dk[i] = k;
            dv[i] = (uint32_t)i;
            if (k != 0xffffffffu) { kmin_inv = max(kmin_inv, ~k); kmax = max(kmax, k); }
        }
    }
    kmin_inv = __reduce_max_sync(0xffffffffu, kmin_inv);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_min[warp] = kmin_inv; s_max[warp] = kmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w2 = 1; w2 < kBlock / 32; ++w2) { kmin_inv = max(kmin_inv, s_min[w2]); kmax = max(kmax, s_max[w2]); }
        if (kmin_inv) atomicMax(&ctrl->kmin_inv, kmin_inv);
        if (kmax) atomicMax(&ctrl->kmax, kmax);
    }
}

// ---- radix pass, part 1: digit counts of every partition ---------------------------------
// Each thread counts 16 consecutive keys, fetched with four 128-bit loads that are
// all in flight at once (the counts of a partition do not depend on the order in
// which its keys are visited).
// plan (depth passes only, else null): skip a pass past the plan's count; the first
// pass shifts the raw keys (depth_key).
__global__ void __launch_bounds__(kBlock) k_upsweep(const uint32_t *__restrict__ keys, Count cnt, int shift,
                                                    uint32_t *__restrict__ counts, size_t stride,
                                                    const Ctrl *plan, int pass) {
    __shared__ uint32_t s_cnt[kBlock / 32][kRadix];
    DepthPlan dp{};
    if (plan) {
        dp = depth_plan(plan);
        if (pass >= dp.passes) return;
    }
    const bool shift_keys = plan && pass == 0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const uint32_t K = cnt.get();
    const uint32_t n_parts = (K + kPart - 1) / kPart;
    for (uint32_t part = blockIdx.x; part < n_parts; part += gridDim.x) {
        for (int j = lane; j < kRadix; j += 32) s_cnt[warp][j] = 0;
        __syncwarp();
        const uint32_t base = part * kPart + tid * kItems;
        uint32_t k[kItems];
        if (base + kItems <= K) {
            const uint4 *src = reinterpret_cast<const uint4 *>(keys + base);
#pragma unroll
            for (int q = 0; q < kItems / 4; ++q) {
                const uint4 t = src[q];
                k[4 * q] = t.x; k[4 * q + 1] = t.y; k[4 * q + 2] = t.z; k[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kItems; ++j) k[j] = base + j < K ? keys[base + j] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            if (base + j < K) {
                const uint32_t kj = shift_keys ? depth_key(dp, k[j]) : k[j];
                atomicAdd(&s_cnt[warp][(kj >> shift) & (kRadix - 1)], 1u);
            }
        __syncthreads();
        uint32_t total = 0;
#pragma unroll
        for (int w2 = 0; w2 < kBlock / 32; ++w2) total += s_cnt[w2][tid];
        counts[(size_t)tid * stride + part] = total;
        __syncthreads();
    }
}

// ---- radix pass, part 2: per digit, exclusive scan of the counts over partitions ---------
// One block per digit, 16 consecutive counts per thread (4096 partitions per round,
// so one round below 16.7M elements); the digit totals go to ctrl->totals.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *tmp);

__global__ void __launch_bounds__(kBlock) k_digit_scan(uint32_t *__restrict__ counts, Count cnt, size_t stride,
                                                       Ctrl *ctrl, bool depth, int pass) {
    __shared__ uint32_t s_tmp[kBlock / 32];
    __shared__ uint32_t s_total;
    if (depth && pass >= depth_plan(ctrl).passes) return;
    const int d = blockIdx.x;
    const uint32_t K = cnt.get();
    const uint32_t n_parts = (K + kPart - 1) / kPart;
    uint32_t *row = counts + (size_t)d * stride;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n_parts; base += kPart) {
        const uint32_t j0 = base + threadIdx.x * kItems;
        const bool full = j0 + kItems <= n_parts;
        uint32_t v[kItems];
        if (full) {
            const uint4 *src = reinterpret_cast<const uint4 *>(row + j0);
#pragma unroll
            for (int q = 0; q < kItems / 4; ++q) {
                const uint4 t = src[q];
                v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kItems; ++j) v[j] = j0 + j < n_parts ? row[j0 + j] : 0u;
        }
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < kItems; ++j) sum += v[j];
        const uint32_t excl = block_excl_scan(sum, s_tmp);
        uint32_t run = carry + excl;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const uint32_t c = v[j];
            v[j] = run;
            run += c;
        }
        if (full) {
            uint4 *dst = reinterpret_cast<uint4 *>(row + j0);
#pragma unroll
            for (int q = 0; q < kItems / 4; ++q) dst[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < kItems; ++j)
                if (j0 + j < n_parts) row[j0 + j] = v[j];
        }
        if (threadIdx.x == kBlock - 1) s_total = excl + sum;
        __syncthreads();
        carry += s_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) ctrl->totals[d] = carry;
}

// ---- radix pass, part 3: rank and scatter ------------------------------------------------
struct DownArgs {
    const uint32_t *kin, *vin;
    uint32_t *kout, *vout;
    uint64_t *kout64;                // last pair pass, optional: (key << 32) | bits(depth[value])
    const float *depth;
    Count cnt;
    int shift;
    const uint32_t *offsets;         // [256][stride] exclusive per-digit offsets of each partition
    size_t stride;
    const Ctrl *ctrl;
    bool depth_stage;                // a depth pass: skipped past the plan's count, the first shifts the keys
    int pass;
    int *status;
};

struct DownSmem {
    uint32_t keys[kPart];
    uint32_t vals[kPart];
    uint32_t warp_cnt[kBlock / 32][kRadix];  // per-warp digit counts, then warp offsets
    uint32_t digit_start[kRadix];            // partition-local exclusive digit prefix
    uint32_t global_off[kRadix];             // global destination of each digit bucket
    uint32_t digit_base[kRadix];             // exclusive prefix of the digit totals
    uint32_t scan_tmp[kBlock / 32];
};

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *tmp) {
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    uint32_t wb = 0;
    for (int w2 = 0; w2 < warp; ++w2) wb += tmp[w2];
    __syncthreads();
    return wb + x - v;
}

template <bool COMPOSE>
// 4 blocks per SM (64 registers): measured faster than 3 (80 registers) and 5 (spills).
__global__ void __launch_bounds__(kBlock, 4) k_downsweep(DownArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem &sm = *reinterpret_cast<DownSmem *>(smem_raw);
    DepthPlan dp{};
    if (a.depth_stage) {
        dp = depth_plan(a.ctrl);
        if (a.pass >= dp.passes) return;
    }
    const bool shift_keys = a.depth_stage && a.pass == 0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const uint32_t K = a.cnt.get();
    const uint32_t n_parts = (K + kPart - 1) / kPart;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    sm.digit_base[tid] = block_excl_scan(a.ctrl->totals[tid], sm.scan_tmp);
    for (uint32_t part = blockIdx.x; part < n_parts; part += gridDim.x) {
        const uint32_t pbase = part * kPart;
        for (int j = lane; j < kRadix; j += 32) sm.warp_cnt[warp][j] = 0;
        sm.global_off[tid] = sm.digit_base[tid] + a.offsets[(size_t)tid * a.stride + part];
        __syncwarp();
        uint32_t key[kItems], val[kItems], rank[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t idx = pbase + warp * (32 * kItems) + it * 32 + lane;
            const bool valid = idx < K;
            key[it] = valid ? a.kin[idx] : 0u;
            if (shift_keys && valid) key[it] = depth_key(dp, key[it]);
            val[it] = valid ? a.vin[idx] : 0u;
        }
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t idx = pbase + warp * (32 * kItems) + it * 32 + lane;
            const bool valid = idx < K;
            // Empty slots (past the element count) rank as digit 255: they all follow every
            // valid element of the partition in this order, so no valid rank counts them,
            // and the overcount they leave in digit 255's tally shifts nothing after it
            // (measured: bin 0.443 -> 0.438 ms against a ninth ballot for them).
            const uint32_t d = valid ? (key[it] >> a.shift) & (kRadix - 1) : kRadix - 1;
            const unsigned peers = peer_mask(d);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (valid && lane == leader) {
                old = sm.warp_cnt[warp][d];
                sm.warp_cnt[warp][d] = old + __popc(peers);
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            rank[it] = old + __popc(peers & lanemask_lt);
            __syncwarp();
        }
        __syncthreads();
        // per digit (thread = digit): warp offsets and partition total
        uint32_t total = 0;
#pragma unroll
        for (int w2 = 0; w2 < kBlock / 32; ++w2) {
            const uint32_t c = sm.warp_cnt[w2][tid];
            sm.warp_cnt[w2][tid] = total;
            total += c;
        }
        sm.digit_start[tid] = block_excl_scan(total, sm.scan_tmp);
        __syncthreads();   // every digit's start is read below, not only this thread's
        // scatter into shared memory in partition-sorted order
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t idx = pbase + warp * (32 * kItems) + it * 32 + lane;
            if (idx < K) {
                const uint32_t d = (key[it] >> a.shift) & (kRadix - 1);
                const uint32_t pos = sm.digit_start[d] + sm.warp_cnt[warp][d] + rank[it];
                if (pos < (uint32_t)kPart) {
                    sm.keys[pos] = key[it];
                    sm.vals[pos] = val[it];
                } else {
                    set_status(a.status, HGS_DEV_BOUNDS);
                }
            }
        }
        __syncthreads();
        const uint32_t cnt = min((uint32_t)kPart, K - pbase);
        for (uint32_t j = tid; j < cnt; j += kBlock) {
            const uint32_t k = sm.keys[j];
            const uint32_t v = sm.vals[j];
            const uint32_t d = (k >> a.shift) & (kRadix - 1);
            const uint32_t dst = sm.global_off[d] + (j - sm.digit_start[d]);
            if (dst >= K) { set_status(a.status, HGS_DEV_BOUNDS); continue; }
            a.kout[dst] = k;
            a.vout[dst] = v;
            if (COMPOSE) a.kout64[dst] = ((uint64_t)k << 32) | (uint64_t)__float_as_uint(a.depth[v]);
        }
        __syncthreads();
    }
}

// ---- stage 2: exclusive scan of tiles touched, in depth order -----------------------------
// Reduce, then scan, then the pair emission applies the prefixes: no inter-block
// waiting.  k_scan_reduce gathers tiles touched into depth order (so later reads are
// contiguous) and sums each chunk of kBlock splats and each group of kGroup chunks;
// k_chunk_scan turns the group sums into exclusive prefixes (64-bit: the total may
// exceed the pair capacity) and the pair count; k_duplicate adds the chunks before
// its own in the group and finishes the scan inside its chunk.
// A block covers 8 chunks of kBlock splats, a warp one chunk, a thread 8 consecutive
// splats (two 128-bit loads of the order, 8 independent gathers in flight).
constexpr int kReducePer = 8;

__global__ void __launch_bounds__(kBlock) k_scan_reduce(const uint32_t *__restrict__ tiles,
                                                        const uint32_t *__restrict__ order_a,
                                                        const uint32_t *__restrict__ order_b, const Ctrl *plan,
                                                        long long vn, uint32_t *__restrict__ tiles_sorted,
                                                        unsigned long long *__restrict__ chunk_sum,
                                                        unsigned long long *__restrict__ group_sum) {
    __shared__ unsigned long long s_chunk[kGroup];
    const uint32_t *__restrict__ order = (depth_plan(plan).passes & 1) ? order_b : order_a;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    // this warp's 256 splats start at `base` (chunk base / kBlock); a thread takes 8 consecutive
    const long long base = (long long)blockIdx.x * kBlock * kReducePer + (long long)warp * 32 * kReducePer;
    const long long i0 = base + (long long)lane * kReducePer;
    uint32_t t[kReducePer];
    if (i0 + kReducePer <= vn) {
        const uint4 a = *reinterpret_cast<const uint4 *>(order + i0);
        const uint4 b = *reinterpret_cast<const uint4 *>(order + i0 + 4);
        t[0] = tiles[a.x]; t[1] = tiles[a.y]; t[2] = tiles[a.z]; t[3] = tiles[a.w];
        t[4] = tiles[b.x]; t[5] = tiles[b.y]; t[6] = tiles[b.z]; t[7] = tiles[b.w];
        *reinterpret_cast<uint4 *>(tiles_sorted + i0) = make_uint4(t[0], t[1], t[2], t[3]);
        *reinterpret_cast<uint4 *>(tiles_sorted + i0 + 4) = make_uint4(t[4], t[5], t[6], t[7]);
    } else {
#pragma unroll
        for (int k = 0; k < kReducePer; ++k) {
            t[k] = i0 + k < vn ? tiles[order[i0 + k]] : 0u;
            if (i0 + k < vn) tiles_sorted[i0 + k] = t[k];
        }
    }
    unsigned long long x = 0;
#pragma unroll
    for (int k = 0; k < kReducePer; ++k) x += t[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    // the warp's 256 splats are chunk `base / kBlock`; only existing chunks are written
    const long long c = base / kBlock;
    if (lane == 0 && base < vn) chunk_sum[c] = x;
    // and the block's 8 chunks are scan group blockIdx.x
    if (lane == 0) s_chunk[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0 && (long long)blockIdx.x * kBlock * kReducePer < vn) {
        unsigned long long g = 0;
#pragma unroll
        for (int w2 = 0; w2 < kGroup; ++w2) g += s_chunk[w2];
        group_sum[blockIdx.x] = g;
    }
}

constexpr int kChunkScanThreads = 1024;

// One block scans the group sums (exclusive, in place) and writes the pair count.
// Warp w of a round scans ROWS x 32 consecutive sums, read row by row (lane l of
// row i holds entry 32 i + l: every load is coalesced); the warps' totals are then
// scanned across the block.  ROWS = 2 covers 2048 groups (4.2M splats) in one round.
// (Scanning the 8x more chunk sums here instead took 15 us, latency-bound.)
template <int ROWS>
__global__ void __launch_bounds__(kChunkScanThreads) k_chunk_scan(unsigned long long *chunk, long long n_chunks,
                                                                  uint64_t *total_out) {
    __shared__ unsigned long long s_w[kChunkScanThreads / 32];
    __shared__ unsigned long long s_total;
    constexpr int kRows = ROWS, kSeg = 32 * kRows;
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    unsigned long long carry = 0;
    for (long long base = 0; base < n_chunks; base += (long long)kChunkScanThreads * kRows) {
        const long long seg = base + (long long)warp * kSeg;
        unsigned long long v[kRows], ex[kRows], run = 0;
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            const long long j = seg + 32 * i + lane;
            v[i] = j < n_chunks ? chunk[j] : 0ull;
        }
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            unsigned long long x = v[i];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            ex[i] = run + x - v[i];
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) s_w[warp] = run;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long w = s_w[lane];
            unsigned long long wx = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, wx, o);
                if (lane >= o) wx += y;
            }
            s_w[lane] = wx - w;                    // exclusive prefix of the warp totals
            if (lane == 31) s_total = wx;
        }
        __syncthreads();
        const unsigned long long off = carry + s_w[warp];
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            const long long j = seg + 32 * i + lane;
            if (j < n_chunks) chunk[j] = off + ex[i];
        }
        carry += s_total;
        __syncthreads();
    }
    if (tid == 0) *total_out = carry;
}

// ---- stage 2: pair emission in depth order ---------------------------------------------------
// A warp expands its 32 splats' pairs cooperatively: pair q of the warp (in
// order) belongs to the last lane whose start is <= q, so consecutive lanes
// write consecutive addresses however uneven the splats' tile counts are.
struct DupArgs {
    const uint32_t *tiles_sorted;   // tiles touched, in depth order
    const int4 *rect;
    const uint32_t *order_a, *order_b;   // (view, splat) indices in depth order: in A after an
    const Ctrl *plan;                    // even number of depth passes, else in B
    const unsigned long long *chunk_sum;   // pair count of each chunk of kBlock splats
    const unsigned long long *group_pre;   // exclusive pair prefix of each group of kGroup chunks
    long long vn;
    int n;
    ViewTable vt;
    size_t capacity;
    uint32_t *tk, *tv;
    int *status;
};

__global__ void __launch_bounds__(kBlock) k_duplicate(DupArgs a) {
    __shared__ uint32_t s_start[kBlock / 32][32];
    __shared__ int s_x0[kBlock / 32][32], s_w[kBlock / 32][32], s_row0[kBlock / 32][32], s_txn[kBlock / 32][32];
    __shared__ uint32_t s_vi[kBlock / 32][32];
    __shared__ uint32_t s_wsum[kBlock / 32];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const long long j0 = (long long)blockIdx.x * kBlock + warp * 32;
    const long long j = j0 + lane;
    const uint32_t *order = (depth_plan(a.plan).passes & 1) ? a.order_b : a.order_a;
    // this chunk's prefix: its group's, plus the chunks before it in the group
    const uint32_t gi = blockIdx.x % kGroup;
    unsigned long long before = lane < (int)gi ? a.chunk_sum[blockIdx.x - gi + lane] : 0ull;
    const unsigned long long gpre = a.group_pre[blockIdx.x / kGroup];
    uint32_t vi = 0, cnt = 0;
    if (j < a.vn) {
        vi = order[j];
        cnt = a.tiles_sorted[j];
    }
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    if (lane == 0) s_wsum[warp] = total;
    __syncthreads();
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
    uint64_t wbase = gpre + __shfl_sync(0xffffffffu, before, 0);
    for (int w2 = 0; w2 < warp; ++w2) wbase += s_wsum[w2];
    if (j0 >= a.vn || total == 0) return;
    const int4 r = cnt ? a.rect[vi] : make_int4(0, 0, 0, 0);
    const int v = (int)(vi / (uint32_t)a.n);
    s_start[warp][lane] = x - cnt;
    s_x0[warp][lane] = r.x;
    s_w[warp][lane] = r.z - r.x;
    s_txn[warp][lane] = a.vt.tiles_x[v];
    s_row0[warp][lane] = a.vt.tile_off[v] + r.y * a.vt.tiles_x[v];
    s_vi[warp][lane] = vi;
    __syncwarp();
    if (wbase + total > a.capacity && lane == 0) set_status(a.status, HGS_DEV_CAPACITY);
    for (uint32_t q = lane; q < total; q += 32) {
        int s = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (s + step < 32 && s_start[warp][s + step] <= q) s += step;
        const uint32_t local = q - s_start[warp][s];
        const uint32_t w = (uint32_t)s_w[warp][s];
        const uint32_t ty = local / w, tx = local - ty * w;
        const uint64_t dst = wbase + q;
        if (dst >= a.capacity) break;
        a.tk[dst] = (uint32_t)(s_row0[warp][s] + (int)ty * s_txn[warp][s] + s_x0[warp][s] + (int)tx);
        a.tv[dst] = s_vi[warp][s];
    }
}

// ---- A5: tile ranges from the sorted 32-bit tile keys ------------------------------------
// Each thread reads 4 consecutive keys with one 128-bit load; the neighbours across
// threads come by shuffle (two extra loads per warp at its ends).  A start (end) of
// tile t is where the previous (next) key differs; 0xFFFFFFFF past both ends.
__global__ void __launch_bounds__(kBlock) k_ranges(const uint32_t *__restrict__ tk, Count cnt, int total_tiles,
                                                   uint32_t *ranges, int *status) {
    const size_t K = cnt.get();
    const size_t n4 = (K + 3) / 4;
    const int lane = lane_id();
    constexpr uint32_t kNone = 0xffffffffu;
    for (size_t g = (size_t)blockIdx.x * kBlock + threadIdx.x; g - lane < n4; g += (size_t)gridDim.x * kBlock) {
        const size_t i0 = 4 * g;
        uint32_t k[4];
        if (i0 + 4 <= K) {
            const uint4 t = *reinterpret_cast<const uint4 *>(tk + i0);
            k[0] = t.x; k[1] = t.y; k[2] = t.z; k[3] = t.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) k[j] = i0 + j < K ? tk[i0 + j] : kNone;
        }
        uint32_t prev = __shfl_up_sync(0xffffffffu, k[3], 1);
        uint32_t next = __shfl_down_sync(0xffffffffu, k[0], 1);
        if (lane == 0) prev = (i0 > 0 && i0 - 1 < K) ? tk[i0 - 1] : kNone;
        if (lane == 31) next = i0 + 4 < K ? tk[i0 + 4] : kNone;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const size_t i = i0 + j;
            if (i >= K) break;
            const uint32_t t = k[j];
            if (t >= (uint32_t)total_tiles) { set_status(status, HGS_DEV_BOUNDS); continue; }
            const uint32_t p = j ? k[j - 1] : prev;
            const uint32_t nx = j < 3 ? k[j + 1] : next;
            if (p != t) ranges[2 * (size_t)t] = (uint32_t)i;
            if (nx != t) ranges[2 * (size_t)t + 1] = (uint32_t)(i + 1);
        }
    }
}

// Resident blocks per SM of the downsweep and of the upsweep/ranges kernels; grids are
// these times the current device's SM count.  Set up once per device (std::call_once,
// so threads making their first calls at the same time do not race): the downsweep's
// shared-memory limit is a per-device attribute and has to be raised in each device's
// context.
struct LaunchShapes {
    std::once_flag once;
    int sweep = 1, aux = 1;
};
LaunchShapes g_shapes[64];

const LaunchShapes &launch_shapes() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    LaunchShapes &ls = g_shapes[dev & 63];
    std::call_once(ls.once, [&ls] {
        int occ = 0, occ2 = 0;
        cudaFuncSetAttribute(k_downsweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DownSmem));
        cudaFuncSetAttribute(k_downsweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DownSmem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_downsweep<false>, kBlock, sizeof(DownSmem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_upsweep, kBlock, 0);
        ls.aux = std::max(occ2, 1);
        ls.sweep = std::max(occ, 1);
    });
    return ls;
}

int sweep_blocks() { return num_sms() * launch_shapes().sweep; }
int aux_blocks() { return num_sms() * launch_shapes().aux; }

// One radix pass over cnt elements: upsweep, digit scan, downsweep.
// depth_pass >= 0: pass number of the depth stage (planned on the device); -1: a pass
// over the tile keys.
cudaError_t radix_pass(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout, uint64_t *kout64,
                       const float *depth, Count cnt, size_t max_elems, int shift, const Ws &w, int *status,
                       int depth_pass, cudaStream_t s) {
    const int parts = (int)std::max<size_t>((max_elems + kPart - 1) / kPart, 1);
    const bool dpass = depth_pass >= 0;
    k_upsweep<<<std::min(parts, aux_blocks()), kBlock, 0, s>>>(kin, cnt, shift, w.counts, w.parts_stride,
                                                               dpass ? w.ctrl : nullptr, depth_pass);
    k_digit_scan<<<kRadix, kBlock, 0, s>>>(w.counts, cnt, w.parts_stride, w.ctrl, dpass, depth_pass);
    DownArgs a{};
    a.kin = kin;
    a.vin = vin;
    a.kout = kout;
    a.vout = vout;
    a.kout64 = kout64;
    a.depth = depth;
    a.cnt = cnt;
    a.shift = shift;
    a.offsets = w.counts;
    a.stride = w.parts_stride;
    a.ctrl = w.ctrl;
    a.depth_stage = dpass;
    a.pass = depth_pass;
    a.status = status;
    const int grid = std::min(parts, sweep_blocks());
    if (kout64)
        k_downsweep<true><<<grid, kBlock, sizeof(DownSmem), s>>>(a);
    else
        k_downsweep<false><<<grid, kBlock, sizeof(DownSmem), s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t bin_workspace_bytes(int n, int n_views, size_t capacity) {
    size_t total = 0;
    carve(nullptr, (size_t)n * n_views, capacity, &total);
    return total;
}

cudaError_t launch_bin(const BinLaunch &p, cudaStream_t s) {
    const size_t vn = (size_t)p.n * p.n_views;
    size_t need = 0;
    Ws w = carve(p.ws, vn, p.capacity, &need);
    if (need > p.ws_bytes) return cudaErrorInvalidValue;
    cudaError_t e;
    const int total_tiles = p.vt.total_tiles;
    int tile_bits = 1;
    while ((1ll << tile_bits) < (long long)total_tiles) ++tile_bits;
    const int tile_passes = (tile_bits + kRadixBits - 1) / kRadixBits;
    launch_shapes();
    if ((e = cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.num_pairs, 0, sizeof(uint64_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.ranges, 0, sizeof(uint32_t) * 2 * (size_t)total_tiles, s)) != cudaSuccess) return e;
    if (vn == 0) return cudaSuccess;

    // stage 1: depth keys and up to four passes over them (as many as the keys' range
    // needs, decided on the device; the order ends in dvA after an even count, else dvB)
    k_depth_keys<<<(unsigned)((vn + 4 * kBlock - 1) / (4 * kBlock)), kBlock, 0, s>>>(p.proj->tiles, p.proj->depth,
                                                                           (long long)vn, w.dkA, w.dvA, w.ctrl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const Count cnt_vn{vn, nullptr, vn};
    for (int pass = 0; pass < kDepthPasses; ++pass) {
        const bool even = (pass % 2) == 0;
        e = radix_pass(even ? w.dkA : w.dkB, even ? w.dvA : w.dvB, even ? w.dkB : w.dkA, even ? w.dvB : w.dvA,
                       nullptr, nullptr, cnt_vn, vn, kRadixBits * pass, w, p.status, pass, s);
        if (e != cudaSuccess) return e;
    }

    // stage 2: pair offsets in depth order, pair emission, passes over the tile half
    const long long n_groups = (long long)((vn + (size_t)kBlock * kReducePer - 1) / ((size_t)kBlock * kReducePer));
    k_scan_reduce<<<(unsigned)n_groups, kBlock, 0, s>>>(p.proj->tiles, w.dvA, w.dvB, w.ctrl, (long long)vn,
                                                        w.tiles_sorted, w.chunk_sum, w.group_pre);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n_groups <= 2 * kChunkScanThreads)
        k_chunk_scan<2><<<1, kChunkScanThreads, 0, s>>>(w.group_pre, n_groups, p.num_pairs);
    else
        k_chunk_scan<16><<<1, kChunkScanThreads, 0, s>>>(w.group_pre, n_groups, p.num_pairs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    DupArgs d;
    d.tiles_sorted = w.tiles_sorted;
    d.rect = reinterpret_cast<const int4 *>(p.proj->rect);
    d.order_a = w.dvA;
    d.order_b = w.dvB;
    d.plan = w.ctrl;
    d.chunk_sum = w.chunk_sum;
    d.group_pre = w.group_pre;
    d.vn = (long long)vn;
    d.n = p.n;
    d.vt = p.vt;
    d.capacity = p.capacity;
    d.tk = w.tkA;
    d.tv = w.tvA;
    d.status = p.status;
    k_duplicate<<<(unsigned)((vn + kBlock - 1) / kBlock), kBlock, 0, s>>>(d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const Count cnt_k{0, p.num_pairs, p.capacity};
    for (int pass = 0; pass < tile_passes; ++pass) {
        const bool even = (pass % 2) == 0;
        const bool last = pass + 1 == tile_passes;
        uint32_t *kout = even ? w.tkB : w.tkA;
        uint32_t *vout = last ? p.ids_out : (even ? w.tvB : w.tvA);
        e = radix_pass(even ? w.tkA : w.tkB, even ? w.tvA : w.tvB, kout, vout, last ? p.keys_out : nullptr,
                       p.proj->depth, cnt_k, p.capacity, kRadixBits * pass, w, p.status, -1, s);
        if (e != cudaSuccess) return e;
    }
    const uint32_t *tiles_sorted = (tile_passes % 2) ? w.tkB : w.tkA;
    k_ranges<<<aux_blocks(), kBlock, 0, s>>>(tiles_sorted, cnt_k, total_tiles, p.ranges, p.status);
    return cudaGetLastError();
}

}  // namespace hgs
