// Tile binning (A3-A5): exclusive scan of tiles touched, key emission, a stable
// LSD onesweep radix sort of the 64-bit (tile | depth) keys, and per-tile ranges.
//
// Scan: single pass with decoupled look-back over 4096-element partitions that
// persistent blocks take in order from an atomic ticket.
// Sort: one histogram pass over all key digits, then one onesweep pass per 8-bit
// digit.  Each pass ranks a 4096-key partition in shared memory (warp-level
// match_any multisplit, stable by construction), publishes per-digit counts,
// resolves its global digit offsets by decoupled look-back over the preceding
// partitions, and scatters through shared memory so that global writes are
// runs of consecutive addresses.  Every spin-wait has an iteration cap; on
// timeout it sets HGS_DEV_TIMEOUT and proceeds with the counts it has.
#include <algorithm>

#include "hgs_internal.cuh"

namespace hgs {
namespace {

constexpr int kBlock = 256;                  // threads per block (8 warps)
constexpr int kItems = 16;                   // items per thread
constexpr int kPart = kBlock * kItems;       // 4096 elements per partition
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;      // 256 digits
constexpr int kMaxPasses = 8;

// look-back word flags (top two bits)
constexpr uint32_t kFlagAgg32 = 1u << 30, kFlagInc32 = 2u << 30, kValMask32 = (1u << 30) - 1u;
constexpr unsigned long long kFlagAgg64 = 1ull << 62, kFlagInc64 = 2ull << 62;
constexpr unsigned long long kValMask64 = (1ull << 62) - 1ull;

struct Ctrl {                                // zeroed at the start of every hgs_bin
    uint32_t hist[kMaxPasses][kRadix];       // global digit histograms
    uint32_t ticket[kMaxPasses];             // partition tickets of each sort pass
    uint32_t scan_ticket;
    uint32_t pad[7];
};

struct Ws {
    uint32_t *offsets;                       // [VN] exclusive scan of tiles
    unsigned long long *scan_state;          // [scan partitions]
    Ctrl *ctrl;
    uint64_t *keys_alt;                      // [capacity]
    uint32_t *ids_alt;                       // [capacity]
    uint32_t *lookback;                      // [2][sort partitions][256]
    size_t scan_parts, sort_parts;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

Ws carve(void *base, size_t vn, size_t cap, size_t *total) {
    Ws w{};
    w.scan_parts = (vn + kPart - 1) / kPart;
    w.sort_parts = (cap + kPart - 1) / kPart;
    size_t off = 0;
    char *b = static_cast<char *>(base);
    auto take = [&](size_t bytes) { char *p = b ? b + off : nullptr; off += align_up(bytes); return p; };
    w.ctrl = reinterpret_cast<Ctrl *>(take(sizeof(Ctrl)));
    w.scan_state = reinterpret_cast<unsigned long long *>(take(8 * std::max<size_t>(w.scan_parts, 1)));
    w.offsets = reinterpret_cast<uint32_t *>(take(4 * std::max<size_t>(vn, 1)));
    w.keys_alt = reinterpret_cast<uint64_t *>(take(8 * std::max<size_t>(cap, 1)));
    w.ids_alt = reinterpret_cast<uint32_t *>(take(4 * std::max<size_t>(cap, 1)));
    w.lookback = reinterpret_cast<uint32_t *>(take(4 * 2 * kRadix * std::max<size_t>(w.sort_parts, 1)));
    if (total) *total = off;
    return w;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// ---- A3: single-pass exclusive scan of tiles touched ---------------------------
__global__ void __launch_bounds__(kBlock) k_scan(const uint32_t *__restrict__ in, long long n,
                                                 uint32_t *__restrict__ out,
                                                 unsigned long long *state, Ctrl *ctrl,
                                                 uint64_t *total_out, int *status) {
    __shared__ unsigned long long s_warp[kBlock / 32];
    __shared__ unsigned long long s_prefix;
    __shared__ uint32_t s_part;
    const long long n_parts = (n + kPart - 1) / kPart;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    for (;;) {
        if (threadIdx.x == 0) s_part = atomicAdd(&ctrl->scan_ticket, 1u);
        __syncthreads();
        const long long part = s_part;
        if (part >= n_parts) break;
        const long long base = part * kPart + (long long)threadIdx.x * kItems;
        uint32_t v[kItems];
        if (base + kItems <= n) {
            const uint4 *src = reinterpret_cast<const uint4 *>(in + base);
#pragma unroll
            for (int j = 0; j < kItems / 4; ++j) {
                uint4 t = src[j];
                v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kItems; ++j) v[j] = (base + j < n) ? in[base + j] : 0u;
        }
        unsigned long long tsum = 0;
#pragma unroll
        for (int j = 0; j < kItems; ++j) tsum += v[j];
        // block exclusive scan of the thread sums
        unsigned long long x = tsum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        unsigned long long wbase = 0, agg = 0;
#pragma unroll
        for (int w2 = 0; w2 < kBlock / 32; ++w2) {
            if (w2 < warp) wbase += s_warp[w2];
            agg += s_warp[w2];
        }
        unsigned long long texcl = wbase + x - tsum;
        // decoupled look-back by warp 0
        if (warp == 0) {
            if (lane == 0)
                st_relaxed_u64(&state[part], (part == 0 ? kFlagInc64 : kFlagAgg64) | agg);
            unsigned long long excl = 0;
            long long j = part - 1;
            unsigned spins = 0;
            bool timed_out = false;
            while (j >= 0) {
                long long idx = j - lane;
                unsigned long long w = idx >= 0 ? ld_relaxed_u64(&state[idx]) : kFlagInc64;
                while (__any_sync(0xffffffffu, (w >> 62) == 0)) {
                    if (++spins > kSpinCap) { timed_out = true; break; }
                    __nanosleep(kSpinSleepNs);
                    if ((w >> 62) == 0) w = ld_relaxed_u64(&state[idx]);
                }
                if (timed_out) { if ((w >> 62) == 0) w = kFlagInc64; }
                unsigned inc = __ballot_sync(0xffffffffu, (w >> 62) == 2);
                int stop = inc ? __ffs(inc) - 1 : 31;
                unsigned long long val = (lane <= stop) ? (w & kValMask64) : 0ull;
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) val += __shfl_xor_sync(0xffffffffu, val, d);
                excl += val;
                if (inc) break;
                j -= 32;
            }
            if (timed_out && lane == 0) set_status(status, HGS_DEV_TIMEOUT);
            if (lane == 0) {
                if (part > 0) st_relaxed_u64(&state[part], kFlagInc64 | (excl + agg));
                s_prefix = excl;
            }
        }
        __syncthreads();
        unsigned long long run = s_prefix + texcl;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (base + j < n) out[base + j] = run > 0xffffffffull ? 0xffffffffu : (uint32_t)run;
            run += v[j];
        }
        if (part == n_parts - 1 && threadIdx.x == kBlock - 1) *total_out = s_prefix + texcl + tsum;
        __syncthreads();
    }
}

// ---- A3: key emission ---------------------------------------------------------------
struct DupArgs {
    const uint32_t *tiles;
    const int4 *rect;
    const float *depth;
    const uint32_t *offsets;
    const uint64_t *num_pairs;
    long long vn;
    int n;
    ViewTable vt;
    size_t capacity;
    uint64_t *keys;
    uint32_t *ids;
    int *status;
};

__global__ void __launch_bounds__(kBlock) k_duplicate(DupArgs a) {
    const long long vi = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (vi >= a.vn) return;
    const uint32_t cnt = a.tiles[vi];
    if (cnt == 0) return;
    const uint64_t off = a.offsets[vi];
    if (off + cnt > a.capacity) set_status(a.status, HGS_DEV_CAPACITY);
    const int v = (int)(vi / a.n);
    const int4 r = a.rect[vi];
    const uint64_t db = __float_as_uint(a.depth[vi]);
    const int tx = a.vt.tiles_x[v];
    const int gbase = a.vt.tile_off[v];
    uint64_t j = off;
    for (int ty = r.y; ty < r.w; ++ty)
        for (int tx2 = r.x; tx2 < r.z; ++tx2, ++j) {
            if (j >= a.capacity) return;
            a.keys[j] = ((uint64_t)(gbase + ty * tx + tx2) << 32) | db;
            a.ids[j] = (uint32_t)vi;
        }
}

// ---- A4: digit histograms for all passes (and look-back region 0 cleared) ------------
__global__ void __launch_bounds__(kBlock) k_hist(const uint64_t *__restrict__ keys,
                                                 const uint64_t *num_pairs, size_t capacity,
                                                 int npass, Ctrl *ctrl, uint32_t *lookback0) {
    __shared__ uint32_t s_hist[kMaxPasses][kRadix];
    for (int j = threadIdx.x; j < kMaxPasses * kRadix; j += kBlock) (&s_hist[0][0])[j] = 0;
    __syncthreads();
    const size_t K = min((size_t)*num_pairs, capacity);
    const size_t parts = (K + kPart - 1) / kPart;
    const size_t stride = (size_t)gridDim.x * kBlock;
    for (size_t j = (size_t)blockIdx.x * kBlock + threadIdx.x; j < parts * kRadix; j += stride) lookback0[j] = 0;
    const size_t rounds = (K + stride - 1) / stride;
    for (size_t r = 0; r < rounds; ++r) {
        const size_t j = r * stride + (size_t)blockIdx.x * kBlock + threadIdx.x;
        const bool valid = j < K;
        const uint64_t key = valid ? keys[j] : 0ull;
        for (int p = 0; p < npass; ++p) {
            const uint32_t d = valid ? (uint32_t)(key >> (kRadixBits * p)) & (kRadix - 1) : kRadix + lane_id();
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&s_hist[p][d], __popc(peers));
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < npass * kRadix; j += kBlock) {
        uint32_t c = (&s_hist[0][0])[j];
        if (c) atomicAdd(&(&ctrl->hist[0][0])[j], c);
    }
}

// ---- A4: one onesweep pass -------------------------------------------------------------
struct SweepSmem {
    uint64_t keys[kPart];
    uint32_t vals[kPart];
    uint32_t warp_cnt[kBlock / 32][kRadix];  // per-warp digit counts, then warp offsets
    uint32_t digit_start[kRadix];            // partition-local exclusive digit prefix
    uint32_t global_off[kRadix];             // global destination of each digit bucket
    uint32_t digit_base[kRadix];             // exclusive prefix of the global histogram
    uint32_t part;
    uint32_t scan_tmp[kBlock / 32];
};

__global__ void __launch_bounds__(kBlock) k_onesweep(int pass, const uint64_t *__restrict__ kin,
                                                     const uint32_t *__restrict__ vin,
                                                     uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                     const uint64_t *num_pairs, size_t capacity,
                                                     Ctrl *ctrl, uint32_t *lookback, uint32_t *lookback_next,
                                                     int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepSmem &sm = *reinterpret_cast<SweepSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const uint32_t K = (uint32_t)min((size_t)*num_pairs, capacity);
    const uint32_t n_parts = (K + kPart - 1) / kPart;
    const int shift = kRadixBits * pass;
    const unsigned lanemask_lt = (1u << lane) - 1u;

    // exclusive prefix of the global histogram of this digit (thread = digit)
    {
        uint32_t c = ctrl->hist[pass][tid];
        uint32_t x = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) sm.scan_tmp[warp] = x;
        __syncthreads();
        uint32_t wb = 0;
        for (int w2 = 0; w2 < warp; ++w2) wb += sm.scan_tmp[w2];
        sm.digit_base[tid] = wb + x - c;
        __syncthreads();
    }

    for (;;) {
        if (tid == 0) sm.part = atomicAdd(&ctrl->ticket[pass], 1u);
        __syncthreads();
        const uint32_t part = sm.part;
        if (part >= n_parts) break;
        // clear this partition's word row in the next pass's look-back region
        if (lookback_next) lookback_next[(size_t)part * kRadix + tid] = 0;
        const uint32_t pbase = part * kPart;
        for (int j = lane; j < kRadix; j += 32) sm.warp_cnt[warp][j] = 0;
        __syncwarp();
        uint64_t key[kItems];
        uint32_t val[kItems];
        uint32_t rank[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t idx = pbase + warp * (32 * kItems) + it * 32 + lane;
            const bool valid = idx < K;
            key[it] = valid ? kin[idx] : 0ull;
            val[it] = valid ? vin[idx] : 0u;
            const uint32_t d = valid ? (uint32_t)(key[it] >> shift) & (kRadix - 1) : kRadix;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
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
            uint32_t c = sm.warp_cnt[w2][tid];
            sm.warp_cnt[w2][tid] = total;
            total += c;
        }
        uint32_t *row = lookback + (size_t)part * kRadix;
        st_relaxed_u32(&row[tid], (part == 0 ? kFlagInc32 : kFlagAgg32) | total);
        // partition-local exclusive prefix over digits
        {
            uint32_t x = total;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += y;
            }
            if (lane == 31) sm.scan_tmp[warp] = x;
            __syncthreads();
            uint32_t wb = 0;
            for (int w2 = 0; w2 < warp; ++w2) wb += sm.scan_tmp[w2];
            sm.digit_start[tid] = wb + x - total;
        }
        // decoupled look-back for this digit
        uint32_t excl = 0;
        if (part > 0) {
            int j = (int)part - 1;
            unsigned spins = 0;
            while (j >= 0) {
                uint32_t w = ld_relaxed_u32(&lookback[(size_t)j * kRadix + tid]);
                uint32_t flag = w & ~kValMask32;
                if (flag == 0) {
                    if (++spins > kSpinCap) { set_status(status, HGS_DEV_TIMEOUT); break; }
                    __nanosleep(kSpinSleepNs);
                    continue;
                }
                excl += w & kValMask32;
                if (flag == kFlagInc32) break;
                --j;
            }
            st_relaxed_u32(&row[tid], kFlagInc32 | ((excl + total) & kValMask32));
        }
        sm.global_off[tid] = sm.digit_base[tid] + excl;
        __syncthreads();
        // scatter into shared memory in partition-sorted order
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t idx = pbase + warp * (32 * kItems) + it * 32 + lane;
            if (idx < K) {
                const uint32_t d = (uint32_t)(key[it] >> shift) & (kRadix - 1);
                const uint32_t pos = sm.digit_start[d] + sm.warp_cnt[warp][d] + rank[it];
                sm.keys[pos] = key[it];
                sm.vals[pos] = val[it];
            }
        }
        __syncthreads();
        const uint32_t cnt = min((uint32_t)kPart, K - pbase);
        for (uint32_t j = tid; j < cnt; j += kBlock) {
            const uint64_t k = sm.keys[j];
            const uint32_t d = (uint32_t)(k >> shift) & (kRadix - 1);
            const uint32_t dst = sm.global_off[d] + (j - sm.digit_start[d]);
            if (dst < capacity) {
                kout[dst] = k;
                vout[dst] = sm.vals[j];
            } else {
                set_status(status, HGS_DEV_BOUNDS);
            }
        }
        __syncthreads();
    }
}

// ---- A5: tile ranges -----------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_ranges(const uint64_t *__restrict__ keys,
                                                   const uint64_t *num_pairs, size_t capacity,
                                                   int total_tiles, uint32_t *ranges, int *status) {
    const size_t K = min((size_t)*num_pairs, capacity);
    for (size_t i = (size_t)blockIdx.x * kBlock + threadIdx.x; i < K; i += (size_t)gridDim.x * kBlock) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        if (t >= (uint32_t)total_tiles) { set_status(status, HGS_DEV_BOUNDS); continue; }
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[2 * (size_t)t] = (uint32_t)i;
        if (i == K - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[2 * (size_t)t + 1] = (uint32_t)(i + 1);
    }
}

int g_sweep_blocks = 0, g_aux_blocks = 0;

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
    // key bits in use: 32 depth bits + enough for the largest global tile id
    int tile_bits = 1;
    while ((1ll << tile_bits) < (long long)total_tiles) ++tile_bits;
    const int key_bits = 32 + tile_bits;
    const int npass = (key_bits + kRadixBits - 1) / kRadixBits;
    // where the unsorted pairs go so that the last pass lands in keys_out/ids_out
    uint64_t *kA = (npass % 2 == 0) ? p.keys_out : w.keys_alt;
    uint32_t *iA = (npass % 2 == 0) ? p.ids_out : w.ids_alt;
    uint64_t *kB = (npass % 2 == 0) ? w.keys_alt : p.keys_out;
    uint32_t *iB = (npass % 2 == 0) ? w.ids_alt : p.ids_out;

    if (g_sweep_blocks == 0) {
        const int sms = num_sms();
        int occ = 0;
        cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SweepSmem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_onesweep, kBlock, sizeof(SweepSmem));
        g_sweep_blocks = sms * std::max(occ, 1);
        int occ2 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_scan, kBlock, 0);
        g_aux_blocks = sms * std::max(occ2, 1);
    }
    if ((e = cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.scan_state, 0, 8 * std::max<size_t>(w.scan_parts, 1), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.num_pairs, 0, sizeof(uint64_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.ranges, 0, sizeof(uint32_t) * 2 * (size_t)total_tiles, s)) != cudaSuccess) return e;
    if (vn == 0) return cudaSuccess;
    {
        int grid = (int)std::min<size_t>(w.scan_parts, (size_t)g_aux_blocks);
        k_scan<<<grid, kBlock, 0, s>>>(p.proj->tiles, (long long)vn, w.offsets, w.scan_state, w.ctrl,
                                       p.num_pairs, p.status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        DupArgs d;
        d.tiles = p.proj->tiles;
        d.rect = reinterpret_cast<const int4 *>(p.proj->rect);
        d.depth = p.proj->depth;
        d.offsets = w.offsets;
        d.num_pairs = p.num_pairs;
        d.vn = (long long)vn;
        d.n = p.n;
        d.vt = p.vt;
        d.capacity = p.capacity;
        d.keys = kA;
        d.ids = iA;
        d.status = p.status;
        k_duplicate<<<(unsigned)((vn + kBlock - 1) / kBlock), kBlock, 0, s>>>(d);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_hist<<<g_aux_blocks, kBlock, 0, s>>>(kA, p.num_pairs, p.capacity, npass, w.ctrl, w.lookback);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t region = (size_t)kRadix * std::max<size_t>(w.sort_parts, 1);
    for (int pass = 0; pass < npass; ++pass) {
        const bool even = (pass % 2) == 0;
        uint32_t *lb = w.lookback + (even ? 0 : region);
        uint32_t *lb_next = (pass + 1 < npass) ? w.lookback + (even ? region : 0) : nullptr;
        k_onesweep<<<g_sweep_blocks, kBlock, sizeof(SweepSmem), s>>>(
            pass, even ? kA : kB, even ? iA : iB, even ? kB : kA, even ? iB : iA, p.num_pairs, p.capacity,
            w.ctrl, lb, lb_next, p.status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_ranges<<<g_aux_blocks, kBlock, 0, s>>>(p.keys_out, p.num_pairs, p.capacity, total_tiles, p.ranges, p.status);
    return cudaGetLastError();
}

}  // namespace hgs
