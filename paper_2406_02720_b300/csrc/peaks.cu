// Issue-rate probes for the compositing roofline: the FP32 FMA rate and the MUFU
// ex2 rate this GPU sustains, measured rather than computed from unit counts.
//
// Each thread runs kChains independent dependency chains (so no instruction waits
// for its predecessor's result) for `iters` rounds; the kernel is launched with
// enough resident warps per SM to keep every scheduler issuing.  The chains'
// final values go to `sink` so the compiler keeps the arithmetic.  One FMA (or
// one ex2) of one lane counts as one lane-operation, the unit of the compositing
// kernels' algorithmic operation counts.
#include "hgs_internal.cuh"

namespace hgs {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 512;

__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma(int iters, float *sink) {
    float x[kChains];
    const float a = 0.999999f, b = 1e-7f * (float)(threadIdx.x & 7);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[0] = s;     // practically never taken; keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(int iters, float *sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.25f + 0.01f * (float)c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                // x <- 2^-x: stays in (0.5, 1), converging to the fixed point ~0.64
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(-x[c]));
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[0] = s;
}

}  // namespace
}  // namespace hgs

extern "C" hgs_status hgs_probe_peak(int kind, int blocks_per_sm, int iters, float *sink, double *lane_ops,
                                     void *stream) {
    if (kind < 0 || kind > 1 || blocks_per_sm < 1 || blocks_per_sm > 4 || iters < 1 || !sink) return HGS_ERR_INVALID;
    const int blocks = hgs::num_sms() * blocks_per_sm;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == 0)
        hgs::k_probe_ffma<<<blocks, hgs::kProbeThreads, 0, s>>>(iters, sink);
    else
        hgs::k_probe_ex2<<<blocks, hgs::kProbeThreads, 0, s>>>(iters, sink);
    if (lane_ops) *lane_ops = (double)blocks * hgs::kProbeThreads * (double)iters * 16.0 * hgs::kChains;
    return cudaGetLastError() == cudaSuccess ? HGS_OK : HGS_ERR_CUDA;
}
