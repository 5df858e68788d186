// Throughput probes of the two SM pipes the CD kernels compute on, for the benchmark's per-pipe
// roofline denominators: packed FP32 fused multiply-add (fma.rn.f32x2, the Gauss-Seidel sweeps) and
// TF32 warp-level MMA (mma.sync m16n8k8, the split-TF32 contractions).  Each thread (warp) runs
// eight independent dependency chains so that neither probe waits on latency; the values stay
// bounded (multipliers within 1e-7 of one) and are summed into a sink so nothing is optimized away.
#include <cuda_runtime.h>

#include "cdmimo.h"
#include "cd_frame_tc.cuh"

namespace cdmimo {
namespace {

constexpr int kProbeThreads = 256, kProbeBlocksPerSm = 4, kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_ffma2_kernel(int iters, float* sink)
{
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(1.f + 1e-3f * k, 1.f - 1e-3f * (threadIdx.x & 7));
    const float2 m = make_float2(1.0000001f, 0.9999999f), c = make_float2(1e-7f, -1e-7f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], m, c);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_mma_tf32_kernel(int iters, float* sink)
{
    const int lane = threadIdx.x & 31;
    uint32_t a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = __float_as_uint(1e-3f * (float)((lane + q) & 7)) & 0xffffe000u;
    const uint32_t b0 = __float_as_uint(1e-3f) & 0xffffe000u, b1 = __float_as_uint(-1e-3f) & 0xffffe000u;
    float d[kChains][4];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) d[k][q] = 0.f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) mma_tf32(d[k], a, b0, b1);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += d[k][0] + d[k][1] + d[k][2] + d[k][3];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace cdmimo

extern "C" {

size_t cdmimo_pipe_probe_sink_floats(void)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return (size_t)sms * cdmimo::kProbeBlocksPerSm * cdmimo::kProbeThreads;
}

int cdmimo_pipe_probe(int kind, int iters, float* sink, size_t sink_floats, double* flops, void* stream)
{
    using namespace cdmimo;
    if (iters < 1 || !sink || !flops) return CDMIMO_ERR_INVALID_ARG;
    const size_t need = cdmimo_pipe_probe_sink_floats();
    if (need == 0) return CDMIMO_ERR_CUDA;
    if (sink_floats < need) return CDMIMO_ERR_WORKSPACE;
    const int blocks = (int)(need / kProbeThreads);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (kind) {
    case CDMIMO_PROBE_FFMA2:
        probe_ffma2_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, sink);
        *flops = (double)need * iters * kChains * 4.0;  // 2 FMAs per fma.rn.f32x2, 2 flop each
        break;
    case CDMIMO_PROBE_MMA_TF32:
        probe_mma_tf32_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, sink);
        *flops = (double)(need / 32) * iters * kChains * (2.0 * 16 * 8 * 8);  // per warp: m16n8k8
        break;
    default:
        return CDMIMO_ERR_INVALID_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

}  // extern "C"
