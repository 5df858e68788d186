// Throughput probes of the two SM pipes the CD kernels compute on, for the benchmark's per-pipe
// roofline denominators: packed FP32 fused multiply-add (fma.rn.f32x2, the Gauss-Seidel sweeps) and
// TF32 warp-level MMA (mma.sync m16n8k8, the split-TF32 contractions).  Each thread (warp) runs
// eight independent dependency chains so that neither probe waits on latency; the values stay
// bounded (multipliers within 1e-7 of one) and are summed into a sink so nothing is optimized away.
#include <cuda_runtime.h>

#include "cdmimo.h"
#include "cd_frame_tc.cuh"
#include "umma.cuh"

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

// One tcgen05 product D = A B^T (tf32, M = M_, N = 32, K = 32) on one CTA: A [M_][32] and B [32][32]
// row-major in global memory, written K-major without swizzle into shared memory (the layout of
// umma.cuh), four chained MMAs into tensor memory, and every one of the 128 lanes x 32 columns read
// back into D [128][32] (lane-major), so that a test sees where each row of the accumulator lands.
template <int M_>
__global__ void __launch_bounds__(128) umma_layout_kernel(const float* A, const float* B, float* D)
{
    constexpr int K = 32, N = 32;
    __shared__ __align__(128) float As[128 * K];
    __shared__ __align__(128) float Bs[N * K];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    auto kmaj = [](int m, int k) { return (m >> 3) * (K / 4) * 32 + (k >> 2) * 32 + (m & 7) * 4 + (k & 3); };
    for (int i = tid; i < 128 * K; i += blockDim.x) As[kmaj(i / K, i % K)] = i / K < M_ ? A[i] : 0.f;
    for (int i = tid; i < N * K; i += blockDim.x) Bs[kmaj(i / K, i % K)] = B[i];
    if (tid == 0) mbar_init(&bar, 1u);
    if (warp == 0) tmem_alloc(&slot, 32u);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = slot;
    if (tid == 0) {
        const uint64_t da = umma_desc(As, 128u, 128u * (K / 4)), db = umma_desc(Bs, 128u, 128u * (K / 4));
#pragma unroll
        for (int ks = 0; ks < K / 8; ++ks) umma_tf32(tb, da + 16u * ks, db + 16u * ks, umma_idesc_tf32(M_, N), ks > 0);
        umma_commit(&bar);
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bar, 0u, 100000000ull);
    tc_fence_after();
    if (ok) {
        float v[32];
        tmem_ld32(tb + ((uint32_t)(32 * warp) << 16), v);
        for (int j = 0; j < 32; ++j) D[(32 * warp + (tid & 31)) * 32 + j] = v[j];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tb, 32u);
    }
}

// Issue cost of back-to-back tcgen05 MMAs (tf32, K = 8, zero operands) from one thread: `n` MMAs of
// M_ x N_ into one accumulator, then a commit and its wait; the best of `reps` runs in SM cycles.
template <int M_>
__global__ void __launch_bounds__(32) umma_rate_kernel(int N_, int n, int reps, long long* cycles)
{
    constexpr int K = 16;                                   // words of K held (two MMA k-steps)
    __shared__ __align__(128) float S[128 * K + 256 * K];   // A: 128 rows; B: up to 256 rows
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    for (int i = threadIdx.x; i < 128 * K + 256 * K; i += 32) S[i] = 0.f;
    if (threadIdx.x == 0) mbar_init(&bar, 1u);
    tmem_alloc(&slot, 256u);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    tc_fence_after();
    const uint32_t tb = slot;
    long long best = -1;
    if (threadIdx.x == 0) {
        const uint64_t da = umma_desc(S, 128u, 128u * (K / 4)), db = umma_desc(S + 128 * K, 128u, 128u * (K / 4));
        const uint32_t idesc = umma_idesc_tf32(M_, N_);
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r) {
            const long long t0 = clock64();
            for (int i = 0; i < n; ++i) umma_tf32(tb, da + 16u * (i & 1), db + 16u * (i & 1), idesc, i > 0);
            umma_commit(&bar);
            ok = mbar_wait_bounded(&bar, (uint32_t)r & 1u, 100000000ull);
            const long long dt = clock64() - t0;
            if (best < 0 || dt < best) best = dt;
        }
        *cycles = ok ? best : -1;
    }
    __syncwarp();
    tc_fence_before();
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tb, 256u);
}

}  // namespace
}  // namespace cdmimo

extern "C" {

int cdmimo_umma_layout_probe(int M, const float* A, const float* B, float* D, void* stream)
{
    using namespace cdmimo;
    if ((M != 64 && M != 128) || !A || !B || !D) return CDMIMO_ERR_INVALID_ARG;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (M == 64) umma_layout_kernel<64><<<1, 128, 0, s>>>(A, B, D);
    else umma_layout_kernel<128><<<1, 128, 0, s>>>(A, B, D);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

int cdmimo_umma_rate_probe(int M, int N, int n, long long* cycles, void* stream)
{
    using namespace cdmimo;
    if ((M != 64 && M != 128) || N < 16 || N > 256 || (N & 15) || n < 1 || n > 4096 || !cycles)
        return CDMIMO_ERR_INVALID_ARG;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (M == 64) umma_rate_kernel<64><<<1, 32, 0, s>>>(N, n, 5, cycles);
    else umma_rate_kernel<128><<<1, 32, 0, s>>>(N, n, 5, cycles);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

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
