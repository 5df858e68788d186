// Host-side launch helpers shared by the library's translation units (each .cu file is compiled
// separately, in parallel, and linked into libcdmimo.so).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "cdmimo.h"
#include "plan.h"
#include "ptx.cuh"

namespace cdmimo {

inline int threads_for(const CdPlan& pl) { return pl.threads; }

// Per-kernel attributes: dynamic shared memory above 48 KB, and the largest shared-memory carveout
// so that several CTAs of one kernel share an SM.
template <typename Kern>
int launch_cd(Kern k, const CdPlan& pl)
{
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    if (pl.smem_bytes > 48u * 1024u) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem_bytes) != cudaSuccess)
            return CDMIMO_ERR_CUDA;
    }
    return CDMIMO_OK;
}

// Grid: one CTA per subcarrier for the scalar kernels; for the persistent kernels (packed and
// Gram form), as many CTAs as fit on the device at once (they walk the subcarriers).
template <typename Kern>
int grid_for(Kern k, const CdPlan& pl)
{
    if (!pl.packed) return pl.n_sc;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return pl.n_sc;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads_for(pl), pl.smem_bytes) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return std::max(1, std::min(pl.n_sc, sms * per_sm));
}

// Launch a persistent CD kernel on plan pl.
template <typename Kern, typename IO>
int launch_persistent(Kern k, const CdPlan& pl, const IO& io, cudaStream_t s)
{
    if (int rc = launch_cd(k, pl)) return rc;
    k<<<grid_for(k, pl), threads_for(pl), pl.smem_bytes, s>>>(pl, io);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

// This translation unit's device status word: OR it into *v, and zero it if clear (the caller has
// synchronized the device).
static inline int module_status(unsigned* v, int clear)
{
    unsigned w = 0;
    if (cudaMemcpyFromSymbol(&w, g_dev_status, sizeof(w)) != cudaSuccess) return CDMIMO_ERR_CUDA;
    *v |= w;
    if (clear) {
        const unsigned z = 0;
        if (cudaMemcpyToSymbol(g_dev_status, &z, sizeof(z)) != cudaSuccess) return CDMIMO_ERR_CUDA;
    }
    return CDMIMO_OK;
}

// Entry points of the Gram-form translation units (gram_detect.cu, gram_precode.cu, gram_frame.cu).
int dispatch_detect_gram(int in_dtype, const CdPlan& pl, const DetectIO& io, cudaStream_t s);
int dispatch_precode_gram(int in_dtype, const CdPlan& pl, const PrecodeIO& io, cudaStream_t s);
int gram_detect_module_status(unsigned* v, int clear);
int gram_precode_module_status(unsigned* v, int clear);
int dispatch_frame_gram(int in_dtype, const CdPlan& pl, const FusedIO& io, cudaStream_t s);
int gram_frame_module_status(unsigned* v, int clear);
// Entry points of the tensor-core translation units (gram_frame_tc.cu: c64 storage;
// gram_frame_tc16.cu: fp16 / bf16 storage); op is CDMIMO_OP_FRAME, CDMIMO_OP_DETECT (io.S, io.Xdl
// unused; learned sweeps and fusion when pl.learned, c64 only) or CDMIMO_OP_PRECODE (only io.d.H and
// io.d.sched of io.d used).
int dispatch_frame_tc(int in_dtype, const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s);
int dispatch_frame_tc16(int in_dtype, const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s);
int frame_tc_module_status(unsigned* v, int clear);
int frame_tc16_module_status(unsigned* v, int clear);
// The warp-specialized tensor-core kernel (gram_frame_ws.cu: c64, gram_frame_ws16.cu: fp16 / bf16),
// for the same plans and ops (not learned); CDMIMO_ERR_UNSUPPORTED, with nothing launched, where it
// does not take the call.
int dispatch_frame_ws(int in_dtype, const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s);
int dispatch_frame_ws16(int in_dtype, const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s);
int frame_ws_module_status(unsigned* v, int clear);
int frame_ws16_module_status(unsigned* v, int clear);
// Tensor-core Gram-form detection for 16 < U <= 32 (gram_tc32.cu), on a plan of build_tc32_plan;
// tc32_layout_fits: CDMIMO_OK where its shared-memory layout fits the device.
int dispatch_detect_tc32(int in_dtype, const CdPlan& pl, const DetectIO& io, cudaStream_t s);
int tc32_layout_fits(const CdPlan& pl, int in_dtype);
int tc32_module_status(unsigned* v, int clear);

}  // namespace cdmimo
