// Translation unit of the tensor-core Gram-form detection kernel for 16 < U <= 32 users
// (cd_detect_tc32.cuh): shared-memory layout, instantiation for clusters of 16, 32 or 64 antennas and
// each storage type, and dispatch.
#include <algorithm>

#include "cd_detect_tc32.cuh"
#include "launch.h"

namespace cdmimo {

namespace {

unsigned tc32_align(unsigned v, unsigned a) { return (v + a - 1u) / a * a; }

// The kernel's layout for plan pl; UNSUPPORTED when it exceeds the device's shared memory per block.
int build_tc32_layout(const CdPlan& pl, int in_dtype, Tc32Layout* tl)
{
    const unsigned C = pl.C, UT = 32, xs = tc_x_stride(pl.n_tiles);
    const unsigned srow = ws_row_words(pl.B, in_dtype);
    unsigned o = 0;
    tl->srow = (int)srow;
    tl->st_H = tc32_align(UT * srow * 4u, 128u);
    tl->off_H = o;
    o += 2u * tl->st_H;
    tl->off_G = o;
    o = tc32_align(o + C * UT * 16u * 16u, 128u);
    tl->off_D = o;
    o = tc32_align(o + C * UT * 4u, 16u);
    tl->off_Z = o;
    o = tc32_align(o + UT * xs * 8u, 16u);
    tl->off_lam = o;
    o = tc32_align(o + C * 4u, 16u);
    tl->off_tab = o;
    o = tc32_align(o + C * (unsigned)sizeof(ClusterTile), 16u);
    tl->off_bar = o;
    o = tc32_align(o + 16u, 16u);
    tl->smem_bytes = o;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    return (int)tl->smem_bytes <= optin ? CDMIMO_OK : CDMIMO_ERR_UNSUPPORTED;
}

template <int BC, int IN>
int launch_tc32(const CdPlan& pl, const Tc32Layout& tl, const DetectIO& io, cudaStream_t s)
{
    auto k = cd_detect_tc32_kernel<BC, IN>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tl.smem_bytes) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTc32Threads, tl.smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return CDMIMO_ERR_UNSUPPORTED;
    const int grid = std::max(1, std::min(pl.n_sc, sms * per_sm));
    k<<<grid, kTc32Threads, tl.smem_bytes, s>>>(pl, tl, io);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

template <int IN>
int dispatch_bc(const CdPlan& pl, const Tc32Layout& tl, const DetectIO& io, cudaStream_t s)
{
    switch (pl.cl[0].size) {
    case 16: return launch_tc32<16, IN>(pl, tl, io, s);
    case 32: return launch_tc32<32, IN>(pl, tl, io, s);
    case 64: return launch_tc32<64, IN>(pl, tl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

}  // namespace

int tc32_layout_fits(const CdPlan& pl, int in_dtype)
{
    Tc32Layout tl{};
    return build_tc32_layout(pl, in_dtype, &tl);
}

int dispatch_detect_tc32(int in_dtype, const CdPlan& pl, const DetectIO& io, cudaStream_t s)
{
    Tc32Layout tl{};
    if (int rc = build_tc32_layout(pl, in_dtype, &tl)) return rc;
    switch (in_dtype) {
    case CDMIMO_C64: return dispatch_bc<CDMIMO_C64>(pl, tl, io, s);
    case CDMIMO_C16F: return dispatch_bc<CDMIMO_C16F>(pl, tl, io, s);
    case CDMIMO_C16BF: return dispatch_bc<CDMIMO_C16BF>(pl, tl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int tc32_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
