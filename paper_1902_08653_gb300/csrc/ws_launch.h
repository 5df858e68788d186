// Host side of the warp-specialized tensor-core kernel (cd_frame_ws.cuh): its shared-memory layout
// for a tensor-core plan, and its launch (one CTA per SM, each walking its subcarriers).  Included
// by the kernel's two translation units (gram_frame_ws.cu, gram_frame_ws16.cu).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "cd_frame_ws.cuh"
#include "launch.h"

namespace cdmimo {

inline unsigned ws_align(unsigned v, unsigned a) { return (v + a - 1u) / a * a; }

// The kernel's layout for plan pl (built by build_tc_plan) and op; UNSUPPORTED where the kernel does
// not take the call: a learned plan, more sweep lanes (C n_sym) than four warps hold, or a layout
// above the device's shared memory per block.
inline int build_ws_layout(const CdPlan& pl, int in_dtype, int op, WsLayout* wl, bool t5 = false)
{
    if (pl.learned || pl.phased) return CDMIMO_ERR_UNSUPPORTED;
    if (pl.n_sym > 16) return CDMIMO_ERR_UNSUPPORTED;
    const int slot = ws_slot(pl.n_sym), cpw = 32 / slot;           // sweep lanes per cluster, clusters per warp
    const int warps = ((pl.C + cpw - 1) / cpw + 3) / 4 * 4;         // warps of a sweep group: four
    if (kWsSweepGroups * warps * 32 + 32 * kWsMmaWarps != kWsMaxThreads) return CDMIMO_ERR_UNSUPPORTED;
    const bool ul = op != CDMIMO_OP_PRECODE, dl = op != CDMIMO_OP_DETECT;
    const unsigned C = pl.C, U = pl.U, UT = kTcUT, n_sym = pl.n_sym, xs = tc_x_stride(pl.n_tiles);
    const unsigned srow = ws_row_words(pl.B, in_dtype);
    const unsigned hbytes = ws_align(UT * srow * 4u, 128u);
    unsigned o = 0;
    auto region = [&](unsigned& off, unsigned& st, unsigned bytes, unsigned align, int n) {
        st = ws_align(bytes, align);
        off = o;
        o += (unsigned)n * st;
    };
    region(wl->off_H, wl->st_H, hbytes, 128u, 3);
    const unsigned bc = (unsigned)pl.cl[0].size, blk = 16u * 2u * bc * 4u;  // T5 operand block bytes
    unsigned st_op = 0;
    wl->off_op = 0;
    if (t5) region(wl->off_op, st_op, std::max(6u * blk, 16384u), 128u, 1);  // also the epilogue's scratch
    region(wl->off_G, wl->st_G, C * UT * (UT / 2) * 16u, 128u, 2);
    region(wl->off_D, wl->st_D, 2u * C * UT * 4u, 16u, 2);
    region(wl->off_Z, wl->st_Z, ul ? UT * xs * 8u : 0u, 16u, 2);
    region(wl->off_W, wl->st_W, dl ? UT * xs * 8u : 0u, 16u, 2);
    region(wl->off_S, wl->st_S, dl ? n_sym * U * 8u : 0u, 16u, 2);
    region(wl->off_lam, wl->st_lam, C * 4u, 16u, 2);
    wl->off_tab = o;
    o = ws_align(o + C * (unsigned)sizeof(ClusterTile), 16u);
    wl->off_bar = o;
    o = ws_align(o + 8u * 8u + 2u * 4u + 16u, 16u);
    wl->smem_bytes = o;
    wl->tmem_cols = 32u;
    while (t5 && wl->tmem_cols < 64u * C) wl->tmem_cols *= 2u;
    wl->sweep_warps = warps;
    wl->slot = slot;
    wl->srow = (int)srow;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    return (int)wl->smem_bytes <= optin ? CDMIMO_OK : CDMIMO_ERR_UNSUPPORTED;
}

template <int BC, int MODE, int IN, bool T5 = false>
int ws_launch(const CdPlan& pl, const WsLayout& wl, const FusedIO& io, cudaStream_t s)
{
    auto k = cd_frame_ws_kernel<BC, MODE, IN, T5>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wl.smem_bytes) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    const int threads = 32 * (kWsMmaWarps + kWsSweepGroups * wl.sweep_warps);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, wl.smem_bytes) != cudaSuccess || per_sm < 1)
        return CDMIMO_ERR_UNSUPPORTED;
    const int grid = std::max(1, std::min(pl.n_sc, sms * per_sm));
    k<<<grid, threads, wl.smem_bytes, s>>>(pl, wl, io);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

// Whether the call runs phase A on the tcgen05 tensor cores: c64 storage, at most 8 clusters, the
// plan asks for it, and (uplink) 16-byte aligned receive samples (read as float4).
template <int IN>
bool ws_use_t5(const CdPlan& pl, const FusedIO& io, int op)
{
    if (IN != CDMIMO_C64 || !pl.umma || pl.C > 8) return false;
    return op == CDMIMO_OP_PRECODE || (reinterpret_cast<uintptr_t>(io.d.Y) & 15u) == 0u;
}

// CDMIMO_ERR_UNSUPPORTED (nothing launched) where the kernel does not take the call; op DETECT also
// needs no per-cluster outputs (io.d.Xc, io.d.lam).
template <int IN>
int ws_dispatch_op(const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s)
{
    const int bc = pl.cl[0].size;
    if (bc != 16 && bc != 32) return CDMIMO_ERR_UNSUPPORTED;
    if (op == CDMIMO_OP_DETECT && (io.d.Xc || io.d.lam)) return CDMIMO_ERR_UNSUPPORTED;
    WsLayout wl{};
    if constexpr (IN == CDMIMO_C64) {
        if (ws_use_t5<IN>(pl, io, op) && build_ws_layout(pl, IN, op, &wl, true) == CDMIMO_OK) {
            switch (op) {
            case CDMIMO_OP_FRAME:
                return bc == 16 ? ws_launch<16, kTcFrame, IN, true>(pl, wl, io, s)
                                : ws_launch<32, kTcFrame, IN, true>(pl, wl, io, s);
            case CDMIMO_OP_DETECT:
                return bc == 16 ? ws_launch<16, kTcDetect, IN, true>(pl, wl, io, s)
                                : ws_launch<32, kTcDetect, IN, true>(pl, wl, io, s);
            case CDMIMO_OP_PRECODE:
                return bc == 16 ? ws_launch<16, kTcPrecode, IN, true>(pl, wl, io, s)
                                : ws_launch<32, kTcPrecode, IN, true>(pl, wl, io, s);
            }
        }
    }
    if (int rc = build_ws_layout(pl, IN, op, &wl)) return rc;
    switch (op) {
    case CDMIMO_OP_FRAME:
        return bc == 16 ? ws_launch<16, kTcFrame, IN>(pl, wl, io, s) : ws_launch<32, kTcFrame, IN>(pl, wl, io, s);
    case CDMIMO_OP_DETECT:
        return bc == 16 ? ws_launch<16, kTcDetect, IN>(pl, wl, io, s) : ws_launch<32, kTcDetect, IN>(pl, wl, io, s);
    case CDMIMO_OP_PRECODE:
        return bc == 16 ? ws_launch<16, kTcPrecode, IN>(pl, wl, io, s) : ws_launch<32, kTcPrecode, IN>(pl, wl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

}  // namespace cdmimo
