// C-ABI entry points of the cdmimo library: argument validation, launch planning and kernel
// dispatch.  Every hot-path call enqueues on the caller's stream and returns; nothing here
// allocates device memory or synchronizes (except cdmimo_device_status, which is documented to).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <vector>

#include "cd_kernels.cuh"
#include "cd_kernels_pp.cuh"
#include "learned_kernels.cuh"
#include "batched_kernel.cuh"
#include "synth_kernels.cuh"
#include "cdmimo.h"
#include "plan.h"
#include "launch.h"

using namespace cdmimo;

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxThreads = 512;             // threads per CTA of the generic CD kernels
constexpr int kMaxSpecializedThreads = 512;  // the compile-time-A variants (96 registers)

int device_smem_optin()
{
    static int cache[kMaxDevices] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 48 * 1024;
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
            v = 48 * 1024;
        cache[dev] = v;
    }
    return cache[dev];
}

int pow2ceil(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

unsigned align16(unsigned v) { return (v + 15u) & ~15u; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int elem_bytes(int dtype) { return dtype == CDMIMO_C64 ? 8 : 4; }

// Structural validation of the problem description (no device pointers involved).
int validate(const cdmimo_params* p)
{
    if (!p) return CDMIMO_ERR_INVALID_ARG;
    if (p->n_sc < 0 || p->n_sym < 1 || p->B < 1 || p->U < 1 || p->C < 1 || p->K < 0) return CDMIMO_ERR_INVALID_ARG;
    if (!(p->Ex > 0.f)) return CDMIMO_ERR_INVALID_ARG;
    if (p->in_dtype != CDMIMO_C64 && p->in_dtype != CDMIMO_C16F && p->in_dtype != CDMIMO_C16BF)
        return CDMIMO_ERR_INVALID_ARG;
    if (p->fuse != CDMIMO_FUSE_EQUAL && p->fuse != CDMIMO_FUSE_COLNORM && p->fuse != CDMIMO_FUSE_LEARNED)
        return CDMIMO_ERR_INVALID_ARG;
    if (p->form != CDMIMO_FORM_AUTO && p->form != CDMIMO_FORM_RESIDUAL && p->form != CDMIMO_FORM_GRAM &&
        p->form != CDMIMO_FORM_GRAM_TC && p->form != CDMIMO_FORM_GRAM_TC_PHASED && p->form != CDMIMO_FORM_GRAM_TC_UMMA)
        return CDMIMO_ERR_INVALID_ARG;
    if (p->U > CDMIMO_MAX_USERS) return CDMIMO_ERR_UNSUPPORTED;
    if (!p->cluster_size || p->C > CDMIMO_MAX_CLUSTERS) return CDMIMO_ERR_BAD_PARTITION;
    long sum = 0;
    for (int c = 0; c < p->C; ++c) {
        if (p->cluster_size[c] < 1) return CDMIMO_ERR_BAD_PARTITION;
        sum += p->cluster_size[c];
    }
    if (sum != p->B) return CDMIMO_ERR_BAD_PARTITION;
    return CDMIMO_OK;
}

// Build the tiling for antennas-per-lane P.  Returns UNSUPPORTED if the CTA would need more than
// kMaxThreads threads or more shared memory than the device grants.
int build_plan(const cdmimo_params* p, int P, bool detect, const void* H, CdPlan* pl)
{
    const bool learned = detect && p->learned != nullptr;
    std::memset(pl, 0, sizeof(*pl));
    pl->n_sc = p->n_sc;
    pl->n_sym = p->n_sym;
    pl->B = p->B;
    pl->U = p->U;
    pl->C = p->C;
    pl->K = p->K;
    pl->P = P;
    pl->fuse = p->fuse;
    pl->inv_Ex = 1.f / p->Ex;
    pl->rho_c = (float)(p->rho / std::sqrt((double)p->C));
    int off = 0, soff = 0;
    bool all_even = true;
    pl->A_uniform = -1;
    for (int c = 0; c < p->C; ++c) {
        ClusterTile& ct = pl->cl[c];
        ct.off = off;
        ct.size = p->cluster_size[c];
        ct.A = pow2ceil((ct.size + P - 1) / P);
        if (ct.A > 32) return CDMIMO_ERR_UNSUPPORTED;
        ct.L = ct.A * P;
        ct.soff = soff;
        if (ct.L != ct.size) pl->padded = 1;
        if (ct.size & 1) all_even = false;
        pl->A_uniform = (pl->A_uniform == -1 || pl->A_uniform == ct.A) ? ct.A : 0;
        off += ct.size;
        soff += p->U * ct.L + 2 * ct.A;  // skew: the next block starts 16*A bytes further in the bank cycle
    }
    pl->h_entries = soff;
    // Lanes: clusters in order of decreasing A so every tile's lane group is A-aligned in its warp.
    int order[CDMIMO_MAX_CLUSTERS];
    for (int c = 0; c < p->C; ++c) order[c] = c;
    std::stable_sort(order, order + p->C, [&](int a, int b) { return pl->cl[a].A > pl->cl[b].A; });
    int lane = 0;
    for (int k = 0; k < p->C; ++k) {
        ClusterTile& ct = pl->cl[order[k]];
        ct.lane0 = lane;
        lane += p->n_sym * ct.A;
    }
    pl->n_lanes = lane;
    pl->n_tiles = p->C * p->n_sym;
    if (pl->n_lanes > kMaxThreads) return CDMIMO_ERR_UNSUPPORTED;
    // Warps: with four or more, a multiple of four with the tiles spread evenly over them, so that
    // each of the SM's four warp schedulers holds the same number of this CTA's warps and the CTA's
    // barriers do not wait on one overloaded scheduler (two 7-warp CTAs on one SM split 4/4/3/3 or
    // worse; two 8-warp CTAs split 4/4/4/4).
    {
        int Amax = 1;
        for (int c = 0; c < p->C; ++c) Amax = std::max(Amax, pl->cl[c].A);
        const int w_min = (pl->n_lanes + 31) / 32;
        pl->lpw = 32;
        if (w_min >= 4) {
            const int W = (w_min + 3) / 4 * 4;
            pl->lpw = ((pl->n_lanes + W - 1) / W + Amax - 1) / Amax * Amax;
        }
        pl->threads = std::max(64, (pl->n_lanes + pl->lpw - 1) / pl->lpw * 32);
    }

    const unsigned U = p->U, C = p->C;
    const unsigned xs = (unsigned)pl->n_tiles | 1u;
    pl->packed = (P == 16 && pl->n_lanes <= kMaxSpecializedThreads &&
                  (pl->A_uniform == 1 || pl->A_uniform == 2 || pl->A_uniform == 4)) ? 1 : 0;
    bool all_mult4 = true;
    for (int c = 0; c < p->C; ++c) all_mult4 = all_mult4 && (p->cluster_size[c] % 4 == 0);
    if (p->in_dtype == CDMIMO_C64) pl->bulk = (all_even && aligned(H, 16)) ? 1 : 0;
    else pl->bulk = (pl->packed && all_mult4 && aligned(H, 16)) ? 1 : 0;
    const unsigned hreg = align16((unsigned)pl->h_entries * 8u);
    unsigned o = hreg;
    // The packed kernels prefetch by bulk copy into a second buffer: the channel itself (c64), or two
    // 16-bit staging buffers of the raw rows (converted into the one channel buffer).  The
    // converting path stages into one buffer (both buffer indices alias it).
    if (pl->packed) {
        pl->off_H2 = 0u;
        pl->off_H3 = 0u;
        if (pl->bulk && p->in_dtype == CDMIMO_C64) {
            pl->off_H2 = o;
            o = align16(o + hreg);
        } else if (pl->bulk) {
            const unsigned sreg = align16(U * (unsigned)p->B * 4u);
            pl->off_H2 = o;
            o = align16(o + sreg);
            pl->off_H3 = o;
            o = align16(o + sreg);
        }
        pl->off_K = o;
        o = align16(o + U * xs * (detect ? 8u : 4u));
    }
    if (detect) {
        pl->off_X = o;
        o = align16(o + U * xs * 8u);
        pl->off_coef = o;
        o = align16(o + C * U * 8u);
        pl->off_lam = o;
        o = align16(o + C * 4u);
    } else {
        pl->off_coef = o;
        o = align16(o + C * U * 4u);
        pl->off_S = o;
        o = align16(o + (unsigned)p->n_sym * (U | 1u) * 8u);
    }
    pl->off_e = o;
    o = align16(o + C * U * 4u);
    pl->learned = learned ? 1 : 0;
    if (learned) {
        pl->off_mlp = o;
        o = align16(o + C * (unsigned)CDMIMO_MAX_HIDDEN * 4u);
    }
    pl->off_tab = o;
    o = align16(o + C * (unsigned)sizeof(ClusterTile));
    pl->off_bar = o;  // two mbarriers, then the two schedule hand-off slots
    o = align16(o + 32u);
    pl->smem_bytes = o;
    if ((int)pl->smem_bytes > device_smem_optin()) return CDMIMO_ERR_UNSUPPORTED;
    if (pl->packed && !detect && p->n_sym * p->U > kSPrefetch * pl->threads)
        pl->packed = 0;  // the packed precoder prefetches at most kSPrefetch entries of s per thread

    return CDMIMO_OK;
}

// Antennas per lane: 16 by default (two lanes per tile at B_c = 32), 8 for tiny clusters, 32 when
// 16 would need more threads than a CTA may have.
int plan_auto(const cdmimo_params* p, bool detect, const void* H, CdPlan* pl)
{
    int maxBc = 0;
    for (int c = 0; c < p->C; ++c) maxBc = std::max(maxBc, p->cluster_size[c]);
    const int first = maxBc <= 8 ? 8 : 16;
    int rc = CDMIMO_ERR_UNSUPPORTED;
    for (int P = first; P <= 32; P *= 2) {
        rc = build_plan(p, P, detect, H, pl);
        if (rc == CDMIMO_OK) return rc;
    }
    return rc;
}



// Gram-form plan: the packed plan's cluster tiles, channel buffers and staging, then the Gram
// regions (rows of G_c, energies, per-tile z / x or w, s).  UNSUPPORTED where the form does not
// apply; with auto_rules also where a cluster has B_c < 2U (conditioning) or where the form would
// need as many complex MACs as the residual form.
int build_gram_plan(const cdmimo_params* p, bool detect, const void* H, bool auto_rules, CdPlan* pl,
                    bool frame = false)
{
    if (p->U > 16 || (frame && p->learned)) return CDMIMO_ERR_UNSUPPORTED;
    if (int rc = build_plan(p, 16, detect, H, pl)) return rc;
    if (!pl->packed) return CDMIMO_ERR_UNSUPPORTED;
    const long U = p->U, n_sym = p->n_sym, K = p->K;
    if (auto_rules) {
        long gram = 0, resid = 0;  // complex MACs per subcarrier
        for (int c = 0; c < p->C; ++c) {
            const long Bc = p->cluster_size[c];
            if (Bc < 2 * U) return CDMIMO_ERR_UNSUPPORTED;
            gram += U * U * Bc + n_sym * U * Bc + n_sym * K * U * U;
            resid += 2 * n_sym * K * U * Bc;
        }
        if (gram >= resid) return CDMIMO_ERR_UNSUPPORTED;
    }
    const int UT = p->U <= 8 ? 8 : 16;
    const int AT = pl->A_uniform;
    // frame: phase A runs symbol pairs and Gram column pairs on disjoint warps; phase B one lane per
    // (cluster, symbol); separate kernels: one phase after the other on the same warps
    const int threads = frame ? std::max(gram_phase_threads(p->C, (p->n_sym + 1) / 2, AT) +
                                             gram_phase_threads(p->C, (p->U + 1) / 2, AT),
                                         gram_phase_threads(p->C, 2 * p->n_sym, 1))
                              : std::max({gram_phase_threads(p->C, p->n_sym, AT), gram_phase_threads(p->C, p->U, AT),
                                          gram_phase_threads(p->C, p->n_sym, 1)});
    if (threads > kMaxSpecializedThreads) return CDMIMO_ERR_UNSUPPORTED;
    if (!detect && p->n_sym * p->U > kSPrefetch * threads) return CDMIMO_ERR_UNSUPPORTED;
    const unsigned C = p->C, xs = (unsigned)pl->n_tiles | 1u, UTu = (unsigned)UT;
    unsigned o = pl->off_K;  // end of the channel buffers / staging of the packed layout
    pl->off_G = o;
    o = align16(o + C * UTu * UTu * 8u);
    pl->off_E = o;
    o = align16(o + C * UTu * 4u);
    pl->off_X = o;  // z / x (uplink) or w (downlink) per tile; UT rows (padded steps read z rows >= U)
    o = align16(o + UTu * xs * 8u);
    if (!detect) {  // s rows, plus UT zero entries past the last row for the padded steps
        pl->off_S = o;
        o = align16(o + ((unsigned)n_sym * ((unsigned)U | 1u) + UTu) * 8u);
    }
    if (frame) {  // the downlink's w per tile, p_u^2, and the subcarrier's s [n_sym][U]
        pl->off_W = o;
        o = align16(o + (unsigned)U * xs * 8u);
        pl->off_E2 = o;
        o = align16(o + C * UTu * 4u);
        pl->off_S = o;
        o = align16(o + (unsigned)n_sym * (unsigned)U * 8u);
    }
    if (pl->learned) {  // ||h_u||^2 per cluster, and the learned fusion's hidden activations
        pl->off_E2 = o;
        o = align16(o + C * UTu * 4u);
        pl->off_mlp = o;
        o = align16(o + C * (unsigned)CDMIMO_MAX_HIDDEN * 4u);
    }
    pl->off_lam = o;
    o = align16(o + C * 4u);
    pl->off_tab = o;
    o = align16(o + C * (unsigned)sizeof(ClusterTile));
    pl->off_bar = o;
    o = align16(o + 32u);
    pl->smem_bytes = o;
    if ((int)pl->smem_bytes > device_smem_optin()) return CDMIMO_ERR_UNSUPPORTED;
    pl->gram = 1;
    pl->UT = UT;
    pl->threads = threads;
    return CDMIMO_OK;
}

// Shared memory per CTA that still lets two CTAs of the tensor-core kernel share an SM (228 KB per
// SM, 1 KB reserved per CTA).
constexpr unsigned kTcTwoCtaSmem = (228u * 1024u - 2u * 1024u) / 2u;

// GRAM and GRAM_TC ask for the Gram form (UNSUPPORTED where it does not apply).
bool is_forced_gram(const cdmimo_params* p)
{
    return p->form == CDMIMO_FORM_GRAM || p->form == CDMIMO_FORM_GRAM_TC || p->form == CDMIMO_FORM_GRAM_TC_PHASED ||
           p->form == CDMIMO_FORM_GRAM_TC_UMMA;
}

// Tensor-core plan (any mode of cd_frame_tc_kernel): the Gram frame plan's cluster table and
// tiling, with the kernel's layout: two channel buffers of C x 16 rows of 2 B_c + 8 floats, the
// Gram rows (later w per tile), m_u and p_u^2, z / x per tile, s.  UNSUPPORTED unless the shape is
// the kernel's (c64 or 16-bit storage by bulk copy, every B_c = 16 or every B_c = 32, 8 < U <= 16,
// n_sym <= 16, 2 C n_sym <= 256; a learned block only for op DETECT with c64) and, for AUTO, the Gram
// form's own rules hold.  p->form must be AUTO or GRAM_TC.
int build_tc_plan(const cdmimo_params* p, const void* H, int op, CdPlan* pl)
{
    if (p->form != CDMIMO_FORM_AUTO && p->form != CDMIMO_FORM_GRAM_TC && p->form != CDMIMO_FORM_GRAM_TC_PHASED &&
        p->form != CDMIMO_FORM_GRAM_TC_UMMA)
        return CDMIMO_ERR_UNSUPPORTED;
    if (p->in_dtype != CDMIMO_C64 && p->learned) return CDMIMO_ERR_UNSUPPORTED;
    if (op != CDMIMO_OP_DETECT && (p->learned || p->fuse == CDMIMO_FUSE_LEARNED)) return CDMIMO_ERR_UNSUPPORTED;
    if (p->U <= 8 || p->U > 16 || p->n_sym > 16 || 2 * p->C * p->n_sym > 256) return CDMIMO_ERR_UNSUPPORTED;
    if (int rc = build_gram_plan(p, true, H, p->form == CDMIMO_FORM_AUTO, pl, op == CDMIMO_OP_FRAME)) return rc;
    const int Bc = p->cluster_size[0];
    if (!pl->bulk || (Bc != 16 && Bc != 32) || pl->A_uniform != Bc / 16) return CDMIMO_ERR_UNSUPPORTED;
    for (int c = 0; c < p->C; ++c)
        if (p->cluster_size[c] != Bc) return CDMIMO_ERR_UNSUPPORTED;
    const unsigned C = p->C, U = p->U, UT = 16, xs = tc_x_stride(pl->n_tiles), n_sym = p->n_sym;
    const unsigned hbytes = align16(C * UT * tc_row_words(Bc, p->in_dtype) * 4u);
    unsigned o = 2u * hbytes;
    pl->off_H2 = hbytes;
    pl->off_H3 = 0u;
    pl->off_G = o;  // Gram rows, then (after the sweeps) w per tile
    o = align16(o + std::max(C * UT * UT * 8u, U * xs * 8u));
    pl->off_E = o;
    o = align16(o + C * UT * 4u);
    pl->off_E2 = o;
    o = align16(o + C * UT * 4u);
    pl->off_X = o;
    o = align16(o + UT * xs * 8u);
    pl->off_W = pl->off_G;
    pl->off_S = o;
    o = align16(o + n_sym * U * 8u);
    if (pl->learned) {  // the learned fusion's logits, and the learned sweep coefficients [C][K][16]
        pl->off_mlp = o;
        o = align16(o + C * 4u);
        pl->off_K = o;
        o = align16(o + C * (unsigned)p->K * UT * 8u);
    }
    pl->off_lam = o;
    o = align16(o + C * 4u);
    pl->off_tab = o;
    o = align16(o + C * (unsigned)sizeof(ClusterTile));
    pl->off_bar = o;
    o = align16(o + 32u);
    pl->smem_bytes = o;
    if ((int)pl->smem_bytes > device_smem_optin()) return CDMIMO_ERR_UNSUPPORTED;
    if (pl->learned && pl->smem_bytes > kTcTwoCtaSmem) return CDMIMO_ERR_UNSUPPORTED;  // long learned schedules
    pl->threads = 256;
    pl->UT = 16;
    pl->phased = p->form == CDMIMO_FORM_GRAM_TC_PHASED;
    pl->umma = p->form == CDMIMO_FORM_GRAM_TC_UMMA;
    return CDMIMO_OK;
}

// Tensor-core plan for 16 < U <= 32 users (cd_detect_tc32_kernel, detection only): every B_c = 16,
// 32 or 64, n_sym <= 16, no learned block, H 16-byte aligned with rows of a multiple of 16 bytes
// (whole-row bulk copies), and a layout that fits shared memory.  With AUTO it also needs
// U <= 2 B_c (the sweeps' FP32 work, K U^2 complex MACs per cluster and vector, at most the residual
// form's 2 K U B_c) and, where B_c < 2U, K <= 8: with few sweeps the Gram-form iterate stays within
// FP32 rounding of the algorithm's even when G_c + (N0/Ex) I is poorly conditioned (an emulation of
// the split-TF32 Gram form gave 6e-7 relative at U = B_c = 32 and 64, K = 5).
int build_tc32_plan(const cdmimo_params* p, const void* H, CdPlan* pl)
{
    if (p->form != CDMIMO_FORM_AUTO && p->form != CDMIMO_FORM_GRAM_TC) return CDMIMO_ERR_UNSUPPORTED;
    if (p->U <= 16 || p->U > 32 || p->n_sym > 16 || p->learned || p->fuse == CDMIMO_FUSE_LEARNED)
        return CDMIMO_ERR_UNSUPPORTED;
    if (p->C > 8 * (32 / (p->n_sym <= 8 ? 8 : 16))) return CDMIMO_ERR_UNSUPPORTED;  // sweep lanes: 8 warps
    const int Bc = p->cluster_size[0];
    if (Bc != 16 && Bc != 32 && Bc != 64) return CDMIMO_ERR_UNSUPPORTED;
    for (int c = 0; c < p->C; ++c)
        if (p->cluster_size[c] != Bc) return CDMIMO_ERR_UNSUPPORTED;
    if (!aligned(H, 16) || ((size_t)p->B * elem_bytes(p->in_dtype)) % 16 != 0) return CDMIMO_ERR_UNSUPPORTED;
    if (p->form == CDMIMO_FORM_AUTO && (p->U > 2 * Bc || (Bc < 2 * p->U && p->K > 8))) return CDMIMO_ERR_UNSUPPORTED;
    std::memset(pl, 0, sizeof(*pl));
    pl->n_sc = p->n_sc;
    pl->n_sym = p->n_sym;
    pl->B = p->B;
    pl->U = p->U;
    pl->C = p->C;
    pl->K = p->K;
    pl->fuse = p->fuse;
    pl->inv_Ex = 1.f / p->Ex;
    pl->rho_c = (float)(p->rho / std::sqrt((double)p->C));
    for (int c = 0; c < p->C; ++c) {
        pl->cl[c].off = c * Bc;
        pl->cl[c].size = Bc;
    }
    pl->n_tiles = p->C * p->n_sym;
    pl->bulk = 1;
    pl->gram = 1;
    pl->UT = 32;
    pl->threads = 256;
    return tc32_layout_fits(*pl, p->in_dtype);
}

// The plan for p->form: GRAM where requested, or (AUTO) where the Gram form applies and pays,
// else the residual form.
int plan_for(const cdmimo_params* p, bool detect, const void* H, CdPlan* pl)
{
    if (p->form != CDMIMO_FORM_RESIDUAL) {
        const int rc = build_gram_plan(p, detect, H, p->form == CDMIMO_FORM_AUTO, pl);
        if (rc == CDMIMO_OK || is_forced_gram(p)) return rc;
    }
    return plan_auto(p, detect, H, pl);
}

template <int P, int IN, int AT>
int launch_detect_t(const CdPlan& pl, const DetectIO& io, cudaStream_t s)
{
    void (*k)(const CdPlan, const DetectIO);
    if constexpr (AT > 0) {
        if constexpr (IN == CDMIMO_C64) k = pl.learned ? cd_detect_pp_kernel<IN, AT, true> : cd_detect_pp_kernel<IN, AT, false>;
        else k = cd_detect_pp_kernel<IN, AT, false>;
    } else {
        k = cd_detect_kernel<P, IN, 0>;
    }
    if (int rc = launch_cd(k, pl)) return rc;
    k<<<grid_for(k, pl), threads_for(pl), pl.smem_bytes, s>>>(pl, io);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

template <int P, int IN, int AT>
int launch_precode_t(const CdPlan& pl, const PrecodeIO& io, cudaStream_t s)
{
    void (*k)(const CdPlan, const PrecodeIO);
    if constexpr (AT > 0) k = cd_precode_pp_kernel<IN, AT>;
    else k = cd_precode_kernel<P, IN, 0>;
    if (int rc = launch_cd(k, pl)) return rc;
    k<<<grid_for(k, pl), threads_for(pl), pl.smem_bytes, s>>>(pl, io);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

// Kernel variant: packed-FP32 kernels with compile-time lanes per tile for uniform partitions at
// P = 16 (B_c in (8, 64]), scalar kernels with run-time lanes per tile otherwise.
template <int IN>
int dispatch_detect(const CdPlan& pl, const DetectIO& io, cudaStream_t s)
{
    if (pl.gram) return dispatch_detect_gram(IN, pl, io, s);
    if (pl.packed) {
        switch (pl.A_uniform) {
        case 1: return launch_detect_t<16, IN, 1>(pl, io, s);
        case 2: return launch_detect_t<16, IN, 2>(pl, io, s);
        case 4: return launch_detect_t<16, IN, 4>(pl, io, s);
        }
    }
    switch (pl.P) {
    case 8: return launch_detect_t<8, IN, 0>(pl, io, s);
    case 16: return launch_detect_t<16, IN, 0>(pl, io, s);
    case 32: return launch_detect_t<32, IN, 0>(pl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

template <int IN>
int dispatch_precode(const CdPlan& pl, const PrecodeIO& io, cudaStream_t s)
{
    if (pl.gram) return dispatch_precode_gram(IN, pl, io, s);
    if (pl.packed) {
        switch (pl.A_uniform) {
        case 1: return launch_precode_t<16, IN, 1>(pl, io, s);
        case 2: return launch_precode_t<16, IN, 2>(pl, io, s);
        case 4: return launch_precode_t<16, IN, 4>(pl, io, s);
        }
    }
    switch (pl.P) {
    case 8: return launch_precode_t<8, IN, 0>(pl, io, s);
    case 16: return launch_precode_t<16, IN, 0>(pl, io, s);
    case 32: return launch_precode_t<32, IN, 0>(pl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

int check_detect_ptrs(const cdmimo_params* p, const void* H, const void* Y, const float* N0, const void* Xhat)
{
    if (p->n_sc == 0) return CDMIMO_OK;
    if (!H || !Y || !N0 || !Xhat) return CDMIMO_ERR_INVALID_ARG;
    const size_t ea = p->in_dtype == CDMIMO_C64 ? 8 : 4;
    if (!aligned(H, ea) || !aligned(Y, ea) || !aligned(N0, 4) || !aligned(Xhat, 8)) return CDMIMO_ERR_INVALID_ARG;
    if (p->in_dtype != CDMIMO_C64 && (!p->h_scale || !p->y_scale)) return CDMIMO_ERR_INVALID_ARG;
    return CDMIMO_OK;
}

// Cluster-group streaming for shapes the whole-channel kernels cannot hold (defined further down).
int streaming_launch(const cdmimo_params* p, int op, const void* H, const void* V, const float* N0, void* out,
                     cudaStream_t s);

int detect_impl(const cdmimo_params* p, const void* H, const void* Y, const float* N0, void* Xhat, void* Xc,
                float* lam, unsigned* sched, cudaStream_t s)
{
    if (int rc = validate(p)) return rc;
    if (int rc = check_detect_ptrs(p, H, Y, N0, Xhat)) return rc;
    if ((Xc && !aligned(Xc, 8)) || (lam && !aligned(lam, 4))) return CDMIMO_ERR_INVALID_ARG;
    if (p->fuse == CDMIMO_FUSE_LEARNED && !p->learned) return CDMIMO_ERR_INVALID_ARG;
    if (p->learned && (p->in_dtype != CDMIMO_C64 || p->K < 1 || p->K > CDMIMO_MAX_LEARNED_SWEEPS ||
                       !aligned(p->learned, 16)))
        return p->in_dtype != CDMIMO_C64 ? CDMIMO_ERR_UNSUPPORTED : CDMIMO_ERR_INVALID_ARG;
    if (p->n_sc == 0) return CDMIMO_OK;
    CdPlan pl;
    if ((!p->learned || (!Xc && !lam)) && build_tc_plan(p, H, CDMIMO_OP_DETECT, &pl) == CDMIMO_OK) {
        const FusedIO io{{H, Y, N0, p->h_scale, p->y_scale, reinterpret_cast<float2*>(Xhat),
                          reinterpret_cast<float2*>(Xc), lam, p->learned, sched},
                         nullptr, nullptr};
        return dispatch_frame_tc(p->in_dtype, pl, io, CDMIMO_OP_DETECT, s);
    }
    if (build_tc32_plan(p, H, &pl) == CDMIMO_OK) {
        const DetectIO io{H, Y, N0, p->h_scale, p->y_scale, reinterpret_cast<float2*>(Xhat),
                          reinterpret_cast<float2*>(Xc), lam, nullptr, sched};
        const int rc = dispatch_detect_tc32(p->in_dtype, pl, io, s);
        if (rc != CDMIMO_ERR_UNSUPPORTED) return rc;
    }
    if (int rc = plan_for(p, true, H, &pl)) {
        if (rc != CDMIMO_ERR_UNSUPPORTED || Xc || lam || is_forced_gram(p)) return rc;
        return streaming_launch(p, CDMIMO_OP_DETECT, H, Y, N0, Xhat, s);
    }
    if (pl.learned && !pl.packed) return CDMIMO_ERR_UNSUPPORTED;  // learned sweeps: uniform B_c <= 64
    DetectIO io{H, Y, N0, p->h_scale, p->y_scale, reinterpret_cast<float2*>(Xhat), reinterpret_cast<float2*>(Xc),
                lam, p->learned, sched};
    switch (p->in_dtype) {
    case CDMIMO_C64: return dispatch_detect<CDMIMO_C64>(pl, io, s);
    case CDMIMO_C16F: return dispatch_detect<CDMIMO_C16F>(pl, io, s);
    case CDMIMO_C16BF: return dispatch_detect<CDMIMO_C16BF>(pl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int precode_impl(const cdmimo_params* p, const void* H, const void* S, void* Xdl, unsigned* sched, cudaStream_t s)
{
    if (int rc = validate(p)) return rc;
    if (p->n_sc == 0) return CDMIMO_OK;
    if (!H || !S || !Xdl) return CDMIMO_ERR_INVALID_ARG;
    const size_t ea = p->in_dtype == CDMIMO_C64 ? 8 : 4;
    if (!aligned(H, ea) || !aligned(S, 8) || !aligned(Xdl, 8)) return CDMIMO_ERR_INVALID_ARG;
    CdPlan pl;
    if (build_tc_plan(p, H, CDMIMO_OP_PRECODE, &pl) == CDMIMO_OK) {
        const FusedIO io{{H, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, sched},
                         reinterpret_cast<const float2*>(S), reinterpret_cast<float2*>(Xdl)};
        return dispatch_frame_tc(p->in_dtype, pl, io, CDMIMO_OP_PRECODE, s);
    }
    if (int rc = plan_for(p, false, H, &pl)) {
        if (rc != CDMIMO_ERR_UNSUPPORTED || is_forced_gram(p)) return rc;
        return streaming_launch(p, CDMIMO_OP_PRECODE, H, S, nullptr, Xdl, s);
    }
    PrecodeIO io{H, reinterpret_cast<const float2*>(S), reinterpret_cast<float2*>(Xdl), sched};
    switch (p->in_dtype) {
    case CDMIMO_C64: return dispatch_precode<CDMIMO_C64>(pl, io, s);
    case CDMIMO_C16F: return dispatch_precode<CDMIMO_C16F>(pl, io, s);
    case CDMIMO_C16BF: return dispatch_precode<CDMIMO_C16BF>(pl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

// Bytes of the optional device workspace of cdmimo_detect / cdmimo_precode: the three schedule
// counters, padded to one 256-byte line.
constexpr size_t kSchedBytes = 256;
constexpr int kHostFrameChunks = 5;  // default chunks of the pipelined host-buffer frame

// The schedule counters in a caller's workspace: NULL -> static schedule; else it must be 16-byte
// aligned and hold kSchedBytes.
int sched_from_workspace(void* ws, size_t ws_bytes, unsigned** sched)
{
    *sched = nullptr;
    if (!ws) return CDMIMO_OK;
    if (!aligned(ws, 16) || ws_bytes < kSchedBytes) return CDMIMO_ERR_WORKSPACE;
    *sched = static_cast<unsigned*>(ws);
    return CDMIMO_OK;
}

}  // namespace

namespace {

// Plan and shared-memory layout of the learned gradient kernel (generic tiling, converting staging).
int grad_plan(const cdmimo_params* p, int hidden, CdPlan* pl, GradLayout* gl)
{
    if (int rc = validate(p)) return rc;
    if (p->in_dtype != CDMIMO_C64 || !cdmimo_learned_param_count(p->K, p->U, hidden)) return CDMIMO_ERR_INVALID_ARG;
    cdmimo_params q = *p;
    q.learned = nullptr;
    if (int rc = plan_auto(&q, true, nullptr, pl)) return rc;
    pl->bulk = 0;
    pl->packed = 0;
    const unsigned U = p->U, C = p->C, K = p->K, T = (unsigned)pl->n_tiles, xs = T | 1u;
    gl->K = p->K;
    gl->Hd = hidden;
    gl->F = p->U + 1;
    gl->n_params = (int)cdmimo_learned_param_count(p->K, p->U, hidden);
    gl->ws_stride = (gl->n_params + 1 + 3) & ~3;
    gl->inv_nvec = 1.f / ((float)p->n_sc * (float)p->n_sym);
    unsigned o = align16((unsigned)pl->h_entries * 8u);
    gl->off_e = o;      o = align16(o + U * C * 4u);
    gl->off_cf = o;     o = align16(o + K * U * C * 8u);
    gl->off_save = o;   o = align16(o + K * U * T * 16u);
    gl->off_X = o;      o = align16(o + U * xs * 8u);
    gl->off_Xb = o;     o = align16(o + U * xs * 8u);
    gl->off_Ab = o;     o = align16(o + K * U * T * 8u);
    gl->off_phi = o;    o = align16(o + C * (U + 1) * 4u);
    gl->off_z = o;      o = align16(o + C * (unsigned)hidden * 4u);
    gl->off_zb = o;     o = align16(o + C * (unsigned)hidden * 4u);
    gl->off_lam = o;    o = align16(o + C * 4u);
    gl->off_lamb = o;   o = align16(o + C * 4u);
    gl->off_lgb = o;    o = align16(o + C * 4u);
    gl->off_gx = o;     o = align16(o + (unsigned)p->n_sym * U * 8u);
    gl->off_tg = o;     o = align16(o + K * C * 8u);
    gl->off_red = o;    o = align16(o + 32u * 4u);
    gl->off_tab = o;    o = align16(o + C * (unsigned)sizeof(ClusterTile));
    gl->smem_bytes = o;
    if ((int)o > device_smem_optin()) return CDMIMO_ERR_UNSUPPORTED;
    return CDMIMO_OK;
}

template <int P>
int launch_grad_t(const CdPlan& pl, const GradLayout& gl, const GradIO& io, cudaStream_t s)
{
    auto k = learned_grad_kernel<P>;
    if (gl.smem_bytes > 48u * 1024u &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gl.smem_bytes) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    k<<<pl.n_sc, threads_for(pl), gl.smem_bytes, s>>>(pl, gl, io);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

}  // namespace

// Scratch of cdmimo_learned_grad_noalloc: a fixed device array owned by the library, for callers
// that cannot allocate device memory.  Host code only ever sees its address through
// cudaGetSymbolAddress (the symbol itself is a host-side stand-in); the address is looked up on every
// call, for the current device and context, so it stays valid across a device or context reset
// (which reloads the module) and needs no shared cache between host threads.
static __device__ __align__(256) float g_noalloc_scratch[CDMIMO_NOALLOC_SCRATCH_BYTES / sizeof(float)];

namespace {

float* noalloc_scratch_address()
{
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return nullptr;
    return static_cast<float*>(ptr);
}

}  // namespace

namespace {

// Host-side split of a batch into cluster groups, and the kernel's shared-memory layout.
struct BatchBuild {
    std::vector<BatchDesc> descs;
    std::vector<BatchGroup> groups;
    std::vector<BatchCluster> clusters;
    BatchLaunch bl{};
};

int batch_split(const cdmimo_batch_desc* d, int n_desc, cdmimo_batch_plan* plan, BatchBuild* bb)
{
    if (!d || n_desc < 1 || !plan) return CDMIMO_ERR_INVALID_ARG;
    const int P = plan->P, T = plan->threads;
    if ((P != 8 && P != 16 && P != 32) || T < 64 || T > (P == 8 ? 384 : 512) || (T & 31) ||
        plan->group_bytes < 4096 || plan->ctas_per_sm < 0)
        return CDMIMO_ERR_INVALID_ARG;
    unsigned h_max = 0, x_max = 0, uc_max = 0, acc_max = 0, s_max = 0;
    int C_max = 1, items = 0;
    // Descriptors enter the table in order of decreasing work per item (K U n_sym B, stable), so the
    // persistent CTAs pop the longest items first and the short ones fill the tail.
    std::vector<int> ord(n_desc);
    for (int i = 0; i < n_desc; ++i) ord[i] = i;
    auto work = [&](int i) { return (double)d[i].K * d[i].U * d[i].n_sym * d[i].B; };
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return work(a) > work(b); });
    for (int oi = 0; oi < n_desc; ++oi) {
        const cdmimo_batch_desc& q = d[ord[oi]];
        if (q.op != CDMIMO_OP_DETECT && q.op != CDMIMO_OP_PRECODE) return CDMIMO_ERR_INVALID_ARG;
        if (q.n_sc < 0 || q.n_sym < 1 || q.B < 1 || q.U < 1 || q.C < 1 || q.K < 0) return CDMIMO_ERR_INVALID_ARG;
        if (q.U > CDMIMO_MAX_USERS) return CDMIMO_ERR_UNSUPPORTED;
        if (!q.cluster_size || q.C > CDMIMO_MAX_CLUSTERS) return CDMIMO_ERR_BAD_PARTITION;
        if (q.op == CDMIMO_OP_DETECT && (!(q.Ex > 0.f) || (q.fuse != CDMIMO_FUSE_EQUAL && q.fuse != CDMIMO_FUSE_COLNORM)))
            return CDMIMO_ERR_INVALID_ARG;
        if (q.n_sc > 0 && (!q.H || !q.V || !q.out || (q.op == CDMIMO_OP_DETECT && !q.N0)))
            return CDMIMO_ERR_INVALID_ARG;
        if (!aligned(q.H, 8) || !aligned(q.V, 8) || !aligned(q.out, 8)) return CDMIMO_ERR_INVALID_ARG;
        long sum = 0;
        bool all_even = (q.B % 2) == 0;
        for (int c = 0; c < q.C; ++c) {
            if (q.cluster_size[c] < 1) return CDMIMO_ERR_BAD_PARTITION;
            sum += q.cluster_size[c];
            if (q.cluster_size[c] & 1) all_even = false;
        }
        if (sum != q.B) return CDMIMO_ERR_BAD_PARTITION;
        BatchDesc bd{};
        bd.H = q.H;
        bd.V = q.V;
        bd.N0 = q.N0;
        bd.out = q.out;
        bd.op = q.op;
        bd.n_sc = q.n_sc;
        bd.n_sym = q.n_sym;
        bd.B = q.B;
        bd.U = q.U;
        bd.C = q.C;
        bd.K = q.K;
        bd.fuse = q.fuse;
        bd.inv_Ex = q.op == CDMIMO_OP_DETECT ? 1.f / q.Ex : 0.f;
        bd.rho_c = (float)(q.rho / std::sqrt((double)q.C));
        bd.item0 = items;
        bd.group0 = (int)bb->groups.size();
        bd.bulk = (all_even && aligned(q.H, 16)) ? 1 : 0;
        items += q.n_sc;
        const unsigned U = q.U, ns = q.n_sym;
        // Greedy groups of consecutive clusters.  With P = 16 (8) a group whose clusters all have
        // A <= 8 (16) runs the packed-FP32 sweeps, which need every warp's active lanes to share one A: each
        // A class then starts at a warp boundary (the gaps are inactive lanes).
        auto lane_count = [&](const std::vector<BatchCluster>& cs_, bool align) {
            std::vector<int> as;
            for (const BatchCluster& x : cs_) as.push_back(x.A);
            std::stable_sort(as.begin(), as.end(), [](int a, int b) { return a > b; });
            unsigned l = 0;
            for (size_t k2 = 0; k2 < as.size(); ++k2) {
                if (align && k2 > 0 && as[k2] != as[k2 - 1]) l = (l + 31u) & ~31u;
                l += ns * (unsigned)as[k2];
            }
            return l;
        };
        int off = 0, c = 0;
        while (c < q.C) {
            BatchGroup g{};
            g.c0 = c;
            g.cl0 = (int)bb->clusters.size();
            unsigned h = 0, tiles = 0, rowb = 0;
            std::vector<BatchCluster> cur;
            while (c < q.C) {
                BatchCluster bc{};
                bc.off = off;
                bc.size = q.cluster_size[c];
                bc.A = pow2ceil((bc.size + P - 1) / P);
                if (bc.A > 32) return CDMIMO_ERR_UNSUPPORTED;
                bc.L = bc.A * P;
                const unsigned h2 = h + U * (unsigned)bc.L + 2u * (unsigned)bc.A;
                std::vector<BatchCluster> trial = cur;
                trial.push_back(bc);
                bool pk = P == 16 || P == 8;
                for (const BatchCluster& x : trial) pk = pk && x.A <= 128 / P;
                const unsigned t2 = tiles + ns, l2 = lane_count(trial, pk), cg2 = (unsigned)cur.size() + 1;
                const unsigned bytes = h2 * 8u + U * (t2 | 1u) * 8u + U * cg2 * 12u;
                if (bytes > (unsigned)plan->group_bytes || l2 > (unsigned)T || cg2 > 64u) {
                    if (cur.empty()) return CDMIMO_ERR_UNSUPPORTED;
                    break;
                }
                bc.soff = (int)h;
                h = h2;
                tiles = t2;
                rowb += U * (unsigned)bc.size * 8u;
                if (bc.L != bc.size) g.padded = 1;
                cur.push_back(bc);
                off += bc.size;
                ++c;
            }
            // Lanes: clusters of the group in order of decreasing A (A-aligned lane groups; packed
            // groups start each A class at a warp boundary).
            bool pk = P == 16 || P == 8;
            for (const BatchCluster& x : cur) pk = pk && x.A <= 128 / P;
            g.packed = pk ? 1 : 0;
            std::vector<int> order(cur.size());
            for (size_t k2 = 0; k2 < cur.size(); ++k2) order[k2] = (int)k2;
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cur[a].A > cur[b].A; });
            int lane = 0, prevA = 0;
            for (int k2 : order) {
                if (pk && prevA && cur[k2].A != prevA) lane = (lane + 31) & ~31;
                prevA = cur[k2].A;
                cur[k2].lane0 = lane;
                lane += (int)ns * cur[k2].A;
            }
            g.c1 = c;
            g.n_lanes = lane;
            g.h_entries = (int)h;
            g.row_bytes = (int)rowb;
            for (const BatchCluster& bc : cur) bb->clusters.push_back(bc);
            bb->groups.push_back(g);
            const unsigned Cg = (unsigned)cur.size();
            h_max = std::max(h_max, h);
            x_max = std::max(x_max, U * (tiles | 1u));
            uc_max = std::max(uc_max, U * Cg);
            C_max = std::max(C_max, (int)Cg);
        }
        bd.n_groups = (int)bb->groups.size() - bd.group0;
        if (q.op == CDMIMO_OP_DETECT) acc_max = std::max(acc_max, 2u * ns * U);
        else s_max = std::max(s_max, ns * (U | 1u));
        bb->descs.push_back(bd);
    }
    BatchLaunch& bl = bb->bl;
    bl.P = P;
    bl.C_max = C_max;
    unsigned o = align16(h_max * 8u);
    bl.off_X = o;    o = align16(o + x_max * 8u);
    bl.off_coef = o; o = align16(o + uc_max * 8u);
    bl.off_e = o;    o = align16(o + uc_max * 4u);
    bl.off_acc = o;  o = align16(o + acc_max * 8u);
    bl.off_w = o;    o = align16(o + (unsigned)(C_max + 1) * 4u);
    bl.off_S = o;    o = align16(o + s_max * 8u);
    bl.off_tab = o;  o = align16(o + (unsigned)C_max * (unsigned)sizeof(ClusterTile));
    bl.off_bar = o;  o = align16(o + 8u);
    bl.off_item = o; o = align16(o + 4u);
    bl.smem_bytes = o;
    plan->n_items = items;
    plan->n_groups = (int)bb->groups.size();
    plan->C_max = C_max;
    plan->smem_bytes = o;
    const unsigned offs[9] = {bl.off_X, bl.off_coef, bl.off_e, bl.off_acc, bl.off_w, bl.off_S, bl.off_tab, bl.off_bar, bl.off_item};
    for (int i = 0; i < 9; ++i) plan->offsets[i] = offs[i];
    const size_t hb = (sizeof(BatchTableHeader) + 15) & ~(size_t)15;
    const size_t db = (bb->descs.size() * sizeof(BatchDesc) + 15) & ~(size_t)15;
    const size_t gb = (bb->groups.size() * sizeof(BatchGroup) + 15) & ~(size_t)15;
    const size_t cb = (bb->clusters.size() * sizeof(BatchCluster) + 15) & ~(size_t)15;
    plan->table_bytes = hb + db + gb + cb;
    return CDMIMO_OK;
}

BatchLaunch launch_from_plan(const cdmimo_batch_plan* plan)
{
    BatchLaunch bl{};
    bl.P = plan->P;
    bl.C_max = plan->C_max;
    bl.off_X = plan->offsets[0];
    bl.off_coef = plan->offsets[1];
    bl.off_e = plan->offsets[2];
    bl.off_acc = plan->offsets[3];
    bl.off_w = plan->offsets[4];
    bl.off_S = plan->offsets[5];
    bl.off_tab = plan->offsets[6];
    bl.off_bar = plan->offsets[7];
    bl.off_item = plan->offsets[8];
    bl.smem_bytes = plan->smem_bytes;
    return bl;
}

template <int P>
int launch_batched_t(const cdmimo_batch_plan* plan, const void* table, int* counter, unsigned long long* stats,
                     cudaStream_t s)
{
    auto k = cd_batched_kernel<P>;
    const BatchLaunch bl = launch_from_plan(plan);
    if ((int)bl.smem_bytes > device_smem_optin()) return CDMIMO_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    if (bl.smem_bytes > 48u * 1024u &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bl.smem_bytes) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, plan->threads, bl.smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return CDMIMO_ERR_UNSUPPORTED;
    if (plan->ctas_per_sm > 0) per_sm = std::min(per_sm, plan->ctas_per_sm);
    const int grid = std::max(1, std::min(plan->n_items, sms * per_sm));
    if (cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    if (stats && (cudaMemsetAsync(stats, 0xff, sizeof(unsigned long long), s) != cudaSuccess ||
                  cudaMemsetAsync(stats + 1, 0, 3 * sizeof(unsigned long long), s) != cudaSuccess))
        return CDMIMO_ERR_CUDA;
    k<<<grid, plan->threads, bl.smem_bytes, s>>>(static_cast<const unsigned char*>(table), bl, counter, stats);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

}  // namespace

namespace {

// cdmimo_detect / cdmimo_precode for shapes whose whole channel does not fit in shared memory (or
// needs more than 512 lanes): the batched kernel's cluster-group streaming, one CTA per subcarrier,
// with the one-descriptor table passed by value.  c64 storage, EQUAL or COLNORM fusion, and no
// per-cluster outputs.
template <int P>
int launch_streaming_t(const SingleTable& t, const cdmimo_batch_plan& plan, cudaStream_t s)
{
    auto k = cd_streaming_kernel<P>;
    const BatchLaunch bl = launch_from_plan(&plan);
    if ((int)bl.smem_bytes > device_smem_optin()) return CDMIMO_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    if (bl.smem_bytes > 48u * 1024u &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bl.smem_bytes) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    k<<<plan.n_items, plan.threads, bl.smem_bytes, s>>>(t, bl);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

int streaming_launch(const cdmimo_params* p, int op, const void* H, const void* V, const float* N0, void* out,
                     cudaStream_t s)
{
    if (p->in_dtype != CDMIMO_C64 || p->learned || (op == CDMIMO_OP_DETECT && p->fuse == CDMIMO_FUSE_LEARNED))
        return CDMIMO_ERR_UNSUPPORTED;
    cdmimo_batch_desc d{};
    d.op = op;
    d.n_sc = p->n_sc;
    d.n_sym = p->n_sym;
    d.B = p->B;
    d.U = p->U;
    d.C = p->C;
    d.K = p->K;
    d.fuse = p->fuse;
    d.Ex = p->Ex;
    d.rho = p->rho;
    d.cluster_size = p->cluster_size;
    d.H = H;
    d.V = V;
    d.N0 = N0;
    d.out = out;
    const int budget = std::min(device_smem_optin() - 16 * 1024, 160 * 1024);
    int rc = CDMIMO_ERR_UNSUPPORTED;
    for (int P = 16; P <= 32; P *= 2) {
        cdmimo_batch_plan plan;
        cdmimo_batch_default_plan(&plan);
        plan.P = P;
        plan.threads = 512;
        plan.group_bytes = budget;
        BatchBuild bb;
        rc = batch_split(&d, 1, &plan, &bb);
        if (rc == CDMIMO_ERR_UNSUPPORTED) continue;
        if (rc) return rc;
        SingleTable t{};
        t.hdr.n_desc = 1;
        t.hdr.n_items = plan.n_items;
        t.hdr.n_groups = (int)bb.groups.size();
        t.hdr.n_clusters = (int)bb.clusters.size();
        t.hdr.off_desc = (unsigned)offsetof(SingleTable, desc);
        t.hdr.off_group = (unsigned)offsetof(SingleTable, groups);
        t.hdr.off_cluster = (unsigned)offsetof(SingleTable, clusters);
        t.hdr.total_bytes = (unsigned)sizeof(SingleTable);
        t.desc = bb.descs[0];
        std::memcpy(t.groups, bb.groups.data(), bb.groups.size() * sizeof(BatchGroup));
        std::memcpy(t.clusters, bb.clusters.data(), bb.clusters.size() * sizeof(BatchCluster));
        switch (P) {
        case 16: return launch_streaming_t<16>(t, plan, s);
        case 32: return launch_streaming_t<32>(t, plan, s);
        }
    }
    return rc;
}

}  // namespace

// One thread waits on an mbarrier that nothing completes, for at most limit_ns, and gives up the way
// every bounded wait of the kernels does (status bit CDMIMO_DEV_TIMEOUT); the kernel then returns.
__global__ void bounded_wait_check_kernel(unsigned long long limit_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_proxy_async_smem();
        mbar_wait_bounded(&bar, 0u, limit_ns);
    }
}

extern "C" {

int cdmimo_check_bounded_wait(unsigned timeout_us, void* stream)
{
    if (timeout_us < 1u || timeout_us > 2000000u) return CDMIMO_ERR_INVALID_ARG;
    bounded_wait_check_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(1000ull * timeout_us);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

int cdmimo_detect(const cdmimo_params* p, const void* H, const void* Y, const float* N0, void* Xhat, void* Xc_opt,
                  float* lambda_opt, void* workspace, size_t ws_bytes, void* stream)
{
    unsigned* sched;
    if (int rc = sched_from_workspace(workspace, ws_bytes, &sched)) return rc;
    return detect_impl(p, H, Y, N0, Xhat, Xc_opt, lambda_opt, sched, static_cast<cudaStream_t>(stream));
}

int cdmimo_precode(const cdmimo_params* p, const void* H, const void* S, void* Xdl, void* workspace, size_t ws_bytes,
                   void* stream)
{
    unsigned* sched;
    if (int rc = sched_from_workspace(workspace, ws_bytes, &sched)) return rc;
    return precode_impl(p, H, S, Xdl, sched, static_cast<cudaStream_t>(stream));
}

namespace {

int frame_impl(const cdmimo_params* p, const void* H, const void* Y, const float* N0, void* Xhat, const void* S,
               void* Xdl, unsigned* sched, cudaStream_t s)
{
    if (int rc = validate(p)) return rc;
    if (int rc = check_detect_ptrs(p, H, Y, N0, Xhat)) return rc;
    if (p->n_sc == 0) return CDMIMO_OK;
    if (!S || !Xdl || !aligned(S, 8) || !aligned(Xdl, 8)) return CDMIMO_ERR_INVALID_ARG;
    CdPlan pl;
    const FusedIO io{{H, Y, N0, p->h_scale, p->y_scale, reinterpret_cast<float2*>(Xhat), nullptr, nullptr, nullptr,
                      sched},
                     reinterpret_cast<const float2*>(S), reinterpret_cast<float2*>(Xdl)};
    if (build_tc_plan(p, H, CDMIMO_OP_FRAME, &pl) == CDMIMO_OK) return dispatch_frame_tc(p->in_dtype, pl, io, CDMIMO_OP_FRAME, s);
    if (p->form != CDMIMO_FORM_RESIDUAL && !p->learned && p->fuse != CDMIMO_FUSE_LEARNED &&
        build_gram_plan(p, true, H, p->form == CDMIMO_FORM_AUTO, &pl, true) == CDMIMO_OK)
        return dispatch_frame_gram(p->in_dtype, pl, io, s);
    // otherwise the two calls, each in the form it selects
    if (int rc = detect_impl(p, H, Y, N0, Xhat, nullptr, nullptr, sched, s)) return rc;
    return precode_impl(p, H, S, Xdl, sched, s);
}

// Per host thread and device, for the pipelined host-buffer frame: a kernel stream and a download
// stream (non-blocking, created on first use) and one event per hand-off (upload -> kernel,
// kernel -> download, download -> caller's stream).  Each record is followed by its wait before the
// event is recorded again, so the events are reused by every chunk and call.
struct HostPipe {
    cudaStream_t sk = nullptr, sd = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    ~HostPipe()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (sk) cudaStreamDestroy(sk);
        if (sd) cudaStreamDestroy(sd);
    }
};
constexpr int kMaxPipeDevices = 64;
thread_local HostPipe t_host_pipe[kMaxPipeDevices];

int host_pipe(HostPipe** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CDMIMO_ERR_CUDA;
    if (dev < 0 || dev >= kMaxPipeDevices) return CDMIMO_ERR_UNSUPPORTED;
    HostPipe& h = t_host_pipe[dev];
    for (cudaEvent_t& e : h.ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return CDMIMO_ERR_CUDA;
    for (cudaStream_t* q : {&h.sk, &h.sd})
        if (!*q && cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) != cudaSuccess) return CDMIMO_ERR_CUDA;
    *out = &h;
    return CDMIMO_OK;
}

}  // namespace

int cdmimo_detect_precode(const cdmimo_params* p, const void* H, const void* Y, const float* N0, void* Xhat,
                          const void* S, void* Xdl, void* workspace, size_t ws_bytes, void* stream)
{
    unsigned* sched;
    if (int rc = sched_from_workspace(workspace, ws_bytes, &sched)) return rc;
    return frame_impl(p, H, Y, N0, Xhat, S, Xdl, sched, static_cast<cudaStream_t>(stream));
}

int cdmimo_detect_precode_host(const cdmimo_params* p, const void* H_host, const void* Y_host, const float* N0_host,
                               const void* S_host, void* Xhat_host, void* Xdl_host, int n_chunks, void* dev_ws,
                               size_t ws_bytes, void* stream)
{
    if (int rc = validate(p)) return rc;
    if (p->n_sc == 0) return CDMIMO_OK;
    if (!H_host || !Y_host || !N0_host || !S_host || !Xhat_host || !Xdl_host || n_chunks < 0)
        return CDMIMO_ERR_INVALID_ARG;
    if (p->in_dtype != CDMIMO_C64 && (!p->h_scale || !p->y_scale)) return CDMIMO_ERR_INVALID_ARG;
    const size_t need = cdmimo_host_workspace_size(p, CDMIMO_OP_FRAME);
    if (!dev_ws || !aligned(dev_ws, 256) || ws_bytes < need) return CDMIMO_ERR_WORKSPACE;
    const int n = p->n_sc, nch = std::min(n_chunks > 0 ? n_chunks : kHostFrameChunks, n);
    cudaStream_t su = static_cast<cudaStream_t>(stream), sk = su, sd = su;
    HostPipe* hp = nullptr;
    if (nch > 1) {
        if (int rc = host_pipe(&hp)) return rc;
        sk = hp->sk;
        sd = hp->sd;
    }
    // per-subcarrier bytes of each staged array, and the staging layout (as in the size query)
    const size_t eb = elem_bytes(p->in_dtype);
    const size_t hs = (size_t)p->U * p->B * eb, ys = (size_t)p->n_sym * p->B * eb;
    const size_t ss = (size_t)p->n_sym * p->U * 8, xs = ss, xds = (size_t)p->n_sym * p->B * 8;
    char* dH = static_cast<char*>(dev_ws);
    char* dY = dH + round256(n * hs);
    char* dN = dY + round256(n * ys);
    char* dS = dN + round256((size_t)n * 4);
    char* dX = dS + round256(n * ss);
    char* dXd = dX + round256(n * xs);
    float* dhs = reinterpret_cast<float*>(dXd + round256(n * xds));
    float* dys = reinterpret_cast<float*>(reinterpret_cast<char*>(dhs) + round256((size_t)n * 4));
    const char* hH = static_cast<const char*>(H_host);
    const char* hY = static_cast<const char*>(Y_host);
    const char* hS = static_cast<const char*>(S_host);
    char* hX = static_cast<char*>(Xhat_host);
    char* hXd = static_cast<char*>(Xdl_host);
    auto hand_off = [&](cudaEvent_t e, cudaStream_t from, cudaStream_t to) {
        return from == to || (cudaEventRecord(e, from) == cudaSuccess && cudaStreamWaitEvent(to, e, 0) == cudaSuccess);
    };
    // the small arrays whole first (a copy has a fixed cost), then H and Y chunk by chunk
    if (cudaMemcpyAsync(dN, N0_host, (size_t)n * 4, cudaMemcpyHostToDevice, su) != cudaSuccess ||
        cudaMemcpyAsync(dS, hS, n * ss, cudaMemcpyHostToDevice, su) != cudaSuccess)
        return CDMIMO_ERR_CUDA;
    if (p->in_dtype != CDMIMO_C64) {
        if (cudaMemcpyAsync(dhs, p->h_scale, (size_t)n * 4, cudaMemcpyHostToDevice, su) != cudaSuccess ||
            cudaMemcpyAsync(dys, p->y_scale, (size_t)n * 4, cudaMemcpyHostToDevice, su) != cudaSuccess)
            return CDMIMO_ERR_CUDA;
    }
    // chunk i starts at subcarrier n 2i / (2 nch - 1): the last chunk is half the size of the others,
    // which shortens the kernel and download that follow the last upload
    const size_t den = 2 * (size_t)nch - 1;
    for (int i = 0; i < nch; ++i) {
        const size_t f0 = (size_t)n * 2 * i / den, f1 = i + 1 < nch ? (size_t)n * 2 * (i + 1) / den : (size_t)n;
        const size_t m = f1 - f0;
        if (m == 0) continue;
        if (cudaMemcpyAsync(dH + f0 * hs, hH + f0 * hs, m * hs, cudaMemcpyHostToDevice, su) != cudaSuccess ||
            cudaMemcpyAsync(dY + f0 * ys, hY + f0 * ys, m * ys, cudaMemcpyHostToDevice, su) != cudaSuccess)
            return CDMIMO_ERR_CUDA;
        if (!hand_off(hp ? hp->ev[0] : nullptr, su, sk)) return CDMIMO_ERR_CUDA;
        cdmimo_params q = *p;
        q.n_sc = (int)m;
        if (p->in_dtype != CDMIMO_C64) {
            q.h_scale = dhs + f0;
            q.y_scale = dys + f0;
        }
        if (int rc = frame_impl(&q, dH + f0 * hs, dY + f0 * ys, reinterpret_cast<const float*>(dN) + f0, dX + f0 * xs,
                                dS + f0 * ss, dXd + f0 * xds, nullptr, sk))
            return rc;
        if (!hand_off(hp ? hp->ev[1] : nullptr, sk, sd)) return CDMIMO_ERR_CUDA;
        if (cudaMemcpyAsync(hX + f0 * xs, dX + f0 * xs, m * xs, cudaMemcpyDeviceToHost, sd) != cudaSuccess ||
            cudaMemcpyAsync(hXd + f0 * xds, dXd + f0 * xds, m * xds, cudaMemcpyDeviceToHost, sd) != cudaSuccess)
            return CDMIMO_ERR_CUDA;
    }
    return hand_off(hp ? hp->ev[2] : nullptr, sd, su) ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

int cdmimo_fuse(int n_sc, int n_sym, int U, int C, const void* Xc, const float* w, int weights_are_lambda, void* Xhat,
                void* stream)
{
    if (n_sc < 0 || n_sym < 1 || U < 1 || C < 1) return CDMIMO_ERR_INVALID_ARG;
    if (n_sc == 0) return CDMIMO_OK;
    if (!Xc || !w || !Xhat || !aligned(Xc, 8) || !aligned(Xhat, 8) || !aligned(w, 4)) return CDMIMO_ERR_INVALID_ARG;
    const size_t total = (size_t)n_sc * n_sym * U;
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((total + threads - 1) / threads, 152 * 16);
    fuse_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        n_sc, n_sym, U, C, reinterpret_cast<const float2*>(Xc), w, weights_are_lambda, reinterpret_cast<float2*>(Xhat));
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

int cdmimo_fusion_weights(const cdmimo_params* p, const void* H, const float* N0, float* w, void* stream)
{
    if (int rc = validate(p)) return rc;
    if (p->fuse == CDMIMO_FUSE_LEARNED) return CDMIMO_ERR_UNSUPPORTED;
    if (p->n_sc == 0) return CDMIMO_OK;
    if (!H || !N0 || !w || !aligned(H, elem_bytes(p->in_dtype)) || !aligned(N0, 4) || !aligned(w, 4))
        return CDMIMO_ERR_INVALID_ARG;
    if (p->in_dtype != CDMIMO_C64 && (!p->h_scale || !aligned(p->h_scale, 4))) return CDMIMO_ERR_INVALID_ARG;
    ClusterTable tab{};  // by value in the kernel's parameters: nothing is allocated
    for (int c = 0, o = 0; c < p->C; o += p->cluster_size[c], ++c) {
        tab.off[c] = o;
        tab.size[c] = p->cluster_size[c];
    }
    const int colnorm = p->fuse == CDMIMO_FUSE_COLNORM;
    const int blocks = std::max(1, std::min(p->n_sc, 152 * 8));
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (p->in_dtype) {
    case CDMIMO_C64:
        fusion_weights_kernel<CDMIMO_C64><<<blocks, 256, 0, s>>>(p->n_sc, p->U, p->B, p->C, tab, H, N0, p->h_scale,
                                                                1.f / p->Ex, colnorm, w);
        break;
    case CDMIMO_C16F:
        fusion_weights_kernel<CDMIMO_C16F><<<blocks, 256, 0, s>>>(p->n_sc, p->U, p->B, p->C, tab, H, N0, p->h_scale,
                                                                 1.f / p->Ex, colnorm, w);
        break;
    default:
        fusion_weights_kernel<CDMIMO_C16BF><<<blocks, 256, 0, s>>>(p->n_sc, p->U, p->B, p->C, tab, H, N0,
                                                                  p->h_scale, 1.f / p->Ex, colnorm, w);
    }
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

int cdmimo_selected_form(const cdmimo_params* p, int op, const void* H)
{
    if (int rc = validate(p)) return rc;
    if (op != CDMIMO_OP_DETECT && op != CDMIMO_OP_PRECODE && op != CDMIMO_OP_FRAME) return CDMIMO_ERR_INVALID_ARG;
    CdPlan pl;
    if (build_tc_plan(p, H, op, &pl) == CDMIMO_OK)
        return (p->form == CDMIMO_FORM_GRAM_TC_PHASED || p->form == CDMIMO_FORM_GRAM_TC_UMMA) ? p->form
                                                                                            : CDMIMO_FORM_GRAM_TC;
    if ((op == CDMIMO_OP_DETECT || op == CDMIMO_OP_FRAME) && build_tc32_plan(p, H, &pl) == CDMIMO_OK)
        return CDMIMO_FORM_GRAM_TC;  // the frame then runs as two calls, the uplink's on this kernel
    if (op == CDMIMO_OP_FRAME) {
        if (p->form != CDMIMO_FORM_RESIDUAL && !p->learned && p->fuse != CDMIMO_FUSE_LEARNED &&
            build_gram_plan(p, true, H, p->form == CDMIMO_FORM_AUTO, &pl, true) == CDMIMO_OK)
            return CDMIMO_FORM_GRAM;
        op = CDMIMO_OP_DETECT;
    }
    const int rc = plan_for(p, op == CDMIMO_OP_DETECT, H, &pl);
    if (rc == CDMIMO_ERR_UNSUPPORTED && !is_forced_gram(p)) return CDMIMO_FORM_RESIDUAL;  // streaming
    if (rc) return rc;
    return pl.gram ? CDMIMO_FORM_GRAM : CDMIMO_FORM_RESIDUAL;
}

size_t cdmimo_workspace_size(const cdmimo_params* p, int op)
{
    (void)op;
    (void)p;
    return kSchedBytes;
}

size_t cdmimo_host_workspace_size(const cdmimo_params* p, int op)
{
    if (validate(p) != CDMIMO_OK) return 0;
    const size_t eb = elem_bytes(p->in_dtype);
    const size_t hb = round256((size_t)p->n_sc * p->U * p->B * eb);
    if (op == CDMIMO_OP_DETECT) {
        size_t v = hb + round256((size_t)p->n_sc * p->n_sym * p->B * eb) + round256((size_t)p->n_sc * 4) +
                   round256((size_t)p->n_sc * p->n_sym * p->U * 8);
        if (p->in_dtype != CDMIMO_C64) v += 2 * round256((size_t)p->n_sc * 4);
        return v + kSchedBytes;
    }
    if (op == CDMIMO_OP_PRECODE)
        return hb + round256((size_t)p->n_sc * p->n_sym * p->U * 8) + round256((size_t)p->n_sc * p->n_sym * p->B * 8) +
               kSchedBytes;
    if (op == CDMIMO_OP_FRAME) {  // H, Y, N0, S, Xhat, Xdl (and the two scale arrays); static schedule
        const size_t su = round256((size_t)p->n_sc * p->n_sym * p->U * 8), nb = round256((size_t)p->n_sc * 4);
        return hb + round256((size_t)p->n_sc * p->n_sym * p->B * eb) + nb + 2 * su +
               round256((size_t)p->n_sc * p->n_sym * p->B * 8) + (p->in_dtype != CDMIMO_C64 ? 2 * nb : 0);
    }
    return 0;
}

int cdmimo_detect_host(const cdmimo_params* p, const void* H_host, const void* Y_host, const float* N0_host,
                       void* Xhat_host, void* dev_ws, size_t ws_bytes, void* stream)
{
    if (int rc = validate(p)) return rc;
    if (p->n_sc == 0) return CDMIMO_OK;
    if (!H_host || !Y_host || !N0_host || !Xhat_host) return CDMIMO_ERR_INVALID_ARG;
    if (p->in_dtype != CDMIMO_C64 && (!p->h_scale || !p->y_scale)) return CDMIMO_ERR_INVALID_ARG;
    const size_t need = cdmimo_host_workspace_size(p, CDMIMO_OP_DETECT);
    if (!dev_ws || !aligned(dev_ws, 256) || ws_bytes < need) return CDMIMO_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t eb = elem_bytes(p->in_dtype);
    const size_t hb = (size_t)p->n_sc * p->U * p->B * eb, yb = (size_t)p->n_sc * p->n_sym * p->B * eb;
    const size_t nb = (size_t)p->n_sc * 4, xb = (size_t)p->n_sc * p->n_sym * p->U * 8;
    char* w = static_cast<char*>(dev_ws);
    char* dH = w;
    char* dY = dH + round256(hb);
    char* dN = dY + round256(yb);
    char* dX = dN + round256(nb);
    // schedule counters: the last kSchedBytes of the workspace, zeroed by every call
    unsigned* sched = reinterpret_cast<unsigned*>(w + need - kSchedBytes);
    if (cudaMemsetAsync(sched, 0, 16, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    cdmimo_params q = *p;
    if (cudaMemcpyAsync(dH, H_host, hb, cudaMemcpyHostToDevice, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    if (cudaMemcpyAsync(dY, Y_host, yb, cudaMemcpyHostToDevice, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    if (cudaMemcpyAsync(dN, N0_host, nb, cudaMemcpyHostToDevice, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    if (p->in_dtype != CDMIMO_C64) {
        char* dhs = dX + round256(xb);
        char* dys = dhs + round256(nb);
        if (cudaMemcpyAsync(dhs, p->h_scale, nb, cudaMemcpyHostToDevice, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
        if (cudaMemcpyAsync(dys, p->y_scale, nb, cudaMemcpyHostToDevice, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
        q.h_scale = reinterpret_cast<const float*>(dhs);
        q.y_scale = reinterpret_cast<const float*>(dys);
    }
    if (int rc = detect_impl(&q, dH, dY, reinterpret_cast<const float*>(dN), dX, nullptr, nullptr, sched, s))
        return rc;
    if (cudaMemcpyAsync(Xhat_host, dX, xb, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    return CDMIMO_OK;
}

int cdmimo_precode_host(const cdmimo_params* p, const void* H_host, const void* S_host, void* Xdl_host, void* dev_ws,
                        size_t ws_bytes, void* stream)
{
    if (int rc = validate(p)) return rc;
    if (p->n_sc == 0) return CDMIMO_OK;
    if (!H_host || !S_host || !Xdl_host) return CDMIMO_ERR_INVALID_ARG;
    const size_t need = cdmimo_host_workspace_size(p, CDMIMO_OP_PRECODE);
    if (!dev_ws || !aligned(dev_ws, 256) || ws_bytes < need) return CDMIMO_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t hb = (size_t)p->n_sc * p->U * p->B * elem_bytes(p->in_dtype);
    const size_t sb = (size_t)p->n_sc * p->n_sym * p->U * 8, xb = (size_t)p->n_sc * p->n_sym * p->B * 8;
    char* dH = static_cast<char*>(dev_ws);
    char* dS = dH + round256(hb);
    char* dX = dS + round256(sb);
    unsigned* sched = reinterpret_cast<unsigned*>(static_cast<char*>(dev_ws) + need - kSchedBytes);
    if (cudaMemsetAsync(sched, 0, 16, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    if (cudaMemcpyAsync(dH, H_host, hb, cudaMemcpyHostToDevice, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    if (cudaMemcpyAsync(dS, S_host, sb, cudaMemcpyHostToDevice, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    if (int rc = precode_impl(p, dH, dS, dX, sched, s)) return rc;
    if (cudaMemcpyAsync(Xdl_host, dX, xb, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CDMIMO_ERR_CUDA;
    return CDMIMO_OK;
}

size_t cdmimo_learned_param_count(int K, int U, int hidden)
{
    if (K < 1 || K > CDMIMO_MAX_LEARNED_SWEEPS || U < 1 || U > CDMIMO_MAX_USERS || hidden < 1 ||
        hidden > CDMIMO_MAX_HIDDEN)
        return 0;
    return (size_t)2 * K + (size_t)hidden * (U + 1) + 2 * (size_t)hidden + 1;
}

int cdmimo_learned_pack(const float* master, int K, int U, int hidden, void* block, void* stream)
{
    if (!cdmimo_learned_param_count(K, U, hidden)) return CDMIMO_ERR_INVALID_ARG;
    if (!master || !block || !aligned(master, 4) || !aligned(block, 16)) return CDMIMO_ERR_INVALID_ARG;
    learned_pack_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(master, K, U, hidden,
                                                                           static_cast<cdmimo_learned*>(block));
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

size_t cdmimo_learned_workspace_size(const cdmimo_params* p, int hidden)
{
    CdPlan pl;
    GradLayout gl;
    if (!p || grad_plan(p, hidden, &pl, &gl) != CDMIMO_OK) return 0;
    return (size_t)p->n_sc * gl.ws_stride * sizeof(float);
}

int cdmimo_learned_grad(const cdmimo_params* p, int hidden, const void* H, const void* Y, const float* N0,
                        const void* Xtarget, float* grad, float* loss, void* workspace, size_t ws_bytes, void* stream)
{
    CdPlan pl;
    GradLayout gl;
    if (int rc = grad_plan(p, hidden, &pl, &gl)) return rc;
    if (!p->learned || !aligned(p->learned, 16) || !grad || !loss) return CDMIMO_ERR_INVALID_ARG;
    if (p->n_sc == 0) return CDMIMO_OK;
    if (!H || !Y || !N0 || !Xtarget || !aligned(H, 8) || !aligned(Y, 8) || !aligned(Xtarget, 8))
        return CDMIMO_ERR_INVALID_ARG;
    if (!workspace || !aligned(workspace, 16) || ws_bytes < (size_t)p->n_sc * gl.ws_stride * sizeof(float))
        return CDMIMO_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GradIO io{static_cast<const float2*>(H), static_cast<const float2*>(Y), N0, static_cast<const float2*>(Xtarget),
              static_cast<const cdmimo_learned*>(p->learned), static_cast<float*>(workspace)};
    int rc = CDMIMO_ERR_UNSUPPORTED;
    switch (pl.P) {
    case 8: rc = launch_grad_t<8>(pl, gl, io, s); break;
    case 16: rc = launch_grad_t<16>(pl, gl, io, s); break;
    case 32: rc = launch_grad_t<32>(pl, gl, io, s); break;
    }
    if (rc) return rc;
    const int threads = 256, blocks = (gl.n_params + 1 + threads - 1) / threads;
    learned_reduce_kernel<<<blocks, threads, 0, s>>>(static_cast<const float*>(workspace), p->n_sc, gl.ws_stride,
                                                     gl.n_params, grad, loss);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

int cdmimo_learned_grad_noalloc(const cdmimo_params* p, int hidden, const void* H, const void* Y, const float* N0,
                                const void* Xtarget, float* grad, float* loss, void* stream)
{
    CdPlan pl;
    GradLayout gl;
    if (int rc = grad_plan(p, hidden, &pl, &gl)) return rc;
    const size_t need = (size_t)p->n_sc * gl.ws_stride * sizeof(float);
    if (need > CDMIMO_NOALLOC_SCRATCH_BYTES) return CDMIMO_ERR_WORKSPACE;
    if (p->n_sc == 0) return cdmimo_learned_grad(p, hidden, H, Y, N0, Xtarget, grad, loss, nullptr, 0, stream);
    float* ws = noalloc_scratch_address();
    if (!ws) return CDMIMO_ERR_CUDA;
    // Every partial-sum entry the reduction reads is written by the gradient kernel first, so the
    // scratch needs no clearing between calls.
    return cdmimo_learned_grad(p, hidden, H, Y, N0, Xtarget, grad, loss, ws, CDMIMO_NOALLOC_SCRATCH_BYTES, stream);
}

int cdmimo_adam_step(float* theta, const float* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                     float eps, int step, void* stream)
{
    if (n < 0 || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return CDMIMO_ERR_INVALID_ARG;
    if (n == 0) return CDMIMO_OK;
    if (!theta || !grad || !m || !v) return CDMIMO_ERR_INVALID_ARG;
    const float c1 = (float)(1.0 - std::pow((double)beta1, step)), c2 = (float)(1.0 - std::pow((double)beta2, step));
    const int threads = 256, blocks = std::min((n + threads - 1) / threads, 1024);
    adam_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(theta, grad, m, v, n, lr, beta1, beta2, eps,
                                                                          c1, c2);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

void cdmimo_batch_default_plan(cdmimo_batch_plan* plan)
{
    if (!plan) return;
    std::memset(plan, 0, sizeof(*plan));
    plan->P = 16;
    plan->threads = 256;
    plan->group_bytes = 64 * 1024;
    plan->ctas_per_sm = 0;
}

int cdmimo_batch_build(const cdmimo_batch_desc* desc, int n_desc, cdmimo_batch_plan* plan, void* table_host,
                       size_t table_bytes)
{
    BatchBuild bb;
    if (int rc = batch_split(desc, n_desc, plan, &bb)) return rc;
    if (!table_host) return CDMIMO_OK;
    if (table_bytes < plan->table_bytes || !aligned(table_host, 16)) return CDMIMO_ERR_WORKSPACE;
    unsigned char* t = static_cast<unsigned char*>(table_host);
    std::memset(t, 0, plan->table_bytes);
    BatchTableHeader hdr{};
    hdr.n_desc = (int)bb.descs.size();
    hdr.n_items = plan->n_items;
    hdr.n_groups = (int)bb.groups.size();
    hdr.n_clusters = (int)bb.clusters.size();
    hdr.off_desc = (unsigned)((sizeof(BatchTableHeader) + 15) & ~(size_t)15);
    hdr.off_group = hdr.off_desc + (unsigned)((bb.descs.size() * sizeof(BatchDesc) + 15) & ~(size_t)15);
    hdr.off_cluster = hdr.off_group + (unsigned)((bb.groups.size() * sizeof(BatchGroup) + 15) & ~(size_t)15);
    hdr.total_bytes = (unsigned)plan->table_bytes;
    std::memcpy(t, &hdr, sizeof(hdr));
    std::memcpy(t + hdr.off_desc, bb.descs.data(), bb.descs.size() * sizeof(BatchDesc));
    std::memcpy(t + hdr.off_group, bb.groups.data(), bb.groups.size() * sizeof(BatchGroup));
    std::memcpy(t + hdr.off_cluster, bb.clusters.data(), bb.clusters.size() * sizeof(BatchCluster));
    return CDMIMO_OK;
}

int cdmimo_detect_batched(const cdmimo_batch_plan* plan, const void* table_dev, int* counter, void* stream)
{
    return cdmimo_detect_batched_stats(plan, table_dev, counter, nullptr, stream);
}

int cdmimo_detect_batched_stats(const cdmimo_batch_plan* plan, const void* table_dev, int* counter,
                                unsigned long long* stats, void* stream)
{
    if (!plan || !table_dev || !counter || !aligned(table_dev, 16) || !aligned(counter, 4) || !aligned(stats, 8))
        return CDMIMO_ERR_INVALID_ARG;
    if (plan->n_items == 0) return CDMIMO_OK;
    if (plan->threads < 64 || plan->threads > (plan->P == 8 ? 384 : 512) || (plan->threads & 31) ||
        plan->smem_bytes == 0)
        return CDMIMO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (plan->P) {
    case 8: return launch_batched_t<8>(plan, table_dev, counter, stats, s);
    case 16: return launch_batched_t<16>(plan, table_dev, counter, stats, s);
    case 32: return launch_batched_t<32>(plan, table_dev, counter, stats, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int cdmimo_synth_uplink(unsigned long long seed, int n_sc, int n_sym, int B, int U, int M, const float* snr_db, void* H,
                        void* X, int* labels, void* Y, float* N0, void* stream)
{
    if (n_sc < 0 || n_sym < 1 || B < 1 || U < 1) return CDMIMO_ERR_INVALID_ARG;
    int L = 0;
    switch (M) {
    case 4: L = 2; break;
    case 16: L = 4; break;
    case 64: L = 8; break;
    case 256: L = 16; break;
    default: return CDMIMO_ERR_INVALID_ARG;
    }
    if (n_sc == 0) return CDMIMO_OK;
    if (!snr_db || !H || !X || !Y || !N0 || !aligned(H, 8) || !aligned(X, 8) || !aligned(Y, 8)) return CDMIMO_ERR_INVALID_ARG;
    SynthArgs a{};
    a.seed = seed;
    a.n_sc = n_sc;
    a.n_sym = n_sym;
    a.B = B;
    a.U = U;
    a.M = M;
    a.L = L;
    a.k = L == 2 ? 1 : L == 4 ? 2 : L == 8 ? 3 : 4;
    a.scale = (float)(1.0 / std::sqrt(2.0 * (L * L - 1) / 3.0));
    a.snr_db = snr_db;
    a.H = static_cast<float2*>(H);
    a.X = static_cast<float2*>(X);
    a.labels = labels;
    a.Y = static_cast<float2*>(Y);
    a.N0 = N0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = 152 * 8;
    synth_channel_kernel<<<blocks, threads, 0, s>>>(a);
    synth_symbol_kernel<<<blocks, threads, 0, s>>>(a);
    synth_receive_kernel<<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? CDMIMO_OK : CDMIMO_ERR_CUDA;
}

const char* cdmimo_status_string(int status)
{
    switch (status) {
    case CDMIMO_OK: return "CDMIMO_OK";
    case CDMIMO_ERR_INVALID_ARG: return "CDMIMO_ERR_INVALID_ARG";
    case CDMIMO_ERR_BAD_PARTITION: return "CDMIMO_ERR_BAD_PARTITION";
    case CDMIMO_ERR_UNSUPPORTED: return "CDMIMO_ERR_UNSUPPORTED";
    case CDMIMO_ERR_CUDA: return "CDMIMO_ERR_CUDA";
    case CDMIMO_ERR_TIMEOUT: return "CDMIMO_ERR_TIMEOUT";
    case CDMIMO_ERR_WORKSPACE: return "CDMIMO_ERR_WORKSPACE";
    }
    return "CDMIMO_UNKNOWN_STATUS";
}

int cdmimo_device_status(int clear)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return CDMIMO_ERR_CUDA;
    unsigned v = 0;
    if (module_status(&v, clear) != CDMIMO_OK || gram_detect_module_status(&v, clear) != CDMIMO_OK ||
        gram_precode_module_status(&v, clear) != CDMIMO_OK || gram_frame_module_status(&v, clear) != CDMIMO_OK ||
        frame_tc_module_status(&v, clear) != CDMIMO_OK || frame_tc16_module_status(&v, clear) != CDMIMO_OK ||
        frame_ws_module_status(&v, clear) != CDMIMO_OK || frame_ws16_module_status(&v, clear) != CDMIMO_OK ||
        tc32_module_status(&v, clear) != CDMIMO_OK)
        return CDMIMO_ERR_CUDA;
    return (int)v;
}

int cdmimo_version(void) { return 0x000100; }

}  // extern "C"
