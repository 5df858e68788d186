// Gram-form CD detection (Algorithm 1 + fusion of Sec. III) on the tensor cores for 16 < U <= 32
// users: the contractions G_c = H_c^H H_c and z = H_c^H y_c as split-TF32 (c64) or exact-TF32
// (fp16 / bf16 storage) mma.sync m16n8k8 tiles, as in cd_frame_tc.cuh but over two 16-row user
// tiles, and the K Gauss-Seidel sweeps in FP32 with one lane per (cluster, symbol) holding its 32
// coordinates in registers.
//
// At U = B_c the sweeps' FP32 work (K U^2 complex MACs per cluster and vector) is half the residual
// form's (2 K U B_c), and 16-bit storage needs one MMA per tile instead of three, so here the
// reduced-precision storage saves arithmetic as well as bytes.
//
// Layout (one CTA per SM, persistent over subcarriers): two channel buffers of 32 whole rows (user u,
// all B antennas, padded to the bank residue of ws_row_words), each arriving as U bulk copies issued
// one subcarrier ahead; G_c as [32][16] pair-planar rows with zero diagonal; m_u; z then x per tile.
// Phase A: one warp per cluster, user tile 0 (rows 0-15) against all 32 columns and tile 1 against
// columns 16-31; rows 16-31 of columns 0-15 are written from tile 0's result as its conjugate
// transpose (G_c is Hermitian).  Phase B: the sweeps.  Phase C: the fusion.
#pragma once
#include "cd_frame_tc.cuh"
#include "cd_frame_ws.cuh"

namespace cdmimo {

constexpr int kTc32Threads = 256;

// Shared-memory layout of cd_detect_tc32_kernel (byte offsets), built on the host (gram_tc32.cu).
struct Tc32Layout {
    unsigned off_H, st_H;  // two channel buffers of [32][srow] words
    unsigned off_G;        // [C][32][16] float4
    unsigned off_D;        // [C][32] floats: m_u
    unsigned off_Z;        // [32][xs] float2: z, then each tile's x
    unsigned off_lam, off_tab, off_bar, smem_bytes;
    int srow;  // 32-bit words per channel row
};

// Phase A of one cluster on one warp (see above).  Hc: the cluster's columns of the 32 channel rows
// (srow words apart); y of symbol n at element ybase + n B of Y.
template <int BC, int IN>
__device__ __forceinline__ void tc32_phase_a(const CdPlan& pl, const float* Hc, int srow, const void* Y, size_t ybase,
                                             float alpha, float4* Gc, float* Dm, float2* Zc, uint32_t xs)
{
    constexpr int NP = 16;
    constexpr int KA = BC / 4;
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int U = pl.U, n_sym = pl.n_sym;
    const float2* Hc2 = reinterpret_cast<const float2*>(Hc);
    const int SR2 = srow / 2;
    auto hget = [&](int row, int e) -> float2 {
        if constexpr (IN == CDMIMO_C64) return Hc2[row * SR2 + e];
        else return Elem<IN>::load_shared(Hc, (size_t)row * srow + e);
    };
    // the lane's receive samples (entry 4 ks + tig of symbols 8 j + gid) for both user tiles
    float2 yv[KA][2];
#pragma unroll
    for (int ks = 0; ks < KA; ++ks)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int n = 8 * j + gid;
            yv[ks][j] = n < n_sym ? Elem<IN>::load(Y, ybase + (size_t)n * pl.B + 4 * ks + tig) : make_float2(0.f, 0.f);
        }
    // c64 (three MMAs and two split operands per product) keeps the user-tile loop rolled: unrolled,
    // its fragments and accumulators pushed the kernel past 255 registers into spills
#pragma unroll(IN == CDMIMO_C64 ? 1 : 2)
    for (int mt = 0; mt < 2; ++mt) {
        const int j0 = mt ? 2 : 0;  // user tile 1: columns 16-31 only
        float accG[8][4], accZ[4][4];
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int q = 0; q < 4; ++q) accG[t][q] = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int q = 0; q < 4; ++q) accZ[t][q] = 0.f;
#pragma unroll
        for (int ks = 0; ks < KA; ++ks) {
            const int e = 4 * ks + tig;
            const int r0 = 16 * mt + gid;
            if constexpr (IN == CDMIMO_C64) {
                uint32_t ah[4], al[4];
                a_frag(hget(r0, e), hget(r0 + 8, e), ah, al);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j < j0) continue;
                    BFrag bp, br;
                    b_frags(hget(8 * j + gid, e), bp, br);
                    mma_3xtf32(accG[j], ah, al, bp);
                    mma_3xtf32(accG[4 + j], ah, al, br);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    BFrag bp, br;
                    b_frags(yv[ks][j], bp, br);
                    mma_3xtf32(accZ[j], ah, al, bp);
                    mma_3xtf32(accZ[2 + j], ah, al, br);
                }
            } else {  // 16-bit storage: every operand exact in TF32, one MMA per tile
                uint32_t a[4];
                a_frag_exact(hget(r0, e), hget(r0 + 8, e), a);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j < j0) continue;
                    const float2 hv = hget(8 * j + gid, e);
                    mma_exact(accG[j], a, hv, false);
                    mma_exact(accG[4 + j], a, hv, true);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    mma_exact(accZ[j], a, yv[ks][j], false);
                    mma_exact(accZ[2 + j], a, yv[ks][j], true);
                }
            }
        }
        // G rows u = 16 mt + gid (+8), columns v = 8 j + 2 tig (+1): pair-planar, zero diagonal, m_u
        // from the diagonal; tile 0's columns 16-31 also give rows 16-31 of columns 0-15 (conjugate).
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j < j0) continue;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int u = 16 * mt + gid + 8 * r, v = 8 * j + 2 * tig;
                float g0 = accG[j][2 * r], g1 = accG[j][2 * r + 1];
                float i0 = accG[4 + j][2 * r], i1 = accG[4 + j][2 * r + 1];
                if (v == u || v + 1 == u) {
                    const float ev = v == u ? g0 : g1, den = ev + alpha;
                    Dm[u] = (u < U && den > 0.f) ? __fdividef(1.f, den) : 0.f;
                    if (v == u) g0 = i0 = 0.f;
                    else g1 = i1 = 0.f;
                }
                Gc[u * NP + (v >> 1)] = make_float4(g0, g1, i0, i1);
                if (mt == 0 && j >= 2) {
                    float* m0 = reinterpret_cast<float*>(Gc + v * NP + (u >> 1));
                    float* m1 = reinterpret_cast<float*>(Gc + (v + 1) * NP + (u >> 1));
                    m0[u & 1] = g0;
                    m0[2 + (u & 1)] = -i0;
                    m1[u & 1] = g1;
                    m1[2 + (u & 1)] = -i1;
                }
            }
        }
        // z rows u = 16 mt + gid (+8), symbols n = 8 j + 2 tig (+1)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int u = 16 * mt + gid + 8 * r, n = 8 * j + 2 * tig;
                if (u < U) {
                    float2* z = Zc + u * xs;
                    if (n < n_sym) z[n] = make_float2(accZ[j][2 * r], accZ[2 + j][2 * r]);
                    if (n + 1 < n_sym) z[n + 1] = make_float2(accZ[j][2 * r + 1], accZ[2 + j][2 * r + 1]);
                }
            }
    }
}

template <int BC, int IN>
__global__ void __launch_bounds__(kTc32Threads, 1) cd_detect_tc32_kernel(const CdPlan pl, const Tc32Layout tl,
                                                                          const DetectIO io)
{
    static_assert(BC == 16 || BC == 32 || BC == 64, "cluster size 16, 32 or 64");
    constexpr int UT = 32, NP = 16;
    constexpr uint32_t eb = IN == CDMIMO_C64 ? 8u : 4u;
    constexpr int ew = IN == CDMIMO_C64 ? 2 : 1;
    constexpr int kWarps = kTc32Threads / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    auto Hb = [&](int b) { return reinterpret_cast<float*>(smem + tl.off_H + (unsigned)b * tl.st_H); };
    float4* Gs = reinterpret_cast<float4*>(smem + tl.off_G);
    float* Dm = reinterpret_cast<float*>(smem + tl.off_D);
    float2* Zs = reinterpret_cast<float2*>(smem + tl.off_Z);
    float* lam = reinterpret_cast<float*>(smem + tl.off_lam);
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + tl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + tl.off_bar);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym, SROW = tl.srow;
    const uint32_t xs = tc_x_stride(pl.n_tiles);

    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0) {
        mbar_init(&bar[0], (uint32_t)kWarps);
        mbar_init(&bar[1], (uint32_t)kWarps);
        fence_proxy_async_smem();
    }
    for (int j = 0; j < 2; ++j) {
        float* hb = Hb(j) + U * SROW;
        for (int i = tid; i < (UT - U) * SROW; i += blockDim.x) hb[i] = 0.f;
    }
    __syncthreads();

    // Subcarrier f's channel rows into buffer b: warp w copies users w, w + 8, ... (whole rows), its
    // lane 0 announcing their bytes (one arrival per warp); warp 0 also brings f's y into L2.
    auto issue_copy = [&](int f, int b) {
        if (lane != 0) return;
        const char* Hf = reinterpret_cast<const char*>(io.H) + (size_t)f * U * pl.B * eb;
        const int rows = warp < U ? (U - 1 - warp) / kWarps + 1 : 0;
        mbar_arrive_expect_tx(&bar[b], (uint32_t)rows * pl.B * eb);
        fence_proxy_async_smem();
        for (int u = warp; u < U; u += kWarps)
            bulk_g2s(Hb(b) + (size_t)u * SROW, Hf + (size_t)u * pl.B * eb, (uint32_t)pl.B * eb, &bar[b]);
        if (warp == 0)
            bulk_prefetch_l2(static_cast<const char*>(io.Y) + (size_t)f * n_sym * pl.B * eb, (uint32_t)n_sym * pl.B * eb);
    };

    // phase B: one lane per (cluster, symbol), each cluster's symbols in their own quarter or half
    // warp so that no quarter warp reads two clusters' Gram rows
    const int slot = ws_slot(n_sym), sc = warp * (32 / slot) + lane / slot, sn = lane % slot;
    const bool sweep_lane = sc < C && sn < n_sym;
    int f = blockIdx.x, done = 0;
    if (f < pl.n_sc) issue_copy(f, 0);
    for (int k = 0; f < pl.n_sc; ++k) {
        const int b = k & 1;
        float alpha = __ldg(io.N0 + f) * pl.inv_Ex, out_scale = 1.f;
        if (!(alpha >= 0.f)) {  // negative or NaN noise variance: this subcarrier's estimate is NaN
            if (tid == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_N0);
            out_scale = __int_as_float(0x7fc00000);
            alpha = 0.f;
        }
        if constexpr (IN != CDMIMO_C64) {  // solve with alpha / a_f^2, scale x by b_f / a_f
            const float hs = __ldg(io.h_scale + f), ys = __ldg(io.y_scale + f);
            alpha = alpha / (hs * hs);
            out_scale = out_scale * (ys / hs);
        }
        const uint32_t parity = (uint32_t)(k >> 1) & 1u;
        const bool ok = mbar_wait_bounded(&bar[b], parity);
        if (__syncthreads_or(!ok)) {  // copy timeout: give it a last bounded wait, then stop
            if (tid == 0) mbar_wait_bounded(&bar[b], parity);
            break;
        }
        const int fn = f + (int)gridDim.x;
        if (fn < pl.n_sc) issue_copy(fn, b ^ 1);  // buffer b ^ 1 was last read before the previous barrier

        // Phase A: G_c, m_u and z per cluster (one warp each).
        for (int c = warp; c < C; c += kWarps) {
            const ClusterTile ct = tab[c];
            tc32_phase_a<BC, IN>(pl, Hb(b) + ct.off * ew, SROW, io.Y, (size_t)f * n_sym * pl.B + ct.off, alpha,
                                 Gs + (size_t)c * UT * NP, Dm + c * UT, Zs + c * n_sym, xs);
        }
        __syncthreads();

        // Phase B: K sweeps per tile; x replaces z.
        if (sweep_lane) {
            const int tile = sc * n_sym + sn;
            const float* dd = Dm + sc * UT;
            float4 x[NP];
            gram_sweeps<UT>(U, pl.K, Gs + (size_t)sc * UT * NP, dd, Zs + tile, xs, x);
#pragma unroll
            for (int u = 0; u < UT; ++u)
                if (u < U) Zs[tile + u * xs] = slice_entry<UT, 1>(x, u);
            if (sn == 0) {
                float msum = 0.f;
                for (int u = 0; u < U; ++u) msum += dd[u] > 0.f ? dd[u] : __int_as_float(0x7f800000);
                lam[sc] = 1.f / msum;
            }
        }
        __syncthreads();

        // Phase C: fusion (Sec. III), with the per-cluster outputs if requested.
        if (io.Xc || io.lam) fuse_subcarrier<false>(pl, io, f, lam, Zs, xs, out_scale);
        else fuse_range(pl, io, f, lam, Zs, xs, out_scale, 0, blockDim.x);
        __syncthreads();
        ++done;
        f = fn;
    }
    sched_finish(io.sched, done, pl.n_sc);
}

}  // namespace cdmimo
