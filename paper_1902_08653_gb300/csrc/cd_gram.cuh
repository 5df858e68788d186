// Gram-form CD kernels: the iterates of Algorithms 1 and 2, evaluated through the cluster Gram
// matrix G_c = H_c^H H_c instead of the running residual.
//
// Uplink.  With r = y_c - H_c x kept implicitly, h_u^H r = z_u - sum_v G_uv x_v (z = H_c^H y_c), and
// Algorithm 1's step x_u <- m h_u^H r + n x_u (n = m ||h_u||^2 = m G_uu) becomes
//   x_u <- m_u (z_u - sum_{v != u} G_uv x_v),
// Gauss-Seidel on (G_c + (N0/Ex) I) x = z, visited u = 1..U ascending, K sweeps from x = 0.
// Downlink.  Algorithm 2 / Eq. (4) only ever adds multiples of h_u to x_c (from x_c = 0), so
// x_c = H_c w with x_c <- x_c - p_u^2 (h_u^H x_c - s_u) h_u acting on w as
//   w_u <- w_u - p_u^2 (sum_v G_uv w_v - s_u) = p_u^2 (s_u - sum_{v != u} G_uv w_v)   (p_u^2 G_uu = 1),
// and w_u stays 0 for a zero column (p_u = 0).  After K sweeps x_c = H_c w is formed once and
// normalized as in Sec. IV-B.
// Same iterates in exact arithmetic; per vector the work drops from 2 K U B_c complex MACs to
// K U^2 + (U^2 B_c) / n_sym + U B_c (Gram matrix shared by the subcarrier's symbols).
//
// Phases per subcarrier (one persistent CTA walks subcarriers as the residual-form kernels do):
//   A  correlations from the channel in shared memory (tiles of AT lanes, as in the packed kernels):
//      tile (c, v) holds h_{v,c} and produces column v of G_c (and ||h_v||^2 on the diagonal);
//      uplink tile (c, n) holds y_{n,c} and produces z.
//   B  one lane per (cluster, symbol) runs the K sweeps with x (or w) in registers, U <= UT
//      complex entries, reading rows of G_c with a zero diagonal from shared memory: four packed
//      FMAs per shared-memory load and no cross-lane reduction.
//   C  uplink: fusion (Sec. III).  Downlink: x_c = H_c w over the tile's antenna lanes, then the
//      per-cluster normalization.
#pragma once
#include "cd_kernels_pp.cuh"

namespace cdmimo {

// A lane of a phase with C x J tiles of AT lanes each.  The phase's lanes are spread evenly over a
// multiple of four warps (whole tiles per warp), so each warp scheduler of the SM holds the same
// share of them; lanes past the end are inactive.
struct GLane {
    bool active;
    int c, j, a;
    unsigned mask;  // the warp's active lanes
};

__device__ __forceinline__ GLane gram_lane(int C, int J, int AT)
{
    const int L = C * J * AT;
    const int W = ((L + 31) / 32 + 3) / 4 * 4;
    const int lpw = ((L + W - 1) / W + AT - 1) / AT * AT;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, v = w * lpw + l;
    GLane g;
    g.active = l < lpw && v < L;
    const int t = g.active ? v / AT : 0;  // inactive lanes get tile (0, 0), lane 0: safe indices
    g.a = g.active ? v - t * AT : 0;
    g.c = t / J;
    g.j = t - g.c * J;
    const int n_act = min(lpw, L - w * lpw);
    g.mask = n_act >= 32 ? 0xffffffffu : (n_act > 0 ? (1u << n_act) - 1u : 0u);
    return g;
}

// Phase A, Gram columns: tile (c, v) correlates h_{v,c} with every h_{u,c}: G_c[u][v] = h_u^H h_v,
// stored in pair-planar rows (row u: (Re G_u,2p, Re G_u,2p+1, Im G_u,2p, Im G_u,2p+1) per pair p)
// with the diagonal replaced by 0; from G_uu = ||h_u||^2 the sweep coefficient
// Ds[c][u] = (||h_u||^2 + alpha)^{-1} (0 when that is not positive: a skipped column) is written
// (uplink: alpha = N0/Ex, m_u of Algorithm 1; downlink: alpha = 0, p_u^2 of Algorithm 2).
template <int AT, int UT>
__device__ __forceinline__ void gram_columns(const GLane& g, int U, const ClusterTile* tab, const float2* Hb,
                                             float alpha, float4* Gs, float* Ds, float* Ds0 = nullptr,
                                             float* Er = nullptr)
{
    constexpr int LP = AT * kPairs;
    if (!g.active) return;
    const ClusterTile ct = tab[g.c];
    const float4* hb = reinterpret_cast<const float4*>(Hb + ct.soff) + g.a;
    float4 hv[kPairs];
    pp_load_h<AT>(hb + g.j * LP, hv);
    float* G = reinterpret_cast<float*>(Gs + (size_t)g.c * UT * (UT / 2));
    const int col = (g.j >> 1) * 4 + (g.j & 1);
#pragma unroll 2
    for (int u = 0; u < U; ++u) {
        float4 hu[kPairs];
        pp_load_h<AT>(hb + u * LP, hu);
        float2 s = pp_partial_corr(hu, hv);
        s.x = tile_sum_c<AT>(s.x, g.mask);
        s.y = tile_sum_c<AT>(s.y, g.mask);
        if (g.a == 0) {
            if (u == g.j) {  // Ds0 (optional): the same with alpha = 0 (downlink p_u^2 beside uplink m_u)
                const float den = s.x + alpha;
                Ds[g.c * UT + u] = den > 0.f ? __fdividef(1.f, den) : 0.f;
                if (Ds0) Ds0[g.c * UT + u] = s.x > 0.f ? __fdividef(1.f, s.x) : 0.f;
                if (Er) Er[g.c * UT + u] = s.x;  // ||h_u||^2 itself (learned sweeps and fusion)
                s = make_float2(0.f, 0.f);
            }
            G[u * (2 * UT) + col] = s.x;
            G[u * (2 * UT) + col + 2] = s.y;
        }
    }
}

// Phase A, uplink right-hand sides: tile (c, n) holds y_{n,c} (pair-planar, in registers) and
// writes z_u = h_{u,c}^H y_{n,c} to Zs[u][c n_sym + n].
template <int AT>
__device__ __forceinline__ void gram_rhs(const GLane& g, int U, int n_sym, uint32_t zs, const ClusterTile* tab,
                                         const float2* Hb, const float4 (&y)[kPairs], float2* Zs)
{
    constexpr int LP = AT * kPairs;
    if (!g.active) return;
    const ClusterTile ct = tab[g.c];
    const float4* hb = reinterpret_cast<const float4*>(Hb + ct.soff) + g.a;
    float2* z = Zs + g.c * n_sym + g.j;
#pragma unroll 2
    for (int u = 0; u < U; ++u) {
        float4 hu[kPairs];
        pp_load_h<AT>(hb + u * LP, hu);
        float2 s = pp_partial_corr(hu, y);
        s.x = tile_sum_c<AT>(s.x, g.mask);
        s.y = tile_sum_c<AT>(s.y, g.mask);
        if (g.a == 0) z[u * zs] = s;
    }
}

// Sum_v Gt_uv x_v over the first npu pairs of row u (Gt zero-diagonal, [UT][UT/2] float4 rows at
// Grow, x pair-planar in registers), as (re, im).  Called from fully unrolled loops over u, where npu
// is a constant and the pair guards fold away.
template <int UT>
__device__ __forceinline__ float2 gram_row_dot(const float4* Grow, int u, int npu, const float4 (&x)[UT / 2])
{
    constexpr int NP = UT / 2;
    const float4* gr = Grow + u * NP;
    float2 R0 = make_float2(0.f, 0.f), I0 = R0, J0 = R0, R1 = R0, I1 = R0, J1 = R0;
#pragma unroll
    for (int i = 0; i < NP; i += 2) {
        if (i < npu) {
            const float4 ga = gr[i];
            R0 = ffma2(lo2(ga), lo2(x[i]), R0);
            J0 = ffma2(hi2(ga), hi2(x[i]), J0);
            I0 = ffma2(lo2(ga), hi2(x[i]), I0);
            I0 = ffma2(hi2(ga), lo2(x[i]), I0);
        }
        if (i + 1 < npu) {
            const float4 gb = gr[i + 1];
            R1 = ffma2(lo2(gb), lo2(x[i + 1]), R1);
            J1 = ffma2(hi2(gb), hi2(x[i + 1]), J1);
            I1 = ffma2(lo2(gb), hi2(x[i + 1]), I1);
            I1 = ffma2(hi2(gb), lo2(x[i + 1]), I1);
        }
    }
    const float2 R = __fadd2_rn(R0, R1), J = __fadd2_rn(J0, J1), I = __fadd2_rn(I0, I1);
    return make_float2((R.x + R.y) - (J.x + J.y), I.x + I.y);
}

__device__ __forceinline__ void set_entry(float4& xp, int u, float re, float im)
{
    if (u & 1) {
        xp.y = re;
        xp.w = im;
    } else {
        xp.x = re;
        xp.z = im;
    }
}

// Phase B: K Gauss-Seidel sweeps x_u <- d_u (b_u - sum_v Gt_uv x_v), u = 0..U-1 ascending, from
// x = 0, with Gt the zero-diagonal rows at Grow ([UT][UT/2] float4), d_u at d[u] and b_u at
// b[u * bs] (all shared memory); one lane per tile holds x in registers (pair-planar).  In the first
// sweep every x_v with v >= u is still 0, so step u sums only the pairs holding some x_v, v < u
// (pairs [0, (u + 1) / 2)): a sixth of the work at K = 3, with the same result (the skipped terms
// are exact zeros).
template <int UT>
__device__ __forceinline__ void gram_sweeps(int U, int K, const float4* Grow, const float* d, const float2* b,
                                            uint32_t bs, float4 (&x)[UT / 2])
{
#pragma unroll
    for (int i = 0; i < UT / 2; ++i) x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (K < 1) return;
#pragma unroll
    for (int u = 0; u < UT; ++u) {
        if (u < U) {
            const float2 dot = gram_row_dot<UT>(Grow, u, (u + 1) / 2, x);
            const float2 bu = b[u * bs];
            const float du = d[u];
            set_entry(x[u >> 1], u, du * (bu.x - dot.x), du * (bu.y - dot.y));
        }
    }
#pragma unroll 1
    for (int t = 1; t < K; ++t) {
#pragma unroll
        for (int u = 0; u < UT; ++u) {
            if (u < U) {
                const float2 dot = gram_row_dot<UT>(Grow, u, UT / 2, x);
                const float2 bu = b[u * bs];
                const float du = d[u];
                set_entry(x[u >> 1], u, du * (bu.x - dot.x), du * (bu.y - dot.y));
            }
        }
    }
}

// Entry u of the tile's x from the slice a lane holds (valid on the lane with a == (u/2) / NPL).
template <int UT, int SB>
__device__ __forceinline__ float2 slice_entry(const float4 (&x)[UT / 2 / SB], int u)
{
    constexpr int NPL = UT / 2 / SB;
    const float4& xp = x[(u >> 1) % NPL];
    return (u & 1) ? make_float2(xp.y, xp.w) : make_float2(xp.x, xp.z);
}

// Phase B of the learned unfolded CD (one lane per tile): sweep t applies
// x_u <- x_u + tau_t (g - gamma_t alpha x_u) / (e_u + gamma_t alpha) with g = h_u^H r =
// b_u - sum_{v != u} Gt_uv x_v - e_u x_u, i.e. x_u <- a (b_u - sum_{v != u} Gt_uv x_v) + (1 - tau_t) x_u
// with a = tau_t / (e_u + gamma_t alpha); a non-positive denominator leaves x_u unchanged.
template <int UT>
__device__ __forceinline__ void gram_sweeps_learned(int U, int K, const float4* Grow, const float* e, float alpha,
                                                    const cdmimo_learned* blk, const float2* b, uint32_t bs,
                                                    float4 (&x)[UT / 2])
{
#pragma unroll
    for (int i = 0; i < UT / 2; ++i) x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    auto step = [&](int u, int npu, float tau, float ga) {
        const float2 dot = gram_row_dot<UT>(Grow, u, npu, x);
        const float2 bu = b[u * bs];
        const float den = e[u] + ga;
        const float a = den > 0.f ? tau * __fdividef(1.f, den) : 0.f;
        const float keep = den > 0.f ? 1.f - tau : 1.f;
        float4& xp = x[u >> 1];
        const float2 xo = (u & 1) ? make_float2(xp.y, xp.w) : make_float2(xp.x, xp.z);
        set_entry(xp, u, fmaf(a, bu.x - dot.x, keep * xo.x), fmaf(a, bu.y - dot.y, keep * xo.y));
    };
    if (K < 1) return;
    {  // first sweep from x = 0: pairs holding some x_v, v < u (as in gram_sweeps)
        const float tau = __ldg(&blk->tau[0]), ga = __ldg(&blk->gamma[0]) * alpha;
#pragma unroll
        for (int u = 0; u < UT; ++u)
            if (u < U) step(u, (u + 1) / 2, tau, ga);
    }
#pragma unroll 1
    for (int t = 1; t < K; ++t) {
        const float tau = __ldg(&blk->tau[t]), ga = __ldg(&blk->gamma[t]) * alpha;
#pragma unroll
        for (int u = 0; u < UT; ++u)
            if (u < U) step(u, UT / 2, tau, ga);
    }
}

// Shared-memory setup common to the Gram kernels: cluster table, barriers, zero padding columns of
// both channel buffers, and zeroed Gram rows / energies (entries past U are never written again).
template <int IN, int UT>
__device__ __forceinline__ void gram_setup(const CdPlan& pl, unsigned char* smem, ClusterTile* tab, uint64_t* bar,
                                           bool detect)
{
    const int tid = threadIdx.x;
    if (tid < pl.C) tab[tid] = pl.cl[tid];
    if (tid == 0 && pl.bulk) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async_smem();
    }
    float* g = reinterpret_cast<float*>(smem + pl.off_G);
    for (int i = tid; i < pl.C * UT * UT * 2; i += blockDim.x) g[i] = 0.f;
    float* e = reinterpret_cast<float*>(smem + pl.off_E);
    for (int i = tid; i < pl.C * UT; i += blockDim.x) e[i] = 0.f;
    // right-hand sides read by the padded steps: z rows U..UT-1 (uplink), or every s entry including
    // the row padding and UT entries past the last row (downlink); none of these is written again
    const uint32_t xs = x_stride(pl);
    float2* rhs = reinterpret_cast<float2*>(smem + (detect ? pl.off_X : pl.off_S));
    const int n_rhs = detect ? (UT - pl.U) * (int)xs : pl.n_sym * (pl.U | 1) + UT;
    if (detect) rhs += pl.U * xs;
    for (int i = tid; i < n_rhs; i += blockDim.x) rhs[i] = make_float2(0.f, 0.f);
    __syncthreads();
    if (IN == CDMIMO_C64 && pl.bulk) {  // 16-bit staging and the converting path write padding themselves
        zero_padding(pl, tab, reinterpret_cast<float2*>(smem));
        zero_padding(pl, tab, reinterpret_cast<float2*>(smem + pl.off_H2));
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Uplink: Algorithm 1 in Gram form + fusion (Sec. III).
// ---------------------------------------------------------------------------------------------
template <int IN, int AT, int UT, bool LEARNED>
__global__ void __maxnreg__(kPPRegs) cd_detect_gram_kernel(const CdPlan pl, const DetectIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    auto Hbuf = [&](int j) { return reinterpret_cast<float2*>(smem + ((IN == CDMIMO_C64 && j) ? pl.off_H2 : 0u)); };
    auto Stg = [&](int j) { return reinterpret_cast<void*>(smem + (j ? pl.off_H3 : pl.off_H2)); };
    auto Dst = [&](int j) { return IN == CDMIMO_C64 ? reinterpret_cast<void*>(Hbuf(j)) : Stg(j); };
    float4* Gs = reinterpret_cast<float4*>(smem + pl.off_G);  // [C][UT][UT/2]
    float* Ds = reinterpret_cast<float*>(smem + pl.off_E);    // [C][UT] m_u
    float2* Zs = reinterpret_cast<float2*>(smem + pl.off_X);  // [U][x_stride]: z, then each tile's x
    float* lam = reinterpret_cast<float*>(smem + pl.off_lam); // [C] w_c = 1 / sum_u m_{u,c}, or lambda_c
    float* Er = reinterpret_cast<float*>(smem + pl.off_E2);   // [C][UT] ||h_u||^2 (learned plans)
    float* mlp = reinterpret_cast<float*>(smem + pl.off_mlp); // [C][hidden] (learned fusion)
    const cdmimo_learned* blk = reinterpret_cast<const cdmimo_learned*>(io.learned);
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);  // [2]
    int* nxt = reinterpret_cast<int*>(smem + pl.off_bar + 16);       // [2] schedule hand-off

    const int tid = threadIdx.x;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    const uint32_t xs_stride = x_stride(pl);
    bool learned_ok = true;
    if (LEARNED) {
        const int hd = __ldg(&blk->hidden);
        learned_ok = __ldg(&blk->K) == pl.K && __ldg(&blk->U) == U && hd >= 1 && hd <= CDMIMO_MAX_HIDDEN;
        if (!learned_ok && tid == 0 && blockIdx.x == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_LEARNED);
    }
    gram_setup<IN, UT>(pl, smem, tab, bar, true);
    const GLane gz = gram_lane(C, n_sym, AT);  // phase A: (cluster, symbol) tiles, y in registers
    const GLane gb = gram_lane(C, n_sym, 1);   // phase B: one lane per (cluster, symbol)
    const GLane gg = gram_lane(C, U, AT);      // phase A: (cluster, user) tiles, Gram columns
    const ClusterTile ctz = tab[gz.c];

    int f = blockIdx.x;
    if (pl.bulk && tid == 0) {
        if (f < pl.n_sc) arm_channel_copy<IN>(pl, &bar[0]);
        if (f + (int)gridDim.x < pl.n_sc) arm_channel_copy<IN>(pl, &bar[1]);
    }
    __syncthreads();
    if (pl.bulk && f < pl.n_sc) issue_channel_copy<IN>(pl, tab, io.H, f, Dst(0), &bar[0]);
    float4 r[kPairs];
    if (gz.active && f < pl.n_sc)
        load_lane_raw<IN, AT>(io.Y, ((size_t)f * n_sym + gz.j) * pl.B + ctz.off, ctz.size, gz.a, r);

    int fn = f + (int)gridDim.x;
    int done = 0;
    for (int k = 0; f < pl.n_sc; ++k) {
        const int b = k & 1;
        const bool draw = fn < pl.n_sc;
        const unsigned ticket = sched_draw(io.sched, draw);
        if (pl.bulk && fn < pl.n_sc) issue_channel_copy<IN>(pl, tab, io.H, fn, Dst(b ^ 1), &bar[b ^ 1]);

        float alpha = __ldg(io.N0 + f) * pl.inv_Ex;
        float out_scale = 1.f;
        if (IN != CDMIMO_C64) {
            const float hs = __ldg(io.h_scale + f), ys = __ldg(io.y_scale + f);
            alpha = alpha / (hs * hs);
            out_scale = ys / hs;
        }
        if (!(alpha >= 0.f)) {
            if (tid == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_N0);
            out_scale = __int_as_float(0x7fc00000);
            alpha = 0.f;
        }
        if (LEARNED && !learned_ok) out_scale = __int_as_float(0x7fc00000);
        if (!acquire_channel<IN>(pl, tab, io.H, f, Hbuf(b), Stg(b), &bar[b], (uint32_t)(k >> 1) & 1u,
                                 io.sched != nullptr || fn + (int)gridDim.x < pl.n_sc)) {
            if (pl.bulk && fn < pl.n_sc && tid == 0) mbar_wait_bounded(&bar[b ^ 1], (uint32_t)((k + 1) >> 1) & 1u);
            break;
        }

        // Phase A: z = H_c^H y and the Gram columns.
        if (gz.active) {
            raw_to_pairs(r);
            gram_rhs<AT>(gz, U, n_sym, xs_stride, tab, Hbuf(b), r, Zs);
        }
        gram_columns<AT, UT>(gg, U, tab, Hbuf(b), alpha, Gs, Ds, nullptr, LEARNED ? Er : nullptr);
        if (tid == 0) nxt[b] = sched_next(io.sched, draw, ticket, fn, pl.n_sc);
        if (gz.active && fn < pl.n_sc)  // next subcarrier's y (r is free now)
            load_lane_raw<IN, AT>(io.Y, ((size_t)fn * n_sym + gz.j) * pl.B + ctz.off, ctz.size, gz.a, r);
        __syncthreads();

        // Phase B: the sweeps; the symbol-0 lane of each cluster also forms the fusion weight
        // w_c = 1 / sum_u m_u (a skipped column, m_u = 0, counts as infinite).  One lane per tile:
        // splitting x over lanes puts a shuffle on the step-to-step dependency chain (measured slower).
        if (gb.active) {
            const int tile = gb.c * n_sym + gb.j;
            const float* d = Ds + gb.c * UT;
            float4 x[UT / 2];
            if (LEARNED)
                gram_sweeps_learned<UT>(U, learned_ok ? pl.K : 0, Gs + (size_t)gb.c * UT * (UT / 2), Er + gb.c * UT,
                                        alpha, blk, Zs + tile, xs_stride, x);
            else
                gram_sweeps<UT>(U, pl.K, Gs + (size_t)gb.c * UT * (UT / 2), d, Zs + tile, xs_stride, x);
#pragma unroll
            for (int u = 0; u < UT; ++u)  // own tile column: z is no longer read
                if (u < U) Zs[u * xs_stride + tile] = slice_entry<UT, 1>(x, u);
            if (gb.j == 0) {
                float msum = 0.f;
                for (int u = 0; u < U; ++u) msum += d[u] > 0.f ? d[u] : __int_as_float(0x7f800000);
                lam[gb.c] = 1.f / msum;
            }
        }
        __syncthreads();

        // Phase C: fusion.  The next writes of Zs, Gs, Ds and lam come after the next acquire's
        // barriers, and the copy into this iteration's channel buffer after the barrier above.
        if (LEARNED && pl.fuse == CDMIMO_FUSE_LEARNED) {
            learned_lambda(pl, blk, learned_ok, alpha, tab, mlp, lam, io.lam, f,
                           [&](int c, int j) { return Er[c * UT + j]; });
            __syncthreads();
            fuse_subcarrier<true>(pl, io, f, lam, Zs, xs_stride, out_scale);
        } else {
            fuse_subcarrier<false>(pl, io, f, lam, Zs, xs_stride, out_scale);
        }
        ++done;
        f = fn;
        fn = nxt[b];
    }
    sched_finish(io.sched, done, pl.n_sc);
}

// ---------------------------------------------------------------------------------------------
// Downlink: Algorithm 2 / Eq. (4) in Gram form + normalization (Sec. IV-B).
// ---------------------------------------------------------------------------------------------
template <int IN, int AT, int UT>
__global__ void __maxnreg__(kPPRegs) cd_precode_gram_kernel(const CdPlan pl, const PrecodeIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    auto Hbuf = [&](int j) { return reinterpret_cast<float2*>(smem + ((IN == CDMIMO_C64 && j) ? pl.off_H2 : 0u)); };
    auto Stg = [&](int j) { return reinterpret_cast<void*>(smem + (j ? pl.off_H3 : pl.off_H2)); };
    auto Dst = [&](int j) { return IN == CDMIMO_C64 ? reinterpret_cast<void*>(Hbuf(j)) : Stg(j); };
    float4* Gs = reinterpret_cast<float4*>(smem + pl.off_G);  // [C][UT][UT/2]
    float* Ds = reinterpret_cast<float*>(smem + pl.off_E);    // [C][UT] p_u^2
    float2* Ws = reinterpret_cast<float2*>(smem + pl.off_X);  // [U][x_stride] w per tile
    float2* Ss = reinterpret_cast<float2*>(smem + pl.off_S);  // [n_sym][U | 1]
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);
    int* nxt = reinterpret_cast<int*>(smem + pl.off_bar + 16);

    const int tid = threadIdx.x;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    const int s_stride = U | 1;
    const int n_s = n_sym * U;
    const uint32_t xs_stride = x_stride(pl);
    constexpr int LP = AT * kPairs;
    gram_setup<IN, UT>(pl, smem, tab, bar, false);
    const GLane gg = gram_lane(C, U, AT);      // phase A
    const GLane gb = gram_lane(C, n_sym, 1);   // phase B: one lane per (cluster, symbol)
    const GLane gx = gram_lane(C, n_sym, AT);  // phase C: (cluster, symbol) tiles over antenna lanes

    int f = blockIdx.x;
    if (pl.bulk && tid == 0) {
        if (f < pl.n_sc) arm_channel_copy<IN>(pl, &bar[0]);
        if (f + (int)gridDim.x < pl.n_sc) arm_channel_copy<IN>(pl, &bar[1]);
    }
    __syncthreads();
    if (pl.bulk && f < pl.n_sc) issue_channel_copy<IN>(pl, tab, io.H, f, Dst(0), &bar[0]);
    float2 sv[kSPrefetch];
#pragma unroll
    for (int q = 0; q < kSPrefetch; ++q) {
        const int i = tid + q * blockDim.x;
        sv[q] = (i < n_s && f < pl.n_sc) ? __ldg(io.S + (size_t)f * n_s + i) : make_float2(0.f, 0.f);
    }

    int fn = f + (int)gridDim.x;
    int done = 0;
    for (int k = 0; f < pl.n_sc; ++k) {
        const int b = k & 1;
        const bool draw = fn < pl.n_sc;
        const unsigned ticket = sched_draw(io.sched, draw);
        if (pl.bulk && fn < pl.n_sc) issue_channel_copy<IN>(pl, tab, io.H, fn, Dst(b ^ 1), &bar[b ^ 1]);
#pragma unroll
        for (int q = 0; q < kSPrefetch; ++q) {
            const int i = tid + q * blockDim.x;
            if (i < n_s) {
                const int n = i / U;
                Ss[n * s_stride + (i - n * U)] = sv[q];
            }
        }
        if (!acquire_channel<IN>(pl, tab, io.H, f, Hbuf(b), Stg(b), &bar[b], (uint32_t)(k >> 1) & 1u,
                                 io.sched != nullptr || fn + (int)gridDim.x < pl.n_sc)) {
            if (pl.bulk && fn < pl.n_sc && tid == 0) mbar_wait_bounded(&bar[b ^ 1], (uint32_t)((k + 1) >> 1) & 1u);
            break;
        }
#pragma unroll
        for (int q = 0; q < kSPrefetch; ++q) {
            const int i = tid + q * blockDim.x;
            if (i < n_s && fn < pl.n_sc) sv[q] = __ldg(io.S + (size_t)fn * n_s + i);
        }

        // Phase A: Gram columns.
        gram_columns<AT, UT>(gg, U, tab, Hbuf(b), 0.f, Gs, Ds);
        if (tid == 0) nxt[b] = sched_next(io.sched, draw, ticket, fn, pl.n_sc);
        __syncthreads();

        // Phase B: sweeps on w with p_u^2 = ||h_u||^{-2} (0 for a zero column).
        if (gb.active) {
            const int tile = gb.c * n_sym + gb.j;
            float4 w[UT / 2];
            gram_sweeps<UT>(U, pl.K, Gs + (size_t)gb.c * UT * (UT / 2), Ds + gb.c * UT, Ss + gb.j * s_stride, 1u, w);
#pragma unroll
            for (int u = 0; u < UT; ++u)
                if (u < U) Ws[u * xs_stride + tile] = slice_entry<UT, 1>(w, u);
        }
        __syncthreads();

        // Phase C: x_c = H_c w, then x_c <- rho_c x_c / ||x_c||.
        if (gx.active) {
            const ClusterTile ct = tab[gx.c];
            const float4* hb = reinterpret_cast<const float4*>(Hbuf(b) + ct.soff) + gx.a;
            const float2* wt = Ws + gx.c * n_sym + gx.j;
            float4 x[kPairs];
#pragma unroll
            for (int i = 0; i < kPairs; ++i) x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
            for (int v = 0; v < U; ++v) {
                float4 h[kPairs];
                pp_load_h<AT>(hb + v * LP, h);
                const float2 wv = wt[v * xs_stride];
                pp_update(h, make_float2(-wv.x, -wv.y), x);  // x += h_v w_v
            }
            float nr = 0.f;
#pragma unroll
            for (int i = 0; i < kPairs; ++i)
                nr = fmaf(x[i].x, x[i].x, fmaf(x[i].y, x[i].y, fmaf(x[i].z, x[i].z, fmaf(x[i].w, x[i].w, nr))));
            nr = tile_sum_c<AT>(nr, gx.mask);
            const float sc = nr > 0.f ? pl.rho_c * rsqrtf(nr) : 0.f;
            float2* out = io.Xdl + ((size_t)f * n_sym + gx.j) * pl.B + ct.off;
#pragma unroll
            for (int i = 0; i < kPairs; ++i) {
                const int col = 2 * (i * AT + gx.a);
                if (col < ct.size) out[col] = make_float2(x[i].x * sc, x[i].z * sc);
                if (col + 1 < ct.size) out[col + 1] = make_float2(x[i].y * sc, x[i].w * sc);
            }
        }
        __syncthreads();  // Ss, Ws and this channel buffer are rewritten next
        ++done;
        f = fn;
        fn = nxt[b];
    }
    sched_finish(io.sched, done, pl.n_sc);
}

}  // namespace cdmimo

