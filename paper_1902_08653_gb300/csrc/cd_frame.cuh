// TDD frame kernel: uplink detection (Algorithm 1 + fusion, Sec. III) and downlink precoding
// (Algorithm 2 + normalization, Sec. IV-B) on one channel per subcarrier (the downlink channel is
// the transpose of the uplink one, Sec. IV), both in Gram form (see cd_gram.cuh), sharing one
// channel copy and one G_c.
//
// Register blocking.  Shared memory delivers 4 bytes per lane and cycle whether or not lanes read
// the same address, so a 16-byte channel pair costs four cycles of the SM's shared-memory pipe
// while the four packed FMAs it feeds take two cycles of its FP32 pipes: loops that use each
// loaded pair for one vector run at half the FP32 rate.  Here every loaded value feeds two vectors:
//   phase A  one lane set correlates h_u with two receive vectors (two symbols) for z, while the
//            other half of the CTA correlates h_u with two channel columns for G_c;
//   phase B  one lane per uplink or downlink (cluster, symbol) runs the sweeps (latency-bound: here
//            one vector per lane on every warp beats two vectors per lane on half of them);
//   phase C  x_c = H_c w for two symbols per lane, while the other half of the CTA fuses the uplink
//            estimates.
#pragma once
#include "cd_gram.cuh"

namespace cdmimo {

// Lane of a phase that runs on the CTA's threads [t0, t0 + 32 W): C x J tiles of AT lanes spread
// evenly over W warps, W the smallest multiple of four that holds them and at least w_min.
__device__ __forceinline__ GLane frame_lane(int t0, int C, int J, int AT, int w_min = 0)
{
    const int L = C * J * AT;
    const int W = max(((L + 31) / 32 + 3) / 4 * 4, w_min);
    const int lpw = ((L + W - 1) / W + AT - 1) / AT * AT;
    const int rel = (int)threadIdx.x - t0;
    const int w = rel >> 5, l = rel & 31, v = w * lpw + l;
    GLane g;
    g.active = rel >= 0 && w < W && l < lpw && v < L;
    const int t = g.active ? v / AT : 0;
    g.a = g.active ? v - t * AT : 0;
    g.c = t / J;
    g.j = t - g.c * J;
    const int n_act = min(lpw, L - w * lpw);
    g.mask = n_act >= 32 ? 0xffffffffu : (n_act > 0 ? (1u << n_act) - 1u : 0u);
    return g;
}

// Lane partials of conj(h)^T v0 and conj(h)^T v1 over the lane's pairs; h is read from shared
// memory one 16-byte pair at a time and feeds eight packed FMAs (one accumulator set per vector:
// with both vectors in registers, a second set would spill).
template <int AT>
__device__ __forceinline__ void corr2(const float4* hr, const float4 (&v0)[kPairs], const float4 (&v1)[kPairs],
                                      float2& s0, float2& s1)
{
    const float2 z = make_float2(0.f, 0.f);
    float2 R0 = z, I0 = z, J0 = z, R1 = z, I1 = z, J1 = z;
#pragma unroll
    for (int i = 0; i < kPairs; ++i) {
        const float4 h = hr[i * AT];
        R0 = ffma2(lo2(h), lo2(v0[i]), R0);
        I0 = ffma2(lo2(h), hi2(v0[i]), I0);
        J0 = ffma2(hi2(h), lo2(v0[i]), J0);
        R1 = ffma2(lo2(h), lo2(v1[i]), R1);
        I1 = ffma2(lo2(h), hi2(v1[i]), I1);
        J1 = ffma2(hi2(h), lo2(v1[i]), J1);
        R0 = ffma2(hi2(h), hi2(v0[i]), R0);
        R1 = ffma2(hi2(h), hi2(v1[i]), R1);
    }
    s0 = make_float2(R0.x + R0.y, (I0.x + I0.y) - (J0.x + J0.y));
    s1 = make_float2(R1.x + R1.y, (I1.x + I1.y) - (J1.x + J1.y));
}

// Data fusion (Sec. III) of one subcarrier on the CTA's threads [t0, t0 + nt): lam holds
// w_c = 1 / sum_u m_{u,c}; lambda_c = w_c / sum w (COLNORM) or 1 / C (EQUAL, or no positive weight).
// final_lam: lam already holds lambda_c (the learned fusion's softmax), used as it is.
__device__ __forceinline__ void fuse_range(const CdPlan& pl, const DetectIO& io, int f, const float* lam,
                                           const float2* Xs, uint32_t xs_stride, float out_scale, int t0, int nt,
                                           bool final_lam = false)
{
    const int r = (int)threadIdx.x - t0, C = pl.C, U = pl.U, n_sym = pl.n_sym;
    if (r < 0 || r >= nt) return;
    float tot = 0.f;
    for (int c = 0; c < C && !final_lam; ++c) tot += lam[c];
    const bool equal = !final_lam && (pl.fuse == CDMIMO_FUSE_EQUAL || !(tot > 0.f));
    const float inv = final_lam ? 1.f : equal ? 1.f / (float)C : 1.f / tot;
    for (int i = r; i < n_sym * U; i += nt) {  // symbols fastest: a warp's loads of x hit distinct banks
        const int u = i / n_sym, n = i - u * n_sym;
        float2 acc = make_float2(0.f, 0.f);
        for (int c = 0; c < C; ++c) {
            const float l = equal ? inv : lam[c] * inv;
            const float2 xv = Xs[u * xs_stride + c * n_sym + n];
            acc.x = fmaf(l, xv.x, acc.x);
            acc.y = fmaf(l, xv.y, acc.y);
        }
        io.Xhat[((size_t)f * n_sym + n) * U + u] = make_float2(acc.x * out_scale, acc.y * out_scale);
    }
}

// x += h_v w for two vectors, h read pair by pair (each 16-byte load feeds eight packed FMAs).
template <int AT>
__device__ __forceinline__ void axpy2(const float4* hr, float2 w0, float2 w1, float4 (&a0)[kPairs], float4 (&a1)[kPairs])
{
    const float2 r0 = make_float2(w0.x, w0.x), i0 = make_float2(w0.y, w0.y), n0 = make_float2(-w0.y, -w0.y);
    const float2 r1 = make_float2(w1.x, w1.x), i1 = make_float2(w1.y, w1.y), n1 = make_float2(-w1.y, -w1.y);
#pragma unroll
    for (int i = 0; i < kPairs; ++i) {
        const float4 h = hr[i * AT];
        // (h_re + i h_im)(w_re + i w_im): re += h_re w_re - h_im w_im, im += h_re w_im + h_im w_re
        float2 re = ffma2(lo2(h), r0, lo2(a0[i]));
        float2 im = ffma2(lo2(h), i0, hi2(a0[i]));
        re = ffma2(hi2(h), n0, re);
        im = ffma2(hi2(h), r0, im);
        a0[i] = cat4(re, im);
        re = ffma2(lo2(h), r1, lo2(a1[i]));
        im = ffma2(lo2(h), i1, hi2(a1[i]));
        re = ffma2(hi2(h), n1, re);
        im = ffma2(hi2(h), r1, im);
        a1[i] = cat4(re, im);
    }
}

// Writes rho_c x / ||x|| (the tile's norm over its AT lanes; a zero x stays zero) for one symbol.
template <int AT>
__device__ __forceinline__ void store_normalized(const float4 (&x)[kPairs], float rho_c, unsigned mask, int a,
                                                 int size, float2* out, bool valid)
{
    float nr = 0.f;
#pragma unroll
    for (int i = 0; i < kPairs; ++i)
        nr = fmaf(x[i].x, x[i].x, fmaf(x[i].y, x[i].y, fmaf(x[i].z, x[i].z, fmaf(x[i].w, x[i].w, nr))));
    nr = tile_sum_c<AT>(nr, mask);
    const float sc = nr > 0.f ? rho_c * rsqrtf(nr) : 0.f;
    if (!valid) return;
#pragma unroll
    for (int i = 0; i < kPairs; ++i) {
        const int col = 2 * (i * AT + a);
        if (col < size) out[col] = make_float2(x[i].x * sc, x[i].z * sc);
        if (col + 1 < size) out[col + 1] = make_float2(x[i].y * sc, x[i].w * sc);
    }
}

// Warps of a phase with L lanes (a multiple of four).
__host__ __device__ inline int frame_warps(int L) { return ((L + 31) / 32 + 3) / 4 * 4; }

template <int IN, int AT, int UT>
__global__ void __maxnreg__(kPPRegs) cd_frame_gram_kernel(const CdPlan pl, const FusedIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    auto Hbuf = [&](int j) { return reinterpret_cast<float2*>(smem + ((IN == CDMIMO_C64 && j) ? pl.off_H2 : 0u)); };
    auto Stg = [&](int j) { return reinterpret_cast<void*>(smem + (j ? pl.off_H3 : pl.off_H2)); };
    auto Dst = [&](int j) { return IN == CDMIMO_C64 ? reinterpret_cast<void*>(Hbuf(j)) : Stg(j); };
    float4* Gs = reinterpret_cast<float4*>(smem + pl.off_G);  // [C][UT][UT/2]
    float* Dm = reinterpret_cast<float*>(smem + pl.off_E);    // [C][UT] m_u
    float* Dp = reinterpret_cast<float*>(smem + pl.off_E2);   // [C][UT] p_u^2
    float2* Zs = reinterpret_cast<float2*>(smem + pl.off_X);  // [U][x_stride]: z, then each tile's x
    float2* Ws = reinterpret_cast<float2*>(smem + pl.off_W);  // [U][x_stride]: w per tile
    float2* Ss = reinterpret_cast<float2*>(smem + pl.off_S);  // [U][n_sym]: s of the subcarrier, transposed
    float* lam = reinterpret_cast<float*>(smem + pl.off_lam);
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);
    int* nxt = reinterpret_cast<int*>(smem + pl.off_bar + 16);
    const DetectIO& d = io.d;

    const int tid = threadIdx.x;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    const uint32_t xs = x_stride(pl);
    constexpr int LP = AT * kPairs;
    gram_setup<IN, UT>(pl, smem, tab, bar, true);
    const int NS2 = (n_sym + 1) / 2, NU2 = (U + 1) / 2;
    const int t_g = 32 * frame_warps(C * NS2 * AT);  // first thread of the Gram-column lanes
    const GLane gz = frame_lane(0, C, NS2, AT);     // symbol pairs: z (phase A), H w (phase C)
    const GLane gg = frame_lane(t_g, C, NU2, AT);   // column pairs of G_c (phase A); fusion (phase C)
    // phase B: one lane per uplink or downlink tile; tile (c, j) is uplink symbol j for j < n_sym and
    // downlink symbol j - n_sym otherwise, so one warp holds both kinds of tiles of a cluster and they
    // read the same rows of G_c.  (One lane sweeping both x and w halves the row loads but leaves half
    // the warps idle; the sweeps are latency-bound and that measured slower.)
    const GLane gb = frame_lane(0, C, 2 * n_sym, 1);
    const ClusterTile ctz = tab[gz.c];
    const int zn0 = 2 * gz.j, zn1 = zn0 + 1;

    // Schedule: CTA i starts with subcarrier i; its next one is decided during the sweeps of the
    // current one (static: + gridDim; dynamic: gridDim + a ticket drawn from the workspace counter),
    // and that channel's copy is issued at the start of phase C into the other buffer, to be waited
    // for at the next acquire.  Deciding this late lets a CTA that runs faster than its SM partner
    // take more of the remaining subcarriers.
    int f = blockIdx.x;
    if (pl.bulk && tid == 0 && f < pl.n_sc) arm_channel_copy<IN>(pl, &bar[0]);
    __syncthreads();
    if (pl.bulk && f < pl.n_sc) issue_channel_copy<IN>(pl, tab, d.H, f, Dst(0), &bar[0]);
    const int n_s = n_sym * U;
    // s is stored [u][n] so that a warp's lanes (consecutive symbols) read consecutive words
    auto put_s = [&](int i, float2 v) { Ss[(i % U) * n_sym + i / U] = v; };
    if (f < pl.n_sc)
        for (int i = tid; i < n_s; i += blockDim.x) put_s(i, io.S[(size_t)f * n_s + i]);
    float4 y0[kPairs], y1[kPairs];
    auto load_y = [&](int fy) {
        const size_t base = (size_t)fy * n_sym * pl.B + ctz.off;
        load_lane_raw<IN, AT>(d.Y, base + (size_t)zn0 * pl.B, ctz.size, gz.a, y0);
        if (zn1 < n_sym) load_lane_raw<IN, AT>(d.Y, base + (size_t)zn1 * pl.B, ctz.size, gz.a, y1);
        else load_lane_raw<IN, AT>(d.Y, base, 0, gz.a, y1);  // size 0: zeros
    };

    int done = 0;
    for (int k = 0; f < pl.n_sc; ++k) {
        const int b = k & 1;

        float alpha = __ldg(d.N0 + f) * pl.inv_Ex;
        float out_scale = 1.f;
        if (IN != CDMIMO_C64) {
            const float hs = __ldg(d.h_scale + f), ys = __ldg(d.y_scale + f);
            alpha = alpha / (hs * hs);
            out_scale = ys / hs;
        }
        if (!(alpha >= 0.f)) {
            if (tid == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_N0);
            out_scale = __int_as_float(0x7fc00000);
            alpha = 0.f;
        }
        if (!acquire_channel<IN>(pl, tab, d.H, f, Hbuf(b), Stg(b), &bar[b], (uint32_t)(k >> 1) & 1u, false)) {
            // copy timeout: no other copy is in flight; give this one a last bounded wait, then stop
            if (pl.bulk && tid == 0) mbar_wait_bounded(&bar[b], (uint32_t)(k >> 1) & 1u);
            break;
        }

        // Phase A: z for two symbols per lane | Gram columns, two per lane, with m_u and p_u^2.  The
        // symbol lanes load their y here (prefetching it across the iteration or the acquire keeps 64
        // more registers live and spills); the Gram-column warps run meanwhile.
        if (gz.active) {
            load_y(f);
            raw_to_pairs(y0);
            raw_to_pairs(y1);
            const float4* hb = reinterpret_cast<const float4*>(Hbuf(b) + ctz.soff) + gz.a;
            float2* z = Zs + gz.c * n_sym;
#pragma unroll 2
            for (int u = 0; u < U; ++u) {
                float2 s0, s1;
                corr2<AT>(hb + u * LP, y0, y1, s0, s1);
                s0.x = tile_sum_c<AT>(s0.x, gz.mask);
                s0.y = tile_sum_c<AT>(s0.y, gz.mask);
                s1.x = tile_sum_c<AT>(s1.x, gz.mask);
                s1.y = tile_sum_c<AT>(s1.y, gz.mask);
                if (gz.a == 0) {
                    z[u * xs + zn0] = s0;
                    if (zn1 < n_sym) z[u * xs + zn1] = s1;
                }
            }
        } else if (gg.active) {
            const ClusterTile ct = tab[gg.c];
            const float4* hb = reinterpret_cast<const float4*>(Hbuf(b) + ct.soff) + gg.a;
            const int v0 = 2 * gg.j, v1 = v0 + 1;
            float4 h0[kPairs], h1[kPairs];
            pp_load_h<AT>(hb + v0 * LP, h0);
            if (v1 < U) pp_load_h<AT>(hb + v1 * LP, h1);
            else {
#pragma unroll
                for (int i = 0; i < kPairs; ++i) h1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float* G = reinterpret_cast<float*>(Gs + (size_t)gg.c * UT * (UT / 2));
            const int col = (v0 >> 1) * 4;  // v0 even: columns v0, v1 are the pair's two halves
#pragma unroll 2
            for (int u = 0; u < U; ++u) {
                float2 s0, s1;
                corr2<AT>(hb + u * LP, h0, h1, s0, s1);
                s0.x = tile_sum_c<AT>(s0.x, gg.mask);
                s0.y = tile_sum_c<AT>(s0.y, gg.mask);
                s1.x = tile_sum_c<AT>(s1.x, gg.mask);
                s1.y = tile_sum_c<AT>(s1.y, gg.mask);
                if (gg.a == 0) {
                    if (u == v0 || u == v1) {  // diagonal: m_u, p_u^2; the stored entry is 0
                        const float e = u == v0 ? s0.x : s1.x, den = e + alpha;
                        Dm[gg.c * UT + u] = den > 0.f ? __fdividef(1.f, den) : 0.f;
                        Dp[gg.c * UT + u] = e > 0.f ? __fdividef(1.f, e) : 0.f;
                        if (u == v0) s0 = make_float2(0.f, 0.f);
                        else s1 = make_float2(0.f, 0.f);
                    }
                    G[u * (2 * UT) + col] = s0.x;
                    G[u * (2 * UT) + col + 2] = s0.y;
                    if (v1 < U) {
                        G[u * (2 * UT) + col + 1] = s1.x;
                        G[u * (2 * UT) + col + 3] = s1.y;
                    }
                }
            }
        }
        __syncthreads();

        // Phase B: uplink sweeps on x (right-hand side z) and downlink sweeps on w (right-hand side s),
        // both read from shared memory.  Thread 0 draws the next
        // subcarrier now and hands it over before the barrier below (the atomic's latency is hidden).
        const unsigned ticket = (d.sched && tid == 0) ? atomicAdd(d.sched, 1u) : 0u;
        if (gb.active) {
            const bool ul = gb.j < n_sym;
            const int n = ul ? gb.j : gb.j - n_sym;
            const int tile = gb.c * n_sym + n;
            const float* dd = (ul ? Dm : Dp) + gb.c * UT;
            const float2* rhs = ul ? Zs + tile : Ss + n;
            float4 x[UT / 2];
            gram_sweeps<UT>(U, pl.K, Gs + (size_t)gb.c * UT * (UT / 2), dd, rhs, ul ? xs : (uint32_t)n_sym, x);
            float2* dst = (ul ? Zs : Ws) + tile;
#pragma unroll
            for (int u = 0; u < UT; ++u)
                if (u < U) dst[u * xs] = slice_entry<UT, 1>(x, u);
            if (ul && n == 0) {
                float msum = 0.f;
                for (int u = 0; u < U; ++u) msum += dd[u] > 0.f ? dd[u] : __int_as_float(0x7f800000);
                lam[gb.c] = 1.f / msum;
            }
        }
        if (tid == 0) {
            int nf = f + (int)gridDim.x;
            if (d.sched) {
                const unsigned v = gridDim.x + ticket;
                nf = v < (unsigned)pl.n_sc ? (int)v : pl.n_sc;
            }
            nxt[b] = nf;
            if (pl.bulk && nf < pl.n_sc) arm_channel_copy<IN>(pl, &bar[b ^ 1]);
        }
        __syncthreads();

        // Phase C: the next subcarrier's channel copy (into the other buffer, last read in the
        // previous iteration) and its y into L2; x_c = H_c w for two symbols per lane, then the
        // normalization | uplink fusion and the next subcarrier's s into shared memory (this one's
        // was last read in phase B; the loads are issued before the fusion and stored after it).
        const int fn = nxt[b];
        if (pl.bulk && fn < pl.n_sc) issue_channel_copy<IN>(pl, tab, d.H, fn, Dst(b ^ 1), &bar[b ^ 1]);
        if (tid == 32 && fn < pl.n_sc) {
            constexpr uint32_t eb = IN == CDMIMO_C64 ? 8u : 4u;
            bulk_prefetch_l2(static_cast<const char*>(d.Y) + (size_t)fn * n_sym * pl.B * eb, (uint32_t)n_sym * pl.B * eb);
        }
        if (gz.active) {
            const float4* hb = reinterpret_cast<const float4*>(Hbuf(b) + ctz.soff) + gz.a;
            const float2* w0 = Ws + gz.c * n_sym + zn0;
            const bool has1 = zn1 < n_sym;
            float4 a0[kPairs], a1[kPairs];
#pragma unroll
            for (int i = 0; i < kPairs; ++i) {
                a0[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                a1[i] = a0[i];
            }
#pragma unroll 1
            for (int v = 0; v < U; ++v)
                axpy2<AT>(hb + v * LP, w0[v * xs], has1 ? w0[v * xs + 1] : make_float2(0.f, 0.f), a0, a1);
            float2* out = io.Xdl + ((size_t)f * n_sym + zn0) * pl.B + ctz.off;
            store_normalized<AT>(a0, pl.rho_c, gz.mask, gz.a, ctz.size, out, true);
            store_normalized<AT>(a1, pl.rho_c, gz.mask, gz.a, ctz.size, out + pl.B, has1);
        } else {
            constexpr int kSv = 2;  // entries of the next s per thread kept in flight across the fusion
            const int r = tid - t_g, nr = (int)blockDim.x - t_g;
            const bool ld = r >= 0 && fn < pl.n_sc;
            const float2* src = io.S + (size_t)min(fn, pl.n_sc - 1) * n_s;
            float2 sv[kSv];
#pragma unroll
            for (int q = 0; q < kSv; ++q)
                sv[q] = (ld && r + q * nr < n_s) ? src[r + q * nr] : make_float2(0.f, 0.f);
            fuse_range(pl, d, f, lam, Zs, xs, out_scale, t_g, nr);
            if (ld) {
#pragma unroll
                for (int q = 0; q < kSv; ++q)
                    if (r + q * nr < n_s) put_s(r + q * nr, sv[q]);
                for (int i = r + kSv * nr; i < n_s; i += nr) put_s(i, src[i]);
            }
        }
        __syncthreads();  // this channel buffer receives the copy issued at the next iteration's start
        ++done;
        f = fn;
    }
    sched_finish(d.sched, done, pl.n_sc);
}

}  // namespace cdmimo
