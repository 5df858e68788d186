// Gram-form CD kernel with the contractions on the tensor cores, for the TDD frame (uplink detection,
// Algorithm 1 + fusion of Sec. III, and downlink precoding, Algorithm 2 + normalization of
// Sec. IV-B, on one channel per subcarrier, like cd_frame_gram_kernel), for either direction alone,
// and for the learned uplink.  In Gram form (see cd_gram.cuh),
//   z = H_c^H y_c,  G_c = H_c^H H_c  (phase A)   and   x_c = H_c w  (phase C)
// are computed by warp-level tensor-core MMAs (mma.sync m16n8k8, TF32 operands, FP32 accumulation),
// one warp per cluster.  The sweeps (phase B) are FP32 Gauss-Seidel steps, one lane per (cluster,
// symbol); in the frame that lane runs the uplink and the downlink vector side by side.
//
// FP32 accuracy from TF32 operands.  Every FP32 operand x is split as x = hi + lo, hi = x with its
// 13 low mantissa bits cleared (a TF32 value) and lo = x - hi (exact in FP32, |lo| < 2^-10 |x|); the
// MMA reads a TF32 operand from its upper 19 bits, so lo enters with an error below 2^-10 of itself,
// 2^-20 of x.  Every product is accumulated as lo_a hi_b + hi_a lo_b + hi_a hi_b (the lo_a lo_b
// term, below 2^-20 |a b|, is dropped): three MMAs per tile, with no conversion instructions.
//
// Complex products as real MMAs.  Each k-step of 8 real values covers four complex entries e:
// k = t is Re of entry e0 + t and k = t + 4 is Im of it (t = 0..3), so a lane's two values of a
// fragment (k = tig and tig + 4) come from one 64-bit load of a complex entry.  Then
//   Re(h_u^H v) = sum_k h_u[k] v[k]            Im(h_u^H v) = sum_k h_u[k] rot(v)[k]
// with rot(v) = (Im v, -Re v) per entry: one contraction gives both parts, the second with the B
// operand rotated (from the same loaded value).  For x_c = H_c w the entries are the users:
// Re x_b = sum_k h^T[b][k] (Re w, -Im w)[k], Im x_b = sum_k h^T[b][k] (Im w, Re w)[k].
//
// Shared memory.  The channel rows of a cluster are UT = 16 rows (rows U..15 zero) of 2 B_c + 8
// floats: with that stride the 64-bit fragment loads of both phases (rows gid x entries tig, and
// users tig x antennas gid) fall on distinct banks.  The rows land in that layout by one bulk copy
// per row, double-buffered one subcarrier ahead as in the SIMT kernel; no permutation pass follows.
// In the frame, the downlink's w per tile takes the place of the Gram rows once the sweeps are over
// (a barrier separates the two), which keeps two CTAs per SM; the downlink alone keeps w where the
// uplink's z and x would be.  Per-tile rows (z, x, w) have a stride of 4 mod 16 entries, so that
// phase C's loads of w (users tig x symbols gid) are conflict-free too.
#pragma once
#include "cd_frame.cuh"

namespace cdmimo {

constexpr int kTcUT = 16;        // users per cluster in the MMA tiles (rows U..15 are zero)
constexpr int kTcThreads = 256;  // eight warps: one per cluster in phases A and C
// What one launch computes: the TDD frame, the uplink alone (cdmimo_detect), the downlink alone
// (cdmimo_precode), or the uplink with the learned sweeps and fusion of a cdmimo_learned block.
// Each mode compiles only its own steps.
constexpr int kTcFrame = 0, kTcDetect = 1, kTcPrecode = 2, kTcDetectLearned = 3;

// x = hi + lo (see above); the negated split of -x is the two values with the sign bit flipped.
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo)
{
    const uint32_t h = __float_as_uint(x) & 0xffffe000u;
    hi = h;
    lo = __float_as_uint(x - __uint_as_float(h));
}

__device__ __forceinline__ uint32_t neg_bits(uint32_t v) { return v ^ 0x80000000u; }

// One B fragment (k = tig, tig + 4) in TF32 halves.
struct BFrag {
    uint32_t h[2], l[2];
};

// d += A B for one m16n8k8 tile (A row-major 16 x 8, B 8 x 8 "col"), TF32 in, FP32 accumulate.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += A B with FP32-accurate operands (three passes, smallest terms first).
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                           const BFrag& b)
{
    mma_tf32(d, al, b.h[0], b.h[1]);
    mma_tf32(d, ah, b.l[0], b.l[1]);
    mma_tf32(d, ah, b.h[0], b.h[1]);
}

// A fragment (rows r0 and r0 + 8 of a k-step) from two complex entries: k = tig is Re, tig + 4 Im.
__device__ __forceinline__ void a_frag(float2 e0, float2 e1, uint32_t (&ah)[4], uint32_t (&al)[4])
{
    tf32_split(e0.x, ah[0], al[0]);
    tf32_split(e1.x, ah[1], al[1]);
    tf32_split(e0.y, ah[2], al[2]);
    tf32_split(e1.y, ah[3], al[3]);
}

// B fragments of a complex entry v for the plain and the rotated operand: (Re v, Im v) and
// (Im v, -Re v) as (k = tig, k = tig + 4) values, split into TF32 halves.
__device__ __forceinline__ void b_frags(float2 v, BFrag& plain, BFrag& rot)
{
    tf32_split(v.x, plain.h[0], plain.l[0]);
    tf32_split(v.y, plain.h[1], plain.l[1]);
    rot.h[0] = plain.h[1];
    rot.l[0] = plain.l[1];
    rot.h[1] = neg_bits(plain.h[0]);
    rot.l[1] = neg_bits(plain.l[0]);
}

// The learned sweeps of gram_sweeps_learned, x_u <- a_{t,u} (b_u - sum_{v != u} Gt_uv x_v) +
// keep_{t,u} x_u, with (a, keep)_{t,u} = (tau_t / (e_u + gamma_t alpha), 1 - tau_t) (or (0, 1) for a
// non-positive denominator) read from the cluster's table co[t][UT] instead of formed at every step.
template <int UT>
__device__ __forceinline__ void gram_sweeps_learned_tab(int U, int K, const float4* Grow, const float2* co,
                                                        const float2* b, uint32_t bs, float4 (&x)[UT / 2])
{
#pragma unroll
    for (int i = 0; i < UT / 2; ++i) x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    auto step = [&](int u, int npu, const float2* ct) {
        const float2 dot = gram_row_dot<UT>(Grow, u, npu, x);
        const float2 bu = b[u * bs];
        const float2 ak = ct[u];
        float4& xp = x[u >> 1];
        const float2 xo = (u & 1) ? make_float2(xp.y, xp.w) : make_float2(xp.x, xp.z);
        set_entry(xp, u, fmaf(ak.x, bu.x - dot.x, ak.y * xo.x), fmaf(ak.x, bu.y - dot.y, ak.y * xo.y));
    };
    if (K < 1) return;
#pragma unroll
    for (int u = 0; u < UT; ++u)  // first sweep from x = 0: pairs holding some x_v, v < u
        if (u < U) step(u, (u + 1) / 2, co);
#pragma unroll 1
    for (int t = 1; t < K; ++t) {
#pragma unroll
        for (int u = 0; u < UT; ++u)
            if (u < U) step(u, UT / 2, co + t * UT);
    }
}

// Learned fusion weights of one subcarrier (the same function as learned_lambda): lambda =
// softmax_c(logit_c), logit_c = b2 + sum_k w2[k] relu(W1[k] . phi_c + b1[k]) with phi_c =
// [||h_{u,c}||^2 / B_c (u < U), log10(max(alpha, 1e-6))], computed by the nw warps starting at warp
// w0 (all of the CTA's, or four that have no sweep lanes).  Warp w0 + i takes clusters i, i + nw, ...;
// each lane computes hidden units lane and lane + 32 with the features in registers, and the logit
// is a warp reduction.  lam[c] is written by warp w0 after one barrier among the nw warps (the CTA
// barrier, or named barrier 1); the caller puts a barrier before reading it.  logit: [C] floats of
// shared scratch.
template <int UT>
__device__ __forceinline__ void tc_learned_lambda(const CdPlan& pl, const cdmimo_learned* blk, bool learned_ok,
                                                  float alpha, const ClusterTile* tab, const float* energy,
                                                  float* logit, float* lam, int w0, int nw)
{
    const int lane = threadIdx.x & 31, warp = (int)(threadIdx.x >> 5) - w0, C = pl.C, U = pl.U;
    const int Hd = learned_ok ? __ldg(&blk->hidden) : 1;
    const int F = U + 1;
    const float la = log10f(fmaxf(alpha, 1e-6f));
    for (int c = warp; c < C; c += nw) {
        const float inv_bc = 1.f / (float)tab[c].size;
        float phi[UT];
#pragma unroll
        for (int j = 0; j < UT; ++j) phi[j] = j < U ? energy[c * UT + j] * inv_bc : 0.f;
        float part = 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            if (k < Hd) {
                const unsigned short* w1 = blk->W1 + (size_t)k * F;
                float z = __ldg(&blk->b1[k]);
#pragma unroll
                for (int j = 0; j < UT; ++j)
                    if (j < U) z = fmaf(bf16_bits_to_float(__ldg(w1 + j)), phi[j], z);
                z = fmaf(bf16_bits_to_float(__ldg(w1 + U)), la, z);
                part = fmaf(bf16_bits_to_float(__ldg(&blk->w2[k])), fmaxf(z, 0.f), part);
            }
        }
        part = warp_sum(part);
        if (lane == 0) logit[c] = __ldg(&blk->b2) + part;
    }
    if (nw * 32 == (int)blockDim.x) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");
    if (warp == 0) {
        float lg[2] = {-__int_as_float(0x7f800000), -__int_as_float(0x7f800000)};
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (lane + 32 * q < C) lg[q] = logit[lane + 32 * q];
        float mx = fmaxf(lg[0], lg[1]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float ex[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) ex[q] = lane + 32 * q < C ? __expf(lg[q] - mx) : 0.f;
        const float tot = warp_sum(ex[0] + ex[1]);
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (lane + 32 * q < C) lam[lane + 32 * q] = ex[q] / tot;
    }
}

// 16-bit storage: an fp16 or bf16 value converted to FP32 has at most 11 significant bits, so its
// FP32 bits are an exact TF32 operand (no split).  A fragment from two such complex entries, and the
// plain and rotated B fragments of one.
__device__ __forceinline__ void a_frag_exact(float2 e0, float2 e1, uint32_t (&a)[4])
{
    a[0] = __float_as_uint(e0.x);
    a[1] = __float_as_uint(e1.x);
    a[2] = __float_as_uint(e0.y);
    a[3] = __float_as_uint(e1.y);
}

__device__ __forceinline__ void mma_exact(float (&d)[4], const uint32_t (&a)[4], float2 v, bool rot)
{
    if (rot) mma_tf32(d, a, __float_as_uint(v.y), __float_as_uint(-v.x));
    else mma_tf32(d, a, __float_as_uint(v.x), __float_as_uint(v.y));
}

// d += A B with A exact and B split: two passes.
__device__ __forceinline__ void mma_2xtf32(float (&d)[4], const uint32_t (&a)[4], const BFrag& b)
{
    mma_tf32(d, a, b.l[0], b.l[1]);
    mma_tf32(d, a, b.h[0], b.h[1]);
}

// Bulk copies of subcarrier f's channel rows into the padded per-cluster layout (row (c, u) at
// 32-bit words (c UT + u) srow); thread i issues row i.  Complex entries of 8 (c64) or 4 bytes.
template <int IN>
__device__ __forceinline__ void issue_channel_copy_tc(const CdPlan& pl, const ClusterTile* tab, const void* H, int f,
                                                      float* dst, int srow, uint64_t* bar)
{
    constexpr uint32_t eb = IN == CDMIMO_C64 ? 8u : 4u;
    const char* Hf = reinterpret_cast<const char*>(H) + (size_t)f * pl.U * pl.B * eb;
    for (int row = threadIdx.x; row < pl.U * pl.C; row += blockDim.x) {
        const int c = row / pl.U, u = row - c * pl.U;
        const ClusterTile ct = tab[c];
        fence_proxy_async_smem();
        bulk_g2s(dst + (size_t)(c * kTcUT + u) * srow, Hf + ((size_t)u * pl.B + ct.off) * eb, (uint32_t)ct.size * eb,
                 bar);
    }
}

// Phase B with two vectors per lane: the uplink x and the downlink w of one (cluster, symbol) tile
// read the same rows of G_c, so each 16-byte pair of a row loaded from shared memory feeds eight
// packed FMAs (four per vector).  The sweeps are bound by the shared-memory pipe (each row pair
// costs four of its cycles whichever lanes read it), and two vectors per lane halve its load.

// Sum_v Gt_uv x_v and Sum_v Gt_uv w_v over the first npu pairs of row gr (as gram_row_dot).  In the
// full sweeps the pairs are visited from the one after the pair holding x_{u-1}, so that only the
// last pair's terms wait for the previous step.
template <int UT>
__device__ __forceinline__ void gram_row_dot2(const float4* gr, int u, int npu, const float4 (&x)[UT / 2],
                                              const float4 (&w)[UT / 2], float2& dx, float2& dw)
{
    constexpr int NP = UT / 2;
    const int s = npu < NP ? 0 : ((((u + UT - 1) % UT) >> 1) + 1) % NP;
    const float2 z = make_float2(0.f, 0.f);
    float2 Rx = z, Jx = z, Ix = z, Kx = z, Rw = z, Jw = z, Iw = z, Kw = z;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        if (k < npu) {
            const int i = (s + k) % NP;
            const float4 g = gr[i];
            Rx = ffma2(lo2(g), lo2(x[i]), Rx);
            Rw = ffma2(lo2(g), lo2(w[i]), Rw);
            Jx = ffma2(hi2(g), hi2(x[i]), Jx);
            Jw = ffma2(hi2(g), hi2(w[i]), Jw);
            Ix = ffma2(lo2(g), hi2(x[i]), Ix);
            Iw = ffma2(lo2(g), hi2(w[i]), Iw);
            Kx = ffma2(hi2(g), lo2(x[i]), Kx);
            Kw = ffma2(hi2(g), lo2(w[i]), Kw);
        }
    }
    dx = make_float2((Rx.x + Rx.y) - (Jx.x + Jx.y), (Ix.x + Ix.y) + (Kx.x + Kx.y));
    dw = make_float2((Rw.x + Rw.y) - (Jw.x + Jw.y), (Iw.x + Iw.y) + (Kw.x + Kw.y));
}

// K Gauss-Seidel sweeps for x (coefficients dx_, right-hand side bx with stride bxs) and for w
// (dw_, bw, bws) on the same Gram rows, from zero, as gram_sweeps does for one vector (the first
// sweep sums only the pairs holding some x_v, v < u).
template <int UT>
__device__ __forceinline__ void gram_sweeps2(int U, int K, const float4* Grow, const float* dx_, const float* dw_,
                                             const float2* bx, uint32_t bxs, const float2* bw, uint32_t bws,
                                             float4 (&x)[UT / 2], float4 (&w)[UT / 2])
{
    constexpr int NP = UT / 2;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        w[i] = x[i];
    }
    if (K < 1) return;
    auto step = [&](int u, int npu) {
        float2 ddx, ddw;
        gram_row_dot2<UT>(Grow + u * NP, u, npu, x, w, ddx, ddw);
        const float2 bxu = bx[u * bxs], bwu = bw[u * bws];
        const float du = dx_[u], eu = dw_[u];
        set_entry(x[u >> 1], u, du * (bxu.x - ddx.x), du * (bxu.y - ddx.y));
        set_entry(w[u >> 1], u, eu * (bwu.x - ddw.x), eu * (bwu.y - ddw.y));
    };
#pragma unroll
    for (int u = 0; u < UT; ++u)
        if (u < U) step(u, (u + 1) / 2);
#pragma unroll 1
    for (int t = 1; t < K; ++t) {
#pragma unroll
        for (int u = 0; u < UT; ++u)
            if (u < U) step(u, NP);
    }
}

// Phase A of one cluster, on one warp: G_c = H_c^H H_c (4 n-tiles: Re and Im of columns 0-7, 8-15)
// and, for the uplink, z = H_c^H y_c (4 n-tiles: Re and Im of symbols 0-7, 8-15), over KA k-steps.
// Hc: the cluster's UT channel rows, srow 32-bit words apart; y of symbol n at element ybase + n B of Y.
// Writes the pair-planar zero-diagonal rows Gc[UT][UT/2], the sweep coefficients Dm[u] = m_u and
// Dp[u] = p_u^2 from the diagonal (learned: Dp[u] = ||h_u||^2 and the per-sweep table LAc[K][UT]),
// and z of the cluster's tiles at Zc[u xs + n].  With ypre, the lane's receive samples (entry
// 4 ks + tig of symbols 8 j + gid, as FP32) were loaded by the caller into ypre[2 ks + j].
template <int BC, int IN, bool UL, bool LEARNED>
__device__ __forceinline__ void tc_phase_a(const CdPlan& pl, const float* Hc, int srow, const void* Y, size_t ybase,
                                           float alpha, float4* Gc, float* Dm, float* Dp, float2* Zc, uint32_t xs,
                                           const cdmimo_learned* blk, float2* LAc, const float2* ypre = nullptr)
{
    constexpr int UT = kTcUT;
    const int SROW = srow, SR2 = srow / 2;
    constexpr int KA = BC / 4;
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int U = pl.U, n_sym = pl.n_sym;
    const float2* Hc2 = reinterpret_cast<const float2*>(Hc);
    const float2* Yc = UL ? reinterpret_cast<const float2*>(Y) + ybase : nullptr;
    float accG[4][4], accZ[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) accG[t][q] = accZ[t][q] = 0.f;
    if constexpr (IN == CDMIMO_C64) {
        // receive samples of the B fragments (entry 4 ks + tig of symbols 8 j + gid), two k-steps
        // ahead: [stage][n-tile]
        float2 yv[2][2];
        auto load_y = [&](int ks, float2 (&dst)[2]) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int n = 8 * j + gid;
                dst[j] = n < n_sym ? __ldg(Yc + (size_t)n * pl.B + 4 * ks + tig) : make_float2(0.f, 0.f);
            }
        };
        if (UL && !ypre) {
            load_y(0, yv[0]);
            if (KA > 1) load_y(1, yv[1]);
        }
#pragma unroll
        for (int ks = 0; ks < KA; ++ks) {
            const int e = 4 * ks + tig;  // the lane's complex entry of this k-step
            uint32_t ah[4], al[4];
            a_frag(Hc2[gid * SR2 + e], Hc2[(gid + 8) * SR2 + e], ah, al);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                BFrag bp, br;
                b_frags(Hc2[(8 * j + gid) * SR2 + e], bp, br);
                mma_3xtf32(accG[j], ah, al, bp);
                mma_3xtf32(accG[2 + j], ah, al, br);
            }
            if constexpr (UL) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    BFrag bp, br;
                    b_frags(ypre ? ypre[2 * ks + j] : yv[ks & 1][j], bp, br);
                    mma_3xtf32(accZ[j], ah, al, bp);
                    mma_3xtf32(accZ[2 + j], ah, al, br);
                }
                if (!ypre && ks + 2 < KA) load_y(ks + 2, yv[ks & 1]);
            }
        }
    } else {  // 16-bit storage: every operand exact in TF32, one MMA per tile
        auto hget = [&](int row, int e) { return Elem<IN>::load_shared(Hc, (size_t)row * SROW + e); };
#pragma unroll
        for (int ks = 0; ks < KA; ++ks) {
            const int e = 4 * ks + tig;
            uint32_t ah[4];
            a_frag_exact(hget(gid, e), hget(gid + 8, e), ah);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float2 hv = hget(8 * j + gid, e);
                mma_exact(accG[j], ah, hv, false);
                mma_exact(accG[2 + j], ah, hv, true);
            }
            if constexpr (UL) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int n = 8 * j + gid;
                    const float2 yy = ypre ? ypre[2 * ks + j]
                                           : (n < n_sym ? Elem<IN>::load(Y, ybase + (size_t)n * pl.B + e) : make_float2(0.f, 0.f));
                    mma_exact(accZ[j], ah, yy, false);
                    mma_exact(accZ[2 + j], ah, yy, true);
                }
            }
        }
    }
    // G rows (pair-planar, zero diagonal) with m_u and p_u^2 from the diagonal; rows u = gid,
    // gid + 8, columns v = 8 j + 2 tig, +1 (accumulator element 2 r + e)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int u = gid + 8 * r, v = 8 * j + 2 * tig;
            float g0 = accG[j][2 * r], g1 = accG[j][2 * r + 1];
            float i0 = accG[2 + j][2 * r], i1 = accG[2 + j][2 * r + 1];
            if (v == u || v + 1 == u) {
                const float e = v == u ? g0 : g1, den = e + alpha;
                Dm[u] = (u < U && den > 0.f) ? __fdividef(1.f, den) : 0.f;
                if constexpr (LEARNED) {
                    Dp[u] = e;
                    for (int t = 0; t < pl.K; ++t) {  // learned coefficients of every sweep
                        const float tau = __ldg(&blk->tau[t]), dl = e + __ldg(&blk->gamma[t]) * alpha;
                        LAc[t * UT + u] = dl > 0.f ? make_float2(tau * __fdividef(1.f, dl), 1.f - tau)
                                                   : make_float2(0.f, 1.f);
                    }
                } else {
                    Dp[u] = (u < U && e > 0.f) ? __fdividef(1.f, e) : 0.f;
                }
                if (v == u) g0 = i0 = 0.f;
                else g1 = i1 = 0.f;
            }
            Gc[u * (UT / 2) + (v >> 1)] = make_float4(g0, g1, i0, i1);
        }
    // z for tile (c, n): rows u = gid, gid + 8, symbols n = 8 j + 2 tig, +1
    if constexpr (UL) {
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int u = gid + 8 * r, n = 8 * j + 2 * tig;
                if (u < U) {
                    float2* z = Zc + u * xs;
                    if (n < n_sym) z[n] = make_float2(accZ[j][2 * r], accZ[2 + j][2 * r]);
                    if (n + 1 < n_sym) z[n + 1] = make_float2(accZ[j][2 * r + 1], accZ[2 + j][2 * r + 1]);
                }
            }
    }
}

// Phase C of one cluster, on one warp: x_c = H_c w for all symbols (MT x 4 tiles) from the cluster's
// channel rows Hc (srow words apart) and its tiles' w at Wc[u xs + n], each symbol's x_c normalized to
// rho_c (a zero x_c stays zero) and written to out[n B + b] (out: the subcarrier's Xdl rows at the
// cluster's offset).
template <int BC, int IN>
__device__ __forceinline__ void tc_phase_c(const CdPlan& pl, const float* Hc, int srow, const float2* Wc, uint32_t xs,
                                           float2* out)
{
    constexpr int UT = kTcUT;
    const int SROW = srow, SR2 = srow / 2;
    constexpr int MT = BC / 16;  // m-tiles (16 antennas each)
    constexpr int KC = UT / 4;   // k-steps (4 users each)
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int U = pl.U, n_sym = pl.n_sym;
    const float2* Hc2 = reinterpret_cast<const float2*>(Hc);
    float acc[MT][4][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][t][q] = 0.f;
    if constexpr (IN == CDMIMO_C64) {
#pragma unroll
        for (int ks = 0; ks < KC; ++ks) {
            const int u = 4 * ks + tig;  // the lane's user of this k-step
            BFrag br[2], bi[2];         // per n-tile: (Re w, -Im w) and (Im w, Re w)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int n = 8 * j + gid;
                const float2 w = (u < U && n < n_sym) ? Wc[u * xs + n] : make_float2(0.f, 0.f);
                b_frags(make_float2(w.y, w.x), bi[j], br[j]);  // rot(Im w, Re w) = (Re w, -Im w)
            }
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                uint32_t ah[4], al[4];
                a_frag(Hc2[u * SR2 + 16 * m + gid], Hc2[u * SR2 + 16 * m + gid + 8], ah, al);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    mma_3xtf32(acc[m][j], ah, al, br[j]);
                    mma_3xtf32(acc[m][2 + j], ah, al, bi[j]);
                }
            }
        }
    } else {  // 16-bit storage: H exact in TF32, w split: two MMAs per tile
#pragma unroll
        for (int ks = 0; ks < KC; ++ks) {
            const int u = 4 * ks + tig;
            BFrag br[2], bi[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int n = 8 * j + gid;
                const float2 w = (u < U && n < n_sym) ? Wc[u * xs + n] : make_float2(0.f, 0.f);
                b_frags(make_float2(w.y, w.x), bi[j], br[j]);
            }
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                uint32_t ah[4];
                a_frag_exact(Elem<IN>::load_shared(Hc, (size_t)u * SROW + 16 * m + gid),
                             Elem<IN>::load_shared(Hc, (size_t)u * SROW + 16 * m + gid + 8), ah);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    mma_2xtf32(acc[m][j], ah, br[j]);
                    mma_2xtf32(acc[m][2 + j], ah, bi[j]);
                }
            }
        }
    }
    // rows b = 16 m + gid (+8), symbols n = 8 j + 2 tig + e; norm over the cluster's antennas
    // (the thread's rows, then the eight lanes of the same tig)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float nr = 0.f;
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float xr = acc[m][j][2 * r + e], xi = acc[m][2 + j][2 * r + e];
                    nr = fmaf(xr, xr, fmaf(xi, xi, nr));
                }
            nr += __shfl_xor_sync(0xffffffffu, nr, 4);
            nr += __shfl_xor_sync(0xffffffffu, nr, 8);
            nr += __shfl_xor_sync(0xffffffffu, nr, 16);
            const float sc = nr > 0.f ? pl.rho_c * rsqrtf(nr) : 0.f;
            const int n = 8 * j + 2 * tig + e;
            if (n < n_sym) {
                float2* o = out + (size_t)n * pl.B;
#pragma unroll
                for (int m = 0; m < MT; ++m)
#pragma unroll
                    for (int r = 0; r < 2; ++r)
                        o[16 * m + 8 * r + gid] = make_float2(acc[m][j][2 * r + e] * sc, acc[m][2 + j][2 * r + e] * sc);
            }
        }
}

template <int BC, int MODE, int IN>
__global__ void __launch_bounds__(kTcThreads, 2) cd_frame_tc_kernel(const CdPlan pl, const FusedIO io)
{
    constexpr bool UL = MODE != kTcPrecode, DL = MODE == kTcFrame || MODE == kTcPrecode;
    constexpr bool LEARNED = MODE == kTcDetectLearned;
    constexpr int UT = kTcUT;
    constexpr int SROW = (int)tc_row_words(BC, IN);  // 32-bit words per channel row
    static_assert(BC == 16 || BC == 32, "cluster size 16 or 32");

    extern __shared__ __align__(128) unsigned char smem[];
    float4* Gs = reinterpret_cast<float4*>(smem + pl.off_G);  // [C][UT][UT/2] pair-planar rows, zero diagonal
    // [U][x_stride] w per tile: over the Gram rows after the sweeps (frame), or where z / x would be
    // (downlink alone: stored as soon as a lane's sweeps end)
    float2* Ws = reinterpret_cast<float2*>(smem + (MODE == kTcPrecode ? pl.off_X : pl.off_G));
    float* Dm = reinterpret_cast<float*>(smem + pl.off_E);    // [C][UT] m_u
    float* Dp = reinterpret_cast<float*>(smem + pl.off_E2);   // [C][UT] p_u^2 (learned: ||h_u||^2)
    float2* Zs = reinterpret_cast<float2*>(smem + pl.off_X);  // [UT][x_stride]: z, then each tile's x
    float2* Ss = reinterpret_cast<float2*>(smem + pl.off_S);  // [U][n_sym]: s of the subcarrier, transposed
    float* lam = reinterpret_cast<float*>(smem + pl.off_lam);
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);
    int* nxt = reinterpret_cast<int*>(smem + pl.off_bar + 16);
    auto Hbuf = [&](int j) { return reinterpret_cast<float*>(smem + (j ? pl.off_H2 : 0u)); };
    const DetectIO& d = io.d;
    const cdmimo_learned* blk = reinterpret_cast<const cdmimo_learned*>(d.learned);
    float* mlp = reinterpret_cast<float*>(smem + pl.off_mlp);  // [C] logits (learned fusion)
    float2* LA = reinterpret_cast<float2*>(smem + pl.off_K);   // [C][K][UT] learned (a, keep) per sweep

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym, n_s = n_sym * U;
    const uint32_t xs = tc_x_stride(pl.n_tiles);
    bool learned_ok = true;
    if constexpr (LEARNED) {
        const int hd = __ldg(&blk->hidden);
        learned_ok = __ldg(&blk->K) == pl.K && __ldg(&blk->U) == U && hd >= 1 && hd <= CDMIMO_MAX_HIDDEN;
        if (!learned_ok && tid == 0 && blockIdx.x == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_LEARNED);
    }

    // Setup: cluster table, barriers, zero channel rows U..UT-1 of both buffers (never copied).
    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async_smem();
    }
    for (int j = 0; j < 2; ++j) {
        float* hb = Hbuf(j);
        const int per_c = (UT - U) * SROW;
        for (int i = tid; i < C * per_c; i += blockDim.x) {
            const int c = i / per_c, r = i - c * per_c;
            hb[(c * UT + U) * SROW + r] = 0.f;
        }
    }
    __syncthreads();

    // Phase B lanes: one per (cluster, symbol), holding that tile's uplink x and (or) downlink w.
    const GLane gb = frame_lane(0, C, n_sym, 1);

    int f = blockIdx.x;
    if (tid == 0 && f < pl.n_sc) arm_channel_copy<IN>(pl, &bar[0]);
    __syncthreads();
    if (f < pl.n_sc) issue_channel_copy_tc<IN>(pl, tab, d.H, f, Hbuf(0), SROW, &bar[0]);
    auto put_s = [&](int i, float2 v) { Ss[(i % U) * n_sym + i / U] = v; };
    if (DL && f < pl.n_sc)
        for (int i = tid; i < n_s; i += blockDim.x) put_s(i, io.S[(size_t)f * n_s + i]);

    int done = 0;
    for (int k = 0; f < pl.n_sc; ++k) {
        const int b = k & 1;
        float alpha = 0.f, out_scale = 1.f;
        if constexpr (UL) {
            alpha = __ldg(d.N0 + f) * pl.inv_Ex;
            if (!(alpha >= 0.f)) {
                if (tid == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_N0);
                out_scale = __int_as_float(0x7fc00000);
                alpha = 0.f;
            }
            if (LEARNED && !learned_ok) out_scale = __int_as_float(0x7fc00000);
            if constexpr (IN != CDMIMO_C64) {  // stored H / a_f, y / b_f: solve with alpha / a_f^2, scale x by b_f / a_f
                const float hs = __ldg(d.h_scale + f), ys = __ldg(d.y_scale + f);
                alpha = alpha / (hs * hs);
                out_scale = out_scale * (ys / hs);
            }
        }
        const uint32_t parity = (uint32_t)(k >> 1) & 1u;
        const bool ok = mbar_wait_bounded(&bar[b], parity);
        if (__syncthreads_or(!ok)) {
            // copy timeout: no other copy is in flight; give this one a last bounded wait, then stop
            if (tid == 0) mbar_wait_bounded(&bar[b], parity);
            break;
        }
        const float* Hb = Hbuf(b);

        // Phase A: per cluster (one warp), G_c and (uplink) z.
        for (int c = warp; c < C; c += kTcThreads / 32) {
            const ClusterTile ct = tab[c];
            tc_phase_a<BC, IN, UL, LEARNED>(pl, Hb + c * UT * SROW, SROW, d.Y, (size_t)f * n_sym * pl.B + ct.off, alpha,
                                           Gs + (size_t)c * UT * (UT / 2), Dm + c * UT, Dp + c * UT, Zs + c * n_sym,
                                           xs, blk, LA + c * pl.K * UT);
        }
        __syncthreads();

        // Phase B: uplink sweeps on x (right-hand side z) and downlink sweeps on w (right-hand side s),
        // in the same lane for the frame; w stays in registers until every lane has finished reading G.
        const unsigned ticket = (d.sched && tid == 0) ? atomicAdd(d.sched, 1u) : 0u;
        float4 x[UT / 2], xw[UT / 2];
        const int n_b = gb.j, tile = gb.c * n_sym + n_b;
        // Learned fusion: its weights need only ||h_u||^2 and N0, so where the sweep lanes leave warps
        // 4-7 free those warps compute them now, during the sweeps.
        const bool mlp_now = LEARNED && pl.fuse == CDMIMO_FUSE_LEARNED && frame_warps(C * n_sym) <= 4;
        if (mlp_now && warp >= 4) tc_learned_lambda<UT>(pl, blk, learned_ok, alpha, tab, Dp, mlp, lam, 4, 4);
        if (gb.active) {
            const float4* Gc = Gs + (size_t)gb.c * UT * (UT / 2);
            const float* dd = Dm + gb.c * UT;
            if constexpr (MODE == kTcFrame)
                gram_sweeps2<UT>(U, pl.K, Gc, dd, Dp + gb.c * UT, Zs + tile, xs, Ss + n_b, (uint32_t)n_sym, x, xw);
            else if constexpr (MODE == kTcDetect)
                gram_sweeps<UT>(U, pl.K, Gc, dd, Zs + tile, xs, x);
            else if constexpr (LEARNED)
                gram_sweeps_learned_tab<UT>(U, learned_ok ? pl.K : 0, Gc, LA + gb.c * pl.K * UT, Zs + tile, xs, x);
            else
                gram_sweeps<UT>(U, pl.K, Gc, Dp + gb.c * UT, Ss + n_b, (uint32_t)n_sym, xw);
            if constexpr (MODE == kTcPrecode) {
#pragma unroll
                for (int u = 0; u < UT; ++u)
                    if (u < U) Ws[tile + u * xs] = slice_entry<UT, 1>(xw, u);
            }
            if constexpr (UL) {
#pragma unroll
                for (int u = 0; u < UT; ++u)
                    if (u < U) Zs[tile + u * xs] = slice_entry<UT, 1>(x, u);
                if (n_b == 0 && !(LEARNED && pl.fuse == CDMIMO_FUSE_LEARNED)) {
                    float msum = 0.f;
                    for (int u = 0; u < U; ++u) msum += dd[u] > 0.f ? dd[u] : __int_as_float(0x7f800000);
                    lam[gb.c] = 1.f / msum;
                }
            }
        }
        if (tid == 0) {
            int nf = f + (int)gridDim.x;
            if (d.sched) {
                const unsigned v = gridDim.x + ticket;
                nf = v < (unsigned)pl.n_sc ? (int)v : pl.n_sc;
            }
            nxt[b] = nf;
            if (nf < pl.n_sc) arm_channel_copy<IN>(pl, &bar[b ^ 1]);
        }
        __syncthreads();
        if constexpr (MODE == kTcFrame) {
            if (gb.active) {
#pragma unroll
                for (int u = 0; u < UT; ++u)
                    if (u < U) Ws[tile + u * xs] = slice_entry<UT, 1>(xw, u);
            }
            __syncthreads();
        }

        // Phase C: the next subcarrier's channel copy (into the other buffer, last read in the
        // previous iteration) and its y into L2; the next s is loaded now and stored at the end.
        // Downlink, per cluster (one warp): x_c = H_c w for all symbols (MT x 4 tiles), normalized
        // per symbol.  Then the uplink fusion.
        const int fn = nxt[b];
        if (fn < pl.n_sc) issue_channel_copy_tc<IN>(pl, tab, d.H, fn, Hbuf(b ^ 1), SROW, &bar[b ^ 1]);
        if (UL && tid == 32 && fn < pl.n_sc) {
            constexpr uint32_t eb = IN == CDMIMO_C64 ? 8u : 4u;
            bulk_prefetch_l2(static_cast<const char*>(d.Y) + (size_t)fn * n_sym * pl.B * eb, (uint32_t)n_sym * pl.B * eb);
        }
        constexpr int kSv = 2;
        const bool ld_s = DL && fn < pl.n_sc;
        const float2* s_src = DL ? io.S + (size_t)min(fn, pl.n_sc - 1) * n_s : nullptr;
        float2 sv[kSv];
#pragma unroll
        for (int q = 0; q < kSv; ++q)
            sv[q] = (ld_s && tid + q * kTcThreads < n_s) ? s_src[tid + q * kTcThreads] : make_float2(0.f, 0.f);

        for (int c = warp; DL && c < C; c += kTcThreads / 32)
            tc_phase_c<BC, IN>(pl, Hb + c * UT * SROW, SROW, Ws + c * n_sym, xs,
                               io.Xdl + (size_t)f * n_sym * pl.B + tab[c].off);
        if constexpr (LEARNED) {
            if (pl.fuse == CDMIMO_FUSE_LEARNED) {  // lambda = softmax of the MLP on ||h_u||^2 / B_c and log10 alpha
                if (!mlp_now) {
                    tc_learned_lambda<UT>(pl, blk, learned_ok, alpha, tab, Dp, mlp, lam, 0, kTcThreads / 32);
                    __syncthreads();
                }
                // (symbols fastest, as for the plain rules: this kernel takes no per-cluster outputs)
                fuse_range(pl, d, f, lam, Zs, xs, out_scale, 0, kTcThreads, true);
            } else {
                fuse_range(pl, d, f, lam, Zs, xs, out_scale, 0, kTcThreads);
            }
        } else if constexpr (MODE == kTcDetect) {
            if (d.Xc || d.lam) fuse_subcarrier<false>(pl, d, f, lam, Zs, xs, out_scale);  // + per-cluster outputs
            else fuse_range(pl, d, f, lam, Zs, xs, out_scale, 0, kTcThreads);
        } else if constexpr (UL) {
            fuse_range(pl, d, f, lam, Zs, xs, out_scale, 0, kTcThreads);
        }
        if (ld_s) {
#pragma unroll
            for (int q = 0; q < kSv; ++q)
                if (tid + q * kTcThreads < n_s) put_s(tid + q * kTcThreads, sv[q]);
            for (int i = tid + kSv * kTcThreads; i < n_s; i += kTcThreads) put_s(i, s_src[i]);
        }
        __syncthreads();  // this channel buffer receives the copy issued at the next iteration's start
        ++done;
        f = fn;
    }
    sched_finish(d.sched, done, pl.n_sc);
}

}  // namespace cdmimo
