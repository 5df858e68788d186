// Warp-specialized tensor-core Gram-form kernel: the TDD frame (uplink detection, Algorithm 1 +
// fusion of Sec. III, and downlink precoding, Algorithm 2 + normalization of Sec. IV-B, on one
// channel per subcarrier), or either direction alone, with the same arithmetic as
// cd_frame_tc_kernel (the contractions z = H_c^H y_c, G_c = H_c^H H_c and x_c = H_c w as split-TF32
// MMAs, the Gauss-Seidel sweeps in FP32; see cd_frame_tc.cuh), but with the phases of consecutive
// subcarriers overlapped inside one CTA per SM instead of run one after the other.
//
// Roles.  Eight "MMA" warps own the clusters (warp c takes clusters c, c + 8, ...): for its clusters
// a warp forms G_c and z of subcarrier s + 1 (phase A) and x_c = H_c w of subcarrier s - 1 (phase C),
// and the MMA warps stage the downlink symbols.  Two groups of four "sweep" warps (one lane per
// (cluster, symbol) tile, 4 warps at C n_sym = 112) take alternate subcarriers: a group runs the K
// sweeps of its subcarrier and then fuses that subcarrier's uplink estimates, so the sweeps of two
// consecutive subcarriers overlap.  A subcarrier then costs about the longest role's work, not the
// sum, with the sweep warps (the FP32 pipes) and the MMA warps (the tensor pipes) issuing on the
// same SM sub-partitions at the same time.  512 threads of 128 registers fill the register file.
//
// Pipeline, for the CTA's subcarriers s = 0, 1, ... (f = blockIdx.x + s gridDim.x, a static schedule;
// calls with schedule counters run the phased kernel):
//   MMA stage j:    [j >= 2] wait done(j - 2); phase C of j - 2; copy the channel of j + 1 into the
//                   buffer j - 2 used;  [j < n] wait channel(j); phase A of j; signal A(j).
//   sweep group g:  for s = g, g + 2, ...: wait A(s); sweeps of s; fusion of s; signal done(s).
// Buffers: the channel rows of subcarrier s live from phase A(s) to phase C(s), two stages later, so
// there are three (s mod 3); G_c, m_u, p_u^2, z / x, w, s and the fusion weights are double
// buffered (s mod 2, the buffers of sweep group s mod 2).  The hand-overs between roles are
// mbarriers (release / acquire), each with a bounded wait; named barriers with reductions (1: the
// MMA warps, 2 and 3: the sweep groups) order the steps within a role and make a timed-out wait leave
// the loop on all of its warps together.
#pragma once
#include "cd_frame_tc.cuh"
#include "umma.cuh"

namespace cdmimo {

constexpr int kWsMmaWarps = 8;
constexpr int kWsSweepGroups = 2;  // sweep groups of four warps, taking alternate subcarriers
constexpr int kWsMaxThreads = 32 * kWsMmaWarps + kWsSweepGroups * 128;  // 512 threads, 128 registers each

// Shared-memory layout of cd_frame_ws_kernel (byte offsets), built on the host.  Buffer i of a
// region starts at off + i * stride (three channel buffers, two of everything else).
struct WsLayout {
    unsigned off_H, st_H;      // channel rows [UT][srow] words: user u's B antennas, all clusters
    unsigned off_G, st_G;      // [C][UT][UT/2] float4 Gram rows with zero diagonal
    unsigned off_D, st_D;      // [2][C][UT] floats: m_u, then p_u^2
    unsigned off_Z, st_Z;      // [UT][xs] float2: z, then each tile's x (uplink)
    unsigned off_W, st_W;      // [UT][xs] float2: w per tile (downlink)
    unsigned off_S, st_S;      // [U][n_sym] float2: s of the subcarrier, transposed (downlink)
    unsigned off_lam, st_lam;  // [C] floats: fusion weights 1 / sum_u m_u
    unsigned off_tab, off_bar, smem_bytes;  // off_bar: [8] mbarriers, then [2] floats: the uplink output
                                            // scale of the subcarrier in each z / x buffer, then (T5) the
                                            // MMA-completion mbarrier and the tensor-memory base address
    unsigned off_op;    // T5: [6][16][2 BC] words of tcgen05 operands (t5_phase_a)
    unsigned tmem_cols; // T5: tensor-memory columns allocated (64 per cluster, a power of two)
    int sweep_warps;  // warps of one sweep group (four); kWsSweepGroups groups run
    int slot;         // sweep lanes per cluster (8 or 16, >= n_sym): a cluster's tiles fill a quarter or
                      // half warp, so that no quarter warp reads two clusters' Gram rows
    int srow;         // 32-bit words per channel row (ws_row_words)
};

// Words per channel row of the warp-specialized kernel: the row's B entries (c64: two words each,
// 16-bit: one) padded to 8 (c64) or 4 (16-bit) mod 32, the residue of tc_row_words, so that the
// fragment loads of phases A and C keep the phased kernel's bank pattern.  Each row arrives by one
// bulk copy of its B entries (16 rows per subcarrier rather than one per cluster and user: the copy
// engine's cost per instruction made 8 U small copies a stage's largest stall).
__host__ __device__ constexpr unsigned ws_row_words(int B, int in_dtype)
{
    return in_dtype == CDMIMO_C64 ? 2u * (unsigned)B + ((8u - 2u * (unsigned)B % 32u) % 32u)
                                  : (unsigned)B + ((36u - (unsigned)B % 32u) % 32u);
}

// Sweep lanes per cluster for n_sym symbols (n_sym <= 16).
__host__ __device__ constexpr int ws_slot(int n_sym) { return n_sym <= 8 ? 8 : 16; }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Named barrier `id` over `n` threads, returning the AND of every participant's `ok`.
__device__ __forceinline__ bool group_and(bool ok, uint32_t id, uint32_t n)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// Named barrier 1 over the MMA warps, returning the AND of every participant's `ok`.
__device__ __forceinline__ bool mma_group_and(bool ok)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok), "n"(32 * kWsMmaWarps)
        : "memory");
    return r != 0;
}

// Phase A on the 5th-generation tensor cores (c64 storage, clusters of BC = 16 or 32, C <= 8): for
// each cluster the MMA warps write six K-major operand blocks of 16 rows x 2 BC FP32 words into `op`
// (the real and imaginary parts of an antenna side by side along K), in this order:
//     0 Y_lo  1 Y_hi  2 H_lo  3 H_hi  4 rot(H)_lo  5 rot(H)_hi
// with H_u the channel row of user u, Y_n the receive samples of symbol n, rot(h) = (Im h, -Re h) per
// antenna, and hi / lo the split-TF32 halves of cd_frame_tc.cuh.  One thread then issues, into
// tensor-memory columns 64 c .. 64 c + 63, the M = 64, N = 64 product D = A B^T with A = blocks 0..3
// and B = blocks 2..5: every pairing of a hi or lo half with a hi or lo half in one instruction per
// 8 words of K (an M = 64, N = 64 tf32 MMA costs the device what an N = 32 one does).  Row by row,
// P_re[v] = D[., v] + D[., 16 + v] and P_im[v] = D[., 32 + v] + D[., 48 + v] sum over B's halves, and
// the sum over A's halves pairs two lane quarters:
//     Re G_uv = P_re(H_lo u) + P_re(H_hi u),  Im G_uv = P_im(H_lo u) + P_im(H_hi u),
//     Re z_vn = P_re(Y_lo n) + P_re(Y_hi n),  Im z_vn = -(P_im(Y_lo n) + P_im(Y_hi n))
// (G_c = H_c^H H_c, z = H_c^H y_c; Sec. III-A).  An M = 64 accumulator keeps A's rows 16 q .. 16 q + 15
// in lanes 32 q .. 32 q + 15, so warps of quarters 1 and 3 (Y_hi, H_hi) pass their partial rows
// through shared memory (the operand buffer, free once the MMAs are done) to the warps of quarters 0
// and 2, which write z and the pair-planar G rows, m_u, p_u^2 and the fusion weight exactly as
// tc_phase_a does.  The operand buffer is reused per cluster (each cluster's MMAs are waited for
// before the next is written).  yq holds this thread's receive samples of every cluster (row tid mod
// 16, words 4 (tid / 16) .. + 3 of the cluster's span).  Returns false, on every MMA thread, when a
// completion wait timed out.
template <int BC, bool UL>
__device__ __forceinline__ bool t5_phase_a(const CdPlan& pl, const ClusterTile* tab, const float* Hj, int srow,
                                           float* op, uint64_t* barT, uint32_t& tpar, uint32_t tbase, float alpha,
                                           float4* Gj, float* Dmj, float* Dpj, float2* Zj, uint32_t xs, float* Lj,
                                           const float4 (&yq)[8])
{
    constexpr int UT = kTcUT, BLK = 32 * BC;             // words per operand block (16 rows x 2 BC)
    constexpr uint32_t LBO = 128u, SBO = 64u * BC;       // bytes: next 4 words of K / next 8 rows
    constexpr uint32_t idesc = umma_idesc_tf32(64, 64);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = tid & 15, kc = tid >> 4;                // this thread's chunk: row r, words 4 kc .. 4 kc + 3
    const bool mine = kc < BC / 2;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    const int cofs = (r >> 3) * (SBO / 4) + kc * 32 + (r & 7) * 4;  // word offset of the chunk in a block
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {  // unrolled: yq[c] stays in registers
        if (c >= C) break;
        if (c > 0) ok = mbar_wait_bounded(barT, (tpar++) & 1u);  // the MMAs of cluster c - 1 read op
        if (mine) {
            const float4 h = *reinterpret_cast<const float4*>(Hj + r * srow + 2 * tab[c].off + 4 * kc);
            const float4 y = yq[c];
            uint32_t hh[4], hl[4], yh[4], yl[4];
            tf32_split(h.x, hh[0], hl[0]);
            tf32_split(h.y, hh[1], hl[1]);
            tf32_split(h.z, hh[2], hl[2]);
            tf32_split(h.w, hh[3], hl[3]);
            tf32_split(y.x, yh[0], yl[0]);
            tf32_split(y.y, yh[1], yl[1]);
            tf32_split(y.z, yh[2], yl[2]);
            tf32_split(y.w, yh[3], yl[3]);
            auto st = [&](int b, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3) {
                *reinterpret_cast<uint4*>(op + b * BLK + cofs) = make_uint4(a0, a1, a2, a3);
            };
            st(0, yl[0], yl[1], yl[2], yl[3]);
            st(1, yh[0], yh[1], yh[2], yh[3]);
            st(2, hl[0], hl[1], hl[2], hl[3]);
            st(3, hh[0], hh[1], hh[2], hh[3]);
            st(4, hl[1], neg_bits(hl[0]), hl[3], neg_bits(hl[2]));
            st(5, hh[1], neg_bits(hh[0]), hh[3], neg_bits(hh[2]));
        }
        fence_proxy_async_smem();
        ok = mma_group_and(ok);
        if (!ok) return false;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t dcol = tbase + 64u * (uint32_t)c;
            // descriptors of k-step 0; k-step ks starts 2 core matrices (256 bytes, 16 address units) on
            const uint64_t da = umma_desc(op, LBO, SBO), db = umma_desc(op + 2 * BLK, LBO, SBO);
#pragma unroll
            for (int ks = 0; ks < BC / 4; ++ks) umma_tf32(dcol, da + 16u * ks, db + 16u * ks, idesc, ks > 0 ? 1u : 0u);
            umma_commit(barT);
        }
        __syncwarp();  // lanes 1..31 of warp 0 wait here, not in a sleeping poll interleaved with the issue
    }
    ok = mma_group_and(mbar_wait_bounded(barT, (tpar++) & 1u));
    if (!ok) return false;
    tc_fence_after();
    // Epilogue, two rounds of four clusters: the warps of each half of the MMA warps take alternate
    // clusters; quarter 3 (H_hi) and 1 (Y_hi) hand their partial rows over in op, quarters 2 and 0
    // finish G and z.
    const int q = warp & 3, half = warp >> 2;
    float* scr = op;  // [4][16][32] G partials, then [4][16][32] z partials
    for (int round = 0; round * 4 < C; ++round) {
        float pr[UT], pi[UT];
        int cs[2];
        cs[0] = 4 * round + half;
        cs[1] = 4 * round + 2 + half;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int c = cs[t];
            if (c < C && (q == 1 || q == 3)) {
                float v[32], w[32];
                const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + 64u * (uint32_t)c;
                tmem_ld32(ta, v);
                tmem_ld32(ta + 32u, w);
                float* dst = scr + ((q == 3 ? 0 : 4) + (c & 3)) * 16 * 32 + (lane & 15) * 32;
                if (lane < 16) {
#pragma unroll
                    for (int i = 0; i < UT; i += 4) {
                        *reinterpret_cast<float4*>(dst + i) =
                            make_float4(v[i] + v[16 + i], v[i + 1] + v[17 + i], v[i + 2] + v[18 + i], v[i + 3] + v[19 + i]);
                        *reinterpret_cast<float4*>(dst + 16 + i) =
                            make_float4(w[i] + w[16 + i], w[i + 1] + w[17 + i], w[i + 2] + w[18 + i], w[i + 3] + w[19 + i]);
                    }
                }
            }
        }
        mma_group_and(true);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int c = cs[t];
            if (c >= C || (q != 0 && q != 2)) continue;
            float v[32], w[32];
            const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + 64u * (uint32_t)c;
            tmem_ld32(ta, v);
            tmem_ld32(ta + 32u, w);
            const float* src = scr + ((q == 2 ? 0 : 4) + (c & 3)) * 16 * 32 + (lane & 15) * 32;
#pragma unroll
            for (int i = 0; i < UT; ++i) {
                pr[i] = v[i] + v[16 + i] + src[i];
                pi[i] = w[i] + w[16 + i] + src[16 + i];
            }
            if (q == 2) {
                const int u = lane;
                float mu = 0.f;
                if (u < UT) {
                    float e = 0.f;  // Re G_uu, selected without a dynamic register index
#pragma unroll
                    for (int i = 0; i < UT; ++i) e = i == u ? pr[i] : e;
                    const float den = e + alpha;
                    mu = (u < U && den > 0.f) ? __fdividef(1.f, den) : 0.f;
                    Dmj[c * UT + u] = mu;
                    Dpj[c * UT + u] = (u < U && e > 0.f) ? __fdividef(1.f, e) : 0.f;
                    float4* Gr = Gj + (size_t)c * UT * (UT / 2) + u * (UT / 2);
#pragma unroll
                    for (int i = 0; i < UT / 2; ++i) {
                        float g0 = pr[2 * i], g1 = pr[2 * i + 1], i0 = pi[2 * i], i1 = pi[2 * i + 1];
                        if (2 * i == u) g0 = i0 = 0.f;
                        if (2 * i + 1 == u) g1 = i1 = 0.f;
                        Gr[i] = make_float4(g0, g1, i0, i1);
                    }
                }
                // fusion weight 1 / sum_u m_u (a skipped column counts as infinite)
                float ms = (lane < U) ? (mu > 0.f ? mu : __int_as_float(0x7f800000)) : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ms += __shfl_xor_sync(0xffffffffu, ms, o);
                if (lane == 0) Lj[c] = 1.f / ms;
            } else if (UL && lane < n_sym) {
                float2* z = Zj + c * n_sym + lane;
#pragma unroll
                for (int u = 0; u < UT; ++u)
                    if (u < U) z[u * xs] = make_float2(pr[u], -pi[u]);
            }
        }
        mma_group_and(true);  // the scratch is read before the next round (or the next cluster's operands) reuse it
    }
    tc_fence_before();
    return true;
}

template <int BC, int MODE, int IN, bool T5 = false>
__global__ void __launch_bounds__(kWsMaxThreads, 1) cd_frame_ws_kernel(const CdPlan pl, const WsLayout wl,
                                                                       const FusedIO io)
{
    constexpr bool UL = MODE != kTcPrecode, DL = MODE != kTcDetect;
    static_assert(MODE == kTcFrame || MODE == kTcDetect || MODE == kTcPrecode, "plain modes only");
    static_assert(BC == 16 || BC == 32, "cluster size 16 or 32");
    static_assert(!T5 || IN == CDMIMO_C64, "tcgen05 phase A: c64 storage");
    constexpr int UT = kTcUT;
    const int SROW = wl.srow;
    constexpr uint32_t eb = IN == CDMIMO_C64 ? 8u : 4u;  // bytes per stored complex entry
    constexpr int ew = IN == CDMIMO_C64 ? 2 : 1;         // 32-bit words per stored complex entry
    constexpr int kMmaThreads = 32 * kWsMmaWarps;

    extern __shared__ __align__(128) unsigned char smem[];
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + wl.off_tab);
    uint64_t* barH = reinterpret_cast<uint64_t*>(smem + wl.off_bar);  // [3] channel copies landed
    uint64_t* barA = barH + 3;                                         // [2] phase A done
    uint64_t* barS = barH + 5;                                         // [2] sweeps done
    uint64_t* barT = barH + 9;                                         // tcgen05 MMAs done (T5)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(barH + 10);          // tensor-memory base (T5)
    auto Hb = [&](int s) { return reinterpret_cast<float*>(smem + wl.off_H + (unsigned)(s % 3) * wl.st_H); };
    auto Gb = [&](int s) { return reinterpret_cast<float4*>(smem + wl.off_G + (unsigned)(s & 1) * wl.st_G); };
    auto Dmb = [&](int s) { return reinterpret_cast<float*>(smem + wl.off_D + (unsigned)(s & 1) * wl.st_D); };
    auto Dpb = [&](int s) { return Dmb(s) + pl.C * UT; };
    auto Zb = [&](int s) { return reinterpret_cast<float2*>(smem + wl.off_Z + (unsigned)(s & 1) * wl.st_Z); };
    auto Wb = [&](int s) { return reinterpret_cast<float2*>(smem + wl.off_W + (unsigned)(s & 1) * wl.st_W); };
    auto Sb = [&](int s) { return reinterpret_cast<float2*>(smem + wl.off_S + (unsigned)(s & 1) * wl.st_S); };
    auto Lb = [&](int s) { return reinterpret_cast<float*>(smem + wl.off_lam + (unsigned)(s & 1) * wl.st_lam); };
    const DetectIO& d = io.d;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym, n_s = n_sym * U;
    const uint32_t xs = tc_x_stride(pl.n_tiles);
    const int n_sw = 32 * wl.sweep_warps;
    // this CTA's subcarriers: f(s) = blockIdx.x + s gridDim.x for s < n_mine (static schedule)
    const int n_mine = (int)blockIdx.x < pl.n_sc ? (pl.n_sc - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto fof = [&](int s) { return (int)blockIdx.x + s * (int)gridDim.x; };

    // Setup: cluster table, barriers, zero channel rows U..UT-1 of the three buffers (never copied).
    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(&barH[i], (uint32_t)kWsMmaWarps);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&barA[i], (uint32_t)kMmaThreads);
            mbar_init(&barS[i], (uint32_t)n_sw);
        }
        if (T5) mbar_init(barT, 1u);
        fence_proxy_async_smem();
    }
    if (T5 && warp == 0) tmem_alloc(tslot, wl.tmem_cols);  // one CTA per SM: the columns are free
    for (int j = 0; j < 3; ++j) {
        float* hb = Hb(j) + U * SROW;
        for (int i = tid; i < (UT - U) * SROW; i += blockDim.x) hb[i] = 0.f;
    }
    if (T5) tc_fence_before();
    __syncthreads();
    if (T5) tc_fence_after();
    const uint32_t tbase = T5 ? *tslot : 0u;
    float* osc = reinterpret_cast<float*>(barH + 8);  // [2] uplink output scale per z / x buffer

    if (warp < kWsMmaWarps) {
        // ------------------------------------------------------------------ MMA role
        // Copies of subcarrier s's channel rows into buffer s mod 3: warp w copies users w, w + 8, ...
        // (whole rows of B entries); its lane 0 announces their bytes on the buffer's barrier (one
        // arrival per MMA warp).
        auto issue_copy = [&](int s) {
            const int f = fof(s);
            const char* Hf = reinterpret_cast<const char*>(d.H) + (size_t)f * U * pl.B * eb;
            float* dst = Hb(s);
            if (lane == 0) {
                const int rows = warp < U ? (U - 1 - warp) / kWsMmaWarps + 1 : 0;
                mbar_arrive_expect_tx(&barH[s % 3], (uint32_t)rows * pl.B * eb);
                fence_proxy_async_smem();
                for (int u = warp; u < U; u += kWsMmaWarps)
                    bulk_g2s(dst + (size_t)u * SROW, Hf + (size_t)u * pl.B * eb, (uint32_t)pl.B * eb, &barH[s % 3]);
                if (warp == 0) {  // this subcarrier's receive samples and downlink symbols into L2
                    if (UL) bulk_prefetch_l2(static_cast<const char*>(d.Y) + (size_t)f * n_sym * pl.B * eb,
                                             (uint32_t)n_sym * pl.B * eb);
                    if (DL) bulk_prefetch_l2(io.S + (size_t)f * n_s, (uint32_t)n_s * 8u);
                }
            }
        };
        uint32_t tpar = 0;           // T5: completions of barT waited for
        int issued = 0, landed = 0;  // channel copies issued / waited for (subcarriers 0 .. issued - 1)
        if (n_mine > 0) issue_copy(issued++);
        bool ok = true;
        for (int j = 0; ok && j < n_mine + 2; ++j) {
            // Loads for phase A of j, issued before phase C and the fusion of j - 2 so that their
            // latency is spent there: N0 (and scales) and the downlink symbols.  Phase A loads its
            // receive samples itself, two k-steps ahead (they are in L2 since the channel copy of j
            // was issued); holding them in registers through phase C would not fit the 128
            // registers a thread has with two sweep groups.
            const bool do_a = j < n_mine;
            const int fa = do_a ? fof(j) : 0;
            float n0 = 0.f, hs = 1.f, ys = 1.f;
            float2 sv = make_float2(0.f, 0.f);
            float4 yq[8];  // T5: this thread's receive samples of every cluster (t5_phase_a)
            if constexpr (T5) {
#pragma unroll
                for (int c = 0; c < 8; ++c) yq[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (do_a) {
                if constexpr (UL) {
                    n0 = __ldg(d.N0 + fa);
                    if constexpr (IN != CDMIMO_C64) {
                        hs = __ldg(d.h_scale + fa);
                        ys = __ldg(d.y_scale + fa);
                    }
                    if constexpr (T5) {
                        const int r = tid & 15, kc = tid >> 4;
                        const float* Yf = static_cast<const float*>(d.Y) + (size_t)fa * n_sym * pl.B * 2;
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (c < C && r < n_sym && kc < BC / 2)
                                yq[c] = __ldg(reinterpret_cast<const float4*>(Yf + ((size_t)r * pl.B + tab[c].off) * 2 + 4 * kc));
                    }
                }
                if (DL && tid < n_s) sv = __ldg(io.S + (size_t)fa * n_s + tid);
            }
            if (j >= 2) {
                const int s = j - 2, f = fof(s);
                ok = mma_group_and(mbar_wait_bounded(&barS[s & 1], (uint32_t)(s >> 1) & 1u));
                if (!ok) break;
                if constexpr (DL) {
                    for (int c = warp; c < C; c += kWsMmaWarps)
                        tc_phase_c<BC, IN>(pl, Hb(s) + tab[c].off * ew, SROW, Wb(s) + c * n_sym, xs,
                                           io.Xdl + (size_t)f * n_sym * pl.B + tab[c].off);
                }
            }
            __syncwarp();
            if (j + 1 < n_mine) issue_copy(issued++);  // into the buffer that phase C of j - 2 released
            if (do_a) {
                float alpha = 0.f;
                if constexpr (UL) {
                    alpha = n0 * pl.inv_Ex;
                    float out_scale = 1.f;
                    if (!(alpha >= 0.f)) {  // negative or NaN noise variance: this subcarrier's estimate is NaN
                        if (lane == 0 && warp == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_N0);
                        out_scale = __int_as_float(0x7fc00000);
                        alpha = 0.f;
                    }
                    if constexpr (IN != CDMIMO_C64) {  // solve with alpha / a_f^2, scale x by b_f / a_f
                        alpha = alpha / (hs * hs);
                        out_scale = out_scale * (ys / hs);
                    }
                    if (tid == 0) osc[j & 1] = out_scale;  // read by the fusion of j, two stages on
                }
                // every MMA warp has finished reading x and the output scale (fusion of j - 2) before
                // phase A overwrites them
                ok = mma_group_and(mbar_wait_bounded(&barH[j % 3], (uint32_t)(j / 3) & 1u));
                if (!ok) break;
                ++landed;
                if constexpr (T5) {
                    if (!t5_phase_a<BC, UL>(pl, tab, Hb(j), SROW, reinterpret_cast<float*>(smem + wl.off_op), barT, tpar,
                                        tbase, alpha, Gb(j), Dmb(j), Dpb(j), Zb(j), xs, Lb(j), yq)) {
                        ok = false;
                        break;
                    }
                }
                for (int c = warp; !T5 && c < C; c += kWsMmaWarps) {
                    const ClusterTile ct = tab[c];
                    float* Dm = Dmb(j) + c * UT;
                    tc_phase_a<BC, IN, UL, false>(pl, Hb(j) + ct.off * ew, SROW, d.Y, (size_t)fa * n_sym * pl.B + ct.off,
                                                  alpha, Gb(j) + (size_t)c * UT * (UT / 2), Dm, Dpb(j) + c * UT,
                                                  Zb(j) + c * n_sym, xs, nullptr, nullptr);
                    if constexpr (UL) {
                        __syncwarp();
                        if (lane == 0) {  // fusion weight 1 / sum_u m_u (a skipped column counts as infinite)
                            float msum = 0.f;
                            for (int u = 0; u < U; ++u) msum += Dm[u] > 0.f ? Dm[u] : __int_as_float(0x7f800000);
                            Lb(j)[c] = 1.f / msum;
                        }
                    }
                }
                if constexpr (DL) {  // s of j, transposed to [u][n]
                    float2* Ss = Sb(j);
                    if (tid < n_s) Ss[(tid % U) * n_sym + tid / U] = sv;
                    for (int i = tid + kMmaThreads; i < n_s; i += kMmaThreads)
                        Ss[(i % U) * n_sym + i / U] = __ldg(io.S + (size_t)fa * n_s + i);
                }
                mbar_arrive(&barA[j & 1]);
            }
        }
        // A copy still in flight (the loop left early): wait for it (bounded) before the CTA exits.
        if (!ok && tid == 0) {
            for (int s = landed; s < issued; ++s) mbar_wait_bounded(&barH[s % 3], (uint32_t)(s / 3) & 1u, 100000000ull);
            // and MMAs (their commit not yet waited for) before the tensor memory is freed
            if (T5) mbar_wait_bounded(barT, tpar & 1u, 100000000ull);
        }
    } else {
        // ------------------------------------------------------------------ sweep role
        // Two groups of four warps take alternate subcarriers (group g sweeps s = g, g + 2, ...; the
        // double-buffered G_c, z / x, w and s of s are group g's), so the sweeps of consecutive
        // subcarriers overlap and each sub-partition holds two sweep warps.  One lane per (cluster,
        // symbol) tile: the uplink x (right-hand side z) and the downlink w (right-hand side s) side
        // by side in the frame, reading the same rows of G_c.  Cluster sc = 32 / slot clusters per
        // warp, each in its own quarter or half warp.
        const int grp = (warp - kWsMmaWarps) / wl.sweep_warps, sw = (warp - kWsMmaWarps) % wl.sweep_warps;
        const int cpw = 32 / wl.slot;
        const int sc = sw * cpw + lane / wl.slot, n_b = lane % wl.slot;
        const bool active = sc < C && n_b < n_sym;
        const int tile = sc * n_sym + n_b;
        const uint32_t gbar = 2u + (uint32_t)grp, gthreads = 32u * (uint32_t)wl.sweep_warps;  // group barrier
        for (int s = grp; s < n_mine; s += kWsSweepGroups) {
            if (!group_and(mbar_wait_bounded(&barA[s & 1], (uint32_t)(s >> 1) & 1u), gbar, gthreads)) break;
            if (active) {
                float4 x[UT / 2], w[UT / 2];
                const float4* Gc = Gb(s) + (size_t)sc * UT * (UT / 2);
                const float* Dm = Dmb(s) + sc * UT;
                const float* Dp = Dpb(s) + sc * UT;
                if constexpr (MODE == kTcFrame)
                    gram_sweeps2<UT>(U, pl.K, Gc, Dm, Dp, Zb(s) + tile, xs, Sb(s) + n_b, (uint32_t)n_sym, x, w);
                else if constexpr (MODE == kTcDetect)
                    gram_sweeps<UT>(U, pl.K, Gc, Dm, Zb(s) + tile, xs, x);
                else
                    gram_sweeps<UT>(U, pl.K, Gc, Dp, Sb(s) + n_b, (uint32_t)n_sym, w);
#pragma unroll
                for (int u = 0; u < UT; ++u) {
                    if (u < U) {
                        if constexpr (UL) Zb(s)[tile + u * xs] = slice_entry<UT, 1>(x, u);
                        if constexpr (DL) Wb(s)[tile + u * xs] = slice_entry<UT, 1>(w, u);
                    }
                }
            }
            if constexpr (UL) {  // the fusion of s (Sec. III), on this group once every tile's x is written
                asm volatile("bar.sync %0, %1;" ::"r"(gbar), "r"(gthreads) : "memory");
                fuse_range(pl, d, fof(s), Lb(s), Zb(s), xs, osc[s & 1], kMmaThreads + grp * (int)gthreads,
                           (int)gthreads);
            }
            mbar_arrive(&barS[s & 1]);
        }
    }
    if (T5) tc_fence_before();
    __syncthreads();
    if (T5 && warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, wl.tmem_cols);
    }
}

}  // namespace cdmimo
