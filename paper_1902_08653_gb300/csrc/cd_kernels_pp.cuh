// Packed-FP32 (FFMA2), persistent, double-buffered CD detection and precoding kernels for uniform
// cluster sizes (every cluster has the same lanes-per-tile AT; P = 16 antennas per lane).
//
// Layout.  Every 16-byte antenna pair is held "pair-planar": (re_0, re_1, im_0, im_1) instead of
// (re_0, im_0, re_1, im_1), in shared memory (channel) and in registers (residual or beamformer).
// Each half of a pair is then a ready 64-bit operand of the sm_100-family packed instruction
// fma.rn.f32x2, and a complex multiply-accumulate over two antennas costs four packed FMAs:
//   correlation  sum conj(h) v:   R += h_re*v_re, R += h_im*v_im, I += h_re*v_im, J += h_im*v_re,
//                                  g = (R.x + R.y) + i((I.x + I.y) - (J.x + J.y));
//   update       v -= h d:         v_re += h_re*(-d_re) + h_im*d_im,  v_im += h_re*(-d_im) + h_im*(-d_re).
// The channel arrives by cp.async.bulk in the interleaved layout and is permuted in place (each
// thread owns whole 16-byte pairs).
//
// Schedule.  A persistent CTA walks subcarriers f = blockIdx.x, blockIdx.x + gridDim.x, ...  Two
// channel buffers alternate: while subcarrier f is computed from buffer k&1, the bulk copy of the
// next subcarrier lands in the other buffer, and the next subcarrier's y (or s) is loaded into
// registers right after the CD loop.  The preprocessing of Algorithm 1 / 2 (||h_{u,c}||^2 and the
// coefficients m, n or p^2) is computed inside the first sweep from the channel pairs each lane
// already holds for the correlation, and kept per tile in shared memory for the later sweeps.
#pragma once
#include "cd_kernels.cuh"

namespace cdmimo {

constexpr int kPP = 16;               // antennas per lane
constexpr int kPairs = kPP / 2;       // antenna pairs per lane
constexpr int kPPRegs = 128;          // register cap of the packed kernels (two 7-warp CTAs per SM)
constexpr int kSPrefetch = 4;         // s entries per thread prefetched by the precoder (n_sym U <= 4 threads)

__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float bf16_bits_to_float(unsigned short v) { return __uint_as_float((unsigned)v << 16); }

// (re0, im0, re1, im1) -> (re0, re1, im0, im1) for every 16-byte pair of one channel buffer.
__device__ __forceinline__ void permute_pairs_in_place(const CdPlan& pl, float2* Hs)
{
    float4* h4 = reinterpret_cast<float4*>(Hs);
    for (int i = threadIdx.x; i < pl.h_entries / 2; i += blockDim.x) {
        const float4 v = h4[i];
        h4[i] = make_float4(v.x, v.z, v.y, v.w);
    }
}

// Arm a buffer's barrier for the next copy: one arrival that announces the copy's byte count.  The
// copy itself is issued later, after the buffer's previous readers have passed a CTA barrier.
template <int IN>
__device__ __forceinline__ void arm_channel_copy(const CdPlan& pl, uint64_t* bar)
{
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, (uint32_t)pl.U * pl.B * (IN == CDMIMO_C64 ? 8u : 4u));
}

// Bulk copies of subcarrier f's channel rows: thread i issues row i (rows are (cluster, user)
// pairs).  64-bit complex rows land in the skewed per-cluster layout of a channel buffer; 16-bit
// rows land densely ([c][u][B_c], cluster c at U o_c) in a staging buffer, converted later.
template <int IN>
__device__ __forceinline__ void issue_channel_copy(const CdPlan& pl, const ClusterTile* tab, const void* H, int f,
                                                   void* dst, uint64_t* bar)
{
    constexpr uint32_t eb = IN == CDMIMO_C64 ? 8u : 4u;
    const char* Hf = reinterpret_cast<const char*>(H) + (size_t)f * pl.U * pl.B * eb;
    for (int row = threadIdx.x; row < pl.U * pl.C; row += blockDim.x) {
        const int c = row / pl.U, u = row - c * pl.U;
        const ClusterTile ct = tab[c];
        const size_t dofs = IN == CDMIMO_C64 ? (size_t)(ct.soff + u * ct.L) : (size_t)pl.U * ct.off + (size_t)u * ct.size;
        fence_proxy_async_smem();
        bulk_g2s(reinterpret_cast<char*>(dst) + dofs * eb, Hf + ((size_t)u * pl.B + ct.off) * eb, (uint32_t)ct.size * eb,
                 bar);
    }
}

// 16-bit staging buffer (dense rows) -> pair-planar FP32 channel rows, padding columns included.
template <int IN>
__device__ __forceinline__ void convert_staged(const CdPlan& pl, const ClusterTile* tab, const void* stg, float2* Hs)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int row = warp; row < pl.U * pl.C; row += nwarps) {
        const int c = row / pl.U, u = row - c * pl.U;
        const ClusterTile ct = tab[c];
        const size_t s0 = (size_t)pl.U * ct.off + (size_t)u * ct.size;
        float4* dst = reinterpret_cast<float4*>(Hs + ct.soff + u * ct.L);
        for (int q = lane; q < ct.L / 2; q += 32) {
            const int j = 2 * q;
            const float2 v0 = j < ct.size ? Elem<IN>::load_shared(stg, s0 + j) : make_float2(0.f, 0.f);
            const float2 v1 = j + 1 < ct.size ? Elem<IN>::load_shared(stg, s0 + j + 1) : make_float2(0.f, 0.f);
            dst[q] = make_float4(v0.x, v1.x, v0.y, v1.y);
        }
    }
}

// Converting channel staging (16-bit storage or odd cluster sizes): writes the pair-planar layout,
// padding columns included, directly.
template <int IN>
__device__ __forceinline__ void stage_H_converting(const CdPlan& pl, const ClusterTile* tab, const void* H, int f,
                                                   float2* Hs)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int row = warp; row < pl.U * pl.C; row += nwarps) {
        const int c = row / pl.U, u = row - c * pl.U;
        const ClusterTile ct = tab[c];
        const size_t g0 = ((size_t)f * pl.U + u) * pl.B + ct.off;
        float4* dst = reinterpret_cast<float4*>(Hs + ct.soff + u * ct.L);
        for (int q = lane; q < ct.L / 2; q += 32) {
            const int j = 2 * q;
            const float2 v0 = j < ct.size ? Elem<IN>::load(H, g0 + j) : make_float2(0.f, 0.f);
            const float2 v1 = j + 1 < ct.size ? Elem<IN>::load(H, g0 + j + 1) : make_float2(0.f, 0.f);
            dst[q] = make_float4(v0.x, v1.x, v0.y, v1.y);
        }
    }
}

// The lane's antenna pairs q = i*AT + a of a length-`size` vector as loaded: (re_j, im_j, re_{j+1}, im_{j+1}) per pair.
template <int IN, int AT>
__device__ __forceinline__ void load_lane_raw(const void* V, size_t base, int size, int a, float4 (&v)[kPairs])
{
    const float2 z = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kPairs; ++i) {
        const int j = 2 * (i * AT + a);
        const float2 v0 = j < size ? Elem<IN>::load(V, base + j) : z;
        const float2 v1 = j + 1 < size ? Elem<IN>::load(V, base + j + 1) : z;
        v[i] = make_float4(v0.x, v0.y, v1.x, v1.y);
    }
}

// To the pair-planar register layout (re_j, re_{j+1}, im_j, im_{j+1}).  The packed adds (of zero)
// write each pair into an aligned register pair, so the loop-carried vector needs no register moves
// in the sweeps' packed FMAs (measured: a third fewer uplink instructions).
__device__ __forceinline__ void raw_to_pairs(float4 (&v)[kPairs])
{
    const float2 z = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kPairs; ++i)
        v[i] = cat4(__fadd2_rn(make_float2(v[i].x, v[i].z), z), __fadd2_rn(make_float2(v[i].y, v[i].w), z));
}

template <int AT, int N>
__device__ __forceinline__ void pp_load_h(const float4* hr, float4 (&h)[N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) h[i] = hr[i * AT];
}

template <int AT>
__device__ __forceinline__ float tile_sum_c(float v, unsigned mask)
{
#pragma unroll
    for (int off = 1; off < AT; off <<= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

// Lane partial of conj(h)^T v over the lane's pairs (two independent accumulator sets; N even).
template <int N>
__device__ __forceinline__ float2 pp_partial_corr(const float4 (&h)[N], const float4 (&v)[N])
{
    static_assert(N % 2 == 0, "pairs per lane must be even");
    float2 R0 = make_float2(0.f, 0.f), I0 = R0, J0 = R0, R1 = R0, I1 = R0, J1 = R0;
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        R0 = ffma2(lo2(h[i]), lo2(v[i]), R0);
        I0 = ffma2(lo2(h[i]), hi2(v[i]), I0);
        J0 = ffma2(hi2(h[i]), lo2(v[i]), J0);
        R1 = ffma2(lo2(h[i + 1]), lo2(v[i + 1]), R1);
        I1 = ffma2(lo2(h[i + 1]), hi2(v[i + 1]), I1);
        J1 = ffma2(hi2(h[i + 1]), lo2(v[i + 1]), J1);
        R0 = ffma2(hi2(h[i]), hi2(v[i]), R0);
        R1 = ffma2(hi2(h[i + 1]), hi2(v[i + 1]), R1);
    }
    const float2 R = __fadd2_rn(R0, R1), I = __fadd2_rn(I0, I1), J = __fadd2_rn(J0, J1);
    return make_float2(R.x + R.y, (I.x + I.y) - (J.x + J.y));
}

// Lane partial of ||h||^2 over the lane's pairs.
__device__ __forceinline__ float pp_partial_energy(const float4 (&h)[kPairs])
{
    float2 E0 = make_float2(0.f, 0.f), E1 = E0;
#pragma unroll
    for (int i = 0; i < kPairs; i += 2) {
        E0 = ffma2(lo2(h[i]), lo2(h[i]), E0);
        E1 = ffma2(lo2(h[i + 1]), lo2(h[i + 1]), E1);
        E0 = ffma2(hi2(h[i]), hi2(h[i]), E0);
        E1 = ffma2(hi2(h[i + 1]), hi2(h[i + 1]), E1);
    }
    const float2 E = __fadd2_rn(E0, E1);
    return E.x + E.y;
}

// v -= h d (packed FMAs).
__device__ __forceinline__ void pp_update(const float4 (&h)[kPairs], float2 d, float4 (&v)[kPairs])
{
    const float2 ndr = make_float2(-d.x, -d.x), pdi = make_float2(d.y, d.y), ndi = make_float2(-d.y, -d.y);
#pragma unroll
    for (int i = 0; i < kPairs; ++i) {
        float2 re = ffma2(lo2(h[i]), ndr, lo2(v[i]));
        float2 im = ffma2(lo2(h[i]), ndi, hi2(v[i]));
        re = ffma2(hi2(h[i]), pdi, re);
        im = ffma2(hi2(h[i]), ndr, im);
        v[i] = cat4(re, im);
    }
}

// pp_update, reloading each h[i] from the next row right after its last use (the loads of the next
// step issue during this step's update without extra registers).
template <int AT, int N>
__device__ __forceinline__ void pp_update_reload(float4 (&h)[N], float2 d, float4 (&v)[N], const float4* next)
{
    const float2 ndr = make_float2(-d.x, -d.x), pdi = make_float2(d.y, d.y), ndi = make_float2(-d.y, -d.y);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float2 re = ffma2(lo2(h[i]), ndr, lo2(v[i]));
        float2 im = ffma2(lo2(h[i]), ndi, hi2(v[i]));
        re = ffma2(hi2(h[i]), pdi, re);
        im = ffma2(hi2(h[i]), ndr, im);
        v[i] = cat4(re, im);
        h[i] = next[i * AT];
    }
}

// Wait for (bulk) or stage (converting) the channel of subcarrier f in buffer Hb, then permute it to
// the pair-planar layout.  Returns false on a copy timeout (the whole CTA then stops).
template <int IN>
__device__ __forceinline__ bool acquire_channel(const CdPlan& pl, const ClusterTile* tab, const void* H, int f,
                                                float2* Hb, const void* stg, uint64_t* bar, uint32_t parity,
                                                bool rearm)
{
    bool ok = true;
    if (pl.bulk) ok = mbar_wait_bounded(bar, parity);
    else stage_H_converting<IN>(pl, tab, H, f, Hb);
    if (__syncthreads_or(!ok)) return false;
    // This buffer next receives the copy issued at the start of the next iteration: arm it now.
    if (pl.bulk && rearm && threadIdx.x == 0) arm_channel_copy<IN>(pl, bar);
    if (pl.bulk) {
        if (IN == CDMIMO_C64) permute_pairs_in_place(pl, Hb);
        else convert_staged<IN>(pl, tab, stg, Hb);
        __syncthreads();
    }
    return true;
}

// Subcarrier schedule of the persistent kernels.  With G CTAs, CTA i starts with subcarriers i and
// i + G.  Static (no counters): it goes on with i + 2G, i + 3G, ...  Dynamic (three counters in the
// caller's workspace): each later subcarrier is 2G + a ticket drawn from counter 0 one iteration
// ahead, so CTAs that run faster take more subcarriers.  A subcarrier's result does not depend on
// the CTA that computes it, so both schedules give the same output bit for bit.
__device__ __forceinline__ unsigned sched_draw(unsigned* sched, bool need)
{
    return (sched && need && threadIdx.x == 0) ? atomicAdd(sched, 1u) : 0u;
}

// The subcarrier after fn (n_sc: none).
__device__ __forceinline__ int sched_next(const unsigned* sched, bool drew, unsigned ticket, int fn, int n_sc)
{
    if (!sched) return fn + (int)gridDim.x;
    const unsigned v = 2u * gridDim.x + ticket;
    return (drew && v < (unsigned)n_sc) ? (int)v : n_sc;
}

// End of a dynamically scheduled launch: counter 1 counts finished CTAs, counter 2 subcarriers
// done.  The last CTA checks that every subcarrier was taken exactly once and zeroes the counters
// for the next call on the same workspace.
__device__ __forceinline__ void sched_finish(unsigned* sched, int done, int n_sc)
{
    if (!sched || threadIdx.x != 0) return;
    atomicAdd(sched + 2, (unsigned)done);
    __threadfence();
    if (atomicAdd(sched + 1, 1u) == gridDim.x - 1u) {
        __threadfence();
        if (atomicAdd(sched + 2, 0u) != (unsigned)n_sc) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_SCHED);
        sched[0] = 0u;
        sched[1] = 0u;
        sched[2] = 0u;
        __threadfence();
    }
}

// Data fusion of one subcarrier (Sec. III): xhat = sum_c lambda_c x_c from the per-tile estimates
// Xs[u][c n_sym + n].  FINAL: lam holds lambda_c.  Otherwise lam holds w_c = 1 / sum_u m_{u,c} and
// lambda_c = w_c / sum_c' w_c' (COLNORM), or 1 / C (EQUAL, or no positive weight).  Optional
// outputs: the per-cluster estimates io.Xc and the weights io.lam (plain rules; the learned fusion
// writes its own).
template <bool FINAL>
__device__ __forceinline__ void fuse_subcarrier(const CdPlan& pl, const DetectIO& io, int f, const float* lam,
                                                const float2* Xs, uint32_t xs_stride, float out_scale)
{
    const int tid = threadIdx.x, C = pl.C, U = pl.U, n_sym = pl.n_sym;
    float inv = 1.f;
    bool equal = false;
    if (!FINAL) {
        float tot = 0.f;
        for (int c = 0; c < C; ++c) tot += lam[c];
        equal = pl.fuse == CDMIMO_FUSE_EQUAL || !(tot > 0.f);
        inv = equal ? 1.f / (float)C : 1.f / tot;
        if (io.lam && tid < C) io.lam[(size_t)f * C + tid] = equal ? inv : lam[tid] * inv;
    }
    for (int i = tid; i < n_sym * U; i += blockDim.x) {
        const int n = i / U, u = i - n * U;
        float2 acc = make_float2(0.f, 0.f);
        for (int c = 0; c < C; ++c) {
            const float l = FINAL ? lam[c] : (equal ? inv : lam[c] * inv);
            const float2 x = Xs[u * xs_stride + c * n_sym + n];
            acc.x = fmaf(l, x.x, acc.x);
            acc.y = fmaf(l, x.y, acc.y);
            if (io.Xc) io.Xc[(((size_t)f * C + c) * n_sym + n) * U + u] = make_float2(x.x * out_scale, x.y * out_scale);
        }
        io.Xhat[((size_t)f * n_sym + n) * U + u] = make_float2(acc.x * out_scale, acc.y * out_scale);
    }
}

// Learned fusion weights of one subcarrier: lambda = softmax_c(logit_c), logit_c = b2 + sum_kk
// w2[kk] relu(z_kk), z_kk = W1[kk] . phi_c + b1[kk] with phi_c = [e(c, u) / B_c (u < U),
// log10(max(alpha, 1e-6))] and e(c, u) = ||h_{u,c}||^2 (from the caller's accessor).  Warp 0 writes
// lam (and lam_out[f] if given): the caller puts a barrier before reading it.  Uses mlp[C][hidden]
// as scratch (one internal barrier).
template <typename EnergyFn>
__device__ __forceinline__ void learned_lambda(const CdPlan& pl, const cdmimo_learned* blk, bool learned_ok, float alpha,
                                               const ClusterTile* tab, float* mlp, float* lam, float* lam_out, int f,
                                               EnergyFn energy)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, C = pl.C, U = pl.U;
    const int Hd = learned_ok ? __ldg(&blk->hidden) : 1;
    const int F = U + 1;
    const float la = log10f(fmaxf(alpha, 1e-6f));
    for (int i = tid; i < C * Hd; i += blockDim.x) {
        const int c = i / Hd, kk = i - c * Hd;
        const float inv_bc = 1.f / (float)tab[c].size;
        const unsigned short* w1 = blk->W1 + (size_t)kk * F;
        float z = __ldg(&blk->b1[kk]);
        for (int j = 0; j < U; ++j) z = fmaf(bf16_bits_to_float(__ldg(w1 + j)), energy(c, j) * inv_bc, z);
        z = fmaf(bf16_bits_to_float(__ldg(w1 + U)), la, z);
        mlp[i] = bf16_bits_to_float(__ldg(&blk->w2[kk])) * fmaxf(z, 0.f);
    }
    __syncthreads();
    if (warp == 0) {
        float lg[2] = {-__int_as_float(0x7f800000), -__int_as_float(0x7f800000)};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c = lane + 32 * q;
            if (c < C) {
                float s = __ldg(&blk->b2);
                for (int kk = 0; kk < Hd; ++kk) s += mlp[c * Hd + kk];
                lg[q] = s;
            }
        }
        float mx = fmaxf(lg[0], lg[1]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float ex[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) ex[q] = lane + 32 * q < C ? __expf(lg[q] - mx) : 0.f;
        const float tot = warp_sum(ex[0] + ex[1]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c = lane + 32 * q;
            if (c < C) {
                lam[c] = ex[q] / tot;
                if (lam_out) lam_out[(size_t)f * C + c] = ex[q] / tot;
            }
        }
    }
}

// Column energies of one cluster from a staged buffer (K = 0 only: no sweep computed them).
__device__ __forceinline__ float row_energy(const float2* row, int L)
{
    float e = 0.f;
    for (int j = 0; j < L; ++j) e = fmaf(row[j].x, row[j].x, fmaf(row[j].y, row[j].y, e));
    return e;
}

// ---------------------------------------------------------------------------------------------
// Uplink: Algorithm 1 + fusion (Sec. III).
// ---------------------------------------------------------------------------------------------
template <int IN, int AT, bool LEARNED>
__global__ void __maxnreg__(kPPRegs) cd_detect_pp_kernel(const CdPlan pl, const DetectIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    // Channel buffer j: 64-bit storage double-buffers the channel itself (buffer 1 at off_H2); 16-bit
    // storage double-buffers the raw copies (staging j at off_H2 / off_H3) and converts into one buffer.
    auto Hbuf = [&](int j) { return reinterpret_cast<float2*>(smem + ((IN == CDMIMO_C64 && j) ? pl.off_H2 : 0u)); };
    auto Stg = [&](int j) { return reinterpret_cast<void*>(smem + (j ? pl.off_H3 : pl.off_H2)); };
    auto Dst = [&](int j) { return IN == CDMIMO_C64 ? reinterpret_cast<void*>(Hbuf(j)) : Stg(j); };
    float2* Xs = reinterpret_cast<float2*>(smem + pl.off_X);  // [U][x_stride] current x per tile
    // [U][x_stride] per tile: (m, n) of Algorithm 1; learned sweeps keep (||h_{u,c}||^2, m) instead
    float2* Ks = reinterpret_cast<float2*>(smem + pl.off_K);
    float* lam = reinterpret_cast<float*>(smem + pl.off_lam); // [C]
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);  // [2]
    int* nxt = reinterpret_cast<int*>(smem + pl.off_bar + 16);       // [2] schedule hand-off

    float* mlp = reinterpret_cast<float*>(smem + pl.off_mlp);   // [C][hidden <= 64] (learned fusion)
    const cdmimo_learned* blk = reinterpret_cast<const cdmimo_learned*>(io.learned);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    const uint32_t xs_stride = x_stride(pl);
    constexpr int LP = AT * kPairs;  // shared-memory row length in pairs
    bool learned_ok = true;
    if (LEARNED) {
        const int hd = __ldg(&blk->hidden);
        learned_ok = __ldg(&blk->K) == pl.K && __ldg(&blk->U) == U && hd >= 1 && hd <= CDMIMO_MAX_HIDDEN;
        if (!learned_ok && tid == 0 && blockIdx.x == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_LEARNED);
    }

    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0 && pl.bulk) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    if (pl.bulk) {  // padding columns are never written by the copies: zero them once in both buffers
        zero_padding(pl, tab, Hbuf(0));
        zero_padding(pl, tab, Hbuf(1));
    }
    __syncthreads();
    const LaneTile lt = map_lane(pl, tab);
    const ClusterTile ct = tab[lt.c];
    const int tile = lt.c * n_sym + lt.n;

    int f = blockIdx.x;
    if (pl.bulk && tid == 0) {  // arm buffer 0 (first subcarrier) and buffer 1 (second)
        if (f < pl.n_sc) arm_channel_copy<IN>(pl, &bar[0]);
        if (f + (int)gridDim.x < pl.n_sc) arm_channel_copy<IN>(pl, &bar[1]);
    }
    __syncthreads();
    if (pl.bulk && f < pl.n_sc) issue_channel_copy<IN>(pl, tab, io.H, f, Dst(0), &bar[0]);
    float4 r[kPairs];
    if (lt.active && f < pl.n_sc) {
        load_lane_raw<IN, AT>(io.Y, ((size_t)f * n_sym + lt.n) * pl.B + ct.off, ct.size, lt.a, r);
        raw_to_pairs(r);
    }

    int fn = f + (int)gridDim.x;  // this CTA's next subcarrier
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
            alpha = alpha / (hs * hs);  // regularizer of the problem in stored units
            out_scale = ys / hs;        // x = (b_f / a_f) x'
        }
        if (!(alpha >= 0.f)) {  // negative or NaN noise variance
            if (tid == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_N0);
            out_scale = __int_as_float(0x7fc00000);
            alpha = 0.f;
        }
        if (LEARNED && !learned_ok) out_scale = __int_as_float(0x7fc00000);
        if (!acquire_channel<IN>(pl, tab, io.H, f, Hbuf(b), Stg(b), &bar[b], (uint32_t)(k >> 1) & 1u,
                                 io.sched != nullptr || fn + (int)gridDim.x < pl.n_sc)) {
            // copy timeout: let the copy in flight into the other buffer land (bounded), then stop
            if (pl.bulk && fn < pl.n_sc && tid == 0) mbar_wait_bounded(&bar[b ^ 1], (uint32_t)((k + 1) >> 1) & 1u);
            break;
        }

        if (LEARNED && lt.active && pl.K > 0) {
            // Learned sweeps: x_u <- a1 h^H r + a2 x_u with a1 = tau_t / (e + gamma_t alpha),
            // a2 = 1 - a1 gamma_t alpha (a skipped column when the denominator is not positive).
            const float4* hb = reinterpret_cast<const float4*>(Hbuf(b) + ct.soff) + lt.a;
            float2* xs = Xs + tile;
            float2* ks = Ks + tile;
            for (int t = 0; t < pl.K; ++t) {
                const float tau = __ldg(&blk->tau[t]), gam = __ldg(&blk->gamma[t]);
                const float ga = gam * alpha;
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    float4 h[kPairs];
                    pp_load_h<AT>(hb + u * LP, h);
                    float2 g = pp_partial_corr(h, r);
                    float e;
                    if (t == 0) {
                        e = pp_partial_energy(h);
#pragma unroll
                        for (int off = 1; off < AT; off <<= 1) e += __shfl_xor_sync(lt.mask, e, off);
                        const float den0 = e + alpha;
                        ks[u * xs_stride] = make_float2(e, den0 > 0.f ? __fdividef(1.f, den0) : 0.f);
                    } else {
                        e = ks[u * xs_stride].x;
                    }
                    g.x = tile_sum_c<AT>(g.x, lt.mask);
                    g.y = tile_sum_c<AT>(g.y, lt.mask);
                    const float den = e + ga;
                    const float a1 = den > 0.f ? tau * __fdividef(1.f, den) : 0.f;
                    const float a2 = 1.f - a1 * ga;
                    const float2 xo = t == 0 ? make_float2(0.f, 0.f) : xs[u * xs_stride];
                    const float2 xn = make_float2(fmaf(a1, g.x, a2 * xo.x), fmaf(a1, g.y, a2 * xo.y));
                    xs[u * xs_stride] = xn;
                    pp_update(h, make_float2(xn.x - xo.x, xn.y - xo.y), r);
                }
            }
        }
        if (!LEARNED && lt.active && pl.K > 0) {
            const float4* hb = reinterpret_cast<const float4*>(Hbuf(b) + ct.soff) + lt.a;
            float2* xs = Xs + tile;
            float2* ks = Ks + tile;
            // Sweep 1 with the preprocessing of Algorithm 1 folded in: e = ||h_{u,c}||^2,
            // m = (e + N0/Ex)^{-1}, n = m e; x starts at 0, so x_u <- m h^H r.  Every lane also sums
            // m over u for the fusion weight of its cluster (a skipped column, m = 0, counts as an
            // infinite (||h||^2 + N0/Ex)^{-1} and gives the cluster weight 0).
            float msum = 0.f;
#pragma unroll 1
            for (int u = 0; u < U; ++u) {
                float4 h[kPairs];
                pp_load_h<AT>(hb + u * LP, h);
                float2 g = pp_partial_corr(h, r);
                float e = pp_partial_energy(h);
#pragma unroll
                for (int off = 1; off < AT; off <<= 1) {
                    g.x += __shfl_xor_sync(lt.mask, g.x, off);
                    g.y += __shfl_xor_sync(lt.mask, g.y, off);
                    e += __shfl_xor_sync(lt.mask, e, off);
                }
                const float den = e + alpha;
                const float m = den > 0.f ? __fdividef(1.f, den) : 0.f;
                msum += m > 0.f ? m : __int_as_float(0x7f800000);
                ks[u * xs_stride] = make_float2(m, m * e);
                const float2 xn = make_float2(m * g.x, m * g.y);
                xs[u * xs_stride] = xn;
                pp_update(h, xn, r);
            }
            for (int t = 1; t < pl.K; ++t) {
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    float4 h[kPairs];
                    pp_load_h<AT>(hb + u * LP, h);
                    float2 g = pp_partial_corr(h, r);
                    g.x = tile_sum_c<AT>(g.x, lt.mask);
                    g.y = tile_sum_c<AT>(g.y, lt.mask);
                    const float2 kc = ks[u * xs_stride];
                    const float2 xo = xs[u * xs_stride];
                    const float2 xn = make_float2(fmaf(kc.x, g.x, kc.y * xo.x), fmaf(kc.x, g.y, kc.y * xo.y));
                    xs[u * xs_stride] = xn;
                    pp_update(h, make_float2(xn.x - xo.x, xn.y - xo.y), r);
                }
            }
            if (lt.n == 0 && lt.a == 0) lam[lt.c] = 1.f / msum;  // w_c, normalized in the fusion
        }
        if (pl.K == 0) {  // no sweep ran: x = 0, and the fusion weights still need m
            for (int i = tid; i < U * (int)xs_stride; i += blockDim.x) Xs[i] = make_float2(0.f, 0.f);
            if (lt.active && lt.a == 0) {
                float msum = 0.f;
                for (int u = 0; u < U; ++u) {
                    const float e = row_energy(Hbuf(b) + ct.soff + u * ct.L, ct.L);
                    const float m = e + alpha > 0.f ? __fdividef(1.f, e + alpha) : 0.f;
                    msum += m > 0.f ? m : __int_as_float(0x7f800000);
                    Ks[u * xs_stride + tile] = LEARNED ? make_float2(e, m) : make_float2(m, 0.f);
                }
                if (!LEARNED && lt.n == 0) lam[lt.c] = 1.f / msum;
            }
        }
        if (tid == 0) nxt[b] = sched_next(io.sched, draw, ticket, fn, pl.n_sc);
        // Prefetch the next subcarrier's receive vector (r is dead from here on).
        if (lt.active && fn < pl.n_sc) {
            load_lane_raw<IN, AT>(io.Y, ((size_t)fn * n_sym + lt.n) * pl.B + ct.off, ct.size, lt.a, r);
            raw_to_pairs(r);  // at load: deferring it to the sweeps costs the 16-bit kernels 20% (measured)
        }
        __syncthreads();

        if (LEARNED) {  // lambda_c from the learned fusion (or from m, below), then a barrier
            if (pl.fuse == CDMIMO_FUSE_LEARNED) {
                learned_lambda(pl, blk, learned_ok, alpha, tab, mlp, lam, io.lam, f,
                               [&](int c, int j) { return Ks[j * xs_stride + c * n_sym].x; });
            } else if (warp == 0) {
                // Fusion weights: lambda_c proportional to 1 / sum_u m_{u,c} (a zero m marks a skipped
                // column, whose (||h||^2 + N0/Ex)^{-1} is infinite).
                float w[2] = {0.f, 0.f};
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = lane + 32 * q;
                    if (c < C) {
                        float s = 0.f;
                        for (int u = 0; u < U; ++u) {
                            const float m = Ks[u * xs_stride + c * n_sym].y;  // learned sweeps keep (e, m)
                            s += m > 0.f ? m : __int_as_float(0x7f800000);
                        }
                        w[q] = 1.f / s;
                    }
                }
                const float tot = warp_sum(w[0] + w[1]);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = lane + 32 * q;
                    if (c < C) {
                        const float l = (pl.fuse == CDMIMO_FUSE_EQUAL || !(tot > 0.f)) ? 1.f / C : w[q] / tot;
                        lam[c] = l;
                        if (io.lam) io.lam[(size_t)f * C + c] = l;
                    }
                }
            }
            __syncthreads();
        }
        fuse_subcarrier<LEARNED>(pl, io, f, lam, Xs, xs_stride, out_scale);
        // No barrier here: the next writes of Xs, Ks and lam come after the next acquire's barriers,
        // and the copy into this iteration's channel buffer is issued after the barrier above.
        ++done;
        f = fn;
        fn = nxt[b];
    }
    sched_finish(io.sched, done, pl.n_sc);
}

// ---------------------------------------------------------------------------------------------
// Downlink: Algorithm 2 (Eq. (4), applied as x -= p^2 (h^H x - s) h) + normalization (Sec. IV-B).
// ---------------------------------------------------------------------------------------------
template <int IN, int AT>
__global__ void __maxnreg__(kPPRegs) cd_precode_pp_kernel(const CdPlan pl, const PrecodeIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    // Channel buffer j: 64-bit storage double-buffers the channel itself (buffer 1 at off_H2); 16-bit
    // storage double-buffers the raw copies (staging j at off_H2 / off_H3) and converts into one buffer.
    auto Hbuf = [&](int j) { return reinterpret_cast<float2*>(smem + ((IN == CDMIMO_C64 && j) ? pl.off_H2 : 0u)); };
    auto Stg = [&](int j) { return reinterpret_cast<void*>(smem + (j ? pl.off_H3 : pl.off_H2)); };
    auto Dst = [&](int j) { return IN == CDMIMO_C64 ? reinterpret_cast<void*>(Hbuf(j)) : Stg(j); };
    float* Qs = reinterpret_cast<float*>(smem + pl.off_K);    // [U][x_stride] p_{u,c}^2 per tile
    float2* Ss = reinterpret_cast<float2*>(smem + pl.off_S);  // [n_sym][U | 1] (odd stride: no bank conflicts)
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);  // [2]
    int* nxt = reinterpret_cast<int*>(smem + pl.off_bar + 16);       // [2] schedule hand-off

    const int tid = threadIdx.x;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    const int s_stride = U | 1;
    const int n_s = n_sym * U;
    const uint32_t xs_stride = x_stride(pl);
    constexpr int LP = AT * kPairs;
    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0 && pl.bulk) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    if (pl.bulk) {
        zero_padding(pl, tab, Hbuf(0));
        zero_padding(pl, tab, Hbuf(1));
    }
    __syncthreads();
    const LaneTile lt = map_lane(pl, tab);
    const ClusterTile ct = tab[lt.c];
    const int tile = lt.c * n_sym + lt.n;

    int f = blockIdx.x;
    if (pl.bulk && tid == 0) {  // arm buffer 0 (first subcarrier) and buffer 1 (second)
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

    int fn = f + (int)gridDim.x;  // this CTA's next subcarrier
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
        // The next subcarrier's s (this one's is in shared memory now).
#pragma unroll
        for (int q = 0; q < kSPrefetch; ++q) {
            const int i = tid + q * blockDim.x;
            if (i < n_s && fn < pl.n_sc) sv[q] = __ldg(io.S + (size_t)fn * n_s + i);
        }

        if (lt.active) {
            float4 x[kPairs];
#pragma unroll
            for (int i = 0; i < kPairs; ++i) x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4* hb = reinterpret_cast<const float4*>(Hbuf(b) + ct.soff) + lt.a;
            float* qs = Qs + tile;
            const float2* s = Ss + lt.n * s_stride;
            if (pl.K > 0) {
                // Sweep 1 with the preprocessing of Algorithm 2 folded in: p^2 = ||h_{u,c}||^{-2}.
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    float4 h[kPairs];
                    pp_load_h<AT>(hb + u * LP, h);
                    float2 g = pp_partial_corr(h, x);
                    float e = pp_partial_energy(h);
#pragma unroll
                    for (int off = 1; off < AT; off <<= 1) {
                        g.x += __shfl_xor_sync(lt.mask, g.x, off);
                        g.y += __shfl_xor_sync(lt.mask, g.y, off);
                        e += __shfl_xor_sync(lt.mask, e, off);
                    }
                    const float q = e > 0.f ? __fdividef(1.f, e) : 0.f;
                    qs[u * xs_stride] = q;
                    const float2 su = s[u];
                    pp_update(h, make_float2(q * (g.x - su.x), q * (g.y - su.y)), x);
                }
            }
            for (int t = 1; t < pl.K; ++t) {
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    float4 h[kPairs];
                    pp_load_h<AT>(hb + u * LP, h);
                    float2 g = pp_partial_corr(h, x);
                    g.x = tile_sum_c<AT>(g.x, lt.mask);
                    g.y = tile_sum_c<AT>(g.y, lt.mask);
                    const float q = qs[u * xs_stride];
                    const float2 su = s[u];
                    pp_update(h, make_float2(q * (g.x - su.x), q * (g.y - su.y)), x);
                }
            }
            // ||x_c|| over the tile, then x_c <- rho_c x_c / ||x_c||.
            float nr = 0.f;
#pragma unroll
            for (int i = 0; i < kPairs; ++i)
                nr = fmaf(x[i].x, x[i].x, fmaf(x[i].y, x[i].y, fmaf(x[i].z, x[i].z, fmaf(x[i].w, x[i].w, nr))));
            nr = tile_sum_c<AT>(nr, lt.mask);
            const float sc = nr > 0.f ? pl.rho_c * rsqrtf(nr) : 0.f;
            float2* out = io.Xdl + ((size_t)f * n_sym + lt.n) * pl.B + ct.off;
#pragma unroll
            for (int i = 0; i < kPairs; ++i) {
                const int col = 2 * (i * AT + lt.a);
                if (col < ct.size) out[col] = make_float2(x[i].x * sc, x[i].z * sc);
                if (col + 1 < ct.size) out[col + 1] = make_float2(x[i].y * sc, x[i].w * sc);
            }
        }
        if (tid == 0) nxt[b] = sched_next(io.sched, draw, ticket, fn, pl.n_sc);
        __syncthreads();
        ++done;
        f = fn;
        fn = nxt[b];
    }
    sched_finish(io.sched, done, pl.n_sc);
}

}  // namespace cdmimo
