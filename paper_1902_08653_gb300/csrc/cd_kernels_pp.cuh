// Packed-FP32 (FFMA2) variants of the CD detection and precoding kernels for uniform cluster sizes.
//
// Same tiling as cd_kernels.cuh (plan.h) with P = 16 antennas per lane and a compile-time number AT
// of lanes per tile, but every 16-byte antenna pair is held "pair-planar": (re_0, re_1, im_0, im_1)
// instead of (re_0, im_0, re_1, im_1), in shared memory (channel) and in registers (residual or
// beamformer).  Then each half of a pair is a ready 64-bit operand of the sm_100-family packed
// instruction fma.rn.f32x2, and a complex multiply-accumulate of two antennas costs four packed FMAs
// with no operand shuffling:
//   correlation  sum conj(h) v:   R += h_re*v_re, R += h_im*v_im, I += h_re*v_im, J += h_im*v_re,
//                                  g = (R.x + R.y) + i((I.x + I.y) - (J.x + J.y));
//   update       v -= h d:         v_re += h_re*(-d_re) + h_im*d_im,  v_im += h_re*(-d_im) + h_im*(-d_re).
// The channel arrives by cp.async.bulk in the interleaved layout and is permuted in place (each
// thread owns whole 16-byte pairs, so the permutation needs no extra buffer).
#pragma once
#include "cd_kernels.cuh"

namespace cdmimo {

constexpr int kPP = 16;               // antennas per lane
constexpr int kPairs = kPP / 2;       // antenna pairs per lane
constexpr int kPPRegs = 128;          // register cap of the packed kernels (two 7-warp CTAs per SM)

__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// (re0, im0, re1, im1) -> (re0, re1, im0, im1) for every 16-byte pair of the channel region.
__device__ __forceinline__ void permute_pairs_in_place(const CdPlan& pl, float2* Hs)
{
    float4* h4 = reinterpret_cast<float4*>(Hs);
    for (int i = threadIdx.x; i < pl.h_entries / 2; i += blockDim.x) {
        const float4 v = h4[i];
        h4[i] = make_float4(v.x, v.z, v.y, v.w);
    }
}

// Channel staging for the packed kernels: bulk copies (permuted after the wait by the caller), or
// converting loads that write the pair-planar layout directly (16-bit storage, odd sizes).
template <int IN>
__device__ __forceinline__ void stage_H_pp(const CdPlan& pl, const ClusterTile* tab, const void* H, int f,
                                           float2* Hs, uint64_t* bar)
{
    if (pl.bulk) {
        stage_H<IN>(pl, tab, H, f, Hs, bar);
        return;
    }
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

// This lane's antenna pairs q = i*AT + a of a length-`size` vector, pair-planar.
template <int IN, int AT>
__device__ __forceinline__ void load_lane_pairs(const void* V, size_t base, int size, int a, float4 (&v)[kPairs])
{
#pragma unroll
    for (int i = 0; i < kPairs; ++i) {
        const int j = 2 * (i * AT + a);
        const float2 v0 = j < size ? Elem<IN>::load(V, base + j) : make_float2(0.f, 0.f);
        const float2 v1 = j + 1 < size ? Elem<IN>::load(V, base + j + 1) : make_float2(0.f, 0.f);
        v[i] = make_float4(v0.x, v1.x, v0.y, v1.y);
    }
}

// g = sum over the tile of conj(h) v (packed FMAs, two independent accumulator sets).
template <int AT>
__device__ __forceinline__ float2 pp_correlate(const float4 (&h)[kPairs], const float4 (&v)[kPairs], unsigned mask)
{
    float2 R0 = make_float2(0.f, 0.f), I0 = R0, J0 = R0, R1 = R0, I1 = R0, J1 = R0;
#pragma unroll
    for (int i = 0; i < kPairs; i += 2) {
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
    float gr = R.x + R.y;
    float gi = (I.x + I.y) - (J.x + J.y);
#pragma unroll
    for (int off = 1; off < AT; off <<= 1) {
        gr += __shfl_xor_sync(mask, gr, off);
        gi += __shfl_xor_sync(mask, gi, off);
    }
    return make_float2(gr, gi);
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

template <int AT>
__device__ __forceinline__ void pp_load_h(const float4* hr, float4 (&h)[kPairs])
{
#pragma unroll
    for (int i = 0; i < kPairs; ++i) h[i] = hr[i * AT];
}

// ---------------------------------------------------------------------------------------------
// Uplink: Algorithm 1 + fusion (Sec. III), packed arithmetic.
// ---------------------------------------------------------------------------------------------
template <int IN, int AT>
__global__ void __maxnreg__(kPPRegs) cd_detect_pp_kernel(const CdPlan pl, const DetectIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float2* Hs = reinterpret_cast<float2*>(smem);
    float2* Xs = reinterpret_cast<float2*>(smem + pl.off_X);     // [U][x_stride] current x per tile
    float2* coef = reinterpret_cast<float2*>(smem + pl.off_coef); // [U][C] (m, n) of Algorithm 1
    float* esum = reinterpret_cast<float*>(smem + pl.off_e);      // [U][C] ||h_{u,c}||^2
    float* lam = reinterpret_cast<float*>(smem + pl.off_lam);     // [C] fusion weights
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    const uint32_t xs_stride = x_stride(pl);
    constexpr int LP = AT * kPairs;  // shared-memory row length in pairs

    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0 && pl.bulk) {
        mbar_init(bar, 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    zero_padding(pl, tab, Hs);
    const LaneTile lt = map_lane(pl, tab);
    const ClusterTile ct = tab[lt.c];
    const int tile = lt.c * n_sym + lt.n;

    uint32_t phase = 0;
    for (int f = blockIdx.x; f < pl.n_sc; f += gridDim.x, phase ^= 1u) {
        stage_H_pp<IN>(pl, tab, io.H, f, Hs, bar);

        float4 r[kPairs];
        if (lt.active) load_lane_pairs<IN, AT>(io.Y, ((size_t)f * n_sym + lt.n) * pl.B + ct.off, ct.size, lt.a, r);

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

        bool ok = true;
        if (pl.bulk) ok = mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(!ok)) return;
        if (pl.bulk) {
            permute_pairs_in_place(pl, Hs);
            __syncthreads();
        }

        // Preprocessing (decentralized): ||h_{u,c}||^2 is the sum of squares of the row's floats,
        // whatever their order, then m and n.
        column_energies(pl, tab, Hs, esum);
        __syncthreads();
        for (int i = tid; i < C * U; i += blockDim.x) {
            const float e = esum[i];
            const float den = e + alpha;
            const float m = den > 0.f ? 1.f / den : 0.f;
            coef[i] = make_float2(m, m * e);
        }
        for (int i = tid; i < U * (int)xs_stride; i += blockDim.x) Xs[i] = make_float2(0.f, 0.f);
        if (warp == 0) {
            float w[2] = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int c = lane + 32 * k;
                if (c < C) {
                    float s = 0.f;
                    for (int u = 0; u < U; ++u) {
                        const float den = esum[u * C + c] + alpha;
                        s += den > 0.f ? 1.f / den : __int_as_float(0x7f800000);
                    }
                    w[k] = 1.f / s;
                }
            }
            const float tot = warp_sum(w[0] + w[1]);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int c = lane + 32 * k;
                if (c < C) {
                    const float l = (pl.fuse == CDMIMO_FUSE_EQUAL || !(tot > 0.f)) ? 1.f / C : w[k] / tot;
                    lam[c] = l;
                    if (io.lam) io.lam[(size_t)f * C + c] = l;
                }
            }
        }
        __syncthreads();

        // CD iterations (decentralized).
        if (lt.active) {
            const float4* hb = reinterpret_cast<const float4*>(Hs + ct.soff) + lt.a;
            float2* xs = Xs + tile;
            const float2* cf = coef + lt.c;
            for (int t = 0; t < pl.K; ++t) {
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    float4 h[kPairs];
                    pp_load_h<AT>(hb + u * LP, h);
                    const float2 g = pp_correlate<AT>(h, r, lt.mask);
                    const float2 k = cf[u * C];
                    const float2 xo = xs[u * xs_stride];
                    const float2 xn = make_float2(fmaf(k.x, g.x, k.y * xo.x), fmaf(k.x, g.y, k.y * xo.y));
                    xs[u * xs_stride] = xn;
                    pp_update(h, make_float2(xn.x - xo.x, xn.y - xo.y), r);
                }
            }
        }
        __syncthreads();

        // Data fusion: xhat = sum_c lambda_c x_c.
        for (int i = tid; i < n_sym * U; i += blockDim.x) {
            const int n = i / U, u = i - n * U;
            float2 acc = make_float2(0.f, 0.f);
            for (int c = 0; c < C; ++c) {
                const float l = lam[c];
                const float2 x = Xs[u * xs_stride + c * n_sym + n];
                acc.x = fmaf(l, x.x, acc.x);
                acc.y = fmaf(l, x.y, acc.y);
                if (io.Xc) io.Xc[(((size_t)f * C + c) * n_sym + n) * U + u] = make_float2(x.x * out_scale, x.y * out_scale);
            }
            io.Xhat[((size_t)f * n_sym + n) * U + u] = make_float2(acc.x * out_scale, acc.y * out_scale);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Downlink: Algorithm 2 (Eq. (4), applied as x -= p^2 (h^H x - s) h) + normalization, packed.
// ---------------------------------------------------------------------------------------------
template <int IN, int AT>
__global__ void __maxnreg__(kPPRegs) cd_precode_pp_kernel(const CdPlan pl, const PrecodeIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float2* Hs = reinterpret_cast<float2*>(smem);
    float* p2 = reinterpret_cast<float*>(smem + pl.off_coef);  // [U][C] p_{u,c}^2
    float* esum = reinterpret_cast<float*>(smem + pl.off_e);
    float2* Ss = reinterpret_cast<float2*>(smem + pl.off_S);   // [n_sym][U]
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);

    const int tid = threadIdx.x;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    constexpr int LP = AT * kPairs;
    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0 && pl.bulk) {
        mbar_init(bar, 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    zero_padding(pl, tab, Hs);
    const LaneTile lt = map_lane(pl, tab);
    const ClusterTile ct = tab[lt.c];

    uint32_t phase = 0;
    for (int f = blockIdx.x; f < pl.n_sc; f += gridDim.x, phase ^= 1u) {
        stage_H_pp<IN>(pl, tab, io.H, f, Hs, bar);
        for (int i = tid; i < n_sym * U; i += blockDim.x) Ss[i] = __ldg(io.S + (size_t)f * n_sym * U + i);

        bool ok = true;
        if (pl.bulk) ok = mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(!ok)) return;
        if (pl.bulk) {
            permute_pairs_in_place(pl, Hs);
            __syncthreads();
        }

        column_energies(pl, tab, Hs, esum);
        __syncthreads();
        for (int i = tid; i < C * U; i += blockDim.x) {
            const float e = esum[i];
            p2[i] = e > 0.f ? 1.f / e : 0.f;
        }
        __syncthreads();

        if (lt.active) {
            float4 x[kPairs];
#pragma unroll
            for (int i = 0; i < kPairs; ++i) x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4* hb = reinterpret_cast<const float4*>(Hs + ct.soff) + lt.a;
            const float* pc = p2 + lt.c;
            const float2* s = Ss + lt.n * U;
            for (int t = 0; t < pl.K; ++t) {
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    float4 h[kPairs];
                    pp_load_h<AT>(hb + u * LP, h);
                    const float2 g = pp_correlate<AT>(h, x, lt.mask);
                    const float q = pc[u * C];
                    const float2 su = s[u];
                    pp_update(h, make_float2(q * (g.x - su.x), q * (g.y - su.y)), x);
                }
            }
            float nr = 0.f;
#pragma unroll
            for (int i = 0; i < kPairs; ++i)
                nr = fmaf(x[i].x, x[i].x, fmaf(x[i].y, x[i].y, fmaf(x[i].z, x[i].z, fmaf(x[i].w, x[i].w, nr))));
#pragma unroll
            for (int off = 1; off < AT; off <<= 1) nr += __shfl_xor_sync(lt.mask, nr, off);
            const float sc = nr > 0.f ? pl.rho_c * rsqrtf(nr) : 0.f;
            float2* out = io.Xdl + ((size_t)f * n_sym + lt.n) * pl.B + ct.off;
#pragma unroll
            for (int i = 0; i < kPairs; ++i) {
                const int col = 2 * (i * AT + lt.a);
                if (col < ct.size) out[col] = make_float2(x[i].x * sc, x[i].z * sc);
                if (col + 1 < ct.size) out[col + 1] = make_float2(x[i].y * sc, x[i].w * sc);
            }
        }
        __syncthreads();
    }
}

}  // namespace cdmimo
