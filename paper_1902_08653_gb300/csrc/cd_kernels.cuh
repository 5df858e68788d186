// CD detection / precoding / fusion kernels for sm_103a (plain FP32 arithmetic, FP32 or 16-bit
// storage).  The tiling and the shared-memory layout are described in plan.h.
//
// Template parameters: P antennas per lane; IN storage type of H (and Y); AT lanes per tile when
// every cluster has the same A (so shuffle counts and shared-memory offsets are compile-time
// constants), or 0 for mixed cluster sizes (per-lane A at run time).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "plan.h"
#include "ptx.cuh"

namespace cdmimo {

// ---------------------------------------------------------------------------------------------
// storage element types
// ---------------------------------------------------------------------------------------------
template <int IN>
struct Elem;
template <>
struct Elem<CDMIMO_C64> {
    static __device__ __forceinline__ float2 load(const void* base, size_t i)
    {
        return __ldg(reinterpret_cast<const float2*>(base) + i);
    }
    static __device__ __forceinline__ float2 load_shared(const void* base, size_t i)
    {
        return reinterpret_cast<const float2*>(base)[i];
    }
};
template <>
struct Elem<CDMIMO_C16F> {
    static __device__ __forceinline__ float2 load(const void* base, size_t i)
    {
        return __half22float2(__ldg(reinterpret_cast<const __half2*>(base) + i));
    }
    static __device__ __forceinline__ float2 load_shared(const void* base, size_t i)
    {
        return __half22float2(reinterpret_cast<const __half2*>(base)[i]);
    }
};
template <>
struct Elem<CDMIMO_C16BF> {
    static __device__ __forceinline__ float2 load(const void* base, size_t i)
    {
        return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(base) + i));
    }
    static __device__ __forceinline__ float2 load_shared(const void* base, size_t i)
    {
        return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(base)[i]);
    }
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------------------------
// per-CTA pieces shared by detection and precoding
// ---------------------------------------------------------------------------------------------
struct LaneTile {
    bool active;     // this thread runs a CD tile
    int c, A, n, a;  // cluster, lanes per tile, symbol, lane within tile
    int Awarp;       // max A over the active lanes of this warp (uniform shuffle trip count)
    unsigned mask;   // active lanes of this warp
};

__device__ __forceinline__ LaneTile map_lane(const CdPlan& pl, const ClusterTile* tab)
{
    LaneTile t{};
    // Tile lane v sits in warp v / lpw at lane v % lpw (lpw = 32 unless the plan spreads the tiles
    // over more warps); the tiles of one warp are whole and A-aligned.
    const int wl = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = w * pl.lpw + wl;
    t.active = wl < pl.lpw && v < pl.n_lanes;
    t.c = 0;
    t.A = 1;
    if (t.active) {
        for (int k = 0; k < pl.C; ++k) {
            const int l0 = tab[k].lane0;
            if (v >= l0 && v < l0 + pl.n_sym * tab[k].A) {
                t.c = k;
                t.A = tab[k].A;
                t.n = (v - l0) / t.A;
                t.a = (v - l0) & (t.A - 1);
            }
        }
    }
    const int n_act = min(pl.lpw, pl.n_lanes - w * pl.lpw);
    t.mask = n_act >= 32 ? 0xffffffffu : (n_act > 0 ? ((1u << n_act) - 1u) : 0u);
    t.Awarp = t.active ? (int)__reduce_max_sync(t.mask, (unsigned)t.A) : 1;
    return t;
}

// Zero the padding columns [B_c, L_c) of every channel row (done once: staging never writes them).
__device__ __forceinline__ void zero_padding(const CdPlan& pl, const ClusterTile* tab, float2* Hs)
{
    if (!pl.padded) return;
    for (int c = 0; c < pl.C; ++c) {
        const ClusterTile ct = tab[c];
        const int w = ct.L - ct.size;
        for (int i = threadIdx.x; i < pl.U * w; i += blockDim.x) {
            const int u = i / w, j = ct.size + (i - u * w);
            Hs[ct.soff + u * ct.L + j] = make_float2(0.f, 0.f);
        }
    }
}

// Stage the channel of subcarrier f into the per-cluster shared-memory blocks.  Bulk path: warp 0
// arms the mbarrier with the total byte count, then its lanes issue one cp.async.bulk per (cluster,
// user) row; the caller waits on the barrier.  Otherwise every warp copies rows with conversion.
template <int IN>
__device__ __forceinline__ void stage_H(const CdPlan& pl, const ClusterTile* tab, const void* H, int f,
                                        float2* Hs, uint64_t* bar)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int rows = pl.U * pl.C;
    if (pl.bulk) {
        if (warp == 0) {
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, (uint32_t)pl.U * pl.B * 8u);
            }
            __syncwarp();
            const float2* Hf = reinterpret_cast<const float2*>(H) + (size_t)f * pl.U * pl.B;
            for (int row = lane; row < rows; row += 32) {
                const int c = row / pl.U, u = row - c * pl.U;
                const ClusterTile ct = tab[c];
                bulk_g2s(Hs + ct.soff + u * ct.L, Hf + (size_t)u * pl.B + ct.off, (uint32_t)ct.size * 8u, bar);
            }
        }
        return;
    }
    for (int row = warp; row < rows; row += nwarps) {
        const int c = row / pl.U, u = row - c * pl.U;
        const ClusterTile ct = tab[c];
        const size_t g0 = ((size_t)f * pl.U + u) * pl.B + ct.off;
        float2* dst = Hs + ct.soff + u * ct.L;
        for (int j = lane; j < ct.size; j += 32) dst[j] = Elem<IN>::load(H, g0 + j);
    }
}

// Column energies esum[u*C + c] = ||h_{u,c}||^2 from the staged rows (sum of squares of the row's
// floats, in either layout): one warp per (c, u) row.
__device__ __forceinline__ void column_energies(const CdPlan& pl, const ClusterTile* tab, const float2* Hs,
                                                float* esum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int row = warp; row < pl.U * pl.C; row += nwarps) {
        const int c = row / pl.U, u = row - c * pl.U;
        const ClusterTile ct = tab[c];
        const float2* hr = Hs + ct.soff + u * ct.L;
        float s = 0.f;
        // The whole row, padding included (zeros): in the pair-planar layout the last valid antenna
        // of an odd-sized cluster shares a 16-byte pair with a padding column.
        for (int j = lane; j < ct.L; j += 32) {
            const float2 h = hr[j];
            s = fmaf(h.x, h.x, fmaf(h.y, h.y, s));
        }
        s = warp_sum(s);
        if (lane == 0) esum[u * pl.C + c] = s;
    }
}

// Load this lane's P antennas (pairs q = i*A + a) of a length-`size` vector starting at `base`.
template <int P, int IN>
__device__ __forceinline__ void load_lane_vec(const void* V, size_t base, int size, int A, int a, float2 (&v)[P])
{
#pragma unroll
    for (int i = 0; i < P / 2; ++i) {
        const int col = 2 * (i * A + a);
        v[2 * i] = col < size ? Elem<IN>::load(V, base + col) : make_float2(0.f, 0.f);
        v[2 * i + 1] = col + 1 < size ? Elem<IN>::load(V, base + col + 1) : make_float2(0.f, 0.f);
    }
}

template <int P>
__device__ __forceinline__ void load_h_pairs(const float2* hr, int A, float2 (&h)[P])
{
#pragma unroll
    for (int i = 0; i < P / 2; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(hr + 2 * i * A);
        h[2 * i] = make_float2(v.x, v.y);
        h[2 * i + 1] = make_float2(v.z, v.w);
    }
}

// Sum of values over the A lanes of a tile (xor butterfly: bitwise-identical on every lane).
template <int AT>
__device__ __forceinline__ float tile_sum(float v, const LaneTile& lt)
{
    if (AT > 0) {
#pragma unroll
        for (int off = 1; off < AT; off <<= 1) v += __shfl_xor_sync(lt.mask, v, off);
        return v;
    }
    for (int off = 1; off < lt.Awarp; off <<= 1) {
        const float o = __shfl_xor_sync(lt.mask, v, off);
        if (off < lt.A) v += o;
    }
    return v;
}

// g = sum_j conj(h_j) v_j over the lane's antennas (four independent accumulator pairs), then over
// the A lanes of the tile.
template <int P, int AT>
__device__ __forceinline__ float2 tile_correlate(const float2 (&h)[P], const float2 (&v)[P], const LaneTile& lt)
{
    float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int q = j & 3;
        ar[q] = fmaf(h[j].x, v[j].x, ar[q]);
        ai[q] = fmaf(h[j].x, v[j].y, ai[q]);
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int q = j & 3;
        ar[q] = fmaf(h[j].y, v[j].y, ar[q]);
        ai[q] = fmaf(-h[j].y, v[j].x, ai[q]);
    }
    float gr = (ar[0] + ar[1]) + (ar[2] + ar[3]);
    float gi = (ai[0] + ai[1]) + (ai[2] + ai[3]);
    if (AT > 0) {
#pragma unroll
        for (int off = 1; off < AT; off <<= 1) {
            gr += __shfl_xor_sync(lt.mask, gr, off);
            gi += __shfl_xor_sync(lt.mask, gi, off);
        }
    } else {
        for (int off = 1; off < lt.Awarp; off <<= 1) {
            const float orr = __shfl_xor_sync(lt.mask, gr, off);
            const float oi = __shfl_xor_sync(lt.mask, gi, off);
            if (off < lt.A) {
                gr += orr;
                gi += oi;
            }
        }
    }
    return make_float2(gr, gi);
}

// v_j -= h_j * d for the lane's antennas.
template <int P>
__device__ __forceinline__ void axpy_update(const float2 (&h)[P], float2 d, float2 (&v)[P])
{
#pragma unroll
    for (int j = 0; j < P; ++j) {
        v[j].x = fmaf(-h[j].x, d.x, v[j].x);
        v[j].y = fmaf(-h[j].x, d.y, v[j].y);
        v[j].x = fmaf(h[j].y, d.y, v[j].x);
        v[j].y = fmaf(-h[j].y, d.x, v[j].y);
    }
}

__device__ __forceinline__ uint32_t x_stride(const CdPlan& pl) { return (uint32_t)pl.n_tiles | 1u; }

// Register budget: the compile-time-A variants are capped at 96 registers so that three CTAs of
// seven warps (the 224-thread tiling of B_c = 32, C = 8, 14 symbols) fit on an SM; the generic
// variant allows 512 threads per CTA.
#define CDMIMO_CD_SPECIALIZED_REGS 96

// ---------------------------------------------------------------------------------------------
// Uplink: Algorithm 1 + fusion (Sec. III), one CTA per subcarrier (grid-stride).
// ---------------------------------------------------------------------------------------------
template <int P, int IN, int AT>
__global__ void __maxnreg__(AT > 0 ? CDMIMO_CD_SPECIALIZED_REGS : 128) cd_detect_kernel(const CdPlan pl, const DetectIO io)
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

    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0 && pl.bulk) {
        mbar_init(bar, 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    zero_padding(pl, tab, Hs);
    __syncthreads();
    const LaneTile lt = map_lane(pl, tab);
    const ClusterTile ct = tab[lt.c];
    const int A = AT > 0 ? AT : lt.A;
    const int L = AT > 0 ? AT * P : ct.L;
    const int tile = lt.c * n_sym + lt.n;

    uint32_t phase = 0;
    for (int f = blockIdx.x; f < pl.n_sc; f += gridDim.x, phase ^= 1u) {
        stage_H<IN>(pl, tab, io.H, f, Hs, bar);

        // r = y_c (registers), overlapping the channel copy.
        float2 r[P];
        if (lt.active) load_lane_vec<P, IN>(io.Y, ((size_t)f * n_sym + lt.n) * pl.B + ct.off, ct.size, A, lt.a, r);

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

        bool ok = true;
        if (pl.bulk) ok = mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(!ok)) {
            // copy timeout: give the copy in flight one last bounded wait so that no CTA leaves with
            // its own bulk copy still writing into its shared memory
            if (threadIdx.x == 0) mbar_wait_bounded(bar, phase);
            return;
        }

        // Preprocessing (decentralized): column energies, then m and n.
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
            // Fusion weights: lambda_c proportional to 1 / sum_u (||h_{u,c}||^2 + alpha)^{-1}.
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

        // CD iterations (decentralized): K cyclic sweeps over the U coordinates.
        if (lt.active) {
            const float2* hb = Hs + ct.soff + 2 * lt.a;
            float2* xs = Xs + tile;
            const float2* cf = coef + lt.c;
            for (int t = 0; t < pl.K; ++t) {
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    float2 h[P];
                    load_h_pairs<P>(hb + u * L, A, h);
                    const float2 g = tile_correlate<P, AT>(h, r, lt);
                    const float2 k = cf[u * C];
                    const float2 xo = xs[u * xs_stride];
                    const float2 xn = make_float2(fmaf(k.x, g.x, k.y * xo.x), fmaf(k.x, g.y, k.y * xo.y));
                    xs[u * xs_stride] = xn;
                    axpy_update<P>(h, make_float2(xn.x - xo.x, xn.y - xo.y), r);
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
// Downlink: Algorithm 2 (Eq. (4)) + per-cluster power normalization (Sec. IV-B).
// The update x -= (hbar^H x - sbar) hbar is applied as x -= p^2 (h^H x - s) h, so hbar is never
// formed: hbar = p h and sbar = p s give the same product.
// ---------------------------------------------------------------------------------------------
template <int P, int IN, int AT>
__global__ void __maxnreg__(AT > 0 ? CDMIMO_CD_SPECIALIZED_REGS : 128) cd_precode_kernel(const CdPlan pl, const PrecodeIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float2* Hs = reinterpret_cast<float2*>(smem);
    float* p2 = reinterpret_cast<float*>(smem + pl.off_coef);  // [U][C] p_{u,c}^2
    float* esum = reinterpret_cast<float*>(smem + pl.off_e);
    float2* Ss = reinterpret_cast<float2*>(smem + pl.off_S);   // [n_sym][U | 1] (odd stride: no bank conflicts)
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + pl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + pl.off_bar);

    const int tid = threadIdx.x;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym;
    const int s_stride = U | 1;
    if (tid < C) tab[tid] = pl.cl[tid];
    if (tid == 0 && pl.bulk) {
        mbar_init(bar, 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    zero_padding(pl, tab, Hs);
    __syncthreads();
    const LaneTile lt = map_lane(pl, tab);
    const ClusterTile ct = tab[lt.c];
    const int A = AT > 0 ? AT : lt.A;
    const int L = AT > 0 ? AT * P : ct.L;

    uint32_t phase = 0;
    for (int f = blockIdx.x; f < pl.n_sc; f += gridDim.x, phase ^= 1u) {
        stage_H<IN>(pl, tab, io.H, f, Hs, bar);
        for (int i = tid; i < n_sym * U; i += blockDim.x) {
            const int n = i / U;
            Ss[n * s_stride + (i - n * U)] = __ldg(io.S + (size_t)f * n_sym * U + i);
        }

        bool ok = true;
        if (pl.bulk) ok = mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(!ok)) {
            // copy timeout: give the copy in flight one last bounded wait so that no CTA leaves with
            // its own bulk copy still writing into its shared memory
            if (threadIdx.x == 0) mbar_wait_bounded(bar, phase);
            return;
        }

        column_energies(pl, tab, Hs, esum);
        __syncthreads();
        for (int i = tid; i < C * U; i += blockDim.x) {
            const float e = esum[i];
            p2[i] = e > 0.f ? 1.f / e : 0.f;
        }
        __syncthreads();

        if (lt.active) {
            float2 x[P];
#pragma unroll
            for (int j = 0; j < P; ++j) x[j] = make_float2(0.f, 0.f);
            const float2* hb = Hs + ct.soff + 2 * lt.a;
            const float* pc = p2 + lt.c;
            const float2* s = Ss + lt.n * s_stride;
            for (int t = 0; t < pl.K; ++t) {
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    float2 h[P];
                    load_h_pairs<P>(hb + u * L, A, h);
                    const float2 g = tile_correlate<P, AT>(h, x, lt);
                    const float q = pc[u * C];
                    const float2 su = s[u];
                    axpy_update<P>(h, make_float2(q * (g.x - su.x), q * (g.y - su.y)), x);
                }
            }
            // ||x_c|| over the tile, then x_c <- rho_c x_c / ||x_c||.
            float nr = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) nr = fmaf(x[j].x, x[j].x, fmaf(x[j].y, x[j].y, nr));
            nr = tile_sum<AT>(nr, lt);
            const float sc = nr > 0.f ? pl.rho_c * rsqrtf(nr) : 0.f;
            float2* out = io.Xdl + ((size_t)f * n_sym + lt.n) * pl.B + ct.off;
#pragma unroll
            for (int i = 0; i < P / 2; ++i) {
                const int col = 2 * (i * A + lt.a);
                if (col < ct.size) out[col] = make_float2(x[2 * i].x * sc, x[2 * i].y * sc);
                if (col + 1 < ct.size) out[col + 1] = make_float2(x[2 * i + 1].x * sc, x[2 * i + 1].y * sc);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Standalone fusion (Sec. III): Xhat[f][n][u] = sum_c lambda_c Xc[f][c][n][u].
// ---------------------------------------------------------------------------------------------
// Unnormalized fusion weights (Sec. III) per (subcarrier, cluster), in the true units of H: COLNORM
// w_c = 1 / sum_u m_{u,c} with m_{u,c} = (||h_{u,c}||^2 + alpha)^{-1} (a user whose denominator is
// not positive counts as infinite, so w_c = 0, as in the fusing kernels); EQUAL w_c = 1.  One warp
// per cluster, users over its lanes; grid-stride over subcarriers.  A negative or NaN N0 gives NaN.
struct ClusterTable {
    int off[CDMIMO_MAX_CLUSTERS];   // antenna offset o_c
    int size[CDMIMO_MAX_CLUSTERS];  // B_c
};

template <int IN>
__global__ void fusion_weights_kernel(int n_sc, int U, int B, int C, const ClusterTable tab, const void* __restrict__ H,
                                      const float* __restrict__ N0, const float* __restrict__ h_scale, float inv_Ex,
                                      int colnorm, float* __restrict__ w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int f = blockIdx.x; f < n_sc; f += gridDim.x) {
        float alpha = __ldg(N0 + f) * inv_Ex;
        const bool bad = !(alpha >= 0.f);
        const float hs2 = IN == CDMIMO_C64 ? 1.f : __ldg(h_scale + f) * __ldg(h_scale + f);
        for (int c = warp; c < C; c += nw) {
            float sum = 0.f;
            if (colnorm) {
                const int off = tab.off[c], bc = tab.size[c];
                for (int u = lane; u < U; u += 32) {
                    const size_t row = ((size_t)f * U + u) * B + off;
                    float e = 0.f;
                    for (int b = 0; b < bc; ++b) {
                        const float2 h = Elem<IN>::load(H, row + b);
                        e = fmaf(h.x, h.x, fmaf(h.y, h.y, e));
                    }
                    const float den = e * hs2 + alpha;
                    sum += den > 0.f ? 1.f / den : __int_as_float(0x7f800000);
                }
                sum = warp_sum(sum);
            }
            if (lane == 0) w[(size_t)f * C + c] = bad ? __int_as_float(0x7fc00000) : (colnorm ? 1.f / sum : 1.f);
        }
    }
}

static __global__ void fuse_kernel(int n_sc, int n_sym, int U, int C, const float2* __restrict__ Xc,
                            const float* __restrict__ w, int is_lambda, float2* __restrict__ Xhat)
{
    const size_t total = (size_t)n_sc * n_sym * U;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t f = i / ((size_t)n_sym * U);
        const size_t nu = i - f * n_sym * U;
        const float* wf = w + f * C;
        float tot = 0.f;
        int zeros = 0;
        if (!is_lambda) {
            for (int c = 0; c < C; ++c) {
                const float s2 = __ldg(wf + c);
                if (s2 == 0.f) ++zeros; else tot += 1.f / s2;
            }
        }
        float2 acc = make_float2(0.f, 0.f);
        for (int c = 0; c < C; ++c) {
            const float s2 = __ldg(wf + c);
            float l;
            if (is_lambda) l = s2;
            else if (zeros) l = s2 == 0.f ? 1.f / zeros : 0.f;
            else l = (1.f / s2) / tot;
            const float2 x = __ldg(Xc + (f * C + c) * n_sym * U + nu);
            acc.x = fmaf(l, x.x, acc.x);
            acc.y = fmaf(l, x.y, acc.y);
        }
        Xhat[i] = acc;
    }
}

}  // namespace cdmimo
