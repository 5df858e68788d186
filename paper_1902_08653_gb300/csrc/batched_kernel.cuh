// Persistent batched CD kernel over a descriptor table of uneven resource blocks (batched.h).
//
// Every CTA pops work items (descriptor, subcarrier) from a device counter until the batch is done,
// so blocks of different sizes balance across SMs inside one launch.  For each item it streams the
// descriptor's cluster groups through shared memory (channel rows by cp.async.bulk when aligned),
// runs Algorithm 1 (detection) or Algorithm 2 (precoding) on every (cluster, symbol) tile of the
// group with the generic run-time lanes-per-tile tiling of cd_kernels.cuh, and, for detection,
// accumulates the fused estimate across groups: xhat = sum_c w_c x_c / sum_c w_c with
// w_c = 1 / sum_u m_{u,c} (COLNORM, the reading of Sec. III) or xhat = sum_c x_c / C (EQUAL).
#pragma once
#include "batched.h"
#include "cd_kernels_pp.cuh"

namespace cdmimo {

// Lane -> tile mapping of one cluster group (same rules as map_lane).  A lane inside no cluster's
// lane range (the gaps that align packed groups' A classes to warps) is inactive; the warp's mask is
// the ballot of its active lanes.  Called by every thread of the CTA.
__device__ __forceinline__ LaneTile map_lane_group(int n_lanes, int Cg, int n_sym, const ClusterTile* tab)
{
    LaneTile t{};
    const int tid = threadIdx.x;
    t.active = false;
    t.c = 0;
    t.A = 1;
    if (tid < n_lanes) {
        for (int k = 0; k < Cg; ++k) {
            const int l0 = tab[k].lane0;
            if (tid >= l0 && tid < l0 + n_sym * tab[k].A) {
                t.active = true;
                t.c = k;
                t.A = tab[k].A;
                t.n = (tid - l0) / t.A;
                t.a = (tid - l0) & (t.A - 1);
            }
        }
    }
    t.mask = __ballot_sync(0xffffffffu, t.active);
    t.Awarp = t.active ? (int)__reduce_max_sync(t.mask, (unsigned)t.A) : 1;
    return t;
}

// Packed-FP32 sweeps of one tile of a packed group (pair-planar channel rows, the lane's AT-strided
// antenna pairs in registers, tile sums over AT lanes): Algorithm 1 with (m, n) from coef, x per
// tile in Xs (zero at the start), the running residual r in registers.  Software-pipelined: the
// rows of step u + 1 are loaded while step u's update consumes the rows of step u (each register
// is reloaded right after its last use), and the step's (m, n) and old x are read before the
// correlation, so neither load latency sits on the step's dependency chain.
template <int AT, int NP>
__device__ __forceinline__ void batched_detect_pp(const float4* hb, int LP, int U, int K, const float2* coef, int Cg,
                                                  int c, float2* xs, int xstride, float4 (&r)[NP], unsigned mask)
{
    if (K <= 0 || U <= 0) return;
    float4 h[NP];
    pp_load_h<AT>(hb, h);
    int u = 0;
#pragma unroll 1
    for (int step = 0; step < K * U; ++step) {
        const float2 k = coef[u * Cg + c];
        const float2 xo = xs[u * xstride];
        float2 g = pp_partial_corr(h, r);
        g.x = tile_sum_c<AT>(g.x, mask);
        g.y = tile_sum_c<AT>(g.y, mask);
        const float2 xn = make_float2(fmaf(k.x, g.x, k.y * xo.x), fmaf(k.x, g.y, k.y * xo.y));
        xs[u * xstride] = xn;
        const int un = u + 1 == U ? 0 : u + 1;
        pp_update_reload<AT>(h, make_float2(xn.x - xo.x, xn.y - xo.y), r, hb + un * LP);
        u = un;
    }
}

// Algorithm 2 on one tile of a packed group (the beamformer x in registers, from zero), p^2 from coef;
// pipelined like batched_detect_pp.
template <int AT, int NP>
__device__ __forceinline__ void batched_precode_pp(const float4* hb, int LP, int U, int K, const float2* coef, int Cg,
                                                   int c, const float2* s, float4 (&x)[NP], unsigned mask)
{
#pragma unroll
    for (int i = 0; i < NP; ++i) x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (K <= 0 || U <= 0) return;
    float4 h[NP];
    pp_load_h<AT>(hb, h);
    int u = 0;
#pragma unroll 1
    for (int step = 0; step < K * U; ++step) {
        const float q = coef[u * Cg + c].x;
        const float2 su = s[u];
        float2 g = pp_partial_corr(h, x);
        g.x = tile_sum_c<AT>(g.x, mask);
        g.y = tile_sum_c<AT>(g.y, mask);
        const int un = u + 1 == U ? 0 : u + 1;
        pp_update_reload<AT>(h, make_float2(q * (g.x - su.x), q * (g.y - su.y)), x, hb + un * LP);
        u = un;
    }
}

// Body shared by the persistent batched kernel (items popped from `counter`) and the single-block
// streaming kernel (counter == nullptr: CTA b processes item b).
template <int P>
__device__ __forceinline__ void batched_body(const unsigned char* __restrict__ table, const BatchLaunch& bl,
                                             int* __restrict__ counter)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const BatchTableHeader hdr = *reinterpret_cast<const BatchTableHeader*>(table);
    const BatchDesc* descs = reinterpret_cast<const BatchDesc*>(table + hdr.off_desc);
    const BatchGroup* groups = reinterpret_cast<const BatchGroup*>(table + hdr.off_group);
    const BatchCluster* clus = reinterpret_cast<const BatchCluster*>(table + hdr.off_cluster);

    float2* Hs = reinterpret_cast<float2*>(smem);
    float2* Xs = reinterpret_cast<float2*>(smem + bl.off_X);      // [U][tiles | 1] of the group
    float2* coef = reinterpret_cast<float2*>(smem + bl.off_coef); // [U][Cg] (m, n) or (p^2, -)
    float* esum = reinterpret_cast<float*>(smem + bl.off_e);      // [U][Cg]
    float2* acc = reinterpret_cast<float2*>(smem + bl.off_acc);   // [2][n_sym][U] weighted / plain sums
    float* wsm = reinterpret_cast<float*>(smem + bl.off_w);       // [C_max] weights, [C_max] running sum
    float2* Ss = reinterpret_cast<float2*>(smem + bl.off_S);      // [n_sym][U | 1]
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + bl.off_tab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + bl.off_bar);
    int* item_sh = reinterpret_cast<int*>(smem + bl.off_item);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    uint32_t phase = 0;

    for (int iter = 0;; ++iter) {
        if (tid == 0) *item_sh = counter ? atomicAdd(counter, 1) : (iter == 0 ? (int)blockIdx.x : 0x7fffffff);
        __syncthreads();
        const int item = *item_sh;
        if (item >= hdr.n_items) break;
        int lo = 0, hi = hdr.n_desc - 1;  // descriptor of the item: last one with item0 <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&descs[mid].item0) <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchDesc D = descs[lo];
        const int f = item - D.item0;
        const int U = D.U, n_sym = D.n_sym, nsu = n_sym * U;
        const bool detect = D.op == CDMIMO_OP_DETECT;
        const int s_stride = U | 1;

        float alpha = 0.f, out_scale = 1.f;
        if (detect) {
            alpha = __ldg(D.N0 + f) * D.inv_Ex;
            if (!(alpha >= 0.f)) {
                if (tid == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_N0);
                out_scale = __int_as_float(0x7fc00000);
                alpha = 0.f;
            }
            for (int i = tid; i < 2 * nsu; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
            if (tid == 0) wsm[bl.C_max] = 0.f;
        } else {
            const float2* S = reinterpret_cast<const float2*>(D.V) + (size_t)f * nsu;
            for (int i = tid; i < nsu; i += blockDim.x) {
                const int n = i / U;
                Ss[n * s_stride + (i - n * U)] = __ldg(S + i);
            }
        }
        __syncthreads();

        for (int g = 0; g < D.n_groups; ++g) {
            const BatchGroup G = groups[D.group0 + g];
            const int Cg = G.c1 - G.c0;
            const int tiles = Cg * n_sym;
            const int xs = tiles | 1;
            if (tid < Cg) {
                const BatchCluster b = clus[G.cl0 + tid];
                tab[tid] = ClusterTile{b.off, b.size, b.A, b.L, b.soff, b.lane0};
            }
            __syncthreads();
            // Padding columns of this group's layout (disjoint from the copied rows).
            if (G.padded) {
                for (int c = 0; c < Cg; ++c) {
                    const ClusterTile ct = tab[c];
                    const int w = ct.L - ct.size;
                    for (int i = tid; i < U * w; i += blockDim.x) {
                        const int u = i / w;
                        Hs[ct.soff + u * ct.L + ct.size + (i - u * w)] = make_float2(0.f, 0.f);
                    }
                }
            }
            const float2* Hf = reinterpret_cast<const float2*>(D.H) + (size_t)f * U * D.B;
            if (D.bulk) {
                if (tid == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(bar, (uint32_t)G.row_bytes);
                }
                __syncthreads();  // armed before any row copy can complete
                for (int row = tid; row < U * Cg; row += blockDim.x) {
                    const int c = row / U, u = row - c * U;
                    const ClusterTile ct = tab[c];
                    fence_proxy_async_smem();
                    bulk_g2s(Hs + ct.soff + u * ct.L, Hf + (size_t)u * D.B + ct.off, (uint32_t)ct.size * 8u, bar);
                }
            } else {
                for (int row = warp; row < U * Cg; row += nwarps) {
                    const int c = row / U, u = row - c * U;
                    const ClusterTile ct = tab[c];
                    for (int j = lane; j < ct.size; j += 32) Hs[ct.soff + u * ct.L + j] = __ldg(Hf + (size_t)u * D.B + ct.off + j);
                }
            }
            const LaneTile lt = map_lane_group(G.n_lanes, Cg, n_sym, tab);
            const ClusterTile ct = tab[lt.c];
            const int tile = lt.c * n_sym + lt.n;
            float2 v[P];
            if (detect && lt.active)
                load_lane_vec<P, CDMIMO_C64>(D.V, ((size_t)f * n_sym + lt.n) * D.B + ct.off, ct.size, lt.A, lt.a, v);
            bool ok = true;
            if (D.bulk) {
                ok = mbar_wait_bounded(bar, phase);
                phase ^= 1u;
            }
            if (__syncthreads_or(!ok)) return;
            constexpr int NP = P / 2;  // antenna pairs per lane
            const bool packed = (P == 16 || P == 8) && G.packed;
            if (packed) {  // (re0, im0, re1, im1) -> (re0, re1, im0, im1) per 16-byte pair of the group's rows
                float4* h4 = reinterpret_cast<float4*>(Hs);
                for (int i = tid; i < G.h_entries / 2; i += blockDim.x) {
                    const float4 q = h4[i];
                    h4[i] = make_float4(q.x, q.z, q.y, q.w);
                }
                __syncthreads();
            }

            // Preprocessing: column energies, then (m, n) of Algorithm 1 or p^2 of Algorithm 2.
            for (int row = warp; row < U * Cg; row += nwarps) {
                const int c = row / U, u = row - c * U;
                const float2* hr = Hs + tab[c].soff + u * tab[c].L;
                float s = 0.f;
                for (int j = lane; j < tab[c].L; j += 32) s = fmaf(hr[j].x, hr[j].x, fmaf(hr[j].y, hr[j].y, s));
                s = warp_sum(s);
                if (lane == 0) esum[u * Cg + c] = s;
            }
            __syncthreads();
            for (int i = tid; i < U * Cg; i += blockDim.x) {
                const float e = esum[i];
                if (detect) {
                    const float den = e + alpha;
                    const float m = den > 0.f ? 1.f / den : 0.f;
                    coef[i] = make_float2(m, m * e);
                } else {
                    coef[i] = make_float2(e > 0.f ? 1.f / e : 0.f, 0.f);
                }
            }
            if (detect)
                for (int i = tid; i < U * xs; i += blockDim.x) Xs[i] = make_float2(0.f, 0.f);
            __syncthreads();

            if (packed && lt.active) {
                // Packed FP32 with the tile width fixed at compile time; every active lane of a warp has
                // the same A (the host aligns each A class of a packed group to a warp).
                const float4* hb4 = reinterpret_cast<const float4*>(Hs + ct.soff) + lt.a;
                const int LP = ct.L / 2;
                float4 w4[NP];
                if (detect) {
#pragma unroll
                    for (int i = 0; i < NP; ++i)  // the receive vector, pair-planar
                        w4[i] = make_float4(v[2 * i].x, v[2 * i + 1].x, v[2 * i].y, v[2 * i + 1].y);
                    float2* xsp = Xs + tile;
                    switch (lt.Awarp) {
                    case 1: batched_detect_pp<1>(hb4, LP, U, D.K, coef, Cg, lt.c, xsp, xs, w4, lt.mask); break;
                    case 2: batched_detect_pp<2>(hb4, LP, U, D.K, coef, Cg, lt.c, xsp, xs, w4, lt.mask); break;
                    case 4: batched_detect_pp<4>(hb4, LP, U, D.K, coef, Cg, lt.c, xsp, xs, w4, lt.mask); break;
                    case 8: batched_detect_pp<8>(hb4, LP, U, D.K, coef, Cg, lt.c, xsp, xs, w4, lt.mask); break;
                    default: batched_detect_pp<16>(hb4, LP, U, D.K, coef, Cg, lt.c, xsp, xs, w4, lt.mask); break;
                    }
                } else {
                    const float2* sp = Ss + lt.n * s_stride;
                    float nr = 0.f;
                    switch (lt.Awarp) {
                    case 1: batched_precode_pp<1>(hb4, LP, U, D.K, coef, Cg, lt.c, sp, w4, lt.mask); break;
                    case 2: batched_precode_pp<2>(hb4, LP, U, D.K, coef, Cg, lt.c, sp, w4, lt.mask); break;
                    case 4: batched_precode_pp<4>(hb4, LP, U, D.K, coef, Cg, lt.c, sp, w4, lt.mask); break;
                    case 8: batched_precode_pp<8>(hb4, LP, U, D.K, coef, Cg, lt.c, sp, w4, lt.mask); break;
                    default: batched_precode_pp<16>(hb4, LP, U, D.K, coef, Cg, lt.c, sp, w4, lt.mask); break;
                    }
#pragma unroll
                    for (int i = 0; i < NP; ++i)
                        nr = fmaf(w4[i].x, w4[i].x, fmaf(w4[i].y, w4[i].y, fmaf(w4[i].z, w4[i].z, fmaf(w4[i].w, w4[i].w, nr))));
                    for (int off = 1; off < lt.Awarp; off <<= 1) nr += __shfl_xor_sync(lt.mask, nr, off);
                    const float sc = nr > 0.f ? D.rho_c * rsqrtf(nr) : 0.f;
                    float2* out = reinterpret_cast<float2*>(D.out) + ((size_t)f * n_sym + lt.n) * D.B + ct.off;
#pragma unroll
                    for (int i = 0; i < NP; ++i) {
                        const int col = 2 * (i * lt.A + lt.a);
                        if (col < ct.size) out[col] = make_float2(w4[i].x * sc, w4[i].z * sc);
                        if (col + 1 < ct.size) out[col + 1] = make_float2(w4[i].y * sc, w4[i].w * sc);
                    }
                }
            } else if (lt.active) {
                const float2* hb = Hs + ct.soff + 2 * lt.a;
                if (detect) {
                    // Algorithm 1 on this tile.
                    for (int t = 0; t < D.K; ++t)
                        for (int u = 0; u < U; ++u) {
                            float2 h[P];
                            load_h_pairs<P>(hb + u * ct.L, lt.A, h);
                            const float2 gc = tile_correlate<P, 0>(h, v, lt);
                            const float2 k = coef[u * Cg + lt.c];
                            const float2 xo = Xs[u * xs + tile];
                            const float2 xn = make_float2(fmaf(k.x, gc.x, k.y * xo.x), fmaf(k.x, gc.y, k.y * xo.y));
                            Xs[u * xs + tile] = xn;
                            axpy_update<P>(h, make_float2(xn.x - xo.x, xn.y - xo.y), v);
                        }
                } else {
                    // Algorithm 2 on this tile, then the per-cluster power normalization.
#pragma unroll
                    for (int j = 0; j < P; ++j) v[j] = make_float2(0.f, 0.f);
                    const float2* s = Ss + lt.n * s_stride;
                    for (int t = 0; t < D.K; ++t)
                        for (int u = 0; u < U; ++u) {
                            float2 h[P];
                            load_h_pairs<P>(hb + u * ct.L, lt.A, h);
                            const float2 gc = tile_correlate<P, 0>(h, v, lt);
                            const float q = coef[u * Cg + lt.c].x;
                            const float2 su = s[u];
                            axpy_update<P>(h, make_float2(q * (gc.x - su.x), q * (gc.y - su.y)), v);
                        }
                    float nr = 0.f;
#pragma unroll
                    for (int j = 0; j < P; ++j) nr = fmaf(v[j].x, v[j].x, fmaf(v[j].y, v[j].y, nr));
                    nr = tile_sum<0>(nr, lt);
                    const float sc = nr > 0.f ? D.rho_c * rsqrtf(nr) : 0.f;
                    float2* out = reinterpret_cast<float2*>(D.out) + ((size_t)f * n_sym + lt.n) * D.B + ct.off;
#pragma unroll
                    for (int i = 0; i < P / 2; ++i) {
                        const int col = 2 * (i * lt.A + lt.a);
                        if (col < ct.size) out[col] = make_float2(v[2 * i].x * sc, v[2 * i].y * sc);
                        if (col + 1 < ct.size) out[col + 1] = make_float2(v[2 * i + 1].x * sc, v[2 * i + 1].y * sc);
                    }
                }
            }
            __syncthreads();

            if (detect) {
                // Fusion, accumulated over the groups of the block.
                if (tid < Cg) {
                    float s = 0.f;
                    for (int u = 0; u < U; ++u) {
                        const float m = coef[u * Cg + tid].x;
                        s += m > 0.f ? m : __int_as_float(0x7f800000);
                    }
                    wsm[tid] = 1.f / s;
                }
                __syncthreads();
                for (int i = tid; i < nsu; i += blockDim.x) {
                    const int n = i / U, u = i - n * U;
                    float2 aw = acc[i], ae = acc[nsu + i];
                    for (int c = 0; c < Cg; ++c) {
                        const float2 x = Xs[u * xs + c * n_sym + n];
                        aw.x = fmaf(wsm[c], x.x, aw.x);
                        aw.y = fmaf(wsm[c], x.y, aw.y);
                        ae.x += x.x;
                        ae.y += x.y;
                    }
                    acc[i] = aw;
                    acc[nsu + i] = ae;
                }
                if (tid == 0) {
                    float s = wsm[bl.C_max];
                    for (int c = 0; c < Cg; ++c) s += wsm[c];
                    wsm[bl.C_max] = s;
                }
                __syncthreads();
            }
        }

        if (detect) {
            const float wsum = wsm[bl.C_max];
            const bool weighted = D.fuse == CDMIMO_FUSE_COLNORM && wsum > 0.f;
            const float sc = out_scale * (weighted ? 1.f / wsum : 1.f / (float)D.C);
            float2* out = reinterpret_cast<float2*>(D.out) + (size_t)f * nsu;
            for (int i = tid; i < nsu; i += blockDim.x) {
                const float2 a = weighted ? acc[i] : acc[nsu + i];
                out[i] = make_float2(a.x * sc, a.y * sc);
            }
        }
        __syncthreads();
    }
}

// P = 8 keeps fewer registers per lane (packed: 4 pairs), so two 384-thread CTAs share an SM.  With
// `stats` non-null every CTA adds its lifetime (global-timer ns) to stats = {earliest start, latest
// end, sum of lifetimes, CTAs}: the load balance of the work queue.
template <int P>
__global__ void __launch_bounds__(P == 8 ? 384 : 512, P == 8 ? 2 : 1)
    cd_batched_kernel(const unsigned char* __restrict__ table, const BatchLaunch bl, int* __restrict__ counter,
                      unsigned long long* __restrict__ stats)
{
    const unsigned long long t0 = stats ? global_ns() : 0ull;
    batched_body<P>(table, bl, counter);
    if (stats && threadIdx.x == 0) {
        const unsigned long long t1 = global_ns();
        atomicMin(&stats[0], t0);
        atomicMax(&stats[1], t1);
        atomicAdd(&stats[2], t1 - t0);
        atomicAdd(&stats[3], 1ull);
    }
}

// A one-descriptor table small enough to travel as a kernel parameter (same format as the device
// table: header offsets point inside this struct).
struct SingleTable {
    BatchTableHeader hdr;
    BatchDesc desc;
    BatchGroup groups[CDMIMO_MAX_CLUSTERS];
    BatchCluster clusters[CDMIMO_MAX_CLUSTERS];
};

// cdmimo_detect / cdmimo_precode for shapes whose whole channel does not fit in shared memory:
// one CTA per subcarrier streams the cluster groups.
template <int P>
__global__ void __launch_bounds__(512) cd_streaming_kernel(const __grid_constant__ SingleTable t, const BatchLaunch bl)
{
    batched_body<P>(reinterpret_cast<const unsigned char*>(&t), bl, nullptr);
}

}  // namespace cdmimo
