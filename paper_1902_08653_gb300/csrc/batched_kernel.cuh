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
#include "cd_kernels.cuh"

namespace cdmimo {

// Lane -> tile mapping of one cluster group (same rules as map_lane).
__device__ __forceinline__ LaneTile map_lane_group(int n_lanes, int Cg, int n_sym, const ClusterTile* tab)
{
    LaneTile t{};
    const int tid = threadIdx.x;
    t.active = tid < n_lanes;
    t.c = 0;
    t.A = 1;
    if (t.active) {
        for (int k = 0; k < Cg; ++k) {
            const int l0 = tab[k].lane0;
            if (tid >= l0 && tid < l0 + n_sym * tab[k].A) {
                t.c = k;
                t.A = tab[k].A;
                t.n = (tid - l0) / t.A;
                t.a = (tid - l0) & (t.A - 1);
            }
        }
    }
    const int n_act = min(32, n_lanes - (tid & ~31));
    t.mask = n_act >= 32 ? 0xffffffffu : (n_act > 0 ? ((1u << n_act) - 1u) : 0u);
    t.Awarp = t.active ? (int)__reduce_max_sync(t.mask, (unsigned)t.A) : 1;
    return t;
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

            if (lt.active) {
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

template <int P>
__global__ void __launch_bounds__(512) cd_batched_kernel(const unsigned char* __restrict__ table, const BatchLaunch bl,
                                                         int* __restrict__ counter)
{
    batched_body<P>(table, bl, counter);
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
