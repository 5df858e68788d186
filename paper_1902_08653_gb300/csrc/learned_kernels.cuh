// Kernels of the learned deep-unfolded CD detector: parameter packing, the loss gradient (forward
// with saved steps, reverse sweep, softmax and perceptron backward), a fixed-order reduction of the
// per-subcarrier partial gradients, and Adam.
//
// Parameter vector ("masters", FP32): [tau (K), graw (K), W1 (Hd x F), b1 (Hd), w2 (Hd), b2],
// F = U + 1, gamma_t = softplus(graw_t).  The inference block (cdmimo_learned) holds tau, gamma,
// b1, b2 in FP32 and W1, w2 rounded to bfloat16; the gradient is taken at the block's values and
// applied to the masters.
#pragma once
#include <cuda_bf16.h>

#include "cd_kernels.cuh"

namespace cdmimo {

__device__ __forceinline__ float bf16_to_f(unsigned short v) { return __uint_as_float((unsigned)v << 16); }

__device__ __forceinline__ unsigned short f_to_bf16(float v)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const unsigned short*>(&b);
}

__device__ __forceinline__ float softplusf(float v) { return v > 30.f ? v : log1pf(expf(v)); }

// Write the inference block from the masters (one CTA).
__global__ void learned_pack_kernel(const float* __restrict__ master, int K, int U, int Hd, cdmimo_learned* blk)
{
    const int F = U + 1;
    const float* tau = master;
    const float* graw = master + K;
    const float* W1 = master + 2 * K;
    const float* b1 = W1 + (size_t)Hd * F;
    const float* w2 = b1 + Hd;
    const float b2 = w2[Hd];
    if (threadIdx.x == 0) {
        blk->K = K;
        blk->U = U;
        blk->hidden = Hd;
        blk->reserved0 = 0;
        blk->b2 = b2;
    }
    for (int t = threadIdx.x; t < CDMIMO_MAX_LEARNED_SWEEPS; t += blockDim.x) {
        blk->tau[t] = t < K ? tau[t] : 0.f;
        blk->gamma[t] = t < K ? softplusf(graw[t]) : 0.f;
    }
    for (int k = threadIdx.x; k < CDMIMO_MAX_HIDDEN; k += blockDim.x) {
        blk->b1[k] = k < Hd ? b1[k] : 0.f;
        blk->w2[k] = k < Hd ? f_to_bf16(w2[k]) : (unsigned short)0;
    }
    for (int i = threadIdx.x; i < CDMIMO_MAX_HIDDEN * (CDMIMO_MAX_USERS + 1); i += blockDim.x)
        blk->W1[i] = i < Hd * F ? f_to_bf16(W1[i]) : (unsigned short)0;
}

// Shared-memory layout of the gradient kernel (byte offsets; the channel rows start at 0).
struct GradLayout {
    int K, Hd, F, n_params, ws_stride;
    float inv_nvec;
    unsigned off_e, off_cf, off_save, off_X, off_Xb, off_Ab, off_phi, off_z, off_zb, off_lam, off_lamb, off_lgb,
        off_gx, off_tg, off_red, off_tab, smem_bytes;
};

struct GradIO {
    const float2* H;
    const float2* Y;
    const float* N0;
    const float2* Xt;
    const cdmimo_learned* blk;
    float* ws;  // [n_sc][ws_stride] partial gradients, loss at index n_params
};

// One CTA per subcarrier: forward (saving h^H r and x_old per step), loss, reverse pass.
template <int P>
__global__ void __launch_bounds__(512) learned_grad_kernel(const CdPlan pl, const GradLayout gl, const GradIO io)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float2* Hs = reinterpret_cast<float2*>(smem);
    float* esum = reinterpret_cast<float*>(smem + gl.off_e);     // [U][C]
    float2* cf = reinterpret_cast<float2*>(smem + gl.off_cf);    // [K][U][C] (a1, a2)
    float4* save = reinterpret_cast<float4*>(smem + gl.off_save); // [K][U][tiles] (g, x_old)
    float2* Xs = reinterpret_cast<float2*>(smem + gl.off_X);     // [U][xs] x per tile
    float2* Xb = reinterpret_cast<float2*>(smem + gl.off_Xb);    // [U][xs] adjoint of x per tile
    float2* Ab = reinterpret_cast<float2*>(smem + gl.off_Ab);    // [K][U][tiles] adjoints of (a1, a2)
    float* phi = reinterpret_cast<float*>(smem + gl.off_phi);    // [C][F]
    float* zs = reinterpret_cast<float*>(smem + gl.off_z);       // [C][Hd]
    float* zb = reinterpret_cast<float*>(smem + gl.off_zb);      // [C][Hd]
    float* lam = reinterpret_cast<float*>(smem + gl.off_lam);    // [C]
    float* lamb = reinterpret_cast<float*>(smem + gl.off_lamb);  // [C]
    float* lgb = reinterpret_cast<float*>(smem + gl.off_lgb);    // [C] adjoint of the logits
    float2* gx = reinterpret_cast<float2*>(smem + gl.off_gx);    // [n_sym][U] dL/dxhat
    float2* tg = reinterpret_cast<float2*>(smem + gl.off_tg);    // [K][C] partial (dtau, dgamma)
    float* red = reinterpret_cast<float*>(smem + gl.off_red);    // [32]
    ClusterTile* tab = reinterpret_cast<ClusterTile*>(smem + gl.off_tab);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int U = pl.U, C = pl.C, n_sym = pl.n_sym, K = gl.K, Hd = gl.Hd, F = gl.F;
    const int tiles = pl.n_tiles;
    const uint32_t xs = x_stride(pl);
    const cdmimo_learned* blk = io.blk;
    const int f = blockIdx.x;

    // A block packed for other dimensions than the caller's (K, U, hidden) would be read with the
    // wrong strides: flag it and give this subcarrier a NaN row, so the gradient and loss are NaN.
    // The test depends only on the block, so every thread of the CTA leaves here or none does.
    if (__ldg(&blk->K) != K || __ldg(&blk->U) != U || __ldg(&blk->hidden) != Hd) {
        if (tid == 0 && f == 0) atomicOr(&g_dev_status, (unsigned)CDMIMO_DEV_BAD_LEARNED);
        float* row = io.ws + (size_t)f * gl.ws_stride;
        for (int i = tid; i <= gl.n_params; i += blockDim.x) row[i] = __int_as_float(0x7fc00000);
        return;
    }

    if (tid < C) tab[tid] = pl.cl[tid];
    __syncthreads();
    zero_padding(pl, tab, Hs);
    __syncthreads();
    const LaneTile lt = map_lane(pl, tab);
    const ClusterTile ct = tab[lt.c];
    const int tile = lt.c * n_sym + lt.n;

    stage_H<CDMIMO_C64>(pl, tab, io.H, f, Hs, nullptr);
    __syncthreads();
    column_energies(pl, tab, Hs, esum);
    __syncthreads();
    const float alpha = __ldg(io.N0 + f) * pl.inv_Ex;

    // Coefficients of every sweep, and the perceptron's features.
    for (int i = tid; i < K * U * C; i += blockDim.x) {
        const int t = i / (U * C), uc = i - t * U * C;
        const float e = esum[uc];
        const float gam = __ldg(&blk->gamma[t]), tau = __ldg(&blk->tau[t]);
        const float den = e + gam * alpha;
        cf[i] = den > 0.f ? make_float2(tau / den, 1.f - tau * gam * alpha / den) : make_float2(0.f, 1.f);
    }
    for (int i = tid; i < C * F; i += blockDim.x) {
        const int c = i / F, j = i - c * F;
        phi[i] = j < U ? esum[j * C + c] / (float)tab[c].size : log10f(fmaxf(alpha, 1e-6f));
    }
    __syncthreads();
    for (int i = tid; i < C * Hd; i += blockDim.x) {
        const int c = i / Hd, k = i - c * Hd;
        float z = __ldg(&blk->b1[k]);
        for (int j = 0; j < F; ++j) z = fmaf(bf16_to_f(__ldg(&blk->W1[k * F + j])), phi[c * F + j], z);
        zs[i] = z;
    }
    __syncthreads();
    if (warp == 0) {
        float lg[2], ex[2];
        float mx = -__int_as_float(0x7f800000);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c = lane + 32 * q;
            lg[q] = -__int_as_float(0x7f800000);
            if (c < C) {
                float s = __ldg(&blk->b2);
                for (int k = 0; k < Hd; ++k) s = fmaf(bf16_to_f(__ldg(&blk->w2[k])), fmaxf(zs[c * Hd + k], 0.f), s);
                lg[q] = s;
                mx = fmaxf(mx, s);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
#pragma unroll
        for (int q = 0; q < 2; ++q) ex[q] = lane + 32 * q < C ? expf(lg[q] - mx) : 0.f;
        const float tot = warp_sum(ex[0] + ex[1]);
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (lane + 32 * q < C) lam[lane + 32 * q] = ex[q] / tot;
    }
    __syncthreads();

    // Forward unfolded sweeps, saving (h^H r, x_old) of every step.
    float2 r[P];
    if (lt.active) {
        load_lane_vec<P, CDMIMO_C64>(io.Y, ((size_t)f * n_sym + lt.n) * pl.B + ct.off, ct.size, lt.A, lt.a, r);
        const float2* hb = Hs + ct.soff + 2 * lt.a;
        for (int t = 0; t < K; ++t)
            for (int u = 0; u < U; ++u) {
                float2 h[P];
                load_h_pairs<P>(hb + u * ct.L, lt.A, h);
                const float2 g = tile_correlate<P, 0>(h, r, lt);
                const float2 xo = t == 0 ? make_float2(0.f, 0.f) : Xs[u * xs + tile];
                if (lt.a == 0) save[(t * U + u) * tiles + tile] = make_float4(g.x, g.y, xo.x, xo.y);
                const float2 k = cf[(t * U + u) * C + lt.c];
                const float2 xn = make_float2(fmaf(k.x, g.x, k.y * xo.x), fmaf(k.x, g.y, k.y * xo.y));
                Xs[u * xs + tile] = xn;
                axpy_update<P>(h, make_float2(xn.x - xo.x, xn.y - xo.y), r);
            }
    }
    __syncthreads();

    // Fusion, loss and dL/dxhat = 2 (xhat - xtarget) / (n_sc n_sym).
    float lpart = 0.f;
    for (int i = tid; i < n_sym * U; i += blockDim.x) {
        const int n = i / U, u = i - n * U;
        float2 xh = make_float2(0.f, 0.f);
        for (int c = 0; c < C; ++c) {
            const float2 x = Xs[u * xs + c * n_sym + n];
            xh.x = fmaf(lam[c], x.x, xh.x);
            xh.y = fmaf(lam[c], x.y, xh.y);
        }
        const float2 tv = __ldg(io.Xt + (size_t)f * n_sym * U + i);
        const float2 d = make_float2(xh.x - tv.x, xh.y - tv.y);
        lpart = fmaf(d.x, d.x, fmaf(d.y, d.y, lpart));
        gx[i] = make_float2(2.f * gl.inv_nvec * d.x, 2.f * gl.inv_nvec * d.y);
    }
    lpart = warp_sum(lpart);
    if (lane == 0) red[warp] = lpart;
    __syncthreads();
    // Adjoint of the fusion weights: lamb_c = sum_{n,u} Re(conj(dL/dxhat) x_c).
    for (int c = warp; c < C; c += nwarps) {
        float s = 0.f;
        for (int i = lane; i < n_sym * U; i += 32) {
            const int n = i / U, u = i - n * U;
            const float2 x = Xs[u * xs + c * n_sym + n];
            s = fmaf(gx[i].x, x.x, fmaf(gx[i].y, x.y, s));
        }
        s = warp_sum(s);
        if (lane == 0) lamb[c] = s;
    }
    __syncthreads();
    if (warp == 0) {
        float d = 0.f;
        for (int c = lane; c < C; c += 32) d = fmaf(lam[c], lamb[c], d);
        d = warp_sum(d);
        for (int c = lane; c < C; c += 32) lgb[c] = lam[c] * (lamb[c] - d);  // softmax adjoint
    }
    __syncthreads();
    for (int i = tid; i < C * Hd; i += blockDim.x) {
        const int c = i / Hd, k = i - c * Hd;
        zb[i] = zs[i] > 0.f ? lgb[c] * bf16_to_f(__ldg(&blk->w2[k])) : 0.f;
    }
    __syncthreads();
    float* row = io.ws + (size_t)f * gl.ws_stride;
    float* gW1 = row + 2 * K;
    float* gb1 = gW1 + Hd * F;
    float* gw2 = gb1 + Hd;
    for (int i = tid; i < Hd * F; i += blockDim.x) {
        const int k = i / F, j = i - k * F;
        float s = 0.f;
        for (int c = 0; c < C; ++c) s = fmaf(zb[c * Hd + k], phi[c * F + j], s);
        gW1[i] = s;
    }
    for (int k = tid; k < Hd; k += blockDim.x) {
        float sb = 0.f, sw = 0.f;
        for (int c = 0; c < C; ++c) {
            sb += zb[c * Hd + k];
            sw = fmaf(lgb[c], fmaxf(zs[c * Hd + k], 0.f), sw);
        }
        gb1[k] = sb;
        gw2[k] = sw;
    }
    if (tid == 0) {
        float sb2 = 0.f, ls = 0.f;
        for (int c = 0; c < C; ++c) sb2 += lgb[c];
        for (int w = 0; w < nwarps; ++w) ls += red[w];
        gw2[Hd] = sb2;                   // b2
        row[gl.n_params] = ls * gl.inv_nvec;  // loss
    }

    // Reverse sweeps: adjoint of the residual in registers, adjoint of x per tile in shared memory.
    if (lt.active) {
        for (int u = 0; u < U; ++u) {
            const float2 gv = gx[lt.n * U + u];
            Xb[u * xs + tile] = make_float2(lam[lt.c] * gv.x, lam[lt.c] * gv.y);
        }
        float2 rb[P];
#pragma unroll
        for (int j = 0; j < P; ++j) rb[j] = make_float2(0.f, 0.f);
        const float2* hb = Hs + ct.soff + 2 * lt.a;
        for (int t = K - 1; t >= 0; --t)
            for (int u = U - 1; u >= 0; --u) {
                float2 h[P];
                load_h_pairs<P>(hb + u * ct.L, lt.A, h);
                const float2 hr = tile_correlate<P, 0>(h, rb, lt);
                const float2 xb = Xb[u * xs + tile];
                const float2 db = make_float2(xb.x - hr.x, xb.y - hr.y);  // adjoint of the step dx
                const float4 sv = save[(t * U + u) * tiles + tile];
                const float2 k = cf[(t * U + u) * C + lt.c];
                if (lt.a == 0)
                    Ab[(t * U + u) * tiles + tile] = make_float2(fmaf(db.x, sv.x, db.y * sv.y), fmaf(db.x, sv.z, db.y * sv.w));
                // r_bar += h (a1 db):  axpy_update subtracts, so pass -a1 db.
                axpy_update<P>(h, make_float2(-k.x * db.x, -k.x * db.y), rb);
                Xb[u * xs + tile] = make_float2(fmaf(k.y - 1.f, db.x, xb.x), fmaf(k.y - 1.f, db.y, xb.y));
            }
    }
    __syncthreads();
    // Chain (a1, a2) -> (tau_t, gamma_t): per (t, c), summed over users and symbols.
    for (int i = tid; i < K * C; i += blockDim.x) {
        const int t = i / C, c = i - t * C;
        const float gam = __ldg(&blk->gamma[t]), tau = __ldg(&blk->tau[t]);
        float gt = 0.f, gg = 0.f;
        for (int u = 0; u < U; ++u) {
            const float e = esum[u * C + c], den = e + gam * alpha;
            if (!(den > 0.f)) continue;
            float a1b = 0.f, a2b = 0.f;
            for (int n = 0; n < n_sym; ++n) {
                const float2 v = Ab[(t * U + u) * tiles + c * n_sym + n];
                a1b += v.x;
                a2b += v.y;
            }
            const float id = 1.f / den;
            gt += (a1b - a2b * gam * alpha) * id;
            gg -= tau * alpha * id * id * (a1b + a2b * e);
        }
        tg[i] = make_float2(gt, gg);
    }
    __syncthreads();
    for (int t = tid; t < K; t += blockDim.x) {
        float gt = 0.f, gg = 0.f;
        for (int c = 0; c < C; ++c) {
            gt += tg[t * C + c].x;
            gg += tg[t * C + c].y;
        }
        const float gam = __ldg(&blk->gamma[t]);
        row[t] = gt;
        row[K + t] = gg * (1.f - expf(-gam));  // d softplus(graw)/d graw = sigmoid(graw) = 1 - exp(-gamma)
    }
}

// grad[i] = sum over subcarriers of the partial rows, in subcarrier order (deterministic).
__global__ void learned_reduce_kernel(const float* __restrict__ ws, int n_rows, int stride, int n_params,
                                      float* __restrict__ grad, float* __restrict__ loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n_params) return;
    float s = 0.f;
    for (int f = 0; f < n_rows; ++f) s += __ldg(ws + (size_t)f * stride + i);
    if (i < n_params) grad[i] = s;
    else *loss = s;
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace cdmimo
