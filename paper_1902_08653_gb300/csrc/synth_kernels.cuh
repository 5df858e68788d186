// Seeded synthetic uplink batches on the device (system model of Sec. II: i.i.d. CN(0,1) Rayleigh
// channel, uniform Gray-labelled QAM symbols, AWGN, y = H x + n).  Input generation only: no step of
// the detection or precoding method is here.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC 2011) keyed by the 64-bit seed; the counter of element i of stream s is
// (lo32(i), hi32(i), s, 0).  Streams: 0 channel, 1 symbol labels, 2 noise.  A complex normal takes
// the first two output words (u = (w + 0.5) / 2^32) through the Box-Muller transform.
#pragma once
#include <cstdint>

namespace cdmimo {

struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t lo0 = M0 * c0, hi0 = __umulhi(M0, c0);
        const uint32_t lo1 = M1 * c2, hi1 = __umulhi(M1, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    return Philox4{{c0, c1, c2, c3}};
}

// CN(0, var) sample of element i of stream s.
__device__ __forceinline__ float2 philox_cnormal(uint64_t i, uint32_t s, uint64_t seed, float var)
{
    const Philox4 w = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), s, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float u1 = ((float)w.v[0] + 0.5f) * 2.3283064365386963e-10f;  // 2^-32
    const float u2 = ((float)w.v[1] + 0.5f) * 2.3283064365386963e-10f;
    const float rad = sqrtf(-2.f * logf(u1) * (0.5f * var));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    return make_float2(rad * cs, rad * sn);
}

__device__ __forceinline__ int gray_inverse(int g)
{
    int b = g;
    for (int sh = 1; sh < 16; sh <<= 1) b ^= b >> sh;
    return b;
}

struct SynthArgs {
    uint64_t seed;
    int n_sc, n_sym, B, U, M;
    int L, k;       // levels per axis, bits per axis
    float scale;    // unit average energy of the square QAM
    const float* snr_db;
    float2* H;
    float2* X;
    int* labels;
    float2* Y;
    float* N0;
};

__global__ void synth_channel_kernel(SynthArgs a)
{
    const uint64_t n = (uint64_t)a.n_sc * a.U * a.B;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        a.H[i] = philox_cnormal(i, 0u, a.seed, 1.f);
}

__global__ void synth_symbol_kernel(SynthArgs a)
{
    const uint64_t n = (uint64_t)a.n_sc * a.n_sym * a.U;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const Philox4 w = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), 1u, 0u, (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        const int lab = (int)(w.v[0] & (uint32_t)(a.M - 1));
        const int li = gray_inverse(lab >> a.k), lq = gray_inverse(lab & (a.L - 1));
        a.X[i] = make_float2((float)(2 * li - (a.L - 1)) * a.scale, (float)(2 * lq - (a.L - 1)) * a.scale);
        if (a.labels) a.labels[i] = lab;
    }
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < a.n_sc; f += gridDim.x * blockDim.x)
        a.N0[f] = (float)a.U * exp10f(-0.1f * __ldg(a.snr_db + f));
}

// y[f][n][b] = sum_u H[f][u][b] x[f][n][u] + n[f][n][b]
__global__ void synth_receive_kernel(SynthArgs a)
{
    const uint64_t n = (uint64_t)a.n_sc * a.n_sym * a.B;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i % a.B);
        const uint64_t fn = i / a.B;
        const int f = (int)(fn / a.n_sym);
        const float2* h = a.H + (size_t)f * a.U * a.B + b;
        const float2* x = a.X + fn * a.U;
        float2 acc = philox_cnormal(i, 2u, a.seed, __ldg(a.N0 + f));
        for (int u = 0; u < a.U; ++u) {
            const float2 hv = h[(size_t)u * a.B], xv = x[u];
            acc.x = fmaf(hv.x, xv.x, fmaf(-hv.y, xv.y, acc.x));
            acc.y = fmaf(hv.x, xv.y, fmaf(hv.y, xv.x, acc.y));
        }
        a.Y[i] = acc;
    }
}

}  // namespace cdmimo
