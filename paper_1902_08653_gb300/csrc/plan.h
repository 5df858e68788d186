// Launch plan shared by the host layer and the CD kernels.
//
// Tiling.  One CTA owns one subcarrier f (grid-stride over subcarriers).  Its work is split into
// tiles (cluster c, OFDM symbol n); each tile is served by A_c lanes (A_c a power of two), and each
// lane keeps P antennas of the tile's residual r (uplink) or beamformer x (downlink) in registers,
// as P/2 antenna pairs: lane a of a tile holds pairs q = i*A_c + a, i = 0..P/2-1, i.e. local antennas
// 2q and 2q+1.  Correlations h^H r are summed in registers over the lane's P antennas and then
// across the A_c lanes with xor-butterfly shuffles.
//
// Shared memory holds the subcarrier's channel once, per cluster as a block of U rows of length
// L_c = A_c P (B_c antennas then zeros): block c starts at soff_c, and consecutive blocks are skewed
// by 2 A_c complex entries (16 A_c bytes) so that lanes of two clusters that share a quarter-warp
// read disjoint shared-memory banks.
#pragma once
#include "cdmimo.h"

namespace cdmimo {

struct ClusterTile {
    int off;    // antenna offset o_c of the cluster in H / Y / Xdl rows
    int size;   // B_c
    int A;      // lanes per (cluster, symbol) tile, power of two, A * P >= B_c
    int L;      // shared-memory row length A * P (complex entries)
    int soff;   // start (complex entries) of the cluster's [U][L] block in shared memory
    int lane0;  // first lane of the cluster's tiles; its n_sym tiles use lanes lane0 + n*A + a
};

struct CdPlan {
    int n_sc, n_sym, B, U, C, K;
    int P;            // antennas per lane (the kernel's template value)
    int A_uniform;    // A shared by every cluster (0 if clusters differ); selects the kernel variant
    int h_entries;    // complex entries of the shared-memory channel region
    int n_lanes;      // lanes that run CD tiles: n_sym * sum A_c
    int lpw;          // tile lanes per warp (whole tiles; the warp's other lanes idle in the sweeps)
    int threads;      // threads per CTA
    int n_tiles;      // C * n_sym
    int bulk;         // 1: channel rows arrive by cp.async.bulk (c64: every B_c even; 16-bit storage,
                      //    packed kernels only: every B_c a multiple of 4; H 16-byte aligned)
    int padded;       // 1: some B_c < A_c P (zero columns must be written once)
    int packed;       // 1: the packed persistent kernels (uniform A in {1, 2, 4}, P = 16) run this plan
    int gram;         // 1: the Gram-form persistent kernels run this plan (packed layout, U <= UT)
    int UT;           // Gram form: users padded to 8 or 16 (compile-time register count of x)
    int fuse;         // cdmimo_fuse_rule
    int learned;      // 1: learned sweeps (and possibly learned fusion) from a cdmimo_learned block
    int phased;       // tensor-core plans: 1 = the phased kernel (cd_frame_tc_kernel) even where the
                      // warp-specialized one (cd_frame_ws_kernel) would take the call
    int umma;         // tensor-core plans: 1 = the warp-specialized kernel forms G_c and z on the tcgen05
                      // tensor cores where it can (c64, C <= 8), 0 = with mma.sync
    float inv_Ex;
    float rho_c;      // downlink per-cluster norm rho / sqrt(C)
    // byte offsets of the shared-memory regions (channel blocks start at 0; the packed kernels keep
    // a second channel buffer at off_H2 and per-tile coefficients at off_K; the tensor-core kernel's
    // learned plans keep the per-sweep coefficient table [C][K][16] at off_K)
    // off_mlp: [C][CDMIMO_MAX_HIDDEN] floats of learned-fusion partial sums (learned plans; the
    // tensor-core kernel keeps only the C logits there)
    // off_G, off_E: Gram form, [C][UT][UT/2] pair-planar rows of G_c with zero diagonal and [C][UT]
    // column energies
    unsigned off_H2, off_H3, off_X, off_K, off_coef, off_e, off_lam, off_S, off_mlp, off_tab, off_bar, smem_bytes;
    unsigned off_G, off_E;
    unsigned off_W, off_E2;  // fused uplink + downlink: w per tile, and p_u^2 beside m_u at off_E
    ClusterTile cl[CDMIMO_MAX_CLUSTERS];
};

struct DetectIO {
    const void* H;
    const void* Y;
    const float* N0;
    const float* h_scale;
    const float* y_scale;
    float2* Xhat;
    float2* Xc;
    float* lam;
    const void* learned;
    unsigned* sched;  // [3] dynamic-schedule counters in the caller's workspace, or nullptr (static)
};

struct PrecodeIO {
    const void* H;
    const float2* S;
    float2* Xdl;
    unsigned* sched;
};

// Fused uplink detection + downlink precoding on one channel (d.H); d.sched drives the schedule.
struct FusedIO {
    DetectIO d;
    const float2* S;
    float2* Xdl;
};

// Threads a Gram-form phase of C x J tiles of AT lanes needs: its lanes spread over a multiple of
// four warps (the kernels' gram_lane mapping uses the same formula).
__host__ __device__ inline int gram_phase_threads(int C, int J, int AT)
{
    const int L = C * J * AT;
    return ((L + 31) / 32 + 3) / 4 * 4 * 32;
}

// Tile-row stride (entries) of z, x and w in the tensor-core frame kernel: at least n_tiles, 4 mod 16.
__host__ __device__ constexpr unsigned tc_x_stride(int n_tiles) { return ((unsigned)n_tiles + 11u) / 16u * 16u + 4u; }

// 32-bit words per shared-memory channel row of the tensor-core kernel for clusters of Bc antennas:
// c64 entries (two words each) padded by 8 words (the fragment loads of both contractions are then
// bank-conflict free), 16-bit complex entries (one word) by 4 (conflict-free for z and G_c, two-way
// for x_c = H_c w).
__host__ __device__ constexpr unsigned tc_row_words(int Bc, int in_dtype)
{
    return in_dtype == CDMIMO_C64 ? 2u * (unsigned)Bc + 8u : (unsigned)Bc + 4u;
}

}  // namespace cdmimo
