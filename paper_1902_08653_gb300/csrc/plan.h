// Launch plan shared by the host layer and the CD kernels.
//
// Tiling.  One CTA owns one subcarrier f (grid-stride over subcarriers).  Its work is split into
// tiles (cluster c, OFDM symbol n); each tile is served by A_c lanes (A_c a power of two), and each
// lane keeps P antennas of the tile's residual r (uplink) or beamformer x (downlink) in registers,
// as P/2 antenna pairs: lane a of a tile holds pairs q = i*A_c + a, i = 0..P/2-1, i.e. local antennas
// 2q and 2q+1.  Correlations h^H r are summed in registers over the lane's P antennas and then
// across the A_c lanes with xor-butterfly shuffles.  The channel block of the subcarrier sits in
// shared memory once, as rows u of length Ltot where cluster c's segment [soff_c, soff_c + A_c P)
// holds its B_c antennas followed by zeros.
#pragma once
#include "cdmimo.h"

namespace cdmimo {

struct ClusterTile {
    int off;    // antenna offset o_c of the cluster in H / Y / Xdl rows
    int size;   // B_c
    int A;      // lanes per (cluster, symbol) tile, power of two, A * P >= B_c
    int soff;   // offset (complex entries) of the cluster's segment in a shared-memory row
    int lane0;  // first lane of the cluster's tiles; its n_sym tiles use lanes lane0 + n*A + a
};

struct CdPlan {
    int n_sc, n_sym, B, U, C, K;
    int P;            // antennas per lane (the kernel's template value)
    int Ltot;         // shared-memory row length in complex entries (sum of A_c P)
    int n_lanes;      // lanes that run CD tiles: n_sym * sum A_c
    int n_tiles;      // C * n_sym
    int bulk;         // 1: H[f] is copied into shared memory by a single bulk copy (c64, unpadded)
    int coef_sweeps;  // 1 for plain CD (coefficients constant over sweeps), K for learned sweeps
    int fuse;         // cdmimo_fuse_rule
    float inv_Ex;
    float rho_c;      // downlink per-cluster norm rho / sqrt(C)
    // byte offsets of the shared-memory regions (H rows start at 0)
    unsigned off_X, off_coef, off_e, off_lam, off_S, off_tab, off_bar, smem_bytes;
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
};

struct PrecodeIO {
    const void* H;
    const float2* S;
    float2* Xdl;
};

}  // namespace cdmimo
