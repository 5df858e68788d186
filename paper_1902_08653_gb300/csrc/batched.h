// Device-side table of the batched (uneven) launch, written by cdmimo_batch_build on the host and
// read by the persistent batched kernel.
//
// Work items are (descriptor d, subcarrier f) pairs, numbered descriptor by descriptor.  A
// descriptor's clusters are processed in groups: each group is a run of consecutive clusters whose
// channel rows (per cluster a [U][L_c] block plus a 16 A_c-byte skew, as in plan.h) and per-tile
// state fit the launch's shared-memory budget, and whose tiles fit the CTA's threads.
#pragma once
#include <cstdint>

namespace cdmimo {

struct BatchDesc {
    const void* H;      // c64 [n_sc][U][B]
    const void* V;      // detect: Y [n_sc][n_sym][B]; precode: S [n_sc][n_sym][U]
    const float* N0;    // detect: [n_sc]
    void* out;          // detect: Xhat [n_sc][n_sym][U]; precode: Xdl [n_sc][n_sym][B]
    int op;             // CDMIMO_OP_DETECT / CDMIMO_OP_PRECODE
    int n_sc, n_sym, B, U, C, K;
    int fuse;           // detect: CDMIMO_FUSE_EQUAL / CDMIMO_FUSE_COLNORM
    float inv_Ex;       // detect
    float rho_c;        // precode: rho / sqrt(C)
    int item0;          // first work item of this descriptor
    int group0, n_groups;
    int bulk;           // 1: channel rows by cp.async.bulk (every B_c even, B even, H 16-byte aligned)
};

struct BatchGroup {
    int c0, c1;         // clusters [c0, c1) of the descriptor
    int cl0;            // index of cluster c0 in the table's cluster array
    int n_lanes;        // n_sym * sum A_c over the group
    int h_entries;      // complex entries of the group's channel region
    int padded;         // 1: some cluster of the group has B_c < A_c P
    int row_bytes;      // bytes of all bulk-copied rows of the group (U * sum B_c * 8)
    int packed;         // 1: packed-FP32 sweeps (P = 16 or 8, every A_c <= 128 / P, each A class warp-aligned)
};

// Cluster entry; soff and lane0 are relative to the cluster's group.
struct BatchCluster {
    int off, size, A, L, soff, lane0;
};

// Table header followed by the descriptor, group and cluster arrays (16-byte aligned sections).
struct BatchTableHeader {
    int n_desc, n_items, n_groups, n_clusters;
    unsigned off_desc, off_group, off_cluster, total_bytes;
};

// Shared-memory layout of the batched kernel, sized for the largest group of the batch.
struct BatchLaunch {
    int P;
    int C_max;  // most clusters in one group
    unsigned off_X, off_coef, off_e, off_acc, off_w, off_S, off_tab, off_bar, off_item, smem_bytes;
};

}  // namespace cdmimo
