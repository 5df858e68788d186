/*
 * cdmimo — GB300 (sm_103a) library for decentralized coordinate-descent (CD) data detection and
 * precoding in massive MU-MIMO, after K. Li, O. Castaneda, C. Jeon, J. R. Cavallaro, C. Studer,
 * "Decentralized Coordinate-Descent Data Detection and Precoding for Massive MU-MIMO"
 * (arXiv 1902.08653).
 *
 * C ABI: plain pointers, sizes and a CUDA stream passed as void*.  Every device buffer is owned by
 * the caller; the hot-path entry points never allocate, free or synchronize: they validate their
 * arguments on the host, enqueue kernels on the given stream and return.  Status codes are
 * negative on error (cdmimo_status_string() names them); no entry point aborts the process.
 *
 * Common layouts (row-major; "c64" = interleaved (re, im) float32 pairs, 8 bytes per entry;
 * "c16" = interleaved (re, im) 16-bit pairs, fp16 or bf16, 4 bytes per entry):
 *   H    [n_sc][U][B]      uplink channel.  Row u is column h_u of the paper's B x U matrix H^ul,
 *                          so cluster c's block h_{u,c} = H[f][u][o_c .. o_c+B_c-1] is contiguous.
 *                          The downlink uses the same array: H^dl_c = (H^ul_c)^H (Sec. II-B).
 *   Y    [n_sc][n_sym][B]  uplink receive vectors y; H is fixed over the n_sym OFDM symbols.
 *   S    [n_sc][n_sym][U]  downlink symbol vectors s (c64).
 *   N0   [n_sc]            float32 noise variance per receive antenna, per subcarrier.
 *   Xhat [n_sc][n_sym][U]  c64 fused uplink estimate.
 *   Xc   [n_sc][C][n_sym][U] c64 per-cluster uplink estimates.
 *   Xdl  [n_sc][n_sym][B]  c64 stacked downlink beamformer [x_1; ...; x_C].
 * Clusters are contiguous antenna ranges in order: o_0 = 0, o_{c+1} = o_c + B_c, sum B_c = B
 * (Sec. II-A).
 */
#ifndef CDMIMO_H
#define CDMIMO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------------------------------- */
/* Status codes.                                                                                   */
/* ---------------------------------------------------------------------------------------------- */
typedef enum {
    CDMIMO_OK = 0,
    CDMIMO_ERR_INVALID_ARG = -1,   /* null pointer, negative size or count, bad enum, misalignment */
    CDMIMO_ERR_BAD_PARTITION = -2, /* some B_c <= 0, or sum B_c != B, or C > CDMIMO_MAX_CLUSTERS */
    CDMIMO_ERR_UNSUPPORTED = -3,   /* shape beyond what the kernels' on-chip tiles can hold */
    CDMIMO_ERR_CUDA = -4,          /* a CUDA runtime call or kernel launch failed */
    CDMIMO_ERR_TIMEOUT = -5,       /* a bounded device-side wait expired (see cdmimo_device_status) */
    CDMIMO_ERR_WORKSPACE = -6      /* workspace pointer missing, misaligned or too small */
} cdmimo_status;

/* Bits of the device-side status word (cdmimo_device_status). */
#define CDMIMO_DEV_TIMEOUT 0x1   /* a bounded wait on an async copy or work queue expired */
#define CDMIMO_DEV_BAD_N0 0x2    /* some N0[f] was negative or NaN: that subcarrier's output is NaN */
#define CDMIMO_DEV_BAD_LEARNED 0x4 /* the learned block does not match p->K, p->U (or hidden): output is NaN */
#define CDMIMO_DEV_BAD_SCHED 0x8  /* a workspace's schedule counters were not zero: output incomplete */

#define CDMIMO_MAX_CLUSTERS 64
#define CDMIMO_MAX_USERS 64

typedef enum { CDMIMO_C64 = 0, CDMIMO_C16F = 1, CDMIMO_C16BF = 2 } cdmimo_dtype;

/*
 * Fusion rule of the uplink (Sec. III: xhat = sum_c lambda_c xhat_c, lambda_c = sigma_c^{-2} /
 * sum_c' sigma_c'^{-2}, sigma_c^2 the post-equalization noise variance of cluster c).
 *   EQUAL   lambda_c = 1 / C.
 *   COLNORM sigma_c^2 = (N0/U) sum_u (||h_{u,c}||^2 + N0/Ex)^{-1}; the paper defines sigma_c^2 only
 *           in words, this is the library's reading.  The factor N0/U cancels in lambda.
 *   LEARNED lambda = softmax_c of a small MLP on per-cluster statistics (see cdmimo_learned).
 */
typedef enum { CDMIMO_FUSE_EQUAL = 0, CDMIMO_FUSE_COLNORM = 1, CDMIMO_FUSE_LEARNED = 2 } cdmimo_fuse_rule;

/*
 * Evaluation form of the CD sweeps (both give the iterates of Algorithms 1 and 2; they differ in
 * rounding only).
 *   RESIDUAL  as the algorithms are written: a running residual r = y_c - H_c x (uplink) or the
 *             beamformer x_c itself (downlink) in registers, 2 U B_c complex MACs per sweep and vector.
 *   GRAM      through G_c = H_c^H H_c, formed once per subcarrier and shared by its n_sym symbols:
 *             x_u <- m_u (z_u - sum_{v != u} G_uv x_v) with z = H_c^H y_c (uplink) and
 *             w_u <- p_u^2 (s_u - sum_{v != u} G_uv w_v), x_c = H_c w (downlink); U^2 complex MACs per
 *             sweep and vector plus U B_c (z or H_c w) and U^2 B_c / n_sym (G_c).  Requires U <= 16,
 *             equal lanes per cluster tile (8 < B_c <= 64 for all clusters, or all B_c <= 16, ...:
 *             the packed-kernel shapes) and no learned block; otherwise CDMIMO_ERR_UNSUPPORTED.
 *   GRAM_TC   GRAM, with the contractions z = H_c^H y_c, G_c = H_c^H H_c and x_c = H_c w on the
 *             tensor cores (TF32 MMAs with each FP32 operand split into a TF32 part and its
 *             remainder, FP32 accumulation; the sweeps stay FP32), for cdmimo_detect (with a
 *             learned block: without Xc_opt / lambda_opt), cdmimo_precode and cdmimo_detect_precode.
 *             That kernel takes
 *             c64, fp16 or bf16 storage (16-bit values are exact TF32 operands: one MMA where both
 *             operands are stored values), every B_c = 16 or every B_c = 32, 8 < U <= 16,
 *             n_sym <= 16 and 2 C n_sym <= 256, and a learned block (c64) in cdmimo_detect only;
 *             elsewhere GRAM_TC is GRAM.  Without a learned block, and where C n_sym <= 128 and
 *             its buffers fit in shared memory (not for cdmimo_detect with Xc_opt / lambda_opt,
 *             nor with a schedule workspace: it walks subcarriers in a static order),
 *             a warp-specialized kernel runs: one CTA per SM whose MMA warps form G_c and z of the
 *             next subcarrier and x_c = H_c w of the previous one while its other warps sweep the
 *             current one; its results equal the phased kernel's bit for bit.
 *   GRAM_TC_PHASED  GRAM_TC always on the phased kernel (the phases of a subcarrier one after the
 *             other, two CTAs per SM), e.g. to compare the two kernels.
 *   GRAM_TC_UMMA  GRAM_TC with G_c and z of the warp-specialized kernel formed on the tcgen05 tensor
 *             cores (c64 storage, C <= 8; one thread issues the MMAs, accumulators in tensor
 *             memory): the same split-TF32 products summed in another order, so results agree with
 *             GRAM_TC to rounding; elsewhere it is GRAM_TC.
 *   AUTO      GRAM where it applies, every B_c >= 2 U (so G_c + (N0/Ex) I stays well conditioned
 *             in FP32) and it needs fewer complex MACs, on the tensor cores where GRAM_TC's kernel
 *             takes the call; else RESIDUAL.
 */
typedef enum {
    CDMIMO_FORM_AUTO = 0,
    CDMIMO_FORM_RESIDUAL = 1,
    CDMIMO_FORM_GRAM = 2,
    CDMIMO_FORM_GRAM_TC = 3,
    CDMIMO_FORM_GRAM_TC_PHASED = 4,
    CDMIMO_FORM_GRAM_TC_UMMA = 5
} cdmimo_form;

/*
 * Problem description shared by detection and precoding.
 *   n_sc, n_sym, B, U, C  dimensions (n_sc >= 0, others >= 1; C <= 64, U <= 64).
 *   cluster_size  HOST array [C] of B_c (each >= 1, sum == B).  Read during the call only.
 *   K             sweeps T_max of the CD loops, K >= 0 (K = 0 gives a zero estimate / beamformer).
 *   Ex            per-user transmit energy, > 0 (the regularizer is N0/Ex, Eq. (1)).
 *   fuse          cdmimo_fuse_rule (uplink only).
 *   rho           downlink total power constraint rho (rho^2 = total power); each cluster gets
 *                 rho_c = rho / sqrt(C) (Sec. IV-B).
 *   in_dtype      storage of H and Y (detection) or H (precoding): CDMIMO_C64, or CDMIMO_C16F /
 *                 CDMIMO_C16BF with per-subcarrier float32 scales: the true values are
 *                 H[f] = h_scale[f] * stored and Y[f] = y_scale[f] * stored.  All arithmetic is FP32.
 *   h_scale, y_scale  DEVICE arrays [n_sc] (16-bit dtypes only, else ignored; may be NULL).
 *   learned       DEVICE pointer to a cdmimo_learned block, else NULL (plain CD).  With a block,
 *                 the sweeps are the learned ones (p->K must equal the block's K; a mismatch sets
 *                 CDMIMO_DEV_BAD_LEARNED and gives NaN output) and fuse may be any rule;
 *                 fuse == CDMIMO_FUSE_LEARNED requires a block.  Learned detection needs equal
 *                 cluster sizes of at most 64 antennas and 64-bit complex storage.
 *   form          cdmimo_form (0 = AUTO).
 */
typedef struct {
    int n_sc, n_sym, B, U, C;
    const int* cluster_size;
    int K;
    float Ex;
    int fuse;
    float rho;
    int in_dtype;
    const float* h_scale;
    const float* y_scale;
    const void* learned;
    int form;
} cdmimo_params;

/* ---------------------------------------------------------------------------------------------- */
/* Hot path.                                                                                       */
/* ---------------------------------------------------------------------------------------------- */

/*
 * Uplink detection: Algorithm 1 (decentralized L-MMSE detection using CD) for every subcarrier,
 * cluster and OFDM symbol, followed by the feedforward fusion of Sec. III, in one launch.
 *   Per cluster: m_{u,c} = (||h_{u,c}||^2 + N0/Ex)^{-1}, n_{u,c} = m_{u,c} ||h_{u,c}||^2;
 *   r = y_c, x_c = 0; for t = 1..K, u = 1..U: x_u <- m h_{u,c}^H r + n x_u, r <- r - h_{u,c} dx.
 *   A column with ||h||^2 + N0/Ex == 0 is skipped (its estimate stays 0).
 * H, Y     DEVICE, layout above, dtype p->in_dtype; 16-byte aligned for c64 (8 for c16).
 * N0       DEVICE float [n_sc], each >= 0 (violations set CDMIMO_DEV_BAD_N0 and give NaN output).
 * Xhat     DEVICE c64 [n_sc][n_sym][U] output, 8-byte aligned.
 * Xc_opt   DEVICE c64 [n_sc][C][n_sym][U] per-cluster estimates, or NULL.
 * lambda_opt DEVICE float [n_sc][C] fusion weights, or NULL.
 * workspace, ws_bytes  optional DEVICE scratch of cdmimo_workspace_size(p, op) (256) bytes, 16-byte
 *          aligned (else CDMIMO_ERR_WORKSPACE), zero-filled before its first use; every call leaves
 *          it zero-filled when its kernel completes.  With it the persistent kernels hand out
 *          subcarriers dynamically (an atomic ticket counter), so CTAs that share an SM and run at
 *          different speeds finish together; with NULL they take a static round-robin schedule.
 *          The output is the same bit for bit.  One workspace serves one call at a time: calls that
 *          may run concurrently (other streams) need their own.  Counters found non-zero at the
 *          start leave subcarriers undone and set CDMIMO_DEV_BAD_SCHED.
 * stream   cudaStream_t (NULL = legacy default stream).
 * Shapes whose per-subcarrier channel does not fit in shared memory (or needs more than 512 lanes
 * per CTA) run by streaming cluster groups through shared memory (one CTA per subcarrier); that
 * path takes c64 storage, EQUAL or COLNORM fusion and no Xc_opt / lambda_opt, else UNSUPPORTED.
 */
int cdmimo_detect(const cdmimo_params* p, const void* H, const void* Y, const float* N0, void* Xhat,
                  void* Xc_opt, float* lambda_opt, void* workspace, size_t ws_bytes, void* stream);

/*
 * Downlink precoding: Algorithm 2 (decentralized ZF precoding using CD, Eq. (4)) plus the
 * per-cluster power normalization of Sec. IV-B, for every subcarrier, cluster and symbol.
 *   p_{u,c} = ||h_{u,c}||^{-1} (0 for a zero column); x_c = 0;
 *   for t = 1..K, u = 1..U: x_c <- x_c - (hbar_{u,c}^H x_c - sbar_{u,c}) hbar_{u,c};
 *   x_c <- rho_c x_c / ||x_c|| (x_c = 0 stays 0).  Output Xdl = [x_1; ...; x_C].
 * H        DEVICE, dtype p->in_dtype (16-bit storage needs no scale: the normalization removes it).
 * S        DEVICE c64 [n_sc][n_sym][U], 8-byte aligned.   Xdl DEVICE c64 [n_sc][n_sym][B].
 * workspace as for cdmimo_detect.
 * Shapes beyond shared memory stream cluster groups as cdmimo_detect does (c64 storage only).
 */
int cdmimo_precode(const cdmimo_params* p, const void* H, const void* S, void* Xdl, void* workspace,
                   size_t ws_bytes, void* stream);

/*
 * One TDD frame on one channel: cdmimo_detect on (H, Y) followed by cdmimo_precode of S on the same
 * H (the downlink channel is the transpose of the uplink one, Sec. IV; precoding uses p->rho),
 * with the same arguments, outputs and results as those two calls (no Xc_opt / lambda_opt).
 * Where the Gram form applies (see cdmimo_form; p->form AUTO, GRAM or GRAM_TC) one kernel does both
 * and shares the channel copy and G_c between the directions (with AUTO and GRAM_TC, on the tensor
 * cores where that kernel takes the shape); otherwise (or with p->form RESIDUAL) it enqueues the two
 * calls.  workspace as for cdmimo_detect.
 */
int cdmimo_detect_precode(const cdmimo_params* p, const void* H, const void* Y, const float* N0, void* Xhat,
                          const void* S, void* Xdl, void* workspace, size_t ws_bytes, void* stream);

/*
 * Standalone fusion (Sec. III): Xhat[f][n][u] = sum_c lambda[f][c] Xc[f][c][n][u].
 * If weights_are_lambda != 0, w is lambda itself; otherwise w holds sigma_c^2 and
 * lambda_c = sigma_c^{-2} / sum_c' sigma_c'^{-2} (a zero sigma^2 gives that cluster all the weight;
 * if several are zero they share it equally).  This is the reduction that a cluster-per-GPU
 * deployment performs across devices.
 * Xc DEVICE c64 [n_sc][C][n_sym][U]; w DEVICE float [n_sc][C]; Xhat DEVICE c64 [n_sc][n_sym][U].
 */
int cdmimo_fuse(int n_sc, int n_sym, int U, int C, const void* Xc, const float* w, int weights_are_lambda,
                void* Xhat, void* stream);

/*
 * Unnormalized fusion weights (Sec. III) of every (subcarrier, cluster) of p, in the true units of H,
 * for fusing estimates made by separate calls or on separate devices (the paper's cluster-per-GPU
 * deployment): lambda_c = w_c / sum_c' w_c' over the clusters of all calls, and the weights of
 * disjoint cluster sets may simply be concatenated.  p->fuse COLNORM: w_c = 1 / sum_u m_{u,c} with
 * m_{u,c} = (||h_{u,c}||^2 + N0/Ex)^{-1} (sigma_c^2 up to the common factor N0/U; a user whose
 * denominator is not positive makes w_c = 0, as in the fusing kernels); EQUAL: w_c = 1; LEARNED:
 * UNSUPPORTED.  If every cluster of a subcarrier has w_c = 0 the fusing kernels use equal weights.
 * H DEVICE [n_sc][U][B] (16-bit storage scaled by p->h_scale); N0 DEVICE float [n_sc] (a negative or
 * NaN N0 gives NaN weights); w DEVICE float [n_sc][C] (written).  Enqueued on `stream`; allocates
 * nothing.
 */
int cdmimo_fusion_weights(const cdmimo_params* p, const void* H, const float* N0, float* w, void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Host-buffer variants (end-to-end calls).                                                        */
/* ---------------------------------------------------------------------------------------------- */

/*
 * Same as cdmimo_detect / cdmimo_precode, but H, Y (or S), N0 and the outputs are HOST buffers
 * (pinned memory makes the copies asynchronous).  The call enqueues on `stream` the host-to-device
 * copies into `dev_ws`, the kernel, and the device-to-host copy of the output, then returns;
 * the caller synchronizes the stream before reading the output.  dev_ws is DEVICE scratch of at
 * least cdmimo_host_workspace_size(p, op) bytes, 256-byte aligned.
 */
int cdmimo_detect_host(const cdmimo_params* p, const void* H_host, const void* Y_host, const float* N0_host,
                       void* Xhat_host, void* dev_ws, size_t ws_bytes, void* stream);
int cdmimo_precode_host(const cdmimo_params* p, const void* H_host, const void* S_host, void* Xdl_host,
                        void* dev_ws, size_t ws_bytes, void* stream);

/*
 * cdmimo_detect_precode with HOST buffers, pipelined over chunks of subcarriers so that the uploads,
 * the kernels and the downloads overlap.  The n_sc subcarriers are split into n_chunks contiguous
 * chunks, the last half the size of the others (chunk i starts at n_sc 2i / (2 n_chunks - 1));
 * n_chunks = 0: the library's default, 5; more chunks than subcarriers: empty chunks are skipped.
 * `stream` first copies N0 and S whole into dev_ws, then per chunk the chunk's H and Y; a kernel
 * stream waits for that copy and runs the frame on the chunk (static schedule); a download stream
 * waits for that kernel and copies the chunk's Xhat and Xdl back.  The uploads thus
 * run back to back on `stream` while earlier chunks compute and download (the two copy directions
 * run concurrently).  Before returning, the call makes `stream` wait for the last download: as for
 * every other entry point, the work is ordered after what `stream` holds and the caller synchronizes
 * `stream` only; the next call's uploads cannot overwrite staging that a download still reads.
 * n_chunks = 1: everything on `stream`, in order.  Results equal cdmimo_detect_precode's bit for bit.
 * H_host, Y_host (dtype p->in_dtype), N0_host, S_host, Xhat_host, Xdl_host: HOST arrays in the
 * layouts of cdmimo_detect_precode; pinned (page-locked) memory is needed for the copies to be
 * asynchronous.  16-bit storage: p->h_scale and p->y_scale are HOST arrays [n_sc] here.
 * dev_ws: DEVICE scratch of at least cdmimo_host_workspace_size(p, CDMIMO_OP_FRAME) bytes, 256-byte
 * aligned (else CDMIMO_ERR_WORKSPACE).
 * The first pipelined call on a host thread creates, for the current device, the two streams
 * (non-blocking) and three CUDA events it uses (released when the thread exits); later calls create
 * nothing.  An error return may leave earlier chunks enqueued.
 */
int cdmimo_detect_precode_host(const cdmimo_params* p, const void* H_host, const void* Y_host, const float* N0_host,
                               const void* S_host, void* Xhat_host, void* Xdl_host, int n_chunks, void* dev_ws,
                               size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Batched uneven launch (an extension beyond the paper).                                          */
/* ---------------------------------------------------------------------------------------------- */
/*
 * A batch is a list of descriptors, each a resource block (or any set of subcarriers) with its own
 * B, U, cluster partition, K and operation; all of it runs in ONE persistent launch whose CTAs pop
 * (descriptor, subcarrier) work items from a device counter.  Per item the clusters are processed in
 * groups that fit the plan's shared-memory budget; detection fuses across groups exactly as
 * cdmimo_detect does (EQUAL or COLNORM), precoding normalizes each cluster (Sec. IV-B).
 * Usage: fill the descriptors, call cdmimo_batch_build (host only) to get the table bytes, copy the
 * table to device memory, then call cdmimo_detect_batched as often as wanted; it only enqueues a
 * 4-byte counter reset and the kernel, so the call can be recorded in a CUDA graph.
 */
typedef struct {
    int op;                   /* CDMIMO_OP_DETECT or CDMIMO_OP_PRECODE */
    int n_sc, n_sym, B, U, C, K;
    int fuse;                 /* detection: CDMIMO_FUSE_EQUAL or CDMIMO_FUSE_COLNORM */
    float Ex;                 /* detection: per-user energy (> 0) */
    float rho;                /* precoding: total power constraint, rho_c = rho / sqrt(C) */
    const int* cluster_size;  /* HOST [C], read by cdmimo_batch_build only */
    const void* H;            /* DEVICE c64 [n_sc][U][B] */
    const void* V;            /* DEVICE c64: detection Y [n_sc][n_sym][B]; precoding S [n_sc][n_sym][U] */
    const float* N0;          /* DEVICE float [n_sc] (detection) */
    void* out;                /* DEVICE c64: detection Xhat [n_sc][n_sym][U]; precoding Xdl [n_sc][n_sym][B] */
} cdmimo_batch_desc;

typedef struct {
    /* tile parameters (inputs; cdmimo_batch_default_plan gives defaults, an autotuner may change them) */
    int P;            /* antennas per lane: 8, 16 or 32 */
    int threads;      /* threads per CTA: multiple of 32 in [64, 512] ([64, 384] for P = 8); every cluster
                         group's tiles fit */
    int group_bytes;  /* shared-memory budget of one cluster group (channel rows + per-tile state) */
    int ctas_per_sm;  /* persistent CTAs per SM, 0 = as many as fit */
    /* filled by cdmimo_batch_build */
    int n_items, n_groups, C_max;
    unsigned smem_bytes;
    unsigned offsets[9];
    size_t table_bytes;
} cdmimo_batch_plan;

/* Default tile parameters: P = 16, 256 threads, 64 KiB groups, all CTAs that fit. */
void cdmimo_batch_default_plan(cdmimo_batch_plan* plan);

/*
 * Host only: validate the descriptors, split every descriptor's clusters into groups, and write the
 * device table (which embeds the descriptors' device pointers) into table_host if it is non-NULL and
 * at least plan->table_bytes long (call once with NULL to learn the size).  Errors: INVALID_ARG,
 * BAD_PARTITION, UNSUPPORTED (a single cluster does not fit the budget or the threads, or more than
 * 32 lanes per tile), WORKSPACE (table_host too small).
 */
int cdmimo_batch_build(const cdmimo_batch_desc* desc, int n_desc, cdmimo_batch_plan* plan, void* table_host,
                       size_t table_bytes);

/*
 * Run the batch: table_dev DEVICE copy of the built table (16-byte aligned), counter DEVICE int
 * scratch (reset by this call), stream as elsewhere.  Returns UNSUPPORTED if the plan's shared
 * memory exceeds the device limit.
 */
int cdmimo_detect_batched(const cdmimo_batch_plan* plan, const void* table_dev, int* counter, void* stream);

/*
 * cdmimo_detect_batched that also measures the work queue's load balance (an instrumentation aid; the
 * paper has no counterpart): stats DEVICE unsigned long long[4], 8-byte aligned, reset by this call,
 * receives {earliest CTA start, latest CTA end, sum of CTA lifetimes, number of CTAs} in global-timer
 * nanoseconds, so sum / (CTAs x (end - start)) is the fraction of the launch's span the persistent
 * CTAs spent working.  stats == NULL is cdmimo_detect_batched.  Same errors.
 */
int cdmimo_detect_batched_stats(const cdmimo_batch_plan* plan, const void* table_dev, int* counter,
                                unsigned long long* stats, void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Learned deep-unfolded CD (an extension beyond the paper; plain CD is the default).              */
/* ---------------------------------------------------------------------------------------------- */
/*
 * Sweep t (t = 0..K-1) of the learned detector replaces Algorithm 1's coordinate update by
 *     x_u <- x_u + tau_t (h_{u,c}^H r - gamma_t alpha x_u) / (||h_{u,c}||^2 + gamma_t alpha),
 * alpha = N0/Ex (over-relaxed Gauss-Seidel with a scaled regularizer; tau_t = gamma_t = 1 is exactly
 * Algorithm 1).  With fuse == CDMIMO_FUSE_LEARNED the fusion weights are lambda = softmax_c(logit_c),
 * logit_c = w2 . relu(W1 phi_c + b1) + b2, on the F = U + 1 cluster features
 * phi_c = [||h_{1,c}||^2 / B_c, ..., ||h_{U,c}||^2 / B_c, log10(max(alpha, 1e-6))].
 *
 * Trainable ("master") parameters, one float32 vector of cdmimo_learned_param_count(K, U, hidden):
 *     [tau (K), graw (K), W1 (hidden x F, row-major), b1 (hidden), w2 (hidden), b2 (1)]
 * with gamma_t = softplus(graw_t).  The detection kernels read the packed inference block below,
 * which cdmimo_learned_pack() writes from the masters (W1 and w2 rounded to bfloat16; all arithmetic
 * FP32).
 */
#define CDMIMO_MAX_LEARNED_SWEEPS 16
#define CDMIMO_MAX_HIDDEN 64

typedef struct {
    int K;                    /* sweeps the parameters were trained for (p->K must match) */
    int U;                    /* users (F = U + 1 features) */
    int hidden;               /* hidden width, 1..CDMIMO_MAX_HIDDEN */
    int reserved0;
    float tau[CDMIMO_MAX_LEARNED_SWEEPS];
    float gamma[CDMIMO_MAX_LEARNED_SWEEPS];  /* softplus(graw), > 0 */
    float b1[CDMIMO_MAX_HIDDEN];
    float b2;
    float reserved1[3];
    unsigned short W1[CDMIMO_MAX_HIDDEN * (CDMIMO_MAX_USERS + 1)]; /* bfloat16 bits, row k: F entries */
    unsigned short w2[CDMIMO_MAX_HIDDEN];                          /* bfloat16 bits */
} cdmimo_learned;

/* Number of master parameters for (K, U, hidden), or 0 if out of range. */
size_t cdmimo_learned_param_count(int K, int U, int hidden);

/*
 * Write the inference block from the masters.  master DEVICE float [param_count];
 * block DEVICE cdmimo_learned.  K in 1..CDMIMO_MAX_LEARNED_SWEEPS, U in 1..CDMIMO_MAX_USERS.
 */
int cdmimo_learned_pack(const float* master, int K, int U, int hidden, void* block, void* stream);

/*
 * Loss L = (1/(n_sc n_sym)) sum ||xhat - xtarget||^2 of the learned detector (p->learned = block
 * packed from the masters, hidden = its hidden width, learned fusion, p->in_dtype = CDMIMO_C64, any
 * cluster partition) and its gradient with respect to the master parameters, by a reverse pass
 * through the K unfolded sweeps, the softmax and the perceptron (p->fuse is ignored).  Xtarget DEVICE c64 [n_sc][n_sym][U]; grad DEVICE float
 * [param_count] (overwritten); loss DEVICE float [1] (overwritten).  workspace DEVICE scratch of
 * cdmimo_learned_workspace_size(p) bytes (per-subcarrier partial sums, reduced in a fixed order, so
 * the result is deterministic).  A block whose K, U or hidden differs from p->K, p->U, hidden sets
 * CDMIMO_DEV_BAD_LEARNED, and grad and loss come out NaN.
 */
int cdmimo_learned_grad(const cdmimo_params* p, int hidden, const void* H, const void* Y, const float* N0,
                        const void* Xtarget, float* grad, float* loss, void* workspace, size_t ws_bytes,
                        void* stream);
size_t cdmimo_learned_workspace_size(const cdmimo_params* p, int hidden);

/*
 * Allocation-free variant of cdmimo_learned_grad (the paper has no counterpart: this is a library
 * convenience).  Same inputs, outputs and result, but no workspace argument: the per-subcarrier
 * partial sums live in a fixed array of CDMIMO_NOALLOC_SCRATCH_BYTES bytes that the library keeps
 * in device memory on every GPU that loads it, until the process exits.  It is for callers that
 * cannot call cudaMalloc or any allocator at the point where they train, for example a real-time
 * baseband pipeline that forbids allocation once it is running, or C code that only receives
 * device pointers from another runtime and has no allocator of its own.
 *   - Limit: n_sc * (cdmimo_learned_param_count(p->K, p->U, hidden) + 1, rounded up to a multiple
 *     of 4) * 4 bytes must not exceed CDMIMO_NOALLOC_SCRATCH_BYTES; larger batches return
 *     CDMIMO_ERR_WORKSPACE (use cdmimo_learned_grad with a workspace, or split the batch).
 *   - Every call looks up the array's device address for the current device and context (so the
 *     entry point stays usable after cudaDeviceReset()); the first call on a device also loads the
 *     module there: make that first call before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents (nothing in it has to
 *     start at zero).  Calls that overlap on the GPU (other streams, other host threads) race on
 *     it: serialize them.
 *   - It allocates nothing and frees nothing.
 *   - A block that does not match (p->K, p->U, hidden) is flagged as in cdmimo_learned_grad.
 */
#define CDMIMO_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
int cdmimo_learned_grad_noalloc(const cdmimo_params* p, int hidden, const void* H, const void* Y, const float* N0,
                                const void* Xtarget, float* grad, float* loss, void* stream);

/*
 * One Adam step (Kingma and Ba, 2015) on n float32 parameters, in place:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   theta -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps),   step >= 1.
 * All pointers DEVICE float [n].
 */
int cdmimo_adam_step(float* theta, const float* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                     float eps, int step, void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Seeded synthetic inputs on the device (the system model of Sec. II; not part of the method).     */
/* ---------------------------------------------------------------------------------------------- */
/*
 * H i.i.d. CN(0, 1) [n_sc][U][B]; X uniform Gray-labelled square M-QAM with unit average energy
 * [n_sc][n_sym][U] (labels_opt [n_sc][n_sym][U] int32, or NULL); N0[f] = U 10^(-snr_db[f]/10)
 * (per-receive-antenna SNR U Ex / N0 with Ex = 1); Y = H x + n with n i.i.d. CN(0, N0[f])
 * [n_sc][n_sym][B].  All DEVICE; c64 outputs.  Random numbers: Philox4x32-10 keyed by `seed`, the
 * counter of element i of stream s (0 channel, 1 labels, 2 noise) being (lo32(i), hi32(i), s, 0); a
 * normal pair comes from the first two words by Box-Muller with u = (w + 0.5) / 2^32.  M in
 * {4, 16, 64, 256}.  Three launches on `stream`.
 */
int cdmimo_synth_uplink(unsigned long long seed, int n_sc, int n_sym, int B, int U, int M, const float* snr_db, void* H,
                        void* X, int* labels_opt, void* Y, float* N0, void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Queries.                                                                                        */
/* ---------------------------------------------------------------------------------------------- */
#define CDMIMO_OP_DETECT 0
#define CDMIMO_OP_PRECODE 1
#define CDMIMO_OP_FRAME 2 /* the TDD frame: cdmimo_host_workspace_size, cdmimo_selected_form */

/* Bytes of the optional device workspace of cdmimo_detect / cdmimo_precode (the schedule counters:
 * 256 for every p). */
size_t cdmimo_workspace_size(const cdmimo_params* p, int op);

/* Device staging bytes that cdmimo_detect_host / cdmimo_precode_host (op DETECT / PRECODE: the last
 * 256 hold the schedule counters, which every host call zeroes before its launch) or
 * cdmimo_detect_precode_host (op FRAME) need for p; 0 for an invalid p or op. */
size_t cdmimo_host_workspace_size(const cdmimo_params* p, int op);

/* The evaluation form (CDMIMO_FORM_RESIDUAL, CDMIMO_FORM_GRAM or CDMIMO_FORM_GRAM_TC) that
 * cdmimo_detect (op = CDMIMO_OP_DETECT) or cdmimo_precode
 * (CDMIMO_OP_PRECODE) would run for p and a channel at H (its alignment decides the staging path), or
 * a negative status (for example UNSUPPORTED for a forced GRAM that does not apply).
 * op = CDMIMO_OP_FRAME: the form of cdmimo_detect_precode's one-kernel frame, or, where it enqueues
 * two calls, the uplink's form.  Host only: nothing is launched. */
int cdmimo_selected_form(const cdmimo_params* p, int op, const void* H);

/*
 * Throughput probes of the SM pipes the CD kernels compute on.  The paper has no counterpart: these
 * give the benchmark its per-pipe roofline denominators, measured on the running GPU.
 *   CDMIMO_PROBE_FFMA2     fma.rn.f32x2 dependency chains (the sweeps' packed FP32 FMA);
 *   CDMIMO_PROBE_MMA_TF32  mma.sync m16n8k8 TF32 chains (the split-TF32 contractions).
 * Enqueues one launch on `stream`: cdmimo_pipe_probe_sink_floats() threads (four 256-thread CTAs
 * per SM) each run `iters` (>= 1) iterations of 8 independent chains and write one float to sink
 * (DEVICE float[sink_floats], at least cdmimo_pipe_probe_sink_floats()).  *flops (HOST) receives
 * the launch's flop count; time the launch with events on `stream`.  Errors: INVALID_ARG (kind,
 * iters, NULL pointers), WORKSPACE (sink too small), CUDA_ERROR.
 */
#define CDMIMO_PROBE_FFMA2 0
#define CDMIMO_PROBE_MMA_TF32 1
size_t cdmimo_pipe_probe_sink_floats(void);
int cdmimo_pipe_probe(int kind, int iters, float* sink, size_t sink_floats, double* flops, void* stream);

/*
 * Probes of the tcgen05 tensor cores behind form GRAM_TC_UMMA (measurement aids; the paper has no
 * counterpart).
 * cdmimo_umma_layout_probe: one CTA forms D = A B^T (tf32 in, FP32 accumulate; M = 64 or 128 rows,
 *   N = 32, K = 32) with the library's operand layout and MMA issue, and copies all 128 tensor-memory
 *   lanes x 32 columns to D.  A DEVICE float[M][32], B DEVICE float[32][32], row-major; D DEVICE
 *   float[128][32] (lane-major; lanes no row maps to keep whatever the accumulator held).
 * cdmimo_umma_rate_probe: one thread issues n (1..4096) back-to-back M x N x 8 tf32 MMAs (M 64 or 128,
 *   N a multiple of 16 in [16, 256]) into one accumulator, commits and waits; *cycles (DEVICE long
 *   long) receives the best of five runs in SM clock cycles, or -1 if a wait timed out.
 * Both enqueue one launch on `stream`.  Errors: INVALID_ARG, CUDA_ERROR.
 */
int cdmimo_umma_layout_probe(int M, const float* A, const float* B, float* D, void* stream);
int cdmimo_umma_rate_probe(int M, int N, int n, long long* cycles, void* stream);

/* Static name of a status code. */
const char* cdmimo_status_string(int status);

/* Device-side status word (CDMIMO_DEV_* bits) accumulated by kernels on the current device since
 * the last clear; synchronizes the device.  clear != 0 resets it to 0.  Returns a negative
 * cdmimo_status if the read itself fails. */
int cdmimo_device_status(int clear);

/* Failure-path check of the kernels' bounded waits (the paper has no counterpart).  Enqueues on
 * `stream` one thread that waits, through the same bounded-wait routine the kernels use for their
 * asynchronous copies, on a barrier that nothing completes.  After timeout_us microseconds the wait
 * gives up, sets CDMIMO_DEV_TIMEOUT in the device status word (read it with cdmimo_device_status) and
 * the kernel returns: no trap, and the context stays usable.  timeout_us must be in
 * [1, 2000000] (else CDMIMO_ERR_INVALID_ARG); CDMIMO_ERR_CUDA if the launch fails. */
int cdmimo_check_bounded_wait(unsigned timeout_us, void* stream);

/* Library version, e.g. 0x000100 for 0.1.0. */
int cdmimo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CDMIMO_H */
