"""Multi-GPU layouts of the decentralized CD path: host logic over torch.distributed.

Two partitionings, one process per GPU:

subcarriers   Subcarriers (and resource blocks) are independent problems, so a batch shards by
              subcarrier with no collective on the data path (``subcarrier_shard``): rank r takes a
              contiguous range, each rank's outputs are its rows of the batch's outputs.

clusters      The paper's deployment (Sec. VI): each GPU owns whole antenna clusters (``cluster_shard``)
              and their channel rows.  Uplink: every rank detects its clusters (Algorithm 1, per-cluster
              estimates x_c) and computes their unnormalized fusion weights w_c (Sec. III,
              ``cdmimo_fusion_weights``); one all-reduce of sum_c w_c per subcarrier gives every rank
              the global lambda_c = w_c / sum_all w, each rank forms its partial sum_local lambda_c x_c
              (``cdmimo_fuse``), and one all-reduce (sum) of U complex values per (subcarrier, symbol)
              gives x_hat -- the reduction the paper does with ncclReduce.  Downlink: the symbols s are
              broadcast from one rank, every rank precodes its clusters (Algorithm 2) with the per-cluster
              norm rho / sqrt(C) of the whole array (it passes rho sqrt(C_local / C) to a call that sees
              C_local clusters), and its antennas' part of the beamformer stays on that rank.

The arithmetic runs in the library's kernels (detection, weights, partial fusion); this module only
moves tensors and calls collectives.  The collectives act on real views of complex tensors, so any
backend (NCCL on GPUs, gloo on CPU) serves.
"""
from __future__ import annotations

import math

import torch
import torch.distributed as dist


def subcarrier_shard(n_sc: int, world: int, rank: int):
    """Contiguous range [lo, hi) of subcarriers for `rank`: sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(int(n_sc), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def cluster_shard(cluster_size, world: int, rank: int):
    """Contiguous clusters [c0, c1) and their antennas [b0, b1) for `rank`: cluster counts differ by at
    most one (a rank may own none if there are fewer clusters than ranks)."""
    C = len(cluster_size)
    c0, c1 = subcarrier_shard(C, world, rank)
    off = [0]
    for b in cluster_size:
        off.append(off[-1] + int(b))
    return c0, c1, off[c0], off[c1]


def _real(t):
    return torch.view_as_real(t) if t.is_complex() else t


def global_lambda(w_local: torch.Tensor, n_clusters: int, group=None):
    """lambda of the local clusters, normalized over the clusters of every rank: w_local [n_sc, C_local]
    unnormalized weights (``cdmimo_fusion_weights``); n_clusters = C of the whole array.  A subcarrier
    whose weights are all zero gets equal weights 1 / C (the fusing kernels' rule)."""
    tot = w_local.sum(dim=1, dtype=torch.float64) if w_local.numel() else torch.zeros(
        w_local.shape[0], dtype=torch.float64, device=w_local.device)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
    lam = torch.where((tot > 0)[:, None], w_local.to(torch.float64) / tot.clamp_min(1e-300)[:, None],
                      torch.full_like(w_local, 1.0 / n_clusters, dtype=torch.float64))
    return lam.to(torch.float32)


def fuse_across(partial: torch.Tensor, group=None):
    """Sum of the ranks' partial estimates sum_local lambda_c x_c (complex [n_sc, n_sym, U]), in place,
    on every rank."""
    dist.all_reduce(_real(partial), op=dist.ReduceOp.SUM, group=group)
    return partial


def detect_clusters(H_local, Y_local, N0, cluster_size_local, n_clusters, K, *, group=None, Ex=1.0,
                    fuse="colnorm", stream=None, **kw):
    """Cluster-parallel uplink detection on this rank's GPU: H_local [n_sc, U, B_local] and Y_local
    [n_sc, n_sym, B_local] hold this rank's antennas (whole clusters, sizes cluster_size_local);
    returns x_hat [n_sc, n_sym, U] (complex64, device), the same on every rank."""
    from . import cdmimo

    n_sc, U = H_local.shape[0], H_local.shape[1]
    n_sym = Y_local.shape[1]
    Cl = len(cluster_size_local)
    partial = torch.zeros((n_sc, n_sym, U), dtype=torch.complex64, device=N0.device)
    if Cl:
        Xc = torch.empty((n_sc, Cl, n_sym, U), dtype=torch.complex64, device=N0.device)
        cdmimo.detect(H_local, Y_local, N0, cluster_size_local, K, Ex=Ex, fuse=fuse, Xc=Xc, stream=stream, **kw)
        w = cdmimo.fusion_weights(H_local, N0, cluster_size_local, Ex=Ex, fuse=fuse,
                                  h_scale=kw.get("h_scale"), stream=stream)
    else:
        w = torch.zeros((n_sc, 0), dtype=torch.float32, device=N0.device)
    lam = global_lambda(w, n_clusters, group)
    if Cl:
        cdmimo.fuse(Xc, lam, weights_are_lambda=True, out=partial, stream=stream)
    return fuse_across(partial, group)


def precode_clusters(H_local, S, cluster_size_local, n_clusters, K, *, rho=1.0, src=0, group=None, stream=None,
                     **kw):
    """Cluster-parallel downlink precoding: S [n_sc, n_sym, U] is broadcast from rank `src`; returns this
    rank's antennas' part [n_sc, n_sym, B_local] of the stacked beamformer, each cluster normalized to
    rho / sqrt(n_clusters)."""
    from . import cdmimo

    dist.broadcast(_real(S), src=src, group=group)
    Cl = len(cluster_size_local)
    if Cl == 0:
        return torch.empty((S.shape[0], S.shape[1], 0), dtype=torch.complex64, device=S.device)
    rho_local = rho * math.sqrt(Cl / n_clusters)  # the call normalizes each of its clusters to rho_local / sqrt(Cl)
    return cdmimo.precode(H_local, S, cluster_size_local, K, rho=rho_local, stream=stream, **kw)
