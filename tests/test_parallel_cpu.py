"""Host logic of the multi-GPU layouts (paper_1902_08653_gb300/parallel.py) on CPU ranks over gloo.

The layouts' arithmetic runs in the library's kernels on a GPU; here each rank stands in for one GPU
with the FP64 oracle computing its local results, and the module's collectives must turn them into
the single-device answer:
  * subcarrier sharding: the ranks' ranges partition the batch, balanced;
  * cluster-per-rank uplink: every rank's local per-cluster estimates and unnormalized fusion weights
    (Sec. III, the COLNORM reading) give, after the module's two all-reduces, the oracle's fused
    estimate over all clusters -- also with a rank that owns no cluster, and for equal weights;
  * cluster-per-rank downlink: s broadcast from rank 0, and the rescaled rho makes each rank's slice
    equal to the corresponding antennas of the oracle's all-cluster precoder (rho / sqrt(C) per cluster).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1902_08653_gb300 import parallel  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_sc,world", [(1200, 8), (7, 3), (2, 4), (0, 2)])
def test_subcarrier_shard_partitions_the_batch(n_sc, world):
    rs = [parallel.subcarrier_shard(n_sc, world, r) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n_sc
    assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    sizes = [hi - lo for lo, hi in rs]
    assert max(sizes) - min(sizes) <= 1


def test_cluster_shard_covers_the_antennas():
    cs = [32, 16, 64, 32, 32]
    parts = [parallel.cluster_shard(cs, 3, r) for r in range(3)]
    assert [p[:2] for p in parts] == [(0, 2), (2, 4), (4, 5)]
    assert [p[2:] for p in parts] == [(0, 48), (48, 144), (144, 176)]
    assert parallel.cluster_shard([32, 32], 3, 2) == (2, 2, 64, 64)  # a rank without clusters


def colnorm_weights(H, N0, cs, Ex=1.0):
    """Unnormalized Sec. III weights w_c = 1 / sum_u (||h_{u,c}||^2 + N0/Ex)^-1 (the library's reading)."""
    o = np.concatenate([[0], np.cumsum(cs)])
    e = np.stack([np.sum(np.abs(H[:, :, o[c]:o[c + 1]]) ** 2, axis=2) for c in range(len(cs))], axis=1)
    return 1.0 / np.sum(1.0 / (e + (N0 / Ex)[:, None, None]), axis=2)


def _rank_main(rank, world, port, cs, fuse, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    from paper_1902_08653_gb300 import workload as wl

    n_sc, n_sym, U, K = 6, 3, 4, 3
    B, C = sum(cs), len(cs)
    d = wl.uplink(2024, n_sc, n_sym, B, U, snr_db=12.0)  # the same batch on every rank
    H, Y, N0 = d["H"], d["Y"], d["N0"]
    c0, c1, b0, b1 = parallel.cluster_shard(cs, world, rank)
    cs_l = cs[c0:c1]
    # uplink: this rank's clusters (the oracle stands in for the GPU's detection)
    if cs_l:
        _, Xc, _ = orc.detect(H[:, :, b0:b1], Y[:, :, b0:b1], N0, cs_l, K, fuse="equal")
        w = colnorm_weights(H[:, :, b0:b1], N0, cs_l) if fuse == "colnorm" else np.ones((n_sc, len(cs_l)))
    else:
        Xc = np.zeros((n_sc, 0, n_sym, U), complex)
        w = np.zeros((n_sc, 0))
    lam = parallel.global_lambda(torch.from_numpy(w).to(torch.float32), C).to(torch.float64).numpy()
    partial = torch.from_numpy(np.einsum("fc,fcnu->fnu", lam, Xc).astype(np.complex128))
    xhat = parallel.fuse_across(partial).numpy()
    ref, _, lam_ref = orc.detect(H, Y, N0, cs, K, fuse=fuse)
    err_ul = float(np.max(np.abs(xhat - ref)) / np.max(np.abs(ref)))
    err_lam = float(np.max(np.abs(lam - lam_ref[:, c0:c1]))) if cs_l else 0.0
    # downlink: s from rank 0, per-rank precoding with rho rescaled to the local cluster count
    S = torch.from_numpy(np.ascontiguousarray(d["X"] * (1.0 + rank)))  # ranks start with different s
    dist.broadcast(torch.view_as_real(S), src=0)
    S0 = d["X"]
    same_s = bool(np.allclose(S.numpy(), S0, rtol=0, atol=0))
    rho = 0.8
    if cs_l:
        part = orc.precode(H[:, :, b0:b1], S.numpy(), cs_l, K, rho=rho * np.sqrt(len(cs_l) / C))
        full = orc.precode(H, S0, cs, K, rho=rho)[:, :, b0:b1]
        err_dl = float(np.max(np.abs(part - full)) / np.max(np.abs(full)))
    else:
        err_dl = 0.0
    out[rank] = (err_ul, err_lam, same_s, err_dl)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,cs,fuse", [(2, [8, 8, 8, 8], "colnorm"), (3, [8, 12, 8, 4], "colnorm"),
                                           (3, [8, 8], "colnorm"), (2, [8, 8, 16], "equal")])
def test_cluster_layout_matches_single_device(world, cs, fuse):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), cs, fuse, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        err_ul, err_lam, same_s, err_dl = out[r]
        assert err_ul < 1e-6, (r, err_ul)   # lambda travels as float32
        assert err_lam < 1e-6, (r, err_lam)
        assert same_s
        assert err_dl < 1e-12, (r, err_dl)
