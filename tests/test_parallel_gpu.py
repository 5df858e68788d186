"""GPU parts of the multi-GPU layouts on one GPU: the fusion weights that cross devices
(cdmimo_fusion_weights) against the oracle's weights, the cluster-per-GPU uplink emulated by two
cluster groups run one after the other with the library's kernels (per-group detection, weights,
partial fusion with cdmimo_fuse) against one all-cluster call and the oracle, and the parallel
module's entry points in a one-rank process group.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist

import oracle as orc
from paper_1902_08653_gb300 import cdmimo, parallel
from paper_1902_08653_gb300 import workload as wl

from _util import assert_vectors_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    orc.build()
    cdmimo.lib()
    cdmimo.device_status(clear=True)
    return torch.device("cuda:0")


def t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("kind", ["c64", "f16"])
@pytest.mark.parametrize("cs,U", [([32] * 8, 16), ([16, 32, 48, 32], 12)])
def test_fusion_weights_normalize_to_the_oracle_lambda(dev, kind, cs, U):
    n_sc = 40
    d = wl.uplink(71, n_sc, 2, sum(cs), U, snr_db=wl.sweep_snr(n_sc))
    N0 = d["N0"].astype(np.float32)
    if kind == "c64":
        H32, H64 = wl.as_c64(d["H"])
        Ht, sc = t(H32, dev), {}
    else:
        qH, sH, H64 = wl.quantize_c16(d["H"], "f16")
        Ht, sc = t(qH.view(np.int16), dev).view(torch.float16), dict(h_scale=t(sH, dev))
    w = cdmimo.fusion_weights(Ht, t(N0, dev), cs, **sc).cpu().numpy().astype(np.float64)
    _, _, lam_o = orc.detect(H64, wl.as_c64(d["Y"])[1], N0.astype(np.float64), cs, 1)
    np.testing.assert_allclose(w / w.sum(axis=1, keepdims=True), lam_o, rtol=2e-6, atol=1e-7)
    we = cdmimo.fusion_weights(Ht, t(N0, dev), cs, fuse="equal", **sc).cpu().numpy()
    assert np.all(we == 1.0)
    N0b = N0.copy()
    N0b[3] = -1.0
    wb = cdmimo.fusion_weights(Ht, t(N0b, dev), cs, **sc).cpu().numpy()
    assert np.all(np.isnan(wb[3])) and np.all(np.isfinite(np.delete(wb, 3, axis=0)))


def test_cluster_groups_fuse_to_the_all_cluster_estimate(dev):
    """Two cluster groups, as two GPUs would hold them: detection with per-cluster outputs, weights,
    global normalization and partial fusion per group, summed -- against one call on all clusters
    (2e-5: the per-group normalization rounds differently) and the oracle (1e-4)."""
    cs, U, n_sc, n_sym, K = [32] * 8, 16, 300, 14, 3
    d = wl.uplink(72, n_sc, n_sym, 256, U, snr_db=wl.sweep_snr(n_sc))
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    N0 = d["N0"].astype(np.float32)
    Ht, Yt, Nt = t(H32, dev), t(Y32, dev), t(N0, dev)
    groups = [(0, 3, 0, 96), (3, 8, 96, 256)]  # uneven split: 3 and 5 clusters
    Xcs, ws = [], []
    for c0, c1, b0, b1 in groups:
        Hl, Yl = Ht[:, :, b0:b1].contiguous(), Yt[:, :, b0:b1].contiguous()
        Xc = torch.empty((n_sc, c1 - c0, n_sym, U), dtype=torch.complex64, device=dev)
        cdmimo.detect(Hl, Yl, Nt, cs[c0:c1], K, Xc=Xc)
        Xcs.append(Xc)
        ws.append(cdmimo.fusion_weights(Hl, Nt, cs[c0:c1]))
    tot = ws[0].sum(dim=1) + ws[1].sum(dim=1)
    X = torch.zeros((n_sc, n_sym, U), dtype=torch.complex64, device=dev)
    for Xc, w in zip(Xcs, ws):
        X += cdmimo.fuse(Xc, (w / tot[:, None]).contiguous(), weights_are_lambda=True)
    Xall = cdmimo.detect(Ht, Yt, Nt, cs, K)
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, threads=8)
    assert_vectors_close(X.cpu().numpy(), Xall.cpu().numpy(), 2e-5, "cluster groups vs one call")
    assert_vectors_close(X.cpu().numpy(), Xo, 1e-4, "cluster groups vs oracle")
    assert cdmimo.device_status(clear=True) == 0


def test_parallel_module_in_a_one_rank_group(dev):
    """detect_clusters / precode_clusters with one rank (NCCL): the whole array on this GPU."""
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        cs, U, n_sc, n_sym, K = [32] * 8, 16, 64, 14, 3
        d = wl.uplink(73, n_sc, n_sym, 256, U, snr_db=wl.sweep_snr(n_sc))
        H32, H64 = wl.as_c64(d["H"])
        Y32, Y64 = wl.as_c64(d["Y"])
        S32, S64 = wl.as_c64(d["X"])
        N0 = d["N0"].astype(np.float32)
        X = parallel.detect_clusters(t(H32, dev), t(Y32, dev), t(N0, dev), cs, 8, K)
        P = parallel.precode_clusters(t(H32, dev), t(S32, dev), cs, 8, K, rho=0.7)
        Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K)
        Po = orc.precode(H64, S64, cs, K, rho=0.7)
        assert_vectors_close(X.cpu().numpy(), Xo, 1e-4, "detect_clusters")
        assert_vectors_close(P.cpu().numpy(), Po, 1e-4, "precode_clusters")
    finally:
        dist.destroy_process_group()
    assert cdmimo.device_status(clear=True) == 0
