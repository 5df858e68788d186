"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Inputs are the exact complex64 (or dequantized 16-bit) values the GPU receives, upcast to FP64, so
the comparison measures kernel arithmetic only.  Acceptance: relative L2 error <= 1e-4 per estimate
vector (U-vector uplink, B-vector downlink); hard decisions identical except where the oracle lies
within 1e-3 of a decision threshold.
"""
import zlib

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo
from paper_1902_08653_gb300 import workload as wl

from _util import assert_decisions_match, assert_vectors_close, offsets

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    orc.build()
    cdmimo.lib()
    cdmimo.device_status(clear=True)
    return torch.device("cuda:0")


def to_dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def run_detect(dev, H, Y, N0, cs, K, fuse="colnorm", Ex=1.0, with_extras=True):
    H32, H64 = wl.as_c64(H)
    Y32, Y64 = wl.as_c64(Y)
    N032 = np.asarray(N0, np.float32)
    n_sc, U, B = H.shape
    C = len(cs)
    Xc = torch.zeros((n_sc, C, Y.shape[1], U), dtype=torch.complex64, device=dev) if with_extras else None
    lam = torch.zeros((n_sc, C), dtype=torch.float32, device=dev) if with_extras else None
    Xg = cdmimo.detect(to_dev(H32, dev), to_dev(Y32, dev), to_dev(N032, dev), cs, K, fuse=fuse, Ex=Ex, Xc=Xc, lam=lam)
    torch.cuda.synchronize()
    ref = orc.detect(H64, Y64, N032.astype(np.float64), cs, K, Ex=Ex, fuse=fuse, threads=8)
    got = (Xg.cpu().numpy(), Xc.cpu().numpy() if with_extras else None, lam.cpu().numpy() if with_extras else None)
    return got, ref


DETECT_CASES = {
    # name: (n_sc, n_sym, cluster sizes, U, K, fuse, M, snr)
    "cfg1_B32_C2_U4_K3": (64, 1, [16, 16], 4, 3, "equal", 4, 10.0),
    "cfg2_shape_ragged_nsc": (37, 14, [32] * 8, 16, 3, "colnorm", 16, "sweep"),
    "uneven_mixed_lanes": (9, 5, [16, 32, 8, 24, 20, 12], 6, 4, "colnorm", 16, 12.0),
    "odd_cluster_sizes": (7, 3, [7, 9, 5], 3, 5, "colnorm", 4, 8.0),
    "centralized_C1_B256": (6, 14, [256], 16, 5, "colnorm", 16, 15.0),
    "Bc64_U32": (5, 14, [64] * 4, 32, 3, "colnorm", 64, 20.0),
    "U64_Bc16": (3, 2, [16] * 4, 64, 2, "colnorm", 4, 25.0),
    "single_user_one_sweep": (8, 4, [16, 16], 1, 1, "equal", 16, 10.0),
    "Bc512_A32": (2, 3, [512], 8, 2, "colnorm", 16, 10.0),
}


@pytest.mark.parametrize("name", list(DETECT_CASES))
def test_detect_parity(dev, name):
    n_sc, n_sym, cs, U, K, fuse, M, snr = DETECT_CASES[name]
    snr = wl.sweep_snr(n_sc) if snr == "sweep" else snr
    d = wl.uplink(zlib.crc32(name.encode()) % 1000, n_sc, n_sym, sum(cs), U, snr_db=snr, M=M)
    (Xg, Xcg, lamg), (Xo, Xco, lamo) = run_detect(dev, d["H"], d["Y"], d["N0"], cs, K, fuse=fuse)
    assert_vectors_close(Xg, Xo, TOL, "Xhat")
    assert_vectors_close(Xcg, Xco, TOL, "Xc")
    np.testing.assert_allclose(lamg, lamo, rtol=1e-5, atol=1e-7)
    assert_decisions_match(Xg, Xo, M)
    assert cdmimo.device_status(clear=True) == 0


def test_detect_K0_and_empty(dev):
    d = wl.uplink(1, 4, 2, 32, 4)
    (Xg, Xcg, _), _ = run_detect(dev, d["H"], d["Y"], d["N0"], [16, 16], 0)
    assert np.all(Xg == 0) and np.all(Xcg == 0)
    e = torch.zeros((0, 4, 32), dtype=torch.complex64, device=dev)
    out = cdmimo.detect(e, torch.zeros((0, 2, 32), dtype=torch.complex64, device=dev),
                        torch.zeros(0, device=dev), [16, 16], 3)
    assert out.shape == (0, 2, 4)


def test_detect_noise_free_and_Ex(dev):
    d = wl.uplink(2, 6, 3, 64, 4, snr_db=np.inf)
    (Xg, _, _), (Xo, _, _) = run_detect(dev, d["H"], d["Y"], d["N0"], [32, 32], 6)
    assert_vectors_close(Xg, Xo, TOL, "N0=0")
    d = wl.uplink(3, 6, 3, 64, 4, snr_db=5.0)
    (Xg, _, _), (Xo, _, _) = run_detect(dev, d["H"], d["Y"], d["N0"], [32, 32], 3, Ex=2.5)
    assert_vectors_close(Xg, Xo, TOL, "Ex=2.5")


def test_detect_zero_column(dev):
    d = wl.uplink(4, 3, 2, 32, 4, snr_db=np.inf)
    H = d["H"].copy()
    H[:, 2, :16] = 0  # user 2 absent from cluster 0
    (Xg, Xcg, _), (Xo, Xco, _) = run_detect(dev, H, d["Y"], d["N0"], [16, 16], 4)
    assert np.all(Xcg[:, 0, :, 2] == 0)
    assert_vectors_close(Xcg, Xco, TOL, "zero column")


def test_detect_bad_noise_variance_flags(dev):
    d = wl.uplink(5, 3, 2, 32, 4)
    N0 = d["N0"].astype(np.float32)
    N0[1] = -1.0
    Xg = cdmimo.detect(to_dev(wl.as_c64(d["H"])[0], dev), to_dev(wl.as_c64(d["Y"])[0], dev), to_dev(N0, dev),
                       [16, 16], 3).cpu().numpy()
    assert cdmimo.device_status(clear=True) & cdmimo.DEV_BAD_N0
    assert np.all(np.isnan(Xg[1])) and np.all(np.isfinite(Xg[[0, 2]]))
    assert cdmimo.device_status(clear=True) == 0


def test_detect_low_precision_storage(dev):
    """16-bit H and y with per-subcarrier scales: parity against the oracle run on the exact
    dequantized values."""
    n_sc, n_sym, B, U, cs = 11, 14, 256, 32, [32] * 8
    d = wl.uplink(8, n_sc, n_sym, B, U, snr_db=wl.sweep_snr(n_sc), M=64)
    N0 = d["N0"].astype(np.float32)
    for kind, tdt in (("f16", torch.float16), ("bf16", torch.bfloat16)):
        qH, sH, dH = wl.quantize_c16(d["H"], kind)
        qY, sY, dY = wl.quantize_c16(d["Y"], kind)
        Ht = torch.from_numpy(qH.view(np.int16)).to(dev).view(tdt)
        Yt = torch.from_numpy(qY.view(np.int16)).to(dev).view(tdt)
        for K in (3, 5):
            Xg = cdmimo.detect(Ht, Yt, to_dev(N0, dev), cs, K, h_scale=to_dev(sH, dev),
                               y_scale=to_dev(sY, dev)).cpu().numpy()
            Xo, _, _ = orc.detect(dH, dY, N0.astype(np.float64), cs, K, threads=8)
            assert_vectors_close(Xg, Xo, TOL, f"{kind} K={K}")


# ------------------------------------------------------------------------------------------
# precoding
# ------------------------------------------------------------------------------------------
PRECODE_CASES = {
    "cfg1_shape": (64, 1, [16, 16], 4, 3, 1.0),
    "cfg2_shape_ragged_nsc": (29, 14, [32] * 8, 16, 3, 1.0),
    "uneven_mixed_lanes": (9, 5, [16, 32, 8, 24, 20, 12], 6, 4, 2.0),
    "odd_cluster_sizes": (7, 3, [7, 9, 5], 3, 5, 0.7),
    "Bc_less_than_U": (5, 4, [16] * 4, 24, 3, 1.0),
    "centralized_C1": (4, 14, [256], 16, 4, 1.0),
    "Bc64_U64": (3, 2, [64] * 2, 64, 2, 1.0),
}


@pytest.mark.parametrize("name", list(PRECODE_CASES))
def test_precode_parity(dev, name):
    n_sc, n_sym, cs, U, K, rho = PRECODE_CASES[name]
    d = wl.downlink(zlib.crc32(name.encode()) % 1000, n_sc, n_sym, sum(cs), U)
    H32, H64 = wl.as_c64(d["H"])
    S32, S64 = wl.as_c64(d["S"])
    Xg = cdmimo.precode(to_dev(H32, dev), to_dev(S32, dev), cs, K, rho=rho).cpu().numpy()
    Xo = orc.precode(H64, S64, cs, K, rho=rho, threads=8)
    assert_vectors_close(Xg, Xo, TOL, "Xdl")
    o = offsets(cs)
    for c in range(len(cs)):
        np.testing.assert_allclose(np.linalg.norm(Xg[..., o[c]:o[c + 1]], axis=-1), rho / np.sqrt(len(cs)), rtol=1e-5)
    assert cdmimo.device_status(clear=True) == 0


def test_precode_K0_and_zero_column(dev):
    d = wl.downlink(6, 4, 2, 32, 4)
    H = d["H"].copy()
    H[:, 1, 16:] = 0
    H32, H64 = wl.as_c64(H)
    S32, S64 = wl.as_c64(d["S"])
    Xg = cdmimo.precode(to_dev(H32, dev), to_dev(S32, dev), [16, 16], 0).cpu().numpy()
    assert np.all(Xg == 0)
    Xg = cdmimo.precode(to_dev(H32, dev), to_dev(S32, dev), [16, 16], 3).cpu().numpy()
    assert_vectors_close(Xg, orc.precode(H64, S64, [16, 16], 3), TOL, "zero column")


# ------------------------------------------------------------------------------------------
# standalone fusion
# ------------------------------------------------------------------------------------------
def test_fuse_parity(dev):
    d = wl.uplink(9, 21, 14, 256, 16, snr_db=wl.sweep_snr(21))
    cs = [32] * 8
    Xo, Xco, lamo = orc.detect(d["H"], d["Y"], d["N0"], cs, 3)
    Xc = to_dev(Xco.astype(np.complex64), dev)
    lam = to_dev(lamo.astype(np.float32), dev)
    got = cdmimo.fuse(Xc, lam, weights_are_lambda=True).cpu().numpy()
    assert_vectors_close(got, Xo, TOL, "fuse lambda")
    sigma2 = to_dev((0.37 / lamo).astype(np.float32), dev)   # any common scale gives the same weights
    got = cdmimo.fuse(Xc, sigma2).cpu().numpy()
    assert_vectors_close(got, Xo, TOL, "fuse sigma2")
    s2 = np.ones((21, 8), np.float32)
    s2[3, 5] = 0.0
    got = cdmimo.fuse(Xc, to_dev(s2, dev)).cpu().numpy()
    np.testing.assert_allclose(got[3], Xco[3, 5], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(got[4], Xco[4].mean(axis=0), rtol=1e-5, atol=1e-6)


# ------------------------------------------------------------------------------------------
# host-buffer (end-to-end) variants
# ------------------------------------------------------------------------------------------
def test_host_variants_match_device_calls(dev):
    n_sc, n_sym, B, U, cs = 40, 14, 256, 16, [32] * 8
    d = wl.uplink(10, n_sc, n_sym, B, U, snr_db=wl.sweep_snr(n_sc))
    H32 = torch.from_numpy(wl.as_c64(d["H"])[0]).pin_memory()
    Y32 = torch.from_numpy(wl.as_c64(d["Y"])[0]).pin_memory()
    N0 = torch.from_numpy(d["N0"].astype(np.float32)).pin_memory()
    X = torch.empty((n_sc, n_sym, U), dtype=torch.complex64).pin_memory()
    ws = torch.empty(cdmimo.host_workspace_size(cdmimo.OP_DETECT, n_sc, n_sym, B, U, cs, 3), dtype=torch.uint8,
                     device=dev)
    cdmimo.detect_host(H32, Y32, N0, cs, 3, X, ws)
    torch.cuda.synchronize()
    ref = cdmimo.detect(H32.to(dev), Y32.to(dev), N0.to(dev), cs, 3).cpu()
    assert torch.equal(X, ref)
    dl = wl.downlink(11, n_sc, n_sym, B, U)
    Hd = torch.from_numpy(wl.as_c64(dl["H"])[0]).pin_memory()
    S = torch.from_numpy(wl.as_c64(dl["S"])[0]).pin_memory()
    Xd = torch.empty((n_sc, n_sym, B), dtype=torch.complex64).pin_memory()
    ws = torch.empty(cdmimo.host_workspace_size(cdmimo.OP_PRECODE, n_sc, n_sym, B, U, cs, 3), dtype=torch.uint8,
                     device=dev)
    cdmimo.precode_host(Hd, S, cs, 3, Xd, ws)
    torch.cuda.synchronize()
    assert torch.equal(Xd, cdmimo.precode(Hd.to(dev), S.to(dev), cs, 3).cpu())


@pytest.mark.parametrize("cs,U", [([20] * 4, 8), ([18] * 2, 5), ([16] * 4, 12), ([64] * 2, 16)])
def test_low_precision_staging_paths(dev, cs, U):
    """16-bit storage: cluster sizes that are multiples of 4 take the bulk-copied staging buffers
    (with padding columns when B_c < A P), others the converting loads; both match the oracle."""
    n_sc, n_sym = 13, 6
    d = wl.uplink(91, n_sc, n_sym, sum(cs), U, snr_db=wl.sweep_snr(n_sc), M=16)
    dl = wl.downlink(92, n_sc, n_sym, sum(cs), U)
    N0 = d["N0"].astype(np.float32)
    for kind, tdt in (("f16", torch.float16), ("bf16", torch.bfloat16)):
        qH, sH, dH = wl.quantize_c16(d["H"], kind)
        qY, sY, dY = wl.quantize_c16(d["Y"], kind)
        Xg = cdmimo.detect(torch.from_numpy(qH.view(np.int16)).to(dev).view(tdt),
                           torch.from_numpy(qY.view(np.int16)).to(dev).view(tdt), to_dev(N0, dev), cs, 3,
                           h_scale=to_dev(sH, dev), y_scale=to_dev(sY, dev)).cpu().numpy()
        Xo, _, _ = orc.detect(dH, dY, N0.astype(np.float64), cs, 3)
        assert_vectors_close(Xg, Xo, TOL, f"{kind} detect {cs}")
        qHd, _, dHd = wl.quantize_c16(dl["H"], kind)
        S32, S64 = wl.as_c64(dl["S"])
        Xd = cdmimo.precode(torch.from_numpy(qHd.view(np.int16)).to(dev).view(tdt), to_dev(S32, dev), cs,
                            3).cpu().numpy()
        assert_vectors_close(Xd, orc.precode(dHd, S64, cs, 3), TOL, f"{kind} precode {cs}")


@pytest.mark.parametrize("kind", ["c64", "f16", "bf16"])
@pytest.mark.parametrize("U", [24, 32, 48, 64])
def test_user_counts_every_storage(dev, U, kind):
    """Detection and precoding at U = 24, 32, 48 and 64 users (B = 256 in clusters of 32, so U > B_c
    for the last two) in every storage format, on whatever form AUTO picks (the tensor-core kernel
    for U <= 32, the residual kernels above): parity with the oracle on the values the GPU receives
    (dequantized for 16-bit storage)."""
    n_sc, n_sym, cs, K = 40, 14, [32] * 8, 3
    d = wl.uplink(500 + U, n_sc, n_sym, sum(cs), U, snr_db=wl.sweep_snr(n_sc), M=16)
    N0 = d["N0"].astype(np.float32)
    if kind == "c64":
        Ht, dH = to_dev(wl.as_c64(d["H"])[0], dev), wl.as_c64(d["H"])[1]
        Yt, dY = to_dev(wl.as_c64(d["Y"])[0], dev), wl.as_c64(d["Y"])[1]
        sc = {}
    else:
        tdt = torch.float16 if kind == "f16" else torch.bfloat16
        qH, sH, dH = wl.quantize_c16(d["H"], kind)
        qY, sY, dY = wl.quantize_c16(d["Y"], kind)
        Ht = torch.from_numpy(qH.view(np.int16)).to(dev).view(tdt)
        Yt = torch.from_numpy(qY.view(np.int16)).to(dev).view(tdt)
        sc = dict(h_scale=to_dev(sH, dev), y_scale=to_dev(sY, dev))
    Xg = cdmimo.detect(Ht, Yt, to_dev(N0, dev), cs, K, **sc).cpu().numpy()
    Xo, _, _ = orc.detect(dH, dY, N0.astype(np.float64), cs, K, threads=8)
    assert_vectors_close(Xg, Xo, TOL, f"detect U={U} {kind}")
    if kind == "c64":
        S32, S64 = wl.as_c64(d["X"])
        Pg = cdmimo.precode(Ht, to_dev(S32, dev), cs, K).cpu().numpy()
        assert_vectors_close(Pg, orc.precode(dH, S64, cs, K, threads=8), TOL, f"precode U={U}")
    assert cdmimo.device_status(clear=True) == 0
