"""GPU parity of the tensor-core Gram-form detection kernel for 16 < U <= 32 users
(cd_detect_tc32_kernel: form GRAM_TC, and AUTO where it applies), against the FP64 oracle.

The kernel evaluates Algorithm 1's iterate through G_c = H_c^H H_c and z = H_c^H y_c formed by
split-TF32 (c64) or exact-TF32 (16-bit storage) MMAs over two 16-user tiles, G_c's lower-left block
mirrored from its upper-right one, and FP32 sweeps with 32 coordinates per lane.  Acceptance as for
every detector: 1e-4 relative L2 per estimate vector, hard decisions equal except within 1e-3 of a
threshold; 16-bit storage against the oracle on the exact dequantized values.  Shapes cover users
below the 32-row tiles (U = 17, 24), clusters of 16, 32 and 64 antennas, one and fourteen symbols,
K = 1 and 5, the pipeline's edges (CTAs with zero, one and two subcarriers), the per-cluster outputs,
and the whole configuration-3 batch (1200 x 14, U = 32, 64-QAM) in every storage.
"""
import os

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo
from paper_1902_08653_gb300 import workload as wl

from _util import assert_decisions_match, assert_vectors_close

pytestmark = pytest.mark.gpu
TOL = 1e-4
THREADS = os.cpu_count() or 8
KINDS = {"c64": (None, cdmimo.C64), "f16": (torch.float16, cdmimo.C16F), "bf16": (torch.bfloat16, cdmimo.C16BF)}


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


def inputs(dev, seed, n_sc, n_sym, cs, U, kind, M=16, snr="sweep"):
    snr = wl.sweep_snr(n_sc) if snr == "sweep" else snr
    d = wl.uplink(seed, n_sc, n_sym, sum(cs), U, snr_db=snr, M=M)
    N0 = d["N0"].astype(np.float32)
    tdt, _ = KINDS[kind]
    if tdt is None:
        H32, H64 = wl.as_c64(d["H"])
        Y32, Y64 = wl.as_c64(d["Y"])
        Ht, Yt, sc = t(H32, dev), t(Y32, dev), {}
    else:
        qH, sH, H64 = wl.quantize_c16(d["H"], kind)
        qY, sY, Y64 = wl.quantize_c16(d["Y"], kind)
        Ht, Yt = t(qH.view(np.int16), dev).view(tdt), t(qY.view(np.int16), dev).view(tdt)
        sc = dict(h_scale=t(sH, dev), y_scale=t(sY, dev))
    return dict(H=Ht, Y=Yt, N0=t(N0, dev), sc=sc, H64=H64, Y64=Y64, N064=N0.astype(np.float64), d=d)


# name: (n_sc, n_sym, cluster sizes, U, K, fuse, storage)
CASES = {
    "U32_Bc32_cfg3_shape": (157, 14, [32] * 8, 32, 3, "colnorm", "c64"),
    "U32_Bc32_fp16_K5": (153, 14, [32] * 8, 32, 5, "colnorm", "f16"),
    "U32_Bc32_bf16": (60, 14, [32] * 8, 32, 3, "colnorm", "bf16"),
    "U24_Bc16_equal": (97, 9, [16] * 8, 24, 3, "equal", "c64"),
    "U17_Bc64_one_symbol": (40, 1, [64] * 4, 17, 5, "colnorm", "c64"),
    "U32_Bc64_K1": (31, 7, [64] * 3, 32, 1, "colnorm", "f16"),
    "one_subcarrier": (1, 14, [32] * 8, 32, 3, "colnorm", "c64"),
    "U20_Bc32_bf16_odd": (11, 5, [32] * 5, 20, 2, "colnorm", "bf16"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_tc32_matches_oracle(dev, name):
    n_sc, n_sym, cs, U, K, fuse, kind = CASES[name]
    x = inputs(dev, 900 + len(name) + n_sc, n_sc, n_sym, cs, U, kind)
    code = KINDS[kind][1]
    assert cdmimo.selected_form(cdmimo.OP_DETECT, n_sc, n_sym, sum(cs), U, cs, K, in_dtype=code, H=x["H"],
                                form="gram_tc") == "gram_tc"
    X = cdmimo.detect(x["H"], x["Y"], x["N0"], cs, K, fuse=fuse, form="gram_tc", **x["sc"])
    torch.cuda.synchronize()
    Xo, _, _ = orc.detect(x["H64"], x["Y64"], x["N064"], cs, K, fuse=fuse, threads=THREADS)
    X = X.cpu().numpy()
    assert_vectors_close(X, Xo, TOL, f"tc32 {name}")
    assert_decisions_match(X, Xo, 16)
    assert cdmimo.device_status(clear=True) == 0


def test_tc32_per_cluster_outputs(dev):
    cs, U, n_sc = [32] * 8, 32, 45
    x = inputs(dev, 41, n_sc, 14, cs, U, "c64")
    Xc = torch.zeros((n_sc, 8, 14, U), dtype=torch.complex64, device=dev)
    lam = torch.zeros((n_sc, 8), dtype=torch.float32, device=dev)
    X = cdmimo.detect(x["H"], x["Y"], x["N0"], cs, 3, form="gram_tc", Xc=Xc, lam=lam)
    Xo, Xco, lamo = orc.detect(x["H64"], x["Y64"], x["N064"], cs, 3, threads=THREADS)
    assert_vectors_close(X.cpu().numpy(), Xo, TOL, "tc32 Xhat")
    assert_vectors_close(Xc.cpu().numpy(), Xco, TOL, "tc32 Xc")
    np.testing.assert_allclose(lam.cpu().numpy(), lamo, rtol=1e-5, atol=1e-7)
    assert cdmimo.device_status(clear=True) == 0


def test_tc32_bad_noise_variance_and_K0(dev):
    cs, U, n_sc = [32] * 8, 32, 9
    x = inputs(dev, 43, n_sc, 14, cs, U, "c64", snr=15.0)
    N0 = x["N0"].clone()
    N0[4] = -1.0
    cdmimo.device_status(clear=True)
    X = cdmimo.detect(x["H"], x["Y"], N0, cs, 3, form="gram_tc").cpu().numpy()
    assert cdmimo.device_status(clear=True) & cdmimo.DEV_BAD_N0
    assert np.all(np.isnan(X[4])) and np.all(np.isfinite(np.delete(X, 4, axis=0)))
    assert not cdmimo.detect(x["H"], x["Y"], x["N0"], cs, 0, form="gram_tc").abs().any()
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("kind", list(KINDS))
def test_config3_full_batch_every_vector(dev, kind):
    """Configuration 3's batch (1200 subcarriers x 14 symbols, B = 256 in 8 x 32, U = 32, 64-QAM, SNR
    sweep) under AUTO, which selects this kernel, at K = 3 and K = 5."""
    cs, U, n_sc = [32] * 8, 32, 1200
    x = inputs(dev, wl.DEFAULT_SEED, n_sc, 14, cs, U, kind, M=64)
    code = KINDS[kind][1]
    for K in (3, 5):
        assert cdmimo.selected_form(cdmimo.OP_DETECT, n_sc, 14, 256, U, cs, K, in_dtype=code, H=x["H"]) == "gram_tc"
        X = cdmimo.detect(x["H"], x["Y"], x["N0"], cs, K, **x["sc"]).cpu().numpy()
        Xo, _, _ = orc.detect(x["H64"], x["Y64"], x["N064"], cs, K, threads=THREADS)
        assert_vectors_close(X, Xo, TOL, f"config 3 {kind} K={K}")
        assert_decisions_match(X, Xo, 64)
    assert cdmimo.device_status(clear=True) == 0


def test_mixed_clusters_fall_back(dev):
    """Unequal cluster sizes are not this kernel's: AUTO runs the residual form, still oracle-exact."""
    cs, U = [32, 64, 32, 128], 24
    x = inputs(dev, 47, 13, 6, cs, U, "c64")
    assert cdmimo.selected_form(cdmimo.OP_DETECT, 13, 6, sum(cs), U, cs, 3, H=x["H"]) == "residual"
    X = cdmimo.detect(x["H"], x["Y"], x["N0"], cs, 3).cpu().numpy()
    Xo, _, _ = orc.detect(x["H64"], x["Y64"], x["N064"], cs, 3, threads=THREADS)
    assert_vectors_close(X, Xo, TOL, "mixed clusters")
