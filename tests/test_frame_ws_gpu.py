"""GPU parity of the warp-specialized tensor-core kernel (cd_frame_ws_kernel), which runs the Gram
form on the tensor cores (form GRAM_TC, and AUTO where it applies) with the phases of consecutive
subcarriers overlapped in one CTA per SM.

With its contractions on mma.sync (form GRAM_TC) it evaluates exactly the operations of the phased
kernel (cd_frame_tc_kernel, form GRAM_TC_PHASED) in the same order, only scheduled differently, so
the two must agree bit for bit.  With G_c and z formed on the tcgen05 tensor cores (form
GRAM_TC_UMMA with c64 storage) the same split-TF32 products are summed in another order: those
results must stay within 1e-5 of the mma.sync ones.  Each case is also held to the FP64
oracle at 1e-4 relative L2 per vector.  The shapes cover the pipeline's edges: CTAs with zero, one,
two and three subcarriers (the fill and drain of a three-stage pipeline), users below the 16-row
tiles, one symbol, K = 1 and K = 5, clusters of 16 and 32 antennas, fewer than eight clusters, and
16-bit storage.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo
from paper_1902_08653_gb300 import workload as wl

from _util import assert_vectors_close

pytestmark = pytest.mark.gpu
TOL = 1e-4
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


def inputs(dev, seed, n_sc, n_sym, cs, U, kind="c64", snr="sweep"):
    snr = wl.sweep_snr(n_sc) if snr == "sweep" else snr
    d = wl.uplink(seed, n_sc, n_sym, sum(cs), U, snr_db=snr)
    S32, S64 = wl.as_c64(d["X"])
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
    return dict(H=Ht, Y=Yt, S=t(S32, dev), N0=t(N0, dev), sc=sc, H64=H64, Y64=Y64, S64=S64, N064=N0.astype(np.float64))


# name: (n_sc, n_sym, cluster sizes, U, K, fuse, storage); n_sc against the GPU's 152 CTAs (one per
# SM): 1..3 leave most CTAs without work and the rest with one subcarrier; 305 gives CTAs two and three
CASES = {
    "cfg2_one_subcarrier": (1, 14, [32] * 8, 16, 3, "colnorm", "c64"),
    "cfg2_three_subcarriers": (3, 14, [32] * 8, 16, 3, "colnorm", "c64"),
    "cfg2_two_and_three_per_cta": (305, 14, [32] * 8, 16, 3, "colnorm", "c64"),
    "cfg2_fp16": (305, 14, [32] * 8, 16, 3, "colnorm", "f16"),
    "cfg2_bf16": (157, 14, [32] * 8, 16, 3, "colnorm", "bf16"),
    "U9_K1_equal": (200, 14, [32] * 8, 9, 1, "equal", "c64"),
    "K5_one_symbol": (170, 1, [32] * 4, 16, 5, "colnorm", "c64"),
    "Bc16_C8_U12_n_sym9": (160, 9, [16] * 8, 12, 3, "colnorm", "c64"),
    "Bc16_C6_bf16_odd": (99, 5, [16] * 6, 13, 2, "colnorm", "bf16"),
    "Bc32_C3_U11_n_sym7": (240, 7, [32] * 3, 11, 3, "colnorm", "c64"),
    "Bc16_C1_U10": (153, 14, [16], 10, 2, "colnorm", "c64"),
    "Bc16_C16_n_sym8": (311, 8, [16] * 16, 12, 3, "colnorm", "c64"),  # four clusters per sweep warp
}


def run_three(x, cs, K, fuse, form):
    args = (x["H"], x["Y"], x["N0"], x["S"], cs, K)
    X, P = cdmimo.detect_precode(*args, fuse=fuse, form=form, **x["sc"])
    D = cdmimo.detect(x["H"], x["Y"], x["N0"], cs, K, fuse=fuse, form=form, **x["sc"])
    Q = cdmimo.precode(x["H"], x["S"], cs, K, form=form)
    torch.cuda.synchronize()
    return X, P, D, Q


@pytest.mark.parametrize("name", list(CASES))
def test_ws_equals_phased_and_matches_oracle(dev, name):
    n_sc, n_sym, cs, U, K, fuse, kind = CASES[name]
    x = inputs(dev, 700 + len(name), n_sc, n_sym, cs, U, kind)
    code = KINDS[kind][1]
    B = sum(cs)
    for form in ("gram_tc", "gram_tc_phased", "gram_tc_umma"):
        assert cdmimo.selected_form(cdmimo.OP_FRAME, n_sc, n_sym, B, U, cs, K, in_dtype=code, H=x["H"],
                                    form=form) == form
    sync = run_three(x, cs, K, fuse, "gram_tc")
    phased = run_three(x, cs, K, fuse, "gram_tc_phased")
    for a, b, what in zip(sync, phased, ("frame Xhat", "frame Xdl", "detect", "precode")):
        assert torch.equal(a, b), f"{what}: warp-specialized (mma.sync) != phased"
    t5 = run_three(x, cs, K, fuse, "gram_tc_umma")
    Xo, _, _ = orc.detect(x["H64"], x["Y64"], x["N064"], cs, K, fuse=fuse, threads=8)
    Po = orc.precode(x["H64"], x["S64"], cs, K, threads=8)
    for got, ref, what in zip(t5, (Xo, Po, Xo, Po), ("frame Xhat", "frame Xdl", "detect", "precode")):
        assert_vectors_close(got.cpu().numpy(), ref, TOL, f"ws {what}")
    for a, b, what in zip(t5, sync, ("frame Xhat", "frame Xdl", "detect", "precode")):
        if kind == "c64":  # tcgen05 contractions: the same products in another order
            assert_vectors_close(a.cpu().numpy(), b.cpu().numpy(), 1e-5, f"tcgen05 vs mma.sync {what}")
        else:
            assert torch.equal(a, b), f"{what}: 16-bit storage runs the mma.sync kernel"
    assert cdmimo.device_status(clear=True) == 0


def test_ws_full_size_equals_phased(dev):
    """The benchmark's batch (1200 x 14, B = 256 in 8 x 32, U = 16, K = 3): the mma.sync kernel (the
    default) and all three modes equal the phased kernel bit for bit, also with a schedule workspace
    (the phased kernel's dynamic schedule, twice in a row so the counters must have reset
    themselves); the tcgen05 variant stays within 1e-5 of them, and repeats its own bits."""
    cs, U, K, n_sc = [32] * 8, 16, 3, 1200
    x = inputs(dev, 20190222, n_sc, 14, cs, U)
    args = (x["H"], x["Y"], x["N0"], x["S"], cs, K)
    ref = cdmimo.detect_precode(*args, form="gram_tc_phased")
    for ws, form in ((None, "auto"), (True, "auto"), (True, "auto")):
        got = cdmimo.detect_precode(*args, workspace=ws, form=form)
        torch.cuda.synchronize()
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
    assert torch.equal(cdmimo.detect(x["H"], x["Y"], x["N0"], cs, K),
                       cdmimo.detect(x["H"], x["Y"], x["N0"], cs, K, form="gram_tc_phased"))
    assert torch.equal(cdmimo.precode(x["H"], x["S"], cs, K),
                       cdmimo.precode(x["H"], x["S"], cs, K, form="gram_tc_phased"))
    t5 = cdmimo.detect_precode(*args, form="gram_tc_umma")
    t5b = cdmimo.detect_precode(*args, form="gram_tc_umma")
    torch.cuda.synchronize()
    assert torch.equal(t5[0], t5b[0]) and torch.equal(t5[1], t5b[1])
    for a, b in zip(t5, ref):
        assert_vectors_close(a.cpu().numpy(), b.cpu().numpy(), 1e-5, "tcgen05 vs mma.sync, full size")
    assert cdmimo.device_status(clear=True) == 0


def test_ws_bad_noise_variance_and_K0(dev):
    """A negative N0 flags CDMIMO_DEV_BAD_N0 and makes only that subcarrier's uplink estimate NaN;
    K = 0 gives zero outputs."""
    cs, U, n_sc = [32] * 8, 16, 310
    x = inputs(dev, 31, n_sc, 14, cs, U, snr=15.0)
    N0 = x["N0"].clone()
    N0[[5, 160]] = -1.0
    cdmimo.device_status(clear=True)
    X, P = cdmimo.detect_precode(x["H"], x["Y"], N0, x["S"], cs, 3)
    assert cdmimo.device_status(clear=True) & cdmimo.DEV_BAD_N0
    X = X.cpu().numpy()
    bad = np.zeros(n_sc, bool)
    bad[[5, 160]] = True
    assert np.all(np.isnan(X[bad])) and np.all(np.isfinite(X[~bad])) and torch.isfinite(P).all()
    X0, P0 = cdmimo.detect_precode(x["H"], x["Y"], x["N0"], x["S"], cs, 0)
    assert not X0.abs().any() and not P0.abs().any()
    assert cdmimo.device_status(clear=True) == 0
