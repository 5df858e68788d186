"""GPU parity of the tensor-core Gram-form kernel (form GRAM_TC, and AUTO where it applies) in its
three modes: the TDD frame (cdmimo_detect_precode), the uplink alone (cdmimo_detect) and the
downlink alone (cdmimo_precode).  z = H_c^H y_c, G_c = H_c^H H_c and x_c = H_c w run on TF32 MMAs
with split FP32 operands; the sweeps are FP32.

Each case is compared with the FP64 oracle (Algorithms 1 and 2 as written) at the 1e-4 relative L2
bound per vector, and the well-conditioned ones with the FP32 Gram-form frame kernel at 2e-5 (the
same iterates, different rounding).
"""
import zlib

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo
from paper_1902_08653_gb300 import workload as wl

from _util import assert_decisions_match, assert_vectors_close

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


def t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


CASES = {
    # name: (n_sc, n_sym, cluster sizes, U, K, fuse, snr, compare with the FP32 Gram frame)
    "cfg2_B256_C8x32_U16": (50, 14, [32] * 8, 16, 3, "colnorm", "sweep", True),
    "more_subcarriers_than_ctas": (333, 14, [32] * 8, 16, 3, "colnorm", 20.0, True),
    "one_subcarrier": (1, 14, [32] * 8, 16, 3, "colnorm", 10.0, True),
    "n_sym16_max_lanes": (23, 16, [32] * 8, 16, 2, "colnorm", 25.0, True),
    "Bc16_C16_U10_n_sym8": (19, 8, [16] * 16, 10, 3, "colnorm", 20.0, False),
    "Bc16_U9_odd_symbols": (13, 5, [16] * 6, 9, 4, "equal", 10.0, False),
    "U12_K1_one_symbol": (29, 1, [32] * 4, 12, 1, "colnorm", 15.0, True),
    "K5_equal": (17, 14, [32] * 8, 16, 5, "equal", 30.0, True),
}


def run_case(dev, n_sc, n_sym, cs, U, K, fuse, snr, seed, tweak=None):
    snr = wl.sweep_snr(n_sc) if snr == "sweep" else snr
    d = wl.uplink(seed, n_sc, n_sym, sum(cs), U, snr_db=snr)
    if tweak:
        tweak(d)
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    S32, S64 = wl.as_c64(d["X"])  # downlink symbols: any U-vectors per (subcarrier, symbol)
    N0 = d["N0"].astype(np.float32)
    Ht, Yt, St, Nt = t(H32, dev), t(Y32, dev), t(S32, dev), t(N0, dev)
    assert cdmimo.selected_form(cdmimo.OP_FRAME, n_sc, n_sym, sum(cs), U, cs, K, form="gram_tc", H=Ht) == "gram_tc"
    X, P = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K, fuse=fuse, form="gram_tc")
    Xg, Pg = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K, fuse=fuse, form="gram")
    torch.cuda.synchronize()
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, fuse=fuse, threads=8)
    Po = orc.precode(H64, S64, cs, K, threads=8)
    return X.cpu().numpy(), P.cpu().numpy(), Xg.cpu().numpy(), Pg.cpu().numpy(), Xo, Po


@pytest.mark.parametrize("name", list(CASES))
def test_frame_tc_matches_oracle(dev, name):
    n_sc, n_sym, cs, U, K, fuse, snr, vs_gram = CASES[name]
    X, P, Xg, Pg, Xo, Po = run_case(dev, n_sc, n_sym, cs, U, K, fuse, snr, zlib.crc32(name.encode()) % 1000)
    assert_vectors_close(X, Xo, TOL, "tc frame Xhat")
    assert_vectors_close(P, Po, TOL, "tc frame Xdl")
    assert_decisions_match(X, Xo, 16)
    if vs_gram:
        assert_vectors_close(X, Xg, 2e-5, "tc vs fp32 gram frame Xhat")
        assert_vectors_close(P, Pg, 2e-5, "tc vs fp32 gram frame Xdl")
    assert cdmimo.device_status(clear=True) == 0


def test_frame_tc_zero_column_and_noise_free(dev):
    """A user with a zero channel in one cluster (the downlink skips it there, p = 0; the uplink's
    m = 1/alpha keeps its estimate 0) and N0 = 0 on some subcarriers (plain Gauss-Seidel LS)."""
    cs, U = [32] * 8, 16

    def tweak(d):
        d["H"][:, 3, 64:96] = 0.0
        d["N0"][::2] = 0.0
        d["Y"][:] = np.einsum("fub,fnu->fnb", d["H"], d["X"])
        d["Y"][1::2] += 0.05 * (np.random.default_rng(5).standard_normal(d["Y"][1::2].shape) + 0j)

    X, P, Xg, Pg, Xo, Po = run_case(dev, 21, 14, cs, U, 3, "colnorm", 20.0, 77, tweak)
    assert_vectors_close(X, Xo, TOL, "tc frame Xhat")
    assert_vectors_close(P, Po, TOL, "tc frame Xdl")
    assert np.isfinite(X).all() and np.isfinite(P).all()
    assert cdmimo.device_status(clear=True) == 0


def test_frame_tc_k0_and_schedules(dev):
    """K = 0 gives zero outputs; the dynamic schedule (workspace) gives the static schedule's result
    bit for bit; AUTO runs the tensor-core kernel at the config-2 shape."""
    cs, U, n_sc, n_sym = [32] * 8, 16, 700, 14
    d = wl.uplink(4242, n_sc, n_sym, 256, U, snr_db=wl.sweep_snr(n_sc))
    H32, _ = wl.as_c64(d["H"])
    Y32, _ = wl.as_c64(d["Y"])
    S32, _ = wl.as_c64(d["X"])
    Ht, Yt, St, Nt = t(H32, dev), t(Y32, dev), t(S32, dev), t(d["N0"].astype(np.float32), dev)
    assert cdmimo.selected_form(cdmimo.OP_FRAME, n_sc, n_sym, 256, U, cs, 3, H=Ht) == "gram_tc"
    assert cdmimo.selected_form(cdmimo.OP_FRAME, n_sc, n_sym, 256, U, cs, 3, form="gram", H=Ht) == "gram"
    X0, P0 = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, 0, form="gram_tc")
    assert not X0.abs().any() and not P0.abs().any()
    a = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, 3)
    b = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, 3, workspace=True)
    c = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, 3, form="gram_tc")
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])
    assert cdmimo.device_status(clear=True) == 0


def test_frame_tc_declines_other_shapes(dev):
    """Shapes outside the kernel's (U <= 8, uneven or other cluster sizes, n_sym > 16) run the FP32
    Gram frame or the two calls; 16-bit storage takes it."""
    for args in ((8, 14, 128, 8, [32] * 4), (8, 14, 192, 16, [64, 64, 64]), (8, 17, 256, 16, [32] * 8),
                 (8, 14, 256, 16, [48, 16] * 4)):
        n_sc, n_sym, B, U, cs = args
        assert cdmimo.selected_form(cdmimo.OP_FRAME, n_sc, n_sym, B, U, cs, 3) != "gram_tc"
    for dt in (cdmimo.C16F, cdmimo.C16BF):
        for op in (cdmimo.OP_FRAME, cdmimo.OP_DETECT, cdmimo.OP_PRECODE):
            assert cdmimo.selected_form(op, 8, 14, 256, 16, [32] * 8, 3, in_dtype=dt) == "gram_tc"


@pytest.mark.parametrize("name", ["cfg2_B256_C8x32_U16", "more_subcarriers_than_ctas", "Bc16_C16_U10_n_sym8",
                                  "Bc16_U9_odd_symbols", "U12_K1_one_symbol", "K5_equal"])
def test_detect_and_precode_tc_match_oracle(dev, name):
    """cdmimo_detect and cdmimo_precode alone on the tensor-core kernel (uplink and downlink modes)."""
    n_sc, n_sym, cs, U, K, fuse, snr, vs_gram = CASES[name]
    snr = wl.sweep_snr(n_sc) if snr == "sweep" else snr
    d = wl.uplink(zlib.crc32(name.encode()) % 1000 + 1, n_sc, n_sym, sum(cs), U, snr_db=snr)
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    S32, S64 = wl.as_c64(d["X"])
    N0 = d["N0"].astype(np.float32)
    Ht, Yt, St, Nt = t(H32, dev), t(Y32, dev), t(S32, dev), t(N0, dev)
    for op in (cdmimo.OP_DETECT, cdmimo.OP_PRECODE):
        assert cdmimo.selected_form(op, n_sc, n_sym, sum(cs), U, cs, K, form="gram_tc", H=Ht) == "gram_tc"
    X = cdmimo.detect(Ht, Yt, Nt, cs, K, fuse=fuse, form="gram_tc").cpu().numpy()
    P = cdmimo.precode(Ht, St, cs, K, form="gram_tc").cpu().numpy()
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, fuse=fuse, threads=8)
    Po = orc.precode(H64, S64, cs, K, threads=8)
    assert_vectors_close(X, Xo, TOL, "tc detect")
    assert_vectors_close(P, Po, TOL, "tc precode")
    if vs_gram:
        Xg = cdmimo.detect(Ht, Yt, Nt, cs, K, fuse=fuse, form="gram").cpu().numpy()
        Pg = cdmimo.precode(Ht, St, cs, K, form="gram").cpu().numpy()
        assert_vectors_close(X, Xg, 2e-5, "tc vs fp32 gram detect")
        assert_vectors_close(P, Pg, 2e-5, "tc vs fp32 gram precode")
    # the frame on the same data gives the same uplink and downlink bits as the two calls
    Xf, Pf = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K, fuse=fuse, form="gram_tc")
    assert_vectors_close(Xf.cpu().numpy(), X, 2e-5, "tc frame vs tc detect")
    assert_vectors_close(Pf.cpu().numpy(), P, 2e-5, "tc frame vs tc precode")
    assert cdmimo.device_status(clear=True) == 0


def test_detect_tc_per_cluster_outputs(dev):
    """Xc_opt / lambda_opt from the tensor-core kernel: the per-cluster estimates and the fusion
    weights agree with the FP32 Gram kernel's (2e-5, 1e-5) and with the oracle's (1e-4)."""
    cs, U, n_sc = [32] * 8, 16, 9
    d = wl.uplink(606, n_sc, 14, 256, U, snr_db=20.0)
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    N0 = d["N0"].astype(np.float32)
    Ht, Yt, Nt = t(H32, dev), t(Y32, dev), t(N0, dev)
    mk = lambda: (torch.empty((n_sc, 8, 14, U), dtype=torch.complex64, device=dev),
                  torch.empty((n_sc, 8), dtype=torch.float32, device=dev))
    Xc_a, lam_a = mk()
    Xc_b, lam_b = mk()
    a = cdmimo.detect(Ht, Yt, Nt, cs, 3, Xc=Xc_a, lam=lam_a, form="gram_tc")
    b = cdmimo.detect(Ht, Yt, Nt, cs, 3, Xc=Xc_b, lam=lam_b, form="gram")
    c = cdmimo.detect(Ht, Yt, Nt, cs, 3, form="gram_tc")
    torch.cuda.synchronize()
    assert torch.equal(a, c)  # the fusion writing the per-cluster outputs computes the same estimate
    assert_vectors_close(a.cpu().numpy(), b.cpu().numpy(), 2e-5, "tc vs gram Xhat")
    assert_vectors_close(Xc_a.cpu().numpy(), Xc_b.cpu().numpy(), 2e-5, "tc vs gram Xc")
    np.testing.assert_allclose(lam_a.cpu().numpy(), lam_b.cpu().numpy(), rtol=1e-5)
    Xo, Xco, lamo = orc.detect(H64, Y64, N0.astype(np.float64), cs, 3, threads=8)
    assert_vectors_close(Xc_a.cpu().numpy(), Xco, TOL, "tc Xc vs oracle")
    np.testing.assert_allclose(lam_a.cpu().numpy(), lamo, rtol=1e-5, atol=1e-7)
    assert cdmimo.device_status(clear=True) == 0


def test_tc_bad_noise_variance_and_K0(dev):
    """A negative N0 sets CDMIMO_DEV_BAD_N0 and gives NaN for that subcarrier's uplink estimate only
    (the downlink does not use N0); K = 0 gives zero outputs in every mode."""
    cs, U, n_sc = [32] * 8, 16, 5
    d = wl.uplink(515, n_sc, 14, 256, U, snr_db=15.0)
    Ht, Yt, St = t(wl.as_c64(d["H"])[0], dev), t(wl.as_c64(d["Y"])[0], dev), t(wl.as_c64(d["X"])[0], dev)
    N0 = d["N0"].astype(np.float32)
    N0[2] = -1.0
    Nt = t(N0, dev)
    cdmimo.device_status(clear=True)
    X = cdmimo.detect(Ht, Yt, Nt, cs, 3, form="gram_tc").cpu().numpy()
    assert cdmimo.device_status(clear=True) & cdmimo.DEV_BAD_N0
    assert np.all(np.isnan(X[2])) and np.all(np.isfinite(X[[0, 1, 3, 4]]))
    Xf, Pf = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, 3, form="gram_tc")
    assert cdmimo.device_status(clear=True) & cdmimo.DEV_BAD_N0
    Xf, Pf = Xf.cpu().numpy(), Pf.cpu().numpy()
    assert np.all(np.isnan(Xf[2])) and np.all(np.isfinite(Xf[[0, 1, 3, 4]])) and np.all(np.isfinite(Pf))
    N0[2] = 0.1
    Nt = t(N0, dev)
    assert not cdmimo.detect(Ht, Yt, Nt, cs, 0, form="gram_tc").abs().any()
    assert not cdmimo.precode(Ht, St, cs, 0, form="gram_tc").abs().any()
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("kind", ["f16", "bf16"])
@pytest.mark.parametrize("n_sc,n_sym,cs,U,K,snr", [(41, 14, [32] * 8, 16, 3, "sweep"), (17, 9, [16] * 6, 12, 2, 20.0)])
def test_tc_16bit_storage(dev, kind, n_sc, n_sym, cs, U, K, snr):
    """fp16 / bf16 channel and receive samples with per-subcarrier scales: each stored value is exact
    in TF32, so z and G_c take one MMA per tile and x_c = H_c w two.  Frame, detection and precoding
    against the FP64 oracle on the dequantized values (1e-4), and against the FP32 Gram kernels on the
    same 16-bit data (2e-5) where B_c >= 2U."""
    snr = wl.sweep_snr(n_sc) if snr == "sweep" else snr
    d = wl.uplink(zlib.crc32(kind.encode()) % 1000 + n_sc, n_sc, n_sym, sum(cs), U, snr_db=snr)
    qH, sH, H64 = wl.quantize_c16(d["H"], kind)
    qY, sY, Y64 = wl.quantize_c16(d["Y"], kind)
    tdt = torch.float16 if kind == "f16" else torch.bfloat16
    Ht = t(qH.view(np.int16), dev).view(tdt)
    Yt = t(qY.view(np.int16), dev).view(tdt)
    S32, S64 = wl.as_c64(d["X"])
    N0 = d["N0"].astype(np.float32)
    sc = dict(h_scale=t(sH, dev), y_scale=t(sY, dev))
    Nt, St = t(N0, dev), t(S32, dev)
    X, P = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K, form="gram_tc", **sc)
    Xd = cdmimo.detect(Ht, Yt, Nt, cs, K, form="gram_tc", **sc)
    Pd = cdmimo.precode(Ht, St, cs, K, form="gram_tc")
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, threads=8)
    Po = orc.precode(H64, S64, cs, K, threads=8)
    for got, ref, what in ((X, Xo, "frame Xhat"), (P, Po, "frame Xdl"), (Xd, Xo, "detect"), (Pd, Po, "precode")):
        assert_vectors_close(got.cpu().numpy(), ref, TOL, f"tc {kind} {what}")
    if min(cs) >= 2 * U:
        Xg, Pg = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K, form="gram", **sc)
        assert_vectors_close(X.cpu().numpy(), Xg.cpu().numpy(), 2e-5, f"tc vs fp32 gram {kind} Xhat")
        assert_vectors_close(P.cpu().numpy(), Pg.cpu().numpy(), 2e-5, f"tc vs fp32 gram {kind} Xdl")
    assert cdmimo.device_status(clear=True) == 0
