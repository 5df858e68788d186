"""GPU parity of the Gram-form CD kernels (cdmimo_form GRAM) and of the form selector.

The Gram form evaluates the iterates of Algorithms 1 and 2 through G_c = H_c^H H_c; it must match
the FP64 oracle (which follows the algorithms step by step in residual form) to the same 1e-4
relative L2 per estimate vector as the residual-form kernels.  Shapes cover every compiled variant
(lanes per tile 1, 2, 4; users padded to 8 or 16), user padding, the converting (non-bulk) staging
path, zero columns, K = 0, 16-bit storage, both subcarrier schedules and the selector's rules.
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
    # name: (n_sc, n_sym, cluster sizes, U, K, fuse, M, snr)
    "cfg2_B256_C8x32_U16": (40, 14, [32] * 8, 16, 3, "colnorm", 16, "sweep"),
    "AT1_Bc16_U8": (23, 14, [16] * 6, 8, 3, "colnorm", 16, 15.0),
    "AT4_Bc64_U16": (11, 14, [64] * 4, 16, 4, "colnorm", 16, 25.0),
    "AT2_U5_padded": (13, 7, [32] * 3, 5, 5, "equal", 4, 10.0),
    "odd_Bc_converting": (9, 6, [31, 27, 29], 12, 3, "colnorm", 16, 20.0),
    "K1_single_sweep": (7, 14, [32] * 4, 16, 1, "colnorm", 16, 30.0),
    "high_snr_K8": (6, 14, [32] * 8, 16, 8, "colnorm", 64, 30.0),
}


def _data(name):
    n_sc, n_sym, cs, U, K, fuse, M, snr = CASES[name]
    snr = wl.sweep_snr(n_sc) if snr == "sweep" else snr
    seed = zlib.crc32(name.encode()) % 1000
    return (wl.uplink(seed, n_sc, n_sym, sum(cs), U, snr_db=snr, M=M),
            wl.downlink(seed + 1, n_sc, n_sym, sum(cs), U, M=M), cs, U, K, fuse, M)


@pytest.mark.parametrize("name", list(CASES))
def test_gram_detect_parity(dev, name):
    d, _, cs, U, K, fuse, M = _data(name)
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    N0 = d["N0"].astype(np.float32)
    n_sc, n_sym, C = H32.shape[0], Y32.shape[1], len(cs)
    Xc = torch.zeros((n_sc, C, n_sym, U), dtype=torch.complex64, device=dev)
    lam = torch.zeros((n_sc, C), dtype=torch.float32, device=dev)
    X = cdmimo.detect(t(H32, dev), t(Y32, dev), t(N0, dev), cs, K, fuse=fuse, Xc=Xc, lam=lam, form="gram")
    Xo, Xco, lamo = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, fuse=fuse, threads=8)
    assert_vectors_close(X.cpu().numpy(), Xo, TOL, "Xhat")
    assert_vectors_close(Xc.cpu().numpy(), Xco, TOL, "Xc")
    np.testing.assert_allclose(lam.cpu().numpy(), lamo, rtol=1e-5, atol=1e-7)
    assert_decisions_match(X.cpu().numpy(), Xo, M)
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("name", list(CASES))
def test_gram_precode_parity(dev, name):
    _, dl, cs, U, K, _, _ = _data(name)
    H32, H64 = wl.as_c64(dl["H"])
    S32, S64 = wl.as_c64(dl["S"])
    X = cdmimo.precode(t(H32, dev), t(S32, dev), cs, K, form="gram")
    Xo = orc.precode(H64, S64, cs, K, threads=8)
    assert_vectors_close(X.cpu().numpy(), Xo, TOL, "Xdl")
    assert cdmimo.device_status(clear=True) == 0


def test_gram_zero_columns_and_K0(dev):
    # user 2 has a zero channel in cluster 1 and N0 = 0 on the first subcarrier: m = 0 / p = 0 there
    cs, U = [32] * 4, 8
    d = wl.uplink(5, 4, 6, 128, U, snr_db=20.0)
    H = d["H"].copy()
    H[:, 2, 32:64] = 0
    N0 = d["N0"].astype(np.float32).copy()
    N0[0] = 0.0
    H32, H64 = wl.as_c64(H)
    Y32, Y64 = wl.as_c64(d["Y"])
    for K in (0, 3):
        X = cdmimo.detect(t(H32, dev), t(Y32, dev), t(N0, dev), cs, K, form="gram").cpu().numpy()
        Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, threads=4)
        if K == 0:
            assert np.all(X == 0)
        else:
            assert_vectors_close(X, Xo, TOL, "detect, zero column")
        S32, S64 = wl.as_c64(d["X"])
        P = cdmimo.precode(t(H32, dev), t(S32, dev), cs, K, form="gram").cpu().numpy()
        Po = orc.precode(H64, S64, cs, K, threads=4)
        if K == 0:
            assert np.all(P == 0)
        else:
            assert_vectors_close(P, Po, TOL, "precode, zero column")
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_gram_low_precision_storage(dev, kind):
    cs, U, K = [32] * 8, 16, 3
    d = wl.uplink(71, 20, 14, 256, U, snr_db=wl.sweep_snr(20))
    qH, sH, H64 = wl.quantize_c16(d["H"], kind)
    qY, sY, Y64 = wl.quantize_c16(d["Y"], kind)
    tdt = torch.float16 if kind == "f16" else torch.bfloat16
    Ht = t(qH.view(np.int16), dev).view(tdt)
    Yt = t(qY.view(np.int16), dev).view(tdt)
    N0 = d["N0"].astype(np.float32)
    X = cdmimo.detect(Ht, Yt, t(N0, dev), cs, K, h_scale=t(sH, dev), y_scale=t(sY, dev), form="gram")
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, threads=8)
    assert_vectors_close(X.cpu().numpy(), Xo, TOL, f"detect {kind}")
    S32, S64 = wl.as_c64(d["X"])
    P = cdmimo.precode(Ht, t(S32, dev), cs, K, form="gram")
    Po = orc.precode(H64, S64, cs, K, threads=8)
    assert_vectors_close(P.cpu().numpy(), Po, TOL, f"precode {kind}")
    assert cdmimo.device_status(clear=True) == 0


def test_gram_full_size_schedules_and_auto(dev):
    """The 1200-subcarrier workload in the persistent launch: dynamic and static schedules agree bit
    for bit, AUTO selects the Gram form on the tensor cores here (within 2e-5 of form="gram", the
    same iterates with other rounding), and sampled subcarriers (first, counter-handed, last) match
    the oracle."""
    cs, U, K, n_sc = [32] * 8, 16, 3, 1200
    d = wl.uplink(20190222, n_sc, 14, 256, U, snr_db=wl.sweep_snr(n_sc))
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    N0 = d["N0"].astype(np.float32)
    Ht, Yt, Nt = t(H32, dev), t(Y32, dev), t(N0, dev)
    a = cdmimo.detect(Ht, Yt, Nt, cs, K, form="gram", workspace=True)
    b = cdmimo.detect(Ht, Yt, Nt, cs, K, form="gram", workspace=False)
    c = cdmimo.detect(Ht, Yt, Nt, cs, K)
    S32, S64 = wl.as_c64(d["X"])
    St = t(S32, dev)
    pa = cdmimo.precode(Ht, St, cs, K, form="gram", workspace=True)
    pb = cdmimo.precode(Ht, St, cs, K, form="gram", workspace=False)
    pc = cdmimo.precode(Ht, St, cs, K)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(pa, pb)
    assert_vectors_close(c.cpu().numpy(), a.cpu().numpy(), 2e-5, "auto (tensor cores) vs gram detect")
    assert_vectors_close(pc.cpu().numpy(), pa.cpu().numpy(), 2e-5, "auto (tensor cores) vs gram precode")
    idx = np.r_[0:3, 700:704, n_sc - 3:n_sc]
    Xo, _, _ = orc.detect(H64[idx], Y64[idx], N0.astype(np.float64)[idx], cs, K, threads=8)
    assert_vectors_close(a.cpu().numpy()[idx], Xo, TOL, "full-size detect")
    Po = orc.precode(H64[idx], S64[idx], cs, K, threads=8)
    assert_vectors_close(pa.cpu().numpy()[idx], Po, TOL, "full-size precode")
    # the residual form on the same inputs: a different rounding order of the same iterates
    r = cdmimo.detect(Ht, Yt, Nt, cs, K, form="residual")
    assert_vectors_close(r.cpu().numpy()[idx], Xo, TOL, "residual form")
    assert cdmimo.device_status(clear=True) == 0


def test_selector_rules(dev):
    z = lambda *s: torch.zeros(s, dtype=torch.complex64, device=dev)
    N0 = torch.ones(2, dtype=torch.float32, device=dev)
    # more than 16 users: no Gram kernel
    with pytest.raises(cdmimo.CdmimoError) as e:
        cdmimo.detect(z(2, 20, 64), z(2, 3, 64), N0, [32, 32], 2, form="gram")
    assert e.value.status == cdmimo.ERR_UNSUPPORTED
    # ... AUTO falls back to the residual form there
    cdmimo.detect(z(2, 20, 64), z(2, 3, 64), N0, [32, 32], 2)
    # unequal lanes per tile: no Gram kernel
    with pytest.raises(cdmimo.CdmimoError) as e:
        cdmimo.precode(z(2, 4, 80), z(2, 3, 4), [16, 64], 2, form="gram")
    assert e.value.status == cdmimo.ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert cdmimo.device_status(clear=True) == 0


def test_selected_form_query(dev):
    H = torch.zeros((4, 16, 256), dtype=torch.complex64, device=dev)
    q = lambda op, **kw: cdmimo.selected_form(op, 4, 14, 256, 16, [32] * 8, 3, H=H, **kw)
    assert q(cdmimo.OP_DETECT) == "gram_tc" and q(cdmimo.OP_PRECODE) == "gram_tc"
    assert q(cdmimo.OP_DETECT, form="gram") == "gram" and q(cdmimo.OP_PRECODE, form="gram") == "gram"
    assert q(cdmimo.OP_DETECT, form="residual") == "residual"
    # one OFDM symbol per subcarrier: the Gram matrix does not pay for itself
    assert cdmimo.selected_form(cdmimo.OP_DETECT, 4, 1, 256, 16, [32] * 8, 3, H=H) == "residual"
    # square clusters (B_c < 2U): AUTO keeps the residual form
    Hs = torch.zeros((4, 16, 128), dtype=torch.complex64, device=dev)
    assert cdmimo.selected_form(cdmimo.OP_DETECT, 4, 14, 128, 16, [16] * 8, 3, H=Hs) == "residual"
