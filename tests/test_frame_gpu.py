"""GPU parity of the TDD frame entry point (cdmimo_detect_precode): uplink detection and downlink
precoding on one channel in one kernel (Gram form), or as two calls where that kernel does not
apply.

The fused kernel evaluates the operations of the separate Gram-form kernels with each loaded value
feeding two vectors (a different summation order), so its outputs agree with theirs to FP32
rounding (2e-5 relative L2 per vector); both are compared with the FP64 oracle (1e-4).
"""
import os
import zlib

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo
from paper_1902_08653_gb300 import workload as wl

from _util import assert_vectors_close

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
    # name: (n_sc, n_sym, cluster sizes, U, K, fuse, snr)
    "cfg2_B256_C8x32_U16": (50, 14, [32] * 8, 16, 3, "colnorm", "sweep"),
    "AT1_Bc16_U8": (17, 14, [16] * 6, 8, 3, "colnorm", 15.0),
    "AT4_Bc64_U16": (9, 14, [64] * 4, 16, 2, "colnorm", 25.0),
    "AT2_U5_padded_equal": (11, 7, [32] * 3, 5, 5, "equal", 10.0),
    "odd_Bc_converting": (7, 6, [31, 27, 29], 12, 3, "colnorm", 20.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_frame_matches_separate_calls_and_oracle(dev, name):
    n_sc, n_sym, cs, U, K, fuse, snr = CASES[name]
    snr = wl.sweep_snr(n_sc) if snr == "sweep" else snr
    d = wl.uplink(zlib.crc32(name.encode()) % 1000, n_sc, n_sym, sum(cs), U, snr_db=snr)
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    S32, S64 = wl.as_c64(d["X"])  # downlink symbols: any U-vectors per (subcarrier, symbol)
    N0 = d["N0"].astype(np.float32)
    Ht, Yt, St, Nt = t(H32, dev), t(Y32, dev), t(S32, dev), t(N0, dev)
    X, P = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K, fuse=fuse, form="gram")
    Xs = cdmimo.detect(Ht, Yt, Nt, cs, K, fuse=fuse, form="gram")
    Ps = cdmimo.precode(Ht, St, cs, K, form="gram")
    torch.cuda.synchronize()
    assert_vectors_close(X.cpu().numpy(), Xs.cpu().numpy(), 2e-5, "frame vs separate Xhat")
    assert_vectors_close(P.cpu().numpy(), Ps.cpu().numpy(), 2e-5, "frame vs separate Xdl")
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, fuse=fuse, threads=8)
    Po = orc.precode(H64, S64, cs, K, threads=8)
    assert_vectors_close(X.cpu().numpy(), Xo, TOL, "frame Xhat")
    assert_vectors_close(P.cpu().numpy(), Po, TOL, "frame Xdl")
    assert cdmimo.device_status(clear=True) == 0


def test_frame_full_size_schedules_and_residual_fallback(dev):
    cs, U, K, n_sc = [32] * 8, 16, 3, 1200
    d = wl.uplink(20190222, n_sc, 14, 256, U, snr_db=wl.sweep_snr(n_sc))
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    S32, S64 = wl.as_c64(d["X"])
    N0 = d["N0"].astype(np.float32)
    Ht, Yt, St, Nt = t(H32, dev), t(Y32, dev), t(S32, dev), t(N0, dev)
    a = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K)
    b = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K, workspace=True)
    c = cdmimo.detect_precode(Ht, Yt, Nt, St, cs, K, form="residual")
    r = (cdmimo.detect(Ht, Yt, Nt, cs, K, form="residual"), cdmimo.precode(Ht, St, cs, K, form="residual"))
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(c[0], r[0]) and torch.equal(c[1], r[1])
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, threads=os.cpu_count() or 8)
    Po = orc.precode(H64, S64, cs, K, threads=os.cpu_count() or 8)
    for X, P, what in ((a[0], a[1], "frame"), (c[0], c[1], "residual calls")):
        assert_vectors_close(X.cpu().numpy(), Xo, TOL, what + " Xhat")
        assert_vectors_close(P.cpu().numpy(), Po, TOL, what + " Xdl")
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_frame_low_precision_storage(dev, kind):
    cs, U, K = [32] * 8, 16, 3
    d = wl.uplink(91, 16, 14, 256, U, snr_db=wl.sweep_snr(16))
    qH, sH, H64 = wl.quantize_c16(d["H"], kind)
    qY, sY, Y64 = wl.quantize_c16(d["Y"], kind)
    tdt = torch.float16 if kind == "f16" else torch.bfloat16
    Ht = t(qH.view(np.int16), dev).view(tdt)
    Yt = t(qY.view(np.int16), dev).view(tdt)
    S32, S64 = wl.as_c64(d["X"])
    N0 = d["N0"].astype(np.float32)
    X, P = cdmimo.detect_precode(Ht, Yt, t(N0, dev), t(S32, dev), cs, K, h_scale=t(sH, dev), y_scale=t(sY, dev))
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, threads=8)
    Po = orc.precode(H64, S64, cs, K, threads=8)
    assert_vectors_close(X.cpu().numpy(), Xo, TOL, f"frame Xhat {kind}")
    assert_vectors_close(P.cpu().numpy(), Po, TOL, f"frame Xdl {kind}")
    assert cdmimo.device_status(clear=True) == 0


def test_frame_edge_cases(dev):
    cs, U = [32] * 4, 8
    z = lambda *s: torch.zeros(s, dtype=torch.complex64, device=dev)
    # empty batch: a no-op that returns the (empty) outputs
    X, P = cdmimo.detect_precode(z(0, U, 128), z(0, 3, 128), torch.zeros(0, device=dev), z(0, 3, U), cs, 3)
    assert X.shape == (0, 3, U) and P.shape == (0, 3, 128)
    d = wl.uplink(12, 5, 1, 128, U, snr_db=15.0)  # one symbol per subcarrier, fewer subcarriers than CTAs
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    S32, S64 = wl.as_c64(d["X"])
    N0 = d["N0"].astype(np.float32)
    for K, form in ((0, "gram"), (2, "gram"), (2, "auto")):
        X, P = cdmimo.detect_precode(t(H32, dev), t(Y32, dev), t(N0, dev), t(S32, dev), cs, K, form=form)
        if K == 0:
            assert not X.abs().any() and not P.abs().any()
            continue
        Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), cs, K, threads=4)
        Po = orc.precode(H64, S64, cs, K, threads=4)
        assert_vectors_close(X.cpu().numpy(), Xo, TOL, f"frame Xhat {form}")
        assert_vectors_close(P.cpu().numpy(), Po, TOL, f"frame Xdl {form}")
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("case,n_chunks,side", [("c64", 0, False), ("c64", 1, False), ("c64", 3, True),
                                                ("c64", 7, False), ("c64", 5000, False), ("bf16", 4, False),
                                                ("residual", 5, True)])
def test_frame_host_pipeline_matches_device_call(dev, case, n_chunks, side):
    """cdmimo_detect_precode_host (host buffers, chunked; uploads, kernels and downloads on three
    streams) returns exactly what cdmimo_detect_precode returns on the same data in device memory,
    on the current stream or on a caller's side stream."""
    cs, U, K, n_sc, n_sym = ([16] * 8, 16, 2, 61, 9) if case == "residual" else ([32] * 8, 16, 3, 203, 14)
    B = sum(cs)
    d = wl.uplink(33, n_sc, n_sym, B, U, snr_db=wl.sweep_snr(n_sc))
    S32, _ = wl.as_c64(d["X"])
    N0 = d["N0"].astype(np.float32)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    if case == "bf16":
        qH, sH, _ = wl.quantize_c16(d["H"], "bf16")
        qY, sY, _ = wl.quantize_c16(d["Y"], "bf16")
        Hh = pin(qH.view(np.int16)).view(torch.bfloat16)
        Yh = pin(qY.view(np.int16)).view(torch.bfloat16)
        sc_dev = dict(h_scale=t(sH, dev), y_scale=t(sY, dev))
        sc_host = dict(h_scale=pin(sH), y_scale=pin(sY))
    else:
        Hh, Yh = pin(wl.as_c64(d["H"])[0]), pin(wl.as_c64(d["Y"])[0])
        sc_dev, sc_host = {}, {}
    Xd, Pd = cdmimo.detect_precode(Hh.to(dev), Yh.to(dev), t(N0, dev), t(S32, dev), cs, K, **sc_dev)
    if case == "residual":
        assert cdmimo.selected_form(cdmimo.OP_DETECT, n_sc, n_sym, B, U, cs, K, H=Hh.to(dev)) == "residual"
    Xh = torch.full((n_sc, n_sym, U), float("nan"), dtype=torch.complex64).pin_memory()
    Ph = torch.full((n_sc, n_sym, B), float("nan"), dtype=torch.complex64).pin_memory()
    dt = cdmimo.C16BF if case == "bf16" else cdmimo.C64
    nb = cdmimo.host_workspace_size(cdmimo.OP_FRAME, n_sc, n_sym, B, U, cs, K, in_dtype=dt)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream() if side else torch.cuda.current_stream()
    st.wait_stream(torch.cuda.current_stream())
    for _ in range(2):  # the second call reuses the staging, the thread's streams and events
        cdmimo.detect_precode_host(Hh, Yh, pin(N0), pin(S32), cs, K, Xh, Ph, ws, n_chunks=n_chunks, stream=st,
                                   **sc_host)
    st.synchronize()
    assert torch.equal(Xh, Xd.cpu()) and torch.equal(Ph, Pd.cpu())
    assert cdmimo.device_status(clear=True) == 0
