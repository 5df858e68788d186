"""GPU parity on every vector of the benchmark's batch, in the launch configuration the benchmark
times: 1200 subcarriers x 14 OFDM symbols, B = 256 antennas in C = 8 clusters of 32, U = 16 users,
K = 3 sweeps, 16-QAM, SNR swept 0..30 dB across subcarriers (the same seeded inputs as bench.py).

The oracle recomputes the whole batch (it takes well under a second on the host's cores), so every
persistent-loop iteration, both channel buffers and the last, ragged share of subcarriers are
compared, not a sample.  Acceptance as everywhere: relative L2 error <= 1e-4 per estimate vector
(U-vector uplink, B-vector downlink), hard decisions equal except within 1e-3 of a threshold.
16-bit storage is compared with the oracle run on the exact dequantized values.
"""
import os

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo, learned
from paper_1902_08653_gb300 import workload as wl

from _util import assert_decisions_match, assert_vectors_close

pytestmark = pytest.mark.gpu
TOL = 1e-4
N_SC, N_SYM, B, U, K, M = 1200, 14, 256, 16, 3, 16
CS = [32] * 8
THREADS = os.cpu_count() or 8
KINDS = {"c64": None, "f16": torch.float16, "bf16": torch.bfloat16}
CODES = {"c64": cdmimo.C64, "f16": cdmimo.C16F, "bf16": cdmimo.C16BF}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    orc.build()
    cdmimo.lib()
    cdmimo.device_status(clear=True)
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def batch(dev):
    """Device inputs per storage kind and the oracle's outputs on the values each kind delivers."""
    up = wl.uplink(wl.DEFAULT_SEED, N_SC, N_SYM, B, U, snr_db=wl.sweep_snr(N_SC), M=M)
    dl = wl.downlink(wl.DEFAULT_SEED, N_SC, N_SYM, B, U, M=M)
    S32, S64 = wl.as_c64(dl["S"])
    N0 = up["N0"].astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out = {"N0": t(N0), "S": t(S32)}
    for kind, tdt in KINDS.items():
        if tdt is None:
            H32, H64 = wl.as_c64(up["H"])
            Y32, Y64 = wl.as_c64(up["Y"])
            dev_in = dict(H=t(H32), Y=t(Y32), sc={})
        else:
            qH, sH, H64 = wl.quantize_c16(up["H"], kind)
            qY, sY, Y64 = wl.quantize_c16(up["Y"], kind)
            dev_in = dict(H=t(qH.view(np.int16)).view(tdt), Y=t(qY.view(np.int16)).view(tdt),
                          sc=dict(h_scale=t(sH), y_scale=t(sY)))
        Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), CS, K, threads=THREADS)
        Po = orc.precode(H64, S64, CS, K, threads=THREADS)
        out[kind] = dict(dev_in, Xo=Xo, Po=Po, H64=H64, Y64=Y64)
    return out


@pytest.mark.parametrize("kind", list(KINDS))
def test_bench_frame_every_vector(dev, batch, kind):
    """cdmimo_detect_precode under the default (AUTO) form, as bench.py calls it: the tensor-core
    frame kernel, one persistent launch over all subcarriers."""
    b = batch[kind]
    assert cdmimo.selected_form(cdmimo.OP_FRAME, N_SC, N_SYM, B, U, CS, K, in_dtype=CODES[kind], H=b["H"]) == "gram_tc"
    X, P = cdmimo.detect_precode(b["H"], b["Y"], batch["N0"], batch["S"], CS, K, **b["sc"])
    torch.cuda.synchronize()
    X, P = X.cpu().numpy(), P.cpu().numpy()
    assert_vectors_close(X, b["Xo"], TOL, f"frame Xhat {kind}")
    assert_vectors_close(P, b["Po"], TOL, f"frame Xdl {kind}")
    assert_decisions_match(X, b["Xo"], M)
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("form", ["auto", "gram", "residual"])
@pytest.mark.parametrize("kind", list(KINDS))
def test_detect_and_precode_every_vector(dev, batch, kind, form):
    """cdmimo_detect and cdmimo_precode on the whole batch, in each evaluation form."""
    b = batch[kind]
    X = cdmimo.detect(b["H"], b["Y"], batch["N0"], CS, K, form=form, **b["sc"])
    P = cdmimo.precode(b["H"], batch["S"], CS, K, form=form)
    torch.cuda.synchronize()
    X, P = X.cpu().numpy(), P.cpu().numpy()
    assert_vectors_close(X, b["Xo"], TOL, f"detect {kind} {form}")
    assert_vectors_close(P, b["Po"], TOL, f"precode {kind} {form}")
    assert_decisions_match(X, b["Xo"], M)
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("form", ["auto", "residual"])
def test_learned_detect_every_vector(dev, batch, form):
    """The learned K = 2 detector (random parameters away from plain CD, learned fusion) on the whole
    batch, against the oracle's learned forward with the parameter values the kernels use."""
    Kl, Hd = 2, 64
    g = np.random.default_rng(17)
    sl = learned.layout(Kl, U, Hd)
    m = np.zeros(cdmimo.learned_param_count(Kl, U, Hd), np.float32)
    m[sl["tau"]] = g.uniform(0.8, 1.3, Kl)
    m[sl["graw"]] = g.uniform(-0.3, 1.0, Kl)
    m[sl["W1"]] = g.standard_normal(Hd * (U + 1)) * 0.3
    m[sl["b1"]] = g.standard_normal(Hd) * 0.3
    m[sl["w2"]] = g.standard_normal(Hd) * 0.3
    m[sl["b2"]] = 0.1
    model = learned.LearnedCD(Kl, U, Hd, master=torch.from_numpy(m), device=dev)
    used = m.astype(np.float64)
    for k in ("W1", "w2"):  # the kernels read W1 and w2 as bfloat16
        used[sl[k]] = wl.bf16_bits_to_f32(wl.f32_to_bf16_bits(m[sl[k]])).astype(np.float64)
    c = batch["c64"]
    X = model.detect(c["H"], c["Y"], batch["N0"], CS, form=form).cpu().numpy()
    Xo, _, _ = orc.learned_forward(c["H64"], c["Y64"], batch["N0"].cpu().numpy().astype(np.float64), CS, Kl, used,
                                   Hd, threads=THREADS)
    assert_vectors_close(X, Xo, TOL, f"learned {form}")
    assert cdmimo.device_status(clear=True) == 0
