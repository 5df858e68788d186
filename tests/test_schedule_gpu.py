"""Dynamic subcarrier schedule of the persistent kernels (counters in the caller's workspace).

The output must not depend on the schedule: dynamic and static launches agree bit for bit, the
subcarriers handed out by the counter (index >= 2 x grid) match the FP64 oracle, the counters are
zero again after every call, and counters that were not zero at the start raise
CDMIMO_DEV_BAD_SCHED (and are zeroed, so the next call is complete).
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo
from paper_1902_08653_gb300 import workload as wl

from _util import assert_vectors_close

pytestmark = pytest.mark.gpu

DEV_BAD_SCHED = 0x8
N_SC, N_SYM, B, U, CS, K = 1500, 14, 256, 16, [32] * 8, 3


@pytest.fixture(scope="module")
def data():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    orc.build()
    cdmimo.device_status(clear=True)
    dev = torch.device("cuda:0")
    up = wl.uplink(77, N_SC, N_SYM, B, U, snr_db=wl.sweep_snr(N_SC))
    dl = wl.downlink(78, N_SC, N_SYM, B, U)
    t = lambda a: torch.from_numpy(wl.as_c64(a)[0]).to(dev)
    return dict(dev=dev, up=up, dl=dl, H=t(up["H"]), Y=t(up["Y"]), Hd=t(dl["H"]), S=t(dl["S"]),
                N0=torch.from_numpy(up["N0"].astype(np.float32)).to(dev))


def test_dynamic_equals_static_and_counters_reset(data):
    d = data
    ws = torch.zeros(256, dtype=torch.uint8, device=d["dev"])
    for _ in range(3):  # repeated calls on one workspace: each leaves the counters zero
        Xd = cdmimo.detect(d["H"], d["Y"], d["N0"], CS, K, workspace=ws)
        Pd = cdmimo.precode(d["Hd"], d["S"], CS, K, workspace=ws)
        torch.cuda.synchronize()
        assert int(ws.count_nonzero()) == 0
    Xs = cdmimo.detect(d["H"], d["Y"], d["N0"], CS, K, workspace=False)
    Ps = cdmimo.precode(d["Hd"], d["S"], CS, K, workspace=False)
    torch.cuda.synchronize()
    assert torch.equal(Xd, Xs)
    assert torch.equal(Pd, Ps)
    assert cdmimo.device_status(clear=True) == 0
    # the binding's own per-stream counters (workspace=True) and its default (static)
    assert torch.equal(cdmimo.detect(d["H"], d["Y"], d["N0"], CS, K, workspace=True), Xs)
    assert torch.equal(cdmimo.detect(d["H"], d["Y"], d["N0"], CS, K), Xs)


def test_counter_handed_subcarriers_match_oracle(data):
    d = data
    X = cdmimo.detect(d["H"], d["Y"], d["N0"], CS, K, workspace=True).cpu().numpy()
    P = cdmimo.precode(d["Hd"], d["S"], CS, K, workspace=True).cpu().numpy()
    # indices past 2 x (152 SMs x 2 CTAs) come from the counter; the last ones are taken last
    idx = np.r_[0:4, 608:616, N_SC - 8:N_SC]
    H64, Y64 = wl.as_c64(d["up"]["H"])[1][idx], wl.as_c64(d["up"]["Y"])[1][idx]
    N0 = d["up"]["N0"].astype(np.float32).astype(np.float64)[idx]
    Xo, _, _ = orc.detect(H64, Y64, N0, CS, K, threads=8)
    assert_vectors_close(X[idx], Xo, 1e-4, "dynamic detect")
    Hd64, S64 = wl.as_c64(d["dl"]["H"])[1][idx], wl.as_c64(d["dl"]["S"])[1][idx]
    Po = orc.precode(Hd64, S64, CS, K, threads=8)
    assert_vectors_close(P[idx], Po, 1e-4, "dynamic precode")


def test_low_precision_storage_dynamic_equals_static(data):
    d = data
    for kind, tdt in (("f16", torch.float16), ("bf16", torch.bfloat16)):
        qH, sH, _ = wl.quantize_c16(d["up"]["H"], kind)
        qY, sY, _ = wl.quantize_c16(d["up"]["Y"], kind)
        Ht = torch.from_numpy(qH.view(np.int16)).to(d["dev"]).view(tdt)
        Yt = torch.from_numpy(qY.view(np.int16)).to(d["dev"]).view(tdt)
        sHt, sYt = torch.from_numpy(sH).to(d["dev"]), torch.from_numpy(sY).to(d["dev"])
        a = cdmimo.detect(Ht, Yt, d["N0"], CS, K, h_scale=sHt, y_scale=sYt, workspace=True)
        b = cdmimo.detect(Ht, Yt, d["N0"], CS, K, h_scale=sHt, y_scale=sYt, workspace=False)
        pa = cdmimo.precode(Ht, d["S"], CS, K, workspace=True)
        pb = cdmimo.precode(Ht, d["S"], CS, K, workspace=False)
        torch.cuda.synchronize()
        assert torch.equal(a, b), kind
        assert torch.equal(pa, pb), kind


def test_nonzero_counters_are_reported_and_cleared(data):
    d = data
    ref = cdmimo.detect(d["H"], d["Y"], d["N0"], CS, K, workspace=False)
    ws = torch.zeros(256, dtype=torch.uint8, device=d["dev"])
    ws.view(torch.int32)[0] = 5  # a stale ticket counter: five counter-handed subcarriers are skipped
    cdmimo.device_status(clear=True)
    out = torch.zeros_like(ref)
    cdmimo.detect(d["H"], d["Y"], d["N0"], CS, K, workspace=ws, out=out)
    torch.cuda.synchronize()
    assert cdmimo.device_status(clear=True) & DEV_BAD_SCHED
    assert int(ws.count_nonzero()) == 0
    assert not torch.equal(out, ref)
    out.zero_()
    cdmimo.detect(d["H"], d["Y"], d["N0"], CS, K, workspace=ws, out=out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert cdmimo.device_status(clear=True) == 0
