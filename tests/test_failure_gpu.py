"""The kernels' bounded waits on the GPU: a wait that nothing completes gives up after its limit,
reports CDMIMO_DEV_TIMEOUT through the device status word, and leaves the context usable (no trap,
no fault: the next call runs and matches the oracle)."""
import time

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo
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


def test_bounded_wait_expires_and_context_stays_usable(dev):
    cdmimo.device_status(clear=True)
    t0 = time.perf_counter()
    cdmimo.check_bounded_wait(20000)  # 20 ms
    st = cdmimo.device_status(clear=True)  # synchronizes
    dt = time.perf_counter() - t0
    assert st & cdmimo.DEV_TIMEOUT
    assert 0.019 <= dt < 2.0
    d = wl.uplink(88, 7, 14, 256, 16, snr_db=15.0)
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    N0 = d["N0"].astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    X = cdmimo.detect(t(H32), t(Y32), t(N0), [32] * 8, 3).cpu().numpy()
    Xo, _, _ = orc.detect(H64, Y64, N0.astype(np.float64), [32] * 8, 3, threads=4)
    assert_vectors_close(X, Xo, 1e-4, "detect after an expired wait")
    assert cdmimo.device_status(clear=True) == 0
