"""The device input generator (cdmimo_synth_uplink) against its host twin (workload.philox_uplink):
labels bit-exact, channel / noise / receive vectors to FP32 rounding of the Box-Muller transform."""
import numpy as np
import pytest
import torch

from paper_1902_08653_gb300 import cdmimo
from paper_1902_08653_gb300 import workload as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,U,B,n_sym", [(16, 8, 64, 3), (4, 16, 256, 1), (64, 5, 48, 2)])
def test_device_generator_matches_host_twin(M, U, B, n_sym):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n_sc = 9
    snr = wl.sweep_snr(n_sc)
    seed = 0x1234_5678_9ABC
    d = cdmimo.synth_uplink(seed, n_sc, n_sym, B, U, torch.from_numpy(snr.astype(np.float32)).cuda(), M=M,
                            labels=True)
    ref = wl.philox_uplink(seed, n_sc, n_sym, B, U, snr, M=M)
    np.testing.assert_array_equal(d["labels"].cpu().numpy(), ref["labels"])
    np.testing.assert_allclose(d["X"].cpu().numpy(), ref["X"], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(d["N0"].cpu().numpy(), ref["N0"], rtol=1e-5)
    np.testing.assert_allclose(d["H"].cpu().numpy(), ref["H"], rtol=2e-5, atol=2e-6)
    err = np.abs(d["Y"].cpu().numpy() - ref["Y"]) / np.sqrt(U + ref["N0"][:, None, None])
    assert err.max() < 1e-5
