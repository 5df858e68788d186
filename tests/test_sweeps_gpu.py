"""BER / MSE sweeps (paper_1902_08653_gb300.sweeps): properties the method must show on seeded
channels: decentralized CD beats the matched filter where interference dominates, more sweeps do
not hurt, centralized CD approaches the L-MMSE solution, and ZF precoding beats MF precoding."""
import numpy as np
import pytest
import torch

from paper_1902_08653_gb300 import sweeps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ul():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return sweeps.uplink_sweep(snrs=(0, 10, 20), U=8, Bc=32, C=4, K_list=(1, 5, 20), n_sc=96, n_sym=14)


def test_uplink_sweep_properties(ul):
    ber, mse = ul["ber"], ul["mse_vs_lmmse"]
    assert mse["lmmse_centralized"] == [0.0, 0.0, 0.0]
    # BER falls with SNR for the optimum linear detector and for decentralized CD
    assert ber["lmmse_centralized"][0] > ber["lmmse_centralized"][2]
    assert ber["cd_decentralized_K5"][0] > ber["cd_decentralized_K5"][2]
    # at 20 dB the matched filter is interference-limited; CD is not
    assert ber["mf"][2] > 2 * ber["cd_decentralized_K5"][2] + 1e-4
    # more sweeps move decentralized and centralized CD toward the L-MMSE estimate
    assert mse["cd_decentralized_K5"][2] < mse["cd_decentralized_K1"][2]
    assert mse["cd_centralized_K20"][2] < 1e-3 * mse["cd_centralized_K1"][2]
    assert mse["cd_centralized_K20"][2] <= mse["cd_decentralized_K20"][2]


def test_downlink_sweep_properties():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dl = sweeps.downlink_sweep(snrs=(0, 20), U=8, Bc=32, C=4, K_list=(1, 5), n_sc=96, n_sym=14)
    ber = dl["ber"]
    assert ber["zf_centralized"][1] < ber["mf"][1]
    assert ber["cd_decentralized_K5"][1] <= ber["cd_decentralized_K1"][1] + 1e-4
    assert all(np.isfinite(v).all() for v in map(np.asarray, ber.values()))
