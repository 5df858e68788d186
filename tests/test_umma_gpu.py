"""GPU checks of the tcgen05 conventions that form GRAM_TC_UMMA builds on (umma.cuh): the K-major
operand layout without swizzle, the instruction descriptor of kind::tf32, the commit / wait and the
tensor-memory read-back.  Small integer operands make every product and sum exact in FP32, so the
accumulator must equal A B^T bit for bit; for an M = 64 accumulator, row 16 q + i must sit in lane
32 q + i (i < 16), the mapping the kernel's epilogue reads."""
import numpy as np
import pytest
import torch

from paper_1902_08653_gb300 import cdmimo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cdmimo.lib()
    return torch.device("cuda:0")


def operands(M, seed):
    g = np.random.default_rng(seed)
    A = g.integers(-8, 9, size=(M, 32)).astype(np.float32)
    B = g.integers(-8, 9, size=(32, 32)).astype(np.float32)
    return A, B


def test_m128_accumulator_is_the_product(dev):
    A, B = operands(128, 1)
    D = cdmimo.umma_layout_probe(128, torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)).cpu().numpy()
    np.testing.assert_array_equal(D, A @ B.T)


def test_m64_rows_sit_in_the_lower_half_of_each_lane_quarter(dev):
    A, B = operands(64, 2)
    D = cdmimo.umma_layout_probe(64, torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)).cpu().numpy()
    ref = A @ B.T
    for q in range(4):
        np.testing.assert_array_equal(D[32 * q:32 * q + 16], ref[16 * q:16 * q + 16])


def test_rate_probe_reports_cycles(dev):
    c = {(M, N): cdmimo.umma_rate_probe(M, N, 64) for M, N in ((64, 32), (128, 64), (128, 256))}
    assert all(v > 0 for v in c.values()), c
    assert c[(128, 256)] >= c[(128, 64)]
    assert cdmimo.device_status(clear=True) == 0
