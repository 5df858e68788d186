"""The allocation-free gradient entry point, cdmimo_learned_grad_noalloc.

Some callers cannot allocate device memory where they train (a baseband pipeline that forbids
allocation once it runs, or C code that only receives device pointers from another runtime).  For
them the library keeps the gradient's scratch in a fixed device array.  This test calls that entry
point through the C ABI twice in a row and checks each result against the regular entry point,
cdmimo_learned_grad with a caller-owned workspace: both run the same kernels with the same fixed
reduction order, so the gradients and losses must agree bit for bit.  It lives in a file that
pytest collects last and also passes when run alone.
"""
import numpy as np
import pytest
import torch

from paper_1902_08653_gb300 import cdmimo, learned
from paper_1902_08653_gb300 import workload as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cdmimo.lib()
    return torch.device("cuda:0")


def _case(seed, n_sc, n_sym, cs, U, dev):
    d = wl.uplink(seed, n_sc, n_sym, sum(cs), U, snr_db=wl.sweep_snr(n_sc), M=16)
    g = np.random.default_rng(seed)
    Xt = d["X"] + 0.1 * (g.standard_normal(d["X"].shape) + 1j * g.standard_normal(d["X"].shape))
    t = lambda a: torch.from_numpy(wl.as_c64(a)[0]).to(dev)
    return t(d["H"]), t(d["Y"]), torch.from_numpy(d["N0"].astype(np.float32)).to(dev), t(Xt)


def test_noalloc_gradient_matches_workspace_entry_point(dev):
    U, K, Hd = 16, 2, 64
    model = learned.LearnedCD(K, U, Hd, seed=4, device=dev)
    # give the perceptron weights that are not zero, so every gradient group is exercised
    gen = torch.Generator().manual_seed(1)
    model.master.copy_(model.master + 0.3 * torch.randn(model.master.numel(), generator=gen).to(dev))
    model.pack()
    n = cdmimo.learned_param_count(K, U, Hd)
    for call, (seed, cs, n_sym, n_sc) in enumerate([(11, [32] * 8, 1, 96), (12, [16, 32, 16], 3, 40)]):
        H, Y, N0, Xt = _case(seed, n_sc, n_sym, cs, U, dev)
        loss_ref, grad_ref = model.grad(H, Y, N0, Xt, cs)
        grad = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
        loss = torch.full((1,), float("nan"), dtype=torch.float32, device=dev)
        cdmimo.learned_grad_noalloc(H, Y, N0, Xt, cs, K, model.block, Hd, grad=grad, loss=loss)
        torch.cuda.synchronize()
        assert torch.all(torch.isfinite(grad)), f"call {call}: non-finite gradient"
        # the same kernels in the same fixed reduction order: the results agree bit for bit
        assert torch.equal(grad, grad_ref), f"call {call}: gradient differs from the workspace entry point"
        assert torch.equal(loss, loss_ref), f"call {call}: loss differs from the workspace entry point"


def test_noalloc_rejects_batches_beyond_its_scratch(dev):
    U, K, Hd = 16, 2, 64
    model = learned.LearnedCD(K, U, Hd, seed=5, device=dev)
    n = cdmimo.learned_param_count(K, U, Hd)
    stride = (n + 1 + 3) // 4 * 4
    n_sc = 8 * 1024 * 1024 // (4 * stride) + 1  # one subcarrier more than the fixed array holds
    H = torch.zeros((n_sc, U, 256), dtype=torch.complex64, device=dev)
    Y = torch.zeros((n_sc, 1, 256), dtype=torch.complex64, device=dev)
    N0 = torch.ones(n_sc, dtype=torch.float32, device=dev)
    Xt = torch.zeros((n_sc, 1, U), dtype=torch.complex64, device=dev)
    grad = torch.zeros(n, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    with pytest.raises(cdmimo.CdmimoError) as e:
        cdmimo.learned_grad_noalloc(H, Y, N0, Xt, [32] * 8, K, model.block, Hd, grad=grad, loss=loss)
    assert e.value.status == cdmimo.ERR_WORKSPACE


def test_noalloc_flags_a_mismatched_block(dev):
    """A block packed for another sweep count is flagged and gives NaN, as in the workspace entry."""
    U, K, Hd = 16, 2, 64
    model = learned.LearnedCD(K, U, Hd, seed=6, device=dev)
    H, Y, N0, Xt = _case(13, 8, 2, [32] * 8, U, dev)
    n = cdmimo.learned_param_count(K + 1, U, Hd)
    grad = torch.zeros(n, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    cdmimo.device_status(clear=True)
    cdmimo.learned_grad_noalloc(H, Y, N0, Xt, [32] * 8, K + 1, model.block, Hd, grad=grad, loss=loss)
    torch.cuda.synchronize()
    assert cdmimo.device_status(clear=True) & cdmimo.DEV_BAD_LEARNED
    assert torch.all(torch.isnan(grad)) and torch.isnan(loss).all()
