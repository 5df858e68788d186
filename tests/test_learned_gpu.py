"""GPU parity of the learned deep-unfolded CD (inference, gradient, packing, Adam) against the FP64
oracle, and a short training run that must beat the untrained (plain CD) model.

The oracle receives exactly the parameter values the kernels use: W1 and w2 rounded to bfloat16.
Tolerances: inference 1e-4 relative L2 per estimate vector (as for plain CD); gradients 1e-3
relative to the largest gradient entry (FP32 accumulation over a batch, vs FP64), and per element
1e-3 relative wherever the entry is above 1e-5 of the largest.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo, learned
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


class Block(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("U", ctypes.c_int), ("hidden", ctypes.c_int), ("r0", ctypes.c_int),
                ("tau", ctypes.c_float * 16), ("gamma", ctypes.c_float * 16), ("b1", ctypes.c_float * 64),
                ("b2", ctypes.c_float), ("r1", ctypes.c_float * 3), ("W1", ctypes.c_uint16 * (64 * 65)),
                ("w2", ctypes.c_uint16 * 64)]


def random_master(seed, K, U, Hd, scale=0.4):
    g = np.random.default_rng(seed)
    sl = learned.layout(K, U, Hd)
    m = np.zeros(cdmimo.learned_param_count(K, U, Hd), np.float32)
    m[sl["tau"]] = g.uniform(0.7, 1.5, K)
    m[sl["graw"]] = g.uniform(-0.5, 1.2, K)
    m[sl["W1"]] = g.standard_normal(Hd * (U + 1)) * scale
    m[sl["b1"]] = g.standard_normal(Hd) * scale
    m[sl["w2"]] = g.standard_normal(Hd) * scale
    m[sl["b2"]] = g.standard_normal() * scale
    return m


def as_used(master, K, U, Hd):
    """The master vector as the kernels see it: W1 and w2 rounded to bfloat16, in FP64."""
    sl = learned.layout(K, U, Hd)
    m = master.astype(np.float64).copy()
    for k in ("W1", "w2"):
        m[sl[k]] = wl.bf16_bits_to_f32(wl.f32_to_bf16_bits(master[sl[k]].astype(np.float32))).astype(np.float64)
    return m


def test_pack(dev):
    K, U, Hd = 3, 16, 64
    m = random_master(1, K, U, Hd)
    mt = torch.from_numpy(m).to(dev)
    blk = torch.zeros(cdmimo.LEARNED_BLOCK_BYTES, dtype=torch.uint8, device=dev)
    cdmimo.learned_pack(mt, K, U, Hd, blk)
    b = Block.from_buffer_copy(blk.cpu().numpy().tobytes())
    sl = learned.layout(K, U, Hd)
    assert (b.K, b.U, b.hidden) == (K, U, Hd)
    np.testing.assert_allclose(np.array(b.tau[:K]), m[sl["tau"]], rtol=0)
    np.testing.assert_allclose(np.array(b.gamma[:K]), np.log1p(np.exp(m[sl["graw"]].astype(np.float64))), rtol=1e-6)
    np.testing.assert_array_equal(np.array(b.W1[:Hd * (U + 1)], dtype=np.uint16), wl.f32_to_bf16_bits(m[sl["W1"]]))
    np.testing.assert_array_equal(np.array(b.w2[:Hd], dtype=np.uint16), wl.f32_to_bf16_bits(m[sl["w2"]]))
    np.testing.assert_allclose(np.array(b.b1[:Hd]), m[sl["b1"]], rtol=0)
    assert b.b2 == np.float32(m[sl["b2"]][0])


def _inputs(seed, n_sc, n_sym, B, U, dev):
    d = wl.uplink(seed, n_sc, n_sym, B, U, snr_db=wl.sweep_snr(n_sc), M=16)
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    N0 = d["N0"].astype(np.float32)
    return d, (torch.from_numpy(H32).to(dev), torch.from_numpy(Y32).to(dev), torch.from_numpy(N0).to(dev)), \
        (H64, Y64, N0.astype(np.float64))


@pytest.mark.parametrize("K,n_sym", [(2, 14), (3, 1), (1, 5)])
def test_learned_inference_parity(dev, K, n_sym):
    U, Hd, cs = 16, 64, [32] * 8
    m = random_master(10 + K, K, U, Hd)
    model = learned.LearnedCD(K, U, Hd, master=torch.from_numpy(m), device=dev)
    _, (H, Y, N0), (H64, Y64, N064) = _inputs(20 + K, 23, n_sym, 256, U, dev)
    lam = torch.zeros((23, 8), dtype=torch.float32, device=dev)
    Xc = torch.zeros((23, 8, n_sym, U), dtype=torch.complex64, device=dev)
    Xg = model.detect(H, Y, N0, cs, lam=lam, Xc=Xc).cpu().numpy()
    Xo, Xco, lamo = orc.learned_forward(H64, Y64, N064, cs, K, as_used(m, K, U, Hd), Hd, threads=8)
    assert_vectors_close(Xc.cpu().numpy(), Xco, 1e-4, "Xc")
    np.testing.assert_allclose(lam.cpu().numpy(), lamo, rtol=2e-5, atol=1e-7)
    assert_vectors_close(Xg, Xo, 1e-4, "Xhat")
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("form", ["gram", "residual"])
@pytest.mark.parametrize("cs,U,K,n_sym,fuse", [([32] * 8, 16, 3, 14, "learned"), ([16] * 6, 8, 2, 9, "learned"),
                                               ([64] * 4, 16, 2, 14, "colnorm"), ([32] * 3, 5, 4, 7, "equal")])
def test_learned_forms_match_oracle(dev, form, cs, U, K, n_sym, fuse):
    """Learned sweeps in both forms: the Gram form sums z_u - sum_v G_uv x_v, the residual form
    h_u^H r (different rounding), both against the FP64 oracle with the same parameters."""
    Hd = 32
    m = random_master(70 + K + U, K, U, Hd)
    model = learned.LearnedCD(K, U, Hd, master=torch.from_numpy(m), device=dev)
    n_sc = 19
    _, (H, Y, N0), (H64, Y64, N064) = _inputs(80 + U, n_sc, n_sym, sum(cs), U, dev)
    assert cdmimo.selected_form(cdmimo.OP_DETECT, n_sc, n_sym, sum(cs), U, cs, K, H=H, form=form) == form
    lam = torch.zeros((n_sc, len(cs)), dtype=torch.float32, device=dev)
    Xc = torch.zeros((n_sc, len(cs), n_sym, U), dtype=torch.complex64, device=dev)
    X = cdmimo.detect(H, Y, N0, cs, K, fuse=fuse, learned=model.block, lam=lam, Xc=Xc, form=form).cpu().numpy()
    Xo, Xco, lamo = orc.learned_forward(H64, Y64, N064, cs, K, as_used(m, K, U, Hd), Hd, threads=8)
    if fuse != "learned":  # learned per-cluster estimates, fused with the plain detector's weights
        lamo = orc.detect(H64, Y64, N064, cs, 0, fuse=fuse, threads=8)[2]
        Xo = np.einsum("fc,fcnu->fnu", lamo, Xco)
    assert_vectors_close(Xc.cpu().numpy(), Xco, 1e-4, f"learned Xc ({form})")
    np.testing.assert_allclose(lam.cpu().numpy(), lamo, rtol=2e-5, atol=1e-7)
    assert_vectors_close(X, Xo, 1e-4, f"learned Xhat ({form}, {fuse})")
    assert cdmimo.device_status(clear=True) == 0


def test_untrained_model_is_plain_cd_with_equal_fusion(dev):
    U, cs = 16, [32] * 8
    model = learned.LearnedCD(2, U, 64, seed=3, device=dev)
    _, (H, Y, N0), _ = _inputs(5, 31, 14, 256, U, dev)
    Xl = model.detect(H, Y, N0, cs)
    Xp = cdmimo.detect(H, Y, N0, cs, 2, fuse="equal")
    assert_vectors_close(Xl.cpu().numpy(), Xp.cpu().numpy(), 1e-5, "reduction")


@pytest.mark.parametrize("cs,U,K,n_sym,fuse,vs_gram", [([32] * 8, 16, 2, 14, "learned", True),
                                                       ([32] * 8, 16, 3, 14, "colnorm", True),
                                                       ([16] * 6, 10, 2, 9, "learned", False),
                                                       ([32] * 4, 9, 4, 7, "equal", True)])
def test_learned_tensor_core_form_matches_oracle(dev, cs, U, K, n_sym, fuse, vs_gram):
    """Learned sweeps and fusion on the tensor-core kernel (z and G_c from split-TF32 MMAs): against
    the FP64 oracle, and against the FP32 Gram-form learned kernel (same iterates, other rounding)."""
    Hd = 32
    m = random_master(90 + K + U, K, U, Hd)
    model = learned.LearnedCD(K, U, Hd, master=torch.from_numpy(m), device=dev)
    n_sc = 37
    _, (H, Y, N0), (H64, Y64, N064) = _inputs(100 + U, n_sc, n_sym, sum(cs), U, dev)
    assert cdmimo.selected_form(cdmimo.OP_DETECT, n_sc, n_sym, sum(cs), U, cs, K, H=H, form="gram_tc") == "gram_tc"
    X = cdmimo.detect(H, Y, N0, cs, K, fuse=fuse, learned=model.block, form="gram_tc").cpu().numpy()
    Xo, Xco, lamo = orc.learned_forward(H64, Y64, N064, cs, K, as_used(m, K, U, Hd), Hd, threads=8)
    if fuse != "learned":  # learned per-cluster estimates, fused with the plain detector's weights
        lamo = orc.detect(H64, Y64, N064, cs, 0, fuse=fuse, threads=8)[2]
        Xo = np.einsum("fc,fcnu->fnu", lamo, Xco)
    assert_vectors_close(X, Xo, 1e-4, f"learned Xhat (gram_tc, {fuse})")
    if vs_gram:
        Xg = cdmimo.detect(H, Y, N0, cs, K, fuse=fuse, learned=model.block, form="gram").cpu().numpy()
        assert_vectors_close(X, Xg, 2e-5, f"learned gram_tc vs gram ({fuse})")
    assert cdmimo.device_status(clear=True) == 0


@pytest.mark.parametrize("form", ["gram", "residual", "gram_tc"])
def test_learned_block_mismatch_is_flagged(dev, form):
    model = learned.LearnedCD(2, 16, 64, device=dev)
    _, (H, Y, N0), _ = _inputs(6, 3, 2, 256, 16, dev)
    X = cdmimo.detect(H, Y, N0, [32] * 8, 3, fuse="learned", learned=model.block, form=form).cpu().numpy()
    assert cdmimo.device_status(clear=True) & cdmimo.DEV_BAD_LEARNED
    assert np.all(np.isnan(X))


@pytest.mark.parametrize("cs,n_sym,K", [([32] * 8, 1, 2), ([16, 32, 16], 3, 2), ([32] * 8, 14, 3)])
def test_gradient_parity(dev, cs, n_sym, K):
    U, Hd = 16, 64
    B = sum(cs)
    m = random_master(40 + K, K, U, Hd)
    model = learned.LearnedCD(K, U, Hd, master=torch.from_numpy(m), device=dev)
    d, (H, Y, N0), (H64, Y64, N064) = _inputs(30 + n_sym, 17, n_sym, B, U, dev)
    g = np.random.default_rng(2)
    Xt = (d["X"] + 0.1 * (g.standard_normal(d["X"].shape) + 1j * g.standard_normal(d["X"].shape)))
    Xt32, Xt64 = wl.as_c64(Xt)
    loss, grad = model.grad(H, Y, N0, torch.from_numpy(Xt32).to(dev), cs)
    lo, go = orc.learned_grad(H64, Y64, N064, cs, K, as_used(m, K, U, Hd), Hd, Xt64)
    np.testing.assert_allclose(loss.item(), lo, rtol=1e-5)
    gg = grad.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(go))
    err = np.abs(gg - go) / scale
    assert err.max() < 1e-3, f"max gradient error {err.max():.2e} at {err.argmax()}"
    # per element: relative 1e-3, except entries that are themselves below 1e-5 of the largest
    # (their absolute error is then at most 1e-8 of it, far under the FP32 accumulation error)
    np.testing.assert_allclose(gg, go, rtol=1e-3, atol=1e-5 * scale)


@pytest.mark.parametrize("what", ["K", "hidden"])
def test_gradient_block_mismatch_is_flagged(dev, what):
    """A block packed for other (K, hidden) than the gradient call's is flagged and gives a NaN
    gradient and loss, like the inference kernels (a mismatched block would otherwise be read with
    the wrong strides)."""
    U, K, Hd = 16, 2, 64
    model = learned.LearnedCD(K, U, Hd, seed=3, device=dev)
    Kc, Hc = (K + 1, Hd) if what == "K" else (K, Hd // 2)
    d, (H, Y, N0), _ = _inputs(8, 5, 2, 256, U, dev)
    Xt = torch.from_numpy(wl.as_c64(d["X"])[0]).to(dev)
    cdmimo.device_status(clear=True)
    loss, grad = cdmimo.learned_grad(H, Y, N0, Xt, [32] * 8, Kc, model.block, Hc)
    torch.cuda.synchronize()
    assert cdmimo.device_status(clear=True) & cdmimo.DEV_BAD_LEARNED
    assert torch.all(torch.isnan(grad)) and torch.isnan(loss).all()


def test_adam_matches_torch(dev):
    g = torch.Generator().manual_seed(0)
    theta = torch.randn(1000, generator=g)
    ref = theta.clone().requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    th = theta.to(dev)
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    for step in range(1, 6):
        grad = torch.randn(1000, generator=g)
        ref.grad = grad.clone()
        opt.step()
        cdmimo.adam_step(th, grad.to(dev), m, v, step, lr=3e-3)
    np.testing.assert_allclose(th.cpu().numpy(), ref.detach().numpy(), rtol=1e-5, atol=1e-6)


def test_training_beats_untrained_model(dev, tmp_path):
    """A short training run (GPU gradient + Adam) lowers the MSE against the centralized L-MMSE on
    held-out channels; the checkpoint round-trips."""
    U, K, cs, B = 16, 2, [32] * 8, 256
    model = learned.LearnedCD(K, U, 64, seed=0, device=dev)

    def batch(seed, n_sc):
        d = wl.uplink(seed, n_sc, 1, B, U, snr_db=np.random.default_rng(seed).uniform(0, 30, n_sc), M=16)
        H = torch.from_numpy(wl.as_c64(d["H"])[0]).to(dev)
        Y = torch.from_numpy(wl.as_c64(d["Y"])[0]).to(dev)
        N0 = torch.from_numpy(d["N0"].astype(np.float32)).to(dev)
        Xt = cdmimo.detect(H, Y, N0, [B], 32, fuse="equal")  # centralized CD, converged: the L-MMSE target
        return H, Y, N0, Xt

    H, Y, N0, Xt = batch(999, 512)
    mse0 = torch.mean(torch.abs(model.detect(H, Y, N0, cs) - Xt) ** 2).item()
    for it in range(150):
        h, y, n0, xt = batch(it, 256)
        model.train_step(h, y, n0, xt, cs, lr=1e-2)
    mse1 = torch.mean(torch.abs(model.detect(H, Y, N0, cs) - Xt) ** 2).item()
    assert mse1 < 0.9 * mse0, (mse0, mse1)
    p = tmp_path / "ckpt.bin"
    model.save(p)
    back = learned.LearnedCD.load(p, device=dev)
    assert back.step == model.step and torch.equal(back.master, model.master)
    assert torch.equal(back.detect(H, Y, N0, cs), model.detect(H, Y, N0, cs))


def test_centralized_cd_target_is_lmmse(dev):
    """The training target (one cluster of all 256 antennas, 32 sweeps) equals the centralized
    L-MMSE of Eq. (1) from the oracle's Cholesky solve."""
    d = wl.uplink(77, 16, 2, 256, 16, snr_db=wl.sweep_snr(16))
    H32, H64 = wl.as_c64(d["H"])
    Y32, Y64 = wl.as_c64(d["Y"])
    N0 = d["N0"].astype(np.float32)
    X = cdmimo.detect(torch.from_numpy(H32).to(dev), torch.from_numpy(Y32).to(dev), torch.from_numpy(N0).to(dev),
                      [256], 32, fuse="equal").cpu().numpy()
    Xm = orc.lmmse(H64, Y64, N0.astype(np.float64))
    assert_vectors_close(X, Xm, 1e-4, "centralized CD vs L-MMSE")
