"""Pins of the oracle's deep-unfolded CD with learned fusion (CPU only).

  * The learned sweep is over-relaxed Gauss-Seidel (SOR, relaxation tau_t) on the normal equations
    with regularizer gamma_t N0/Ex; checked against the SOR matrix splitting solved with a library
    triangular solve.
  * tau = gamma = 1 with a constant fusion logit reduces exactly to Algorithm 1 with equal fusion.
  * The analytic reverse pass matches central finite differences of the forward loss.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1902_08653_gb300 import workload as wl

GRAW_ONE = np.log(np.e - 1.0)  # softplus(GRAW_ONE) = 1


def crandn(g, *shape):
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / np.sqrt(2)


def make_master(g, K, U, Hd, tau=None, gamma_raw=None, scale=0.5, w2_zero=False):
    F = U + 1
    tau = g.uniform(0.6, 1.6, K) if tau is None else np.full(K, tau, float)
    graw = g.uniform(-1.0, 1.5, K) if gamma_raw is None else np.full(K, gamma_raw, float)
    W1 = g.standard_normal((Hd, F)) * scale
    b1 = g.standard_normal(Hd) * scale
    w2 = np.zeros(Hd) if w2_zero else g.standard_normal(Hd) * scale
    b2 = np.array([g.standard_normal() * scale])
    return np.concatenate([tau, graw, W1.ravel(), b1, w2, b2])


def sor_reference(Hc, y, alpha, taus, gammas):
    z = np.conj(Hc) @ y
    x = np.zeros(Hc.shape[0], complex)
    for tau, gam in zip(taus, gammas):
        A = np.conj(Hc) @ Hc.T + gam * alpha * np.eye(Hc.shape[0])
        D = np.diag(np.diag(A))
        Lo = np.tril(A, -1)
        Up = np.triu(A, 1)
        x = sla.solve_triangular(D + tau * Lo, tau * z - (tau * Up + (tau - 1) * D) @ x, lower=True)
    return x


@pytest.mark.parametrize("seed", range(4))
def test_learned_sweeps_are_sor(oracle, seed):
    g = np.random.default_rng(300 + seed)
    U, K, Hd = int(g.integers(1, 6)), int(g.integers(1, 4)), 4
    cs = [int(v) for v in g.integers(max(1, U - 1), 10, size=3)]
    H = crandn(g, 2, U, sum(cs))
    Y = crandn(g, 2, 2, sum(cs))
    N0 = g.uniform(0.1, 1.5, 2)
    master = make_master(g, K, U, Hd)
    _, Xc, lam = oracle.learned_forward(H, Y, N0, cs, K, master, Hd)
    taus = master[:K]
    gammas = np.log1p(np.exp(master[K:2 * K]))
    o = np.concatenate([[0], np.cumsum(cs)])
    for f in range(2):
        for c in range(3):
            for n in range(2):
                ref = sor_reference(H[f, :, o[c]:o[c + 1]], Y[f, n, o[c]:o[c + 1]], N0[f], taus, gammas)
                np.testing.assert_allclose(Xc[f, c, n], ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(lam.sum(axis=1), 1.0, atol=1e-14)
    assert np.all(lam > 0)


@pytest.mark.parametrize("seed", range(3))
def test_learned_fusion_is_cluster_permutation_equivariant(oracle, seed):
    """Relabelling equal-size clusters (permuting their antenna blocks) permutes the per-cluster
    estimates and the fusion weights the same way and leaves the fused estimate unchanged: the MLP
    sees each cluster's own features, and the softmax runs over clusters."""
    g = np.random.default_rng(500 + seed)
    U, K, Hd, C, Bc = 3, 2, 6, 4, 5
    cs = [Bc] * C
    H = crandn(g, 3, U, C * Bc)
    Y = crandn(g, 3, 2, C * Bc)
    N0 = g.uniform(0.1, 1.0, 3)
    master = make_master(g, K, U, Hd)
    X, Xc, lam = oracle.learned_forward(H, Y, N0, cs, K, master, Hd)
    perm = np.roll(np.arange(C), 1 + seed)  # a non-trivial relabelling
    cols = np.concatenate([np.arange(p * Bc, (p + 1) * Bc) for p in perm])
    Xp, Xcp, lamp = oracle.learned_forward(H[:, :, cols], Y[:, :, cols], N0, cs, K, master, Hd)
    np.testing.assert_allclose(lamp, lam[:, perm], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Xcp, Xc[:, perm], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Xp, X, rtol=1e-12, atol=1e-14)
    assert np.ptp(lam, axis=1).min() > 1e-3  # the weights do differ between clusters


def test_reduces_to_plain_cd_with_equal_fusion(oracle):
    g = np.random.default_rng(7)
    d = wl.uplink(3, 5, 3, 64, 8, snr_db=wl.sweep_snr(5))
    cs = [16] * 4
    master = make_master(g, 3, 8, 16, tau=1.0, gamma_raw=GRAW_ONE, w2_zero=True)
    Xl, Xcl, lam = oracle.learned_forward(d["H"], d["Y"], d["N0"], cs, 3, master, 16)
    Xp, Xcp, _ = oracle.detect(d["H"], d["Y"], d["N0"], cs, 3, fuse="equal")
    np.testing.assert_allclose(lam, 0.25, rtol=1e-14)
    np.testing.assert_allclose(Xcl, Xcp, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Xl, Xp, rtol=1e-12, atol=1e-14)


def test_loss_matches_forward(oracle):
    g = np.random.default_rng(11)
    d = wl.uplink(4, 3, 2, 24, 4, snr_db=10.0)
    cs = [8, 8, 8]
    master = make_master(g, 2, 4, 6)
    Xt = crandn(g, 3, 2, 4)
    Xl, _, _ = oracle.learned_forward(d["H"], d["Y"], d["N0"], cs, 2, master, 6)
    loss, _ = oracle.learned_grad(d["H"], d["Y"], d["N0"], cs, 2, master, 6, Xt)
    np.testing.assert_allclose(loss, np.mean(np.sum(np.abs(Xl - Xt) ** 2, axis=-1)), rtol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_central_differences(oracle, seed):
    g = np.random.default_rng(500 + seed)
    U, K, Hd = 3, 2, 5
    cs = [4, 6]
    H = crandn(g, 2, U, 10)
    Y = crandn(g, 2, 2, 10)
    N0 = np.array([0.3, 0.8])
    master = make_master(g, K, U, Hd)
    Xt = crandn(g, 2, 2, U)
    loss, grad = oracle.learned_grad(H, Y, N0, cs, K, master, Hd, Xt)
    num = np.zeros_like(master)
    eps = 1e-6
    for i in range(master.size):
        mp = master.copy()
        mp[i] += eps
        mm = master.copy()
        mm[i] -= eps
        num[i] = (oracle.learned_grad(H, Y, N0, cs, K, mp, Hd, Xt)[0] -
                  oracle.learned_grad(H, Y, N0, cs, K, mm, Hd, Xt)[0]) / (2 * eps)
    scale = np.max(np.abs(num))
    assert scale > 0
    np.testing.assert_allclose(grad, num, rtol=1e-5, atol=1e-7 * scale)
    # every parameter group receives gradient
    F = U + 1
    groups = np.split(grad, np.cumsum([K, K, Hd * F, Hd, Hd]))
    assert all(np.any(np.abs(gr) > 0) for gr in groups)


# --- Hand-computed pins of the learned fusion (features, MLP, ReLU, softmax) -------------------------
#
# A 3-subcarrier case whose cluster energies are small integers, with hand-set weights, so that every
# logit is a number derived by hand below.  U = 2, clusters of B_c = 2, 4, 2 antennas (uneven, so a
# dropped 1/B_c changes the features), F = U + 1 = 3 features phi_c = [e_{0,c}/B_c, e_{1,c}/B_c,
# log10(max(alpha, 1e-6))], hidden width 4.
#
#   user 0:  cluster 0 [1, 1j] -> e = 2, /2 = 1.0;  cluster 1 [1, 0, 0, 1] -> 2, /4 = 0.5;
#            cluster 2 [2, 0] -> 4, /2 = 2.0
#   user 1:  cluster 0 [0, 1] -> 1, /2 = 0.5;  cluster 1 [1, 1, 1, 1] -> 4, /4 = 1.0;
#            cluster 2 [1j, 1] -> 2, /2 = 1.0
#
# Hidden units (W1 row, b1) and output weights w2, b2 = -0.5:
#   k = 0: [1, 0, 0],  0   -> relu(phi_0)                            w2 = 1
#   k = 1: [0, 1, 1],  2   -> relu(phi_1 + log10 alpha + 2)          w2 = 2
#   k = 2: [-1, 0, 0], -0.25 -> always negative: ReLU off            w2 = 10
#   k = 3: [1, 0, -1], -7  -> relu(phi_0 - log10 alpha - 7)          w2 = 1
# Subcarrier 0, N0 = 0.01 (log10 alpha = -2): units 0, 1, 3 give [1, .5, 2], [.5, 1, 1], 0
#   -> logits [1 + 1, .5 + 2, 2 + 2] - 0.5 = [1.5, 2.0, 3.5]
# Subcarrier 1, N0 = 0 (alpha clamped to 1e-6, feature -6): unit 1 gives relu(phi_1 - 4) = 0, unit 3
#   relu(phi_0 - 1) = [0, 0, 1] -> logits [1, .5, 2 + 1] - 0.5 = [0.5, 0.0, 2.5]
# Subcarrier 2, N0 = 10 (feature 1): unit 1 gives [3.5, 4, 4], unit 3 is off
#   -> logits [1 + 7, .5 + 8, 2 + 8] - 0.5 = [7.5, 8.0, 9.5]
HAND_CS = [2, 4, 2]
HAND_N0 = np.array([0.01, 0.0, 10.0])
HAND_LOGITS = np.array([[1.5, 2.0, 3.5], [0.5, 0.0, 2.5], [7.5, 8.0, 9.5]])


def hand_channel():
    row0 = [1, 1j, 1, 0, 0, 1, 2, 0]
    row1 = [0, 1, 1, 1, 1, 1, 1j, 1]
    return np.tile(np.array([row0, row1], complex), (3, 1, 1))


def hand_master(K, tau=1.0, graw=GRAW_ONE):
    W1 = np.array([[1, 0, 0], [0, 1, 1], [-1, 0, 0], [1, 0, -1]], float)
    b1 = np.array([0.0, 2.0, -0.25, -7.0])
    w2 = np.array([1.0, 2.0, 10.0, 1.0])
    return np.concatenate([np.full(K, tau), np.full(K, graw), W1.ravel(), b1, w2, [-0.5]])


def softmax_rows(z):
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def test_learned_fusion_hand_computed_weights(oracle):
    """The fusion weights of the hand-set MLP equal the softmax of the logits derived by hand above:
    this fixes the features (1/B_c, log10 and its clamp at 1e-6), the row-major W1, the ReLU, w2, b2
    and the softmax over clusters."""
    g = np.random.default_rng(41)
    H = hand_channel()
    Y = crandn(g, 3, 2, 8)
    _, _, lam = oracle.learned_forward(H, Y, HAND_N0, HAND_CS, 1, hand_master(1), 4)
    np.testing.assert_allclose(lam, softmax_rows(HAND_LOGITS), rtol=1e-13, atol=1e-15)
    # the literal values of subcarrier 0: exp([0, .5, 2]) / (1 + e^0.5 + e^2)
    np.testing.assert_allclose(lam[0], [0.09962364, 0.16425163, 0.73612473], rtol=1e-7)


@pytest.mark.parametrize("K", [1, 3])
def test_learned_fused_estimate_hand_computed(oracle, K):
    """With tau = gamma = 1 the per-cluster estimates are Gauss-Seidel iterates (library triangular
    solves of the splitting), and the fused estimate is their combination with the hand-derived
    weights."""
    g = np.random.default_rng(43 + K)
    H = hand_channel()
    Y = crandn(g, 3, 2, 8)
    X, Xc, lam = oracle.learned_forward(H, Y, HAND_N0, HAND_CS, K, hand_master(K), 4)
    lam_ref = softmax_rows(HAND_LOGITS)
    o = np.concatenate([[0], np.cumsum(HAND_CS)])
    for f in range(3):
        want = np.zeros((2, 2), complex)
        for c in range(3):
            for n in range(2):
                xc = sor_reference(H[f, :, o[c]:o[c + 1]], Y[f, n, o[c]:o[c + 1]], HAND_N0[f], [1.0] * K, [1.0] * K)
                np.testing.assert_allclose(Xc[f, c, n], xc, rtol=1e-11, atol=1e-12)
                want[n] += lam_ref[f, c] * xc
        np.testing.assert_allclose(X[f], want, rtol=1e-11, atol=1e-12)


def test_learned_fusion_scaled_cluster_closed_form(oracle):
    """Random channels, a single hidden unit selecting user j's normalized energy: lambda_c is
    proportional to exp(w ||h_{j,c}||^2 / B_c), with the energies summed directly from H."""
    g = np.random.default_rng(47)
    U, K, Hd, cs = 4, 2, 3, [6, 10, 8, 12]
    B = sum(cs)
    H = crandn(g, 2, U, B)
    o = np.concatenate([[0], np.cumsum(cs)])
    for c, s in enumerate([0.5, 1.0, 1.3, 0.8]):  # distinct cluster gains
        H[:, :, o[c]:o[c + 1]] *= s
    Y = crandn(g, 2, 3, B)
    N0 = np.array([0.2, 0.05])
    j, w = 2, 0.7
    F = U + 1
    W1 = np.zeros((Hd, F))
    W1[1, j] = 1.0                      # hidden unit 1 = relu(e_{j,c} / B_c) = e_{j,c} / B_c
    b1 = np.array([-1.0, 0.0, -3.0])    # units 0 and 2 have zero weights and negative bias: off
    w2 = np.array([5.0, w, -4.0])
    master = np.concatenate([g.uniform(0.8, 1.2, K), g.uniform(-0.5, 0.5, K), W1.ravel(), b1, w2, [0.9]])
    _, _, lam = oracle.learned_forward(H, Y, N0, cs, K, master, Hd)
    energy = np.array([[np.sum(np.abs(H[f, j, o[c]:o[c + 1]]) ** 2) / cs[c] for c in range(4)] for f in range(2)])
    np.testing.assert_allclose(lam, softmax_rows(w * energy), rtol=1e-12, atol=1e-15)
