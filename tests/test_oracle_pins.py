"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Nothing here re-types the oracle's loops.  Each test checks the oracle against an independent
formulation or a consequence of the method:
  * Algorithm 1 is exact coordinate minimization of Eq. (1)'s objective, i.e. Gauss-Seidel on the
    normal equations (H^H H + a I) x = H^H y; the matrix-splitting form of Gauss-Seidel
    x <- (D + L)^{-1} (H^H y - L^H x) is solved with a library triangular solve.
  * Algorithm 2 is cyclic coordinate descent on the dual (2) with the primal map x = Hbar^H z
    (Eqs. (3)-(4)), i.e. unit-diagonal Gauss-Seidel on (Hbar Hbar^H) z = sbar, again as a splitting.
  * Limits: K -> infinity gives the local L-MMSE (library solve) / local min-norm ZF (library pinv).
  * Closed forms (U = 1, orthogonal columns), invariants (objective non-increasing in K, sum of
    fusion weights, per-cluster transmit power), special cases (C = 1, K = 0), brute-force ML.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

from paper_1902_08653_gb300 import workload as wl


def crandn(g, *shape):
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / np.sqrt(2)


def offsets(cs):
    return np.concatenate([[0], np.cumsum(cs)]).astype(int)


def gs_detect_reference(Hc, y, alpha, K):
    """K Gauss-Seidel sweeps (ascending coordinates) on (Hc Hc^H... in uplink form) by splitting.

    Hc: [U][Bc] rows = columns h_u of the local uplink matrix; y: [Bc].
    """
    A = np.conj(Hc) @ Hc.T + alpha * np.eye(Hc.shape[0])   # A_uv = h_u^H h_v + a delta_uv
    z = np.conj(Hc) @ y                                      # z_u = h_u^H y
    DL = np.tril(A)
    Up = np.triu(A, 1)
    x = np.zeros(Hc.shape[0], complex)
    for _ in range(K):
        x = sla.solve_triangular(DL, z - Up @ x, lower=True)
    return x


def gs_precode_reference(Hc, s, K):
    """K cyclic dual-CD sweeps of Eqs. (3)-(4) by splitting; returns the unnormalized primal x."""
    e = np.sum(np.abs(Hc) ** 2, axis=1)
    p = np.where(e > 0, 1 / np.sqrt(np.where(e > 0, e, 1)), 0.0)
    Hb = Hc * p[:, None]                                      # rows hbar_u (uplink columns)
    G = np.conj(Hb) @ Hb.T                                    # Gbar_uv = hbar_u^H hbar_v
    sb = p * s
    DL = np.tril(G)
    Up = np.triu(G, 1)
    z = np.zeros(Hc.shape[0], complex)
    for _ in range(K):
        z = sla.solve_triangular(DL, sb - Up @ z, lower=True)
    return Hb.T @ z                                           # x = sum_u hbar_u z_u


# ------------------------------------------------------------------------------------------
# Algorithm 1: detection
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_detect_equals_gauss_seidel_splitting(oracle, seed):
    g = np.random.default_rng(100 + seed)
    U = int(g.integers(1, 7))
    C = int(g.integers(1, 4))
    cs = [int(v) for v in g.integers(max(1, U - 1), 12, size=C)]  # includes B_c < U
    B = sum(cs)
    n_sc, n_sym, K = 3, 2, int(g.integers(1, 5))
    H = crandn(g, n_sc, U, B)
    Y = crandn(g, n_sc, n_sym, B)
    N0 = g.uniform(0.05, 2.0, n_sc)
    Xhat, Xc, lam = oracle.detect(H, Y, N0, cs, K, fuse="colnorm")
    o = offsets(cs)
    for f in range(n_sc):
        for c in range(C):
            for n in range(n_sym):
                ref = gs_detect_reference(H[f, :, o[c]:o[c + 1]], Y[f, n, o[c]:o[c + 1]], N0[f], K)
                np.testing.assert_allclose(Xc[f, c, n], ref, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(Xhat[f], np.einsum("c,cnu->nu", lam[f], Xc[f]), rtol=1e-12, atol=1e-14)


def test_detect_Ex_enters_only_through_regularizer(oracle):
    g = np.random.default_rng(7)
    H = crandn(g, 2, 4, 16)
    Y = crandn(g, 2, 3, 16)
    N0 = np.array([0.3, 0.9])
    a = oracle.detect(H, Y, N0, [8, 8], 3, Ex=2.0)[1]
    b = oracle.detect(H, Y, N0 / 2.0, [8, 8], 3, Ex=1.0)[1]
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("Bc,U", [(16, 4), (8, 8), (32, 16)])
def test_detect_converges_to_local_lmmse(oracle, Bc, U):
    g = np.random.default_rng(Bc * 100 + U)
    C = 2
    H = crandn(g, 2, U, C * Bc)
    Y = crandn(g, 2, 2, C * Bc)
    N0 = np.array([0.5, 0.1])
    K = 4000 if Bc == U else 400
    _, Xc, _ = oracle.detect(H, Y, N0, [Bc] * C, K)
    for f in range(2):
        for c in range(C):
            Hc = H[f, :, c * Bc:(c + 1) * Bc]
            A = np.conj(Hc) @ Hc.T + N0[f] * np.eye(U)
            for n in range(2):
                ref = np.linalg.solve(A, np.conj(Hc) @ Y[f, n, c * Bc:(c + 1) * Bc])
                np.testing.assert_allclose(Xc[f, c, n], ref, rtol=1e-9, atol=1e-11)


def test_lmmse_oracle_matches_library_solve(oracle):
    g = np.random.default_rng(11)
    H = crandn(g, 3, 6, 20)
    Y = crandn(g, 3, 4, 20)
    N0 = np.array([0.0, 0.2, 1.5])
    X = oracle.lmmse(H, Y, N0)
    Xl = oracle.lmmse(H, Y, N0, rows=(5, 10))
    for f in range(3):
        A = np.conj(H[f]) @ H[f].T + N0[f] * np.eye(6)
        Al = np.conj(H[f, :, 5:15]) @ H[f, :, 5:15].T + N0[f] * np.eye(6)
        for n in range(4):
            np.testing.assert_allclose(X[f, n], np.linalg.solve(A, np.conj(H[f]) @ Y[f, n]), rtol=1e-10)
            np.testing.assert_allclose(Xl[f, n], np.linalg.solve(Al, np.conj(H[f, :, 5:15]) @ Y[f, n, 5:15]),
                                       rtol=1e-10)


def test_single_user_closed_form(oracle):
    """U = 1: one coordinate step is exact, x = h^H y / (||h||^2 + N0/Ex), for every K >= 1."""
    g = np.random.default_rng(3)
    H = crandn(g, 4, 1, 12)
    Y = crandn(g, 4, 2, 12)
    N0 = np.array([0.0, 0.1, 1.0, 10.0])
    for K in (1, 2, 5):
        _, Xc, _ = oracle.detect(H, Y, N0, [5, 7], K)
        for f in range(4):
            for c, (a, b) in enumerate([(0, 5), (5, 12)]):
                h = H[f, 0, a:b]
                ref = (np.conj(h) @ Y[f, :, a:b].T) / (np.vdot(h, h).real + N0[f])
                np.testing.assert_allclose(Xc[f, c, :, 0], ref, rtol=1e-13)


def test_orthogonal_columns_exact_after_one_sweep(oracle):
    """Orthogonal columns decouple the normal equations: one sweep reaches the L-MMSE solution."""
    Bc, U = 16, 6
    F = np.exp(-2j * np.pi * np.outer(np.arange(U), np.arange(Bc)) / Bc)  # DFT rows: orthogonal
    gains = np.array([1.0, 0.5, 2.0, 1.5, 0.7, 3.0])
    H = (F * gains[:, None])[None]
    g = np.random.default_rng(5)
    Y = crandn(g, 1, 3, Bc)
    N0 = np.array([0.4])
    _, Xc, _ = oracle.detect(H, Y, N0, [Bc], 1)
    ref = (np.conj(H[0]) @ Y[0].T).T / (gains ** 2 * Bc + 0.4)
    np.testing.assert_allclose(Xc[0, 0], ref, rtol=1e-12)


def test_objective_non_increasing_in_sweeps(oracle):
    """Each coordinate step minimizes ||y - H x||^2 + a ||x||^2 exactly, so the objective never grows."""
    g = np.random.default_rng(9)
    U, Bc = 8, 12
    H = crandn(g, 1, U, Bc)
    Y = crandn(g, 1, 1, Bc)
    N0 = np.array([0.3])
    prev = np.inf
    for K in range(0, 12):
        x = oracle.detect(H, Y, N0, [Bc], K)[1][0, 0, 0]
        J = np.linalg.norm(Y[0, 0] - H[0].T @ x) ** 2 + 0.3 * np.linalg.norm(x) ** 2
        assert J <= prev * (1 + 1e-14)
        prev = J


def test_K0_gives_zero(oracle):
    g = np.random.default_rng(1)
    H = crandn(g, 2, 3, 8)
    Y = crandn(g, 2, 2, 8)
    S = crandn(g, 2, 2, 3)
    Xhat, Xc, _ = oracle.detect(H, Y, np.array([0.1, 0.1]), [4, 4], 0)
    assert np.all(Xhat == 0) and np.all(Xc == 0)
    assert np.all(oracle.precode(H, S, [4, 4], 0) == 0)


def test_single_cluster_is_centralized_cd(oracle):
    """C = 1 is centralized CD (Sec. III): lambda = 1 and, as K grows, the centralized L-MMSE (1)."""
    g = np.random.default_rng(21)
    U, B = 8, 64
    H = crandn(g, 2, U, B)
    Y = crandn(g, 2, 3, B)
    N0 = np.array([0.2, 1.0])
    Xhat, Xc, lam = oracle.detect(H, Y, N0, [B], 3)
    assert np.all(lam == 1.0)
    np.testing.assert_array_equal(Xhat, Xc[:, 0])
    for f in range(2):
        for n in range(3):
            np.testing.assert_allclose(Xhat[f, n], gs_detect_reference(H[f], Y[f, n], N0[f], 3), rtol=1e-11)
    Xinf = oracle.detect(H, Y, N0, [B], 200)[0]
    np.testing.assert_allclose(Xinf, oracle.lmmse(H, Y, N0), rtol=1e-10, atol=1e-12)


def test_noise_free_least_squares_recovers_x(oracle):
    """N0 = 0 and B_c >= U: CD converges to the local least-squares solution, which is x itself."""
    d = wl.uplink(3, 2, 2, 32, 4, snr_db=np.inf, M=16)
    assert np.all(d["N0"] == 0)
    _, Xc, _ = oracle.detect(d["H"], d["Y"], d["N0"], [16, 16], 300)
    for c in range(2):
        np.testing.assert_allclose(Xc[:, c], d["X"], rtol=0, atol=1e-10)


def test_zero_column_skipped_without_regularizer(oracle):
    g = np.random.default_rng(4)
    H = crandn(g, 1, 3, 10)
    H[0, 1, :] = 0
    Y = crandn(g, 1, 1, 10)
    x = oracle.detect(H, Y, np.array([0.0]), [10], 200)[0][0, 0]
    assert x[1] == 0
    Hk = H[0][[0, 2]]
    ls = np.linalg.lstsq(Hk.T, Y[0, 0], rcond=None)[0]
    np.testing.assert_allclose(x[[0, 2]], ls, rtol=1e-10)


# ------------------------------------------------------------------------------------------
# Fusion (Sec. III)
# ------------------------------------------------------------------------------------------
def test_fusion_weights_sum_to_one_and_equal_rule(oracle):
    g = np.random.default_rng(12)
    H = crandn(g, 5, 4, 40)
    Y = crandn(g, 5, 2, 40)
    N0 = g.uniform(0.0, 1.0, 5)
    cs = [8, 12, 4, 16]
    for rule in ("colnorm", "equal"):
        Xhat, Xc, lam = oracle.detect(H, Y, N0, cs, 2, fuse=rule)
        np.testing.assert_allclose(lam.sum(axis=1), 1.0, rtol=0, atol=1e-15)
        assert np.all(lam > 0)
        if rule == "equal":
            assert np.all(lam == 0.25)
            np.testing.assert_allclose(Xhat, Xc.mean(axis=1), rtol=1e-13)


def test_antenna_and_cluster_relabelling(oracle):
    """Permuting the antennas inside each cluster leaves detection (estimates, per-cluster estimates,
    fusion weights) unchanged and permutes the precoder's output the same way; relabelling
    equal-size clusters permutes the per-cluster outputs and weights and leaves the fused estimate
    unchanged.  The algorithms see a cluster's antennas only through inner products over them."""
    g = np.random.default_rng(41)
    cs = [6, 9, 6, 5]
    o = offsets(cs)
    B, U = sum(cs), 4
    H = crandn(g, 3, U, B)
    Y = crandn(g, 3, 2, B)
    S = crandn(g, 3, 2, U)
    N0 = g.uniform(0.05, 0.8, 3)
    cols = np.concatenate([o[c] + g.permutation(cs[c]) for c in range(len(cs))])  # within clusters
    X, Xc, lam = oracle.detect(H, Y, N0, cs, 3)
    Xp, Xcp, lamp = oracle.detect(H[:, :, cols], Y[:, :, cols], N0, cs, 3)
    np.testing.assert_allclose(Xp, X, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Xcp, Xc, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(lamp, lam, rtol=1e-12)
    P = oracle.precode(H, S, cs, 3)
    Pp = oracle.precode(H[:, :, cols], S, cs, 3)
    np.testing.assert_allclose(Pp, P[:, :, cols], rtol=1e-12, atol=1e-14)
    # equal-size clusters relabelled (blocks 0 and 2 swapped)
    cs2 = [6, 6, 6]
    H2, Y2 = H[:, :, :18], Y[:, :, :18]
    blocks = np.concatenate([np.arange(12, 18), np.arange(6, 12), np.arange(0, 6)])
    X2, Xc2, lam2 = oracle.detect(H2, Y2, N0, cs2, 3)
    X2p, Xc2p, lam2p = oracle.detect(H2[:, :, blocks], Y2[:, :, blocks], N0, cs2, 3)
    np.testing.assert_allclose(lam2p, lam2[:, ::-1], rtol=1e-12)
    np.testing.assert_allclose(Xc2p, Xc2[:, ::-1], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(X2p, X2, rtol=1e-12, atol=1e-14)
    assert np.ptp(lam2, axis=1).min() > 1e-4  # the clusters do get different weights


def test_fusion_identical_clusters(oracle):
    g = np.random.default_rng(13)
    Hh = crandn(g, 2, 4, 8)
    Yh = crandn(g, 2, 3, 8)
    H = np.concatenate([Hh, Hh, Hh], axis=2)
    Y = np.concatenate([Yh, Yh, Yh], axis=2)
    Xhat, Xc, lam = oracle.detect(H, Y, np.array([0.1, 0.7]), [8, 8, 8], 3)
    np.testing.assert_allclose(lam, 1 / 3, rtol=1e-15)
    np.testing.assert_allclose(Xhat, Xc[:, 0], rtol=1e-14)


def test_fusion_scaled_cluster_closed_form(oracle):
    """Cluster 2 = sqrt(2) x cluster 1 and N0 = 0: its column energies double, so its
    post-equalization noise variance halves and lambda = (1/3, 2/3)."""
    g = np.random.default_rng(14)
    Hh = crandn(g, 1, 4, 8)
    H = np.concatenate([Hh, np.sqrt(2) * Hh], axis=2)
    Y = crandn(g, 1, 1, 16)
    _, _, lam = oracle.detect(H, Y, np.array([0.0]), [8, 8], 1)
    np.testing.assert_allclose(lam[0], [1 / 3, 2 / 3], rtol=1e-14)


# ------------------------------------------------------------------------------------------
# Algorithm 2: precoding
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_precode_equals_dual_gauss_seidel(oracle, seed):
    g = np.random.default_rng(200 + seed)
    U = int(g.integers(1, 7))
    C = int(g.integers(1, 4))
    cs = [int(v) for v in g.integers(max(1, U - 2), 12, size=C)]
    B = sum(cs)
    K = int(g.integers(1, 5))
    rho = float(g.uniform(0.5, 2.0))
    H = crandn(g, 2, U, B)
    S = crandn(g, 2, 3, U)
    X = oracle.precode(H, S, cs, K, rho=rho)
    o = offsets(cs)
    for f in range(2):
        for n in range(3):
            for c in range(C):
                ref = gs_precode_reference(H[f, :, o[c]:o[c + 1]], S[f, n], K)
                ref = rho / np.sqrt(C) * ref / np.linalg.norm(ref)
                np.testing.assert_allclose(X[f, n, o[c]:o[c + 1]], ref, rtol=1e-11, atol=1e-13)


def test_precode_power_per_cluster(oracle):
    g = np.random.default_rng(31)
    cs = [8, 16, 8]
    H = crandn(g, 3, 4, 32)
    S = crandn(g, 3, 2, 4)
    X = oracle.precode(H, S, cs, 3, rho=1.7)
    o = offsets(cs)
    for c in range(3):
        np.testing.assert_allclose(np.linalg.norm(X[..., o[c]:o[c + 1]], axis=-1), 1.7 / np.sqrt(3), rtol=1e-13)
    np.testing.assert_allclose(np.sum(np.abs(X) ** 2, axis=-1), 1.7 ** 2, rtol=1e-13)


@pytest.mark.parametrize("Bc,U", [(16, 4), (32, 16)])
def test_precode_converges_to_local_zf(oracle, Bc, U):
    g = np.random.default_rng(Bc + U)
    H = crandn(g, 2, U, 2 * Bc)
    S = crandn(g, 2, 2, U)
    X = oracle.precode(H, S, [Bc, Bc], 3000, rho=1.0)
    for c in range(2):
        Zo = oracle.zf(H, S, rows=(c * Bc, Bc))
        for f in range(2):
            Hdl = np.conj(H[f, :, c * Bc:(c + 1) * Bc])       # H^dl_c = (H^ul_c)^H, U x Bc
            for n in range(2):
                zf = np.linalg.pinv(Hdl) @ S[f, n]
                np.testing.assert_allclose(Zo[f, n], zf, rtol=1e-10)
                np.testing.assert_allclose(Hdl @ zf, S[f, n], rtol=1e-10)
                ref = zf / np.linalg.norm(zf) / np.sqrt(2)
                np.testing.assert_allclose(X[f, n, c * Bc:(c + 1) * Bc], ref, rtol=1e-8, atol=1e-10)


def test_precode_single_user_is_matched_filter(oracle):
    """U = 1: one projection makes hbar^H x = sbar exactly, so x is parallel to h (conjugate beamforming)."""
    g = np.random.default_rng(8)
    H = crandn(g, 1, 1, 12)
    S = crandn(g, 1, 2, 1)
    X = oracle.precode(H, S, [12], 4, rho=1.0)
    for n in range(2):
        ref = H[0, 0] * S[0, n, 0]
        np.testing.assert_allclose(X[0, n], ref / np.linalg.norm(ref), rtol=1e-13)


# ------------------------------------------------------------------------------------------
# ML floor
# ------------------------------------------------------------------------------------------
def test_ml_matches_python_brute_force(oracle):
    g = np.random.default_rng(41)
    pts, _, _ = wl.qam(4)
    U, B = 3, 6
    H = crandn(g, 5, U, B)
    Y = crandn(g, 5, B)
    lab = oracle.ml(H, Y, pts)
    for v in range(5):
        best = min(itertools.product(range(4), repeat=U),
                   key=lambda idx: np.linalg.norm(Y[v] - H[v].T @ pts[list(idx)]))
        assert tuple(lab[v]) == best


def test_ml_error_rate_is_a_floor_for_cd(oracle):
    """Exhaustive ML on tiny QPSK systems makes no more bit errors than decentralized CD."""
    n_vec, U, B = 1500, 3, 8
    d = wl.uplink(77, n_vec, 1, B, U, snr_db=4.0, M=4)
    pts, _, _ = wl.qam(4)
    ml_lab = oracle.ml(d["H"], d["Y"][:, 0], pts)
    Xhat, _, _ = oracle.detect(d["H"], d["Y"], d["N0"], [4, 4], 3)
    cd_lab, _ = wl.hard_decision(Xhat[:, 0], 4)
    e_ml = wl.bit_errors(ml_lab, d["labels"][:, 0])
    e_cd = wl.bit_errors(cd_lab, d["labels"][:, 0])
    assert e_ml > 0 and e_ml <= e_cd


def test_decentralized_cd_snr_loss_is_small(oracle):
    """Qualitative check of Sec. V (U = 8, B_c = 32, C = 4, 16-QAM, K = 3): near BER 1e-3 the
    decentralized CD detector needs less than 2 dB more SNR than the centralized L-MMSE (1)
    (the paper reports about 1 dB; its fusion and slicing details are not given)."""
    nb = 400 * 4 * 8 * 4
    d5 = wl.uplink(5, 400, 4, 128, 8, snr_db=5.0, M=16)
    e_mm = wl.bit_errors(wl.hard_decision(oracle.lmmse(d5["H"], d5["Y"], d5["N0"]), 16)[0], d5["labels"])
    d7 = wl.uplink(5, 400, 4, 128, 8, snr_db=7.0, M=16)
    Xhat, _, _ = oracle.detect(d7["H"], d7["Y"], d7["N0"], [32] * 4, 3)
    e_cd = wl.bit_errors(wl.hard_decision(Xhat, 16)[0], d7["labels"])
    assert 3e-4 < e_mm / nb < 3e-3
    assert e_cd <= e_mm
