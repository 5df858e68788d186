"""The seeded input generator and the 16-bit storage format (CPU only)."""
import numpy as np
import pytest
import torch

from paper_1902_08653_gb300 import workload as wl


@pytest.mark.parametrize("M", [4, 16, 64])
def test_qam_unit_energy_and_gray_labels(M):
    pts, L, scale = wl.qam(M)
    assert pts.size == M and len(set(np.round(pts, 12))) == M
    np.testing.assert_allclose(np.mean(np.abs(pts) ** 2), 1.0, rtol=1e-14)
    # Gray labelling: nearest neighbours (distance 2*scale) differ in exactly one bit.
    for a in range(M):
        for b in range(M):
            if abs(abs(pts[a] - pts[b]) - 2 * scale) < 1e-12:
                assert bin(a ^ b).count("1") == 1
    lab, margin = wl.hard_decision(pts, M)
    np.testing.assert_array_equal(lab, np.arange(M))
    np.testing.assert_allclose(margin, scale, rtol=1e-12)


def test_hard_decision_noisy_points():
    g = np.random.default_rng(0)
    pts, _, scale = wl.qam(16)
    lab = g.integers(0, 16, 1000)
    x = pts[lab] + (g.uniform(-0.9, 0.9, 1000) + 1j * g.uniform(-0.9, 0.9, 1000)) * scale
    got, _ = wl.hard_decision(x, 16)
    np.testing.assert_array_equal(got, lab)
    assert wl.bit_errors(got, lab) == 0
    assert wl.bit_errors(np.array([0b1010]), np.array([0b0110])) == 2


def test_uplink_statistics_and_model():
    d = wl.uplink(1, 64, 14, 64, 8, snr_db=10.0, M=16)
    H, X, Y, N0 = d["H"], d["X"], d["Y"], d["N0"]
    assert H.shape == (64, 8, 64) and Y.shape == (64, 14, 64) and X.shape == (64, 14, 8)
    assert abs(np.mean(np.abs(H) ** 2) - 1.0) < 0.02
    assert abs(np.mean(H)) < 0.02
    noise = Y - np.einsum("fub,fnu->fnb", H, X)
    np.testing.assert_allclose(N0, 8 * 10 ** -1.0)
    assert abs(np.mean(np.abs(noise) ** 2) / N0[0] - 1.0) < 0.03
    # SNR = U Ex / N0 per receive antenna
    snr = np.mean(np.abs(Y - noise) ** 2) / np.mean(np.abs(noise) ** 2)
    assert abs(10 * np.log10(snr) - 10.0) < 0.2
    d2 = wl.uplink(1, 64, 14, 64, 8, snr_db=10.0, M=16)
    np.testing.assert_array_equal(d2["Y"], Y)


def test_sweep_snr_and_partition():
    s = wl.sweep_snr(10)
    np.testing.assert_array_equal(s, [0, 5, 10, 15, 20, 25, 30, 0, 5, 10])
    assert wl.partition(256, 8) == [32] * 8
    with pytest.raises(ValueError):
        wl.partition(10, 3)


def test_bf16_rounding_matches_torch():
    g = np.random.default_rng(2)
    x = (g.standard_normal(4096) * np.exp(g.uniform(-20, 20, 4096))).astype(np.float32)
    ours = wl.f32_to_bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    np.testing.assert_array_equal(wl.bf16_bits_to_f32(ours), torch.from_numpy(x).to(torch.bfloat16).float().numpy())


@pytest.mark.parametrize("kind,eps", [("f16", 2 ** -11), ("bf16", 2 ** -8)])
def test_quantize_c16(kind, eps):
    d = wl.uplink(4, 6, 2, 32, 4)
    q, scale, deq = wl.quantize_c16(d["H"], kind)
    assert q.shape == d["H"].shape + (2,) and q.dtype == np.uint16 and scale.dtype == np.float32
    rel = np.abs(deq - d["H"]) / np.maximum(np.abs(d["H"]), 1e-3)
    assert np.max(rel) < 2 * eps
    np.testing.assert_allclose(np.sqrt(np.mean(np.abs(d["H"].reshape(6, -1)) ** 2, axis=1)), scale, rtol=1e-6)


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 published with the algorithm's reference
    implementation (Salmon et al., SC 2011)."""
    f = 0xFFFFFFFF
    cases = [((0, 0, 0, 0, 0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((f, f, f, f, f, f), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for args, want in cases:
        got = wl.philox4x32_10(*[[a] for a in args])
        assert tuple(int(w[0]) for w in got) == want


def test_philox_uplink_statistics():
    d = wl.philox_uplink(123, 64, 4, 64, 8, snr_db=10.0, M=16)
    assert abs(np.mean(np.abs(d["H"]) ** 2) - 1) < 0.03 and abs(np.mean(d["H"])) < 0.03
    assert np.all((d["labels"] >= 0) & (d["labels"] < 16))
    assert abs(np.mean(np.abs(d["noise"]) ** 2) / d["N0"][0] - 1) < 0.05
    hist = np.bincount(d["labels"].ravel(), minlength=16) / d["labels"].size
    assert np.all(np.abs(hist - 1 / 16) < 0.02)
