"""bench.py's per-form tables cover every evaluation form the library reports (cdmimo_selected_form:
residual, gram, gram_tc), so that a step that runs any of them can be reported; and the algorithmic
counts restate the forms' definitions at the config-2 shape."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1902_08653_gb300 import cdmimo  # noqa: E402


def test_every_reported_form_has_kernels_and_flops():
    for form in cdmimo.FORM:
        if form == "auto":
            continue  # never reported: the query resolves it
        assert form in bench.KERNELS and len(bench.KERNELS[form]) == 2, form
        assert form in bench.FLOP_PER_VEC and bench.FLOP_PER_VEC[form] > 0, form
    assert set(bench.FRAME_KERNELS) <= set(cdmimo.FORM)
    names = {n for pair in bench.KERNELS.values() for n in pair} | set(bench.FRAME_KERNELS.values())
    assert set(bench.NCU_TRAFFIC) <= names


def test_algorithmic_counts_at_config2():
    U, B, C, K, n_sym = bench.U, bench.B, bench.C, bench.K, bench.N_SYM
    assert (U, B, C, K, n_sym) == (16, 256, 8, 3, 14)
    # residual form: 2 K U B complex MACs per vector, 8 flop each
    assert bench.FLOP_PER_VEC["residual"] == 2 * K * U * B * 8
    # Gram form per vector: K C U^2 (sweeps) + U B (z or H w) + C U (U + 1) / 2 B_c / n_sym (Hermitian G_c)
    g = K * C * U * U + U * B + C * U * (U + 1) / 2 * (B // C) / n_sym
    assert bench.FLOP_PER_VEC["gram"] == pytest.approx(8 * g)
    assert bench.FLOP_PER_VEC["gram_tc"] == bench.FLOP_PER_VEC["gram"]
    # frame: both directions' sweeps and z / H w, one G_c
    assert bench.FRAME_FLOP_PER_VEC["gram"] == pytest.approx(8 * (2 * K * C * U * U + 2 * U * B + (g - K * C * U * U - U * B)))
    # algorithmic bytes: H once per subcarrier (shared by its symbols), y in, xhat out (uplink)
    assert bench.UL_BYTES_PER_VEC == pytest.approx(U * B * 8 / n_sym + B * 8 + U * 8)
    assert bench.FRAME_BYTES_PER_VEC == pytest.approx(U * B * 8 / n_sym + 2 * (B * 8 + U * 8))
