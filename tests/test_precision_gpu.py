"""Reduced-precision storage: error of the 16-bit detection path against the FP64 oracle run on the
unquantized inputs, per SNR and K (config-3 shape: B = 256 in 8 x 32, U = 32, 64-QAM, 14 symbols).

This is the total error of storing H and y in fp16 / bf16 (with per-subcarrier scales) and
computing in FP32.  Asserted: the median relative L2 error per vector stays below a per-type bound
of the order of that type's unit roundoff times the conditioning (BOUNDS below), and the hard-decision
BER stays within 5% (plus 1e-4) of the oracle's; set CDMIMO_REPORT_DIR to write the per-SNR table as
JSON.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1902_08653_gb300 import cdmimo
from paper_1902_08653_gb300 import workload as wl

from _util import rel_l2

pytestmark = pytest.mark.gpu

BOUNDS = {"c64": 1e-5, "f16": 2e-3, "bf16": 2e-2}  # median relative L2 error per estimate vector


def test_precision_per_snr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    snrs = np.arange(0, 31, 5, dtype=float)
    per = 12
    n_sc, n_sym, B, U, cs, M = per * len(snrs), 14, 256, 32, [32] * 8, 64
    d = wl.uplink(31415, n_sc, n_sym, B, U, snr_db=np.repeat(snrs, per), M=M)
    N0 = d["N0"].astype(np.float32)
    report = {}
    for K in (3, 5):
        ref, _, _ = orc.detect(d["H"], d["Y"], N0.astype(np.float64), cs, K, threads=8)  # FP64, unquantized
        lab_ref, _ = wl.hard_decision(ref, M)
        for kind in ("c64", "f16", "bf16"):
            if kind == "c64":
                Ht = torch.from_numpy(wl.as_c64(d["H"])[0]).to(dev)
                Yt = torch.from_numpy(wl.as_c64(d["Y"])[0]).to(dev)
                sH = sY = None
            else:
                tdt = torch.float16 if kind == "f16" else torch.bfloat16
                qH, sHn, _ = wl.quantize_c16(d["H"], kind)
                qY, sYn, _ = wl.quantize_c16(d["Y"], kind)
                Ht = torch.from_numpy(qH.view(np.int16)).to(dev).view(tdt)
                Yt = torch.from_numpy(qY.view(np.int16)).to(dev).view(tdt)
                sH, sY = torch.from_numpy(sHn).to(dev), torch.from_numpy(sYn).to(dev)
            X = cdmimo.detect(Ht, Yt, torch.from_numpy(N0).to(dev), cs, K, h_scale=sH, y_scale=sY).cpu().numpy()
            e = rel_l2(X, ref)
            lab, _ = wl.hard_decision(X, M)
            row = {}
            for i, s in enumerate(snrs):
                sel = slice(i * per, (i + 1) * per)
                nb = lab[sel].size * 6
                row[f"{int(s)}dB"] = {
                    "rel_l2_median": float(np.median(e[sel])), "rel_l2_max": float(np.max(e[sel])),
                    "ber": wl.bit_errors(lab[sel], d["labels"][sel]) / nb,
                    "ber_fp64": wl.bit_errors(lab_ref[sel], d["labels"][sel]) / nb}
            report[f"{kind}_K{K}"] = row
            assert np.median(e) < BOUNDS[kind], (kind, K, float(np.median(e)))
            # decisions: the 16-bit path may flip only decisions the FP64 result itself places near a
            # threshold; overall BER within 5% (relative) + 1e-4 of the FP64 oracle's
            ber = wl.bit_errors(lab, d["labels"]) / (lab.size * 6)
            ber_ref = wl.bit_errors(lab_ref, d["labels"]) / (lab.size * 6)
            assert abs(ber - ber_ref) <= 0.05 * ber_ref + 1e-4, (kind, K, ber, ber_ref)
    out = os.environ.get("CDMIMO_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_report.json"), "w") as f:
            json.dump(report, f, indent=1)
