"""Train and evaluate the learned deep-unfolded CD detector on device-generated channels.

    python -m paper_1902_08653_gb300.train_learned --channels 1000000 --out learned.ckpt

Training data: seeded synthetic uplink batches from cdmimo_synth_uplink (B = 256 antennas in C = 8
clusters of 32, U = 16, 16-QAM, one OFDM symbol per channel, SNR uniform in [0, 30] dB).  Target:
the centralized L-MMSE estimate of Eq. (1), computed by the library's own CD with one cluster of
all B antennas and K_target sweeps (Gauss-Seidel on the well-conditioned normal equations converges
to the solve; a GPU test checks it against the oracle's Cholesky solution).  Loss: mean squared
error to the target.  Optimizer: Adam with a cosine learning-rate decay.  All arithmetic runs in
the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import cdmimo
from .learned import LearnedCD


def snr_batch(seed, n, lo=0.0, hi=30.0):
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), 7])))
    return g.uniform(lo, hi, n).astype(np.float32)


def batch(seed, n_sc, B, U, device, snr=None, target_K=32, n_sym=1):
    snr = snr_batch(seed, n_sc) if snr is None else np.asarray(snr, np.float32)
    d = cdmimo.synth_uplink(seed, n_sc, n_sym, B, U, torch.from_numpy(snr).to(device), M=16, device=device)
    d["target"] = cdmimo.detect(d["H"], d["Y"], d["N0"], [B], target_K, fuse="equal")
    d["snr"] = snr
    return d


def train(K=2, U=16, B=256, C=8, hidden=64, channels=1_000_000, batch_size=4096, lr=3e-3, seed=20190222,
          target_K=32, device="cuda", log=None):
    dev = torch.device(device)
    cs = [B // C] * C
    model = LearnedCD(K, U, hidden, seed=seed, device=dev)
    steps = max(1, channels // batch_size)
    ws = torch.empty(cdmimo.learned_workspace_size(batch_size, 1, B, U, cs, K, hidden), dtype=torch.uint8, device=dev)
    hist = []
    t0 = time.perf_counter()
    for it in range(steps):
        d = batch(seed * 7919 + it, batch_size, B, U, dev, target_K=target_K)
        lr_t = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * it / steps)))
        loss = model.train_step(d["H"], d["Y"], d["N0"], d["target"], cs, lr=lr_t, workspace=ws)
        if it % max(1, steps // 20) == 0 or it == steps - 1:
            hist.append((it, float(loss.item())))
            if log:
                log(f"step {it}/{steps} loss {hist[-1][1]:.5f}")
    torch.cuda.synchronize()
    return model, {"steps": steps, "channels": steps * batch_size, "batch": batch_size, "lr": lr,
                   "wall_s": time.perf_counter() - t0, "loss": hist}


def evaluate(model, B=256, C=8, seed=987654321, n_sc=4096, snrs=(0, 5, 10, 15, 20, 25, 30), plain_K=(2, 3, 5),
             device="cuda", target_K=32):
    """MSE per user against the centralized L-MMSE on held-out channels, per SNR, for the learned
    model and for plain CD (COLNORM fusion) with several sweep counts."""
    dev = torch.device(device)
    cs = [B // C] * C
    out = {"learned": {}, **{f"plain_K{k}": {} for k in plain_K}}
    for s in snrs:
        d = batch(seed + int(s), n_sc, B, model.U, dev, snr=np.full(n_sc, s, np.float32), target_K=target_K)
        mse = lambda x: float(torch.mean(torch.abs(x - d["target"]) ** 2).item())
        out["learned"][f"{s}dB"] = mse(model.detect(d["H"], d["Y"], d["N0"], cs))
        for k in plain_K:
            out[f"plain_K{k}"][f"{s}dB"] = mse(cdmimo.detect(d["H"], d["Y"], d["N0"], cs, k, fuse="colnorm"))
    for key in list(out):
        out[key]["mean"] = float(np.mean([v for k2, v in out[key].items()]))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--channels", type=int, default=1_000_000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--K", type=int, default=2)
    ap.add_argument("--hidden", type=int, default=64)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=20190222)
    ap.add_argument("--out", default="learned_cd.ckpt")
    ap.add_argument("--report", default=None)
    args = ap.parse_args()
    model, info = train(K=args.K, hidden=args.hidden, channels=args.channels, batch_size=args.batch, lr=args.lr,
                        seed=args.seed, log=print)
    model.save(args.out)
    rep = {"train": info, "eval_mse_vs_mmse": evaluate(model)}
    print(json.dumps(rep))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
