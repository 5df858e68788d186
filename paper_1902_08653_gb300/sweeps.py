"""BER and MSE against SNR for decentralized CD detection and precoding (the shape of the paper's
Sec. V study, on seeded synthetic Rayleigh channels).

    python -m paper_1902_08653_gb300.sweeps --C 4 8 --out sweeps.json

Uplink, per SNR point: decentralized CD (C clusters of B_c antennas, K sweeps, COLNORM fusion),
centralized CD (one cluster of B antennas, i.e. Algorithm 1 with C = 1), and two host-side
comparators evaluated in FP64: the centralized L-MMSE estimate of Eq. (1) and the matched filter
x_u = h_u^H y / ||h_u||^2.  Reported: uncoded BER against the transmitted bits (Gray QAM, nearest-
point slicing) and the MSE to the centralized L-MMSE estimate.

Downlink, per SNR point: decentralized CD precoding (Algorithm 2 + per-cluster normalization), and
as host comparators centralized ZF x = H (H^H H)^{-1} s and matched-filter precoding x = H s, both
normalized to the total power.  Each user receives r_u = h_u^H x + n_u; the noise variance sets the
SNR against the mean received signal power of the subcarrier, and the user divides by the
noise-free gain g_u = mean_n (h_u^H x)_n / s_{u,n} of its subcarrier before slicing (the paper does
not say how a user scales its sample; this genie gain is the library's reading, evaluation only).

The CD estimates come from the library's kernels; only the comparators and the channel model run
on the host.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import cdmimo
from . import workload as wl


def _lmmse(H, Y, N0):
    """Centralized L-MMSE of Eq. (1): (H^H H + N0 I)^{-1} H^H y per subcarrier (Ex = 1), FP64."""
    U = H.shape[1]
    A = np.einsum("fub,fvb->fuv", np.conj(H), H) + N0[:, None, None] * np.eye(U)[None]
    Z = np.einsum("fub,fnb->fun", np.conj(H), Y)
    return np.linalg.solve(A, Z).transpose(0, 2, 1)


def _mf(H, Y):
    """Matched filter: x_u = h_u^H y / ||h_u||^2."""
    e = np.sum(np.abs(H) ** 2, axis=2)  # [f][u]
    return np.einsum("fub,fnb->fnu", np.conj(H), Y) / e[:, None, :]


def _ber(X, labels, M):
    lab, _ = wl.hard_decision(X, M)
    return wl.bit_errors(lab, labels) / (lab.size * int(np.log2(M)))


def uplink_sweep(snrs=(0, 4, 8, 12, 16, 20), U=8, Bc=32, C=4, K_list=(1, 2, 3, 5), n_sc=256, n_sym=14, M=16,
                 seed=20190222, device="cuda"):
    dev = torch.device(device)
    B = Bc * C
    out = {"U": U, "B": B, "C": C, "B_c": Bc, "M": M, "n_vectors": n_sc * n_sym, "snr_db": list(snrs), "ber": {},
           "mse_vs_lmmse": {}}

    def put(name, s, X, d, Xm):
        out["ber"].setdefault(name, []).append(_ber(X, d["labels"], M))
        out["mse_vs_lmmse"].setdefault(name, []).append(float(np.mean(np.sum(np.abs(X - Xm) ** 2, -1) / U)))

    for i, s in enumerate(snrs):
        d = wl.uplink(seed + 101 * i, n_sc, n_sym, B, U, snr_db=float(s), M=M)
        H32, H64 = wl.as_c64(d["H"])
        Y32, Y64 = wl.as_c64(d["Y"])
        N0 = d["N0"].astype(np.float32)
        Ht, Yt, Nt = (torch.from_numpy(a).to(dev) for a in (H32, Y32, N0))
        Xm = _lmmse(H64, Y64, N0.astype(np.float64))
        put("lmmse_centralized", s, Xm, d, Xm)
        put("mf", s, _mf(H64, Y64), d, Xm)
        for K in K_list:
            X = cdmimo.detect(Ht, Yt, Nt, [Bc] * C, K).cpu().numpy().astype(np.complex128)
            put(f"cd_decentralized_K{K}", s, X, d, Xm)
            X = cdmimo.detect(Ht, Yt, Nt, [B], K).cpu().numpy().astype(np.complex128)
            put(f"cd_centralized_K{K}", s, X, d, Xm)
    return out


def _dl_ber(H, X, S, labels, M, snr_db, g):
    """BER of the users' sliced samples r = H^dl x + n, with H^dl = H^H, the noise set against the
    subcarrier's mean received signal power, and the genie gain of the module docstring."""
    R0 = np.einsum("fub,fnb->fnu", np.conj(H), X)  # noise-free received samples [f][n][u]
    p = np.mean(np.abs(R0) ** 2, axis=(1, 2))
    n0 = p * 10.0 ** (-snr_db / 10.0)
    noise = (g.standard_normal(R0.shape) + 1j * g.standard_normal(R0.shape)) * np.sqrt(n0 / 2)[:, None, None]
    gain = np.mean(R0 / S, axis=1, keepdims=True)
    return _ber((R0 + noise) / gain, labels, M)


def downlink_sweep(snrs=(0, 4, 8, 12, 16, 20), U=8, Bc=32, C=4, K_list=(1, 2, 3, 5), n_sc=256, n_sym=14, M=16,
                   seed=20190222, device="cuda"):
    dev = torch.device(device)
    B = Bc * C
    d = wl.downlink(seed, n_sc, n_sym, B, U, M=M)
    H32, H64 = wl.as_c64(d["H"])
    S32, S64 = wl.as_c64(d["S"])
    Ht, St = torch.from_numpy(H32).to(dev), torch.from_numpy(S32).to(dev)
    Hm = H64.transpose(0, 2, 1)  # [f][b][u]: column u is h_u; user u receives h_u^H x
    W = np.linalg.solve(np.einsum("fub,fvb->fuv", np.conj(H64), H64), S64.transpose(0, 2, 1)).transpose(0, 2, 1)
    Xzf = np.einsum("fbu,fnu->fnb", Hm, W)
    Xmf = np.einsum("fbu,fnu->fnb", Hm, S64)
    norm = lambda X: X / np.linalg.norm(X, axis=-1, keepdims=True)
    schemes = {"zf_centralized": norm(Xzf), "mf": norm(Xmf)}
    for K in K_list:
        schemes[f"cd_decentralized_K{K}"] = cdmimo.precode(Ht, St, [Bc] * C, K).cpu().numpy().astype(np.complex128)
    out = {"U": U, "B": B, "C": C, "B_c": Bc, "M": M, "n_vectors": n_sc * n_sym, "snr_db": list(snrs), "ber": {}}
    for name, X in schemes.items():
        g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 99])))
        out["ber"][name] = [_dl_ber(H64, X, S64, d["labels"], M, float(s), g) for s in snrs]
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--C", type=int, nargs="+", default=[4, 8])
    ap.add_argument("--U", type=int, default=8)
    ap.add_argument("--Bc", type=int, default=32)
    ap.add_argument("--n-sc", type=int, default=256)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    rep = {f"C{C}": {"uplink": uplink_sweep(U=args.U, Bc=args.Bc, C=C, n_sc=args.n_sc),
                     "downlink": downlink_sweep(U=args.U, Bc=args.Bc, C=C, n_sc=args.n_sc)} for C in args.C}
    print(json.dumps(rep))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
