#!/usr/bin/env python3
"""Throughput benchmark of the decentralized CD hot path on GB300.

Workload (one "step"): uplink CD detection with feedforward fusion (Algorithm 1, Sec. III) followed
by downlink CD ZF precoding with per-cluster power normalization (Algorithm 2, Sec. IV-B), over one
batch of 1200 subcarriers x 14 OFDM symbols, B = 256 antennas in C = 8 clusters of 32, U = 16 users,
K = 3 sweeps, i.i.d. CN(0,1) channels fixed per subcarrier, 16-QAM, SNR swept 0..30 dB across
subcarriers.  Inputs are resident in HBM; L2 is flushed (256 MB write) between timed steps, outside
the timed brackets.  value = vectors (subcarrier-symbol pairs, each detected and precoded) per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload (the oracle is the reference implementation of this path).  Under torchrun (N > 1) every
rank runs its own batch (weak scaling, no collective on the data path) and rank 0 prints one JSON
line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "detected vectors/s & Gb/s at B=256,U=16,C=8,K=3; % HBM roofline; MSE vs MMSE"
N_SC, N_SYM, B, U, C, K, M = 1200, 14, 256, 16, 8, 3, 16
CS = [B // C] * C
BITS = U * 4  # 16-QAM bits per vector
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# FP32 ALU peak (FFMA = 2 flop): SMs x FP32 lanes per SM x 2 x max SM clock.
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
# Algorithmic work per vector, residual-form CD (SURVEY / DESIGN): 2 K U B complex MACs x 8 flop.
FLOP_PER_VEC = 2 * K * U * B * 8
# Algorithmic HBM bytes per vector: uplink H/14 + y + xhat; downlink H/14 + s + x.
UL_BYTES_PER_VEC = U * B * 8 / N_SYM + B * 8 + U * 8
DL_BYTES_PER_VEC = U * B * 8 / N_SYM + U * 8 + B * 8
# DRAM traffic per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) for the
# kernel version named in the key; None until a capture of the current kernel exists.
NCU_TRAFFIC = {}

WORKLOAD = ("UL CD detect + fusion, then DL CD ZF precode + normalization; B=256 (C=8 x 32), U=16, "
            "K=3, 1200 subcarriers x 14 OFDM symbols, i.i.d. CN(0,1), 16-QAM, SNR sweep 0-30 dB")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def make_inputs(seed):
    from paper_1902_08653_gb300 import workload as wl

    up = wl.uplink(seed, N_SC, N_SYM, B, U, snr_db=wl.sweep_snr(N_SC), M=M)
    dl = wl.downlink(seed, N_SC, N_SYM, B, U, M=M)
    return up, dl


def mse_vs_mmse(up, Xhat):
    """Mean ||xhat - x_MMSE||^2 / U per SNR point, x_MMSE the centralized L-MMSE of Eq. (1)
    (library solve in FP64 on the host, evaluation only)."""
    H = up["H"]
    A = np.einsum("fub,fvb->fuv", np.conj(H), H) + up["N0"][:, None, None] * np.eye(U)[None]
    Z = np.einsum("fub,fnb->fun", np.conj(H), up["Y"])
    Xm = np.linalg.solve(A, Z).transpose(0, 2, 1)
    err = np.sum(np.abs(Xhat - Xm) ** 2, axis=-1) / U
    out = {}
    for s in np.unique(up["snr_db"]):
        out[f"{int(s)}dB"] = float(np.mean(err[up["snr_db"] == s]))
    from paper_1902_08653_gb300 import workload as wl

    ber = {}
    for s in np.unique(up["snr_db"]):
        sel = up["snr_db"] == s
        lab, _ = wl.hard_decision(Xhat[sel], M)
        ber[f"{int(s)}dB"] = wl.bit_errors(lab, up["labels"][sel]) / (lab.size * 4)
    return out, ber


def run_cuda(args, rank, world, local_rank):
    import torch

    from paper_1902_08653_gb300 import cdmimo
    from paper_1902_08653_gb300 import workload as wl

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cdmimo.lib()
    up, dl = make_inputs(20190222 + rank)
    H = torch.from_numpy(wl.as_c64(up["H"])[0]).to(dev)
    Y = torch.from_numpy(wl.as_c64(up["Y"])[0]).to(dev)
    N0 = torch.from_numpy(up["N0"].astype(np.float32)).to(dev)
    Hd = torch.from_numpy(wl.as_c64(dl["H"])[0]).to(dev)
    S = torch.from_numpy(wl.as_c64(dl["S"])[0]).to(dev)
    Xhat = torch.empty((N_SC, N_SYM, U), dtype=torch.complex64, device=dev)
    Xdl = torch.empty((N_SC, N_SYM, B), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        cdmimo.detect(H, Y, N0, CS, K, out=Xhat, stream=stream)
        cdmimo.precode(Hd, S, CS, K, out=Xdl, stream=stream)

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    cdmimo.device_status(clear=True)

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local_rank)
    if rank == 0:
        sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        e = ev[i]
        e[0].record(stream)
        cdmimo.detect(H, Y, N0, CS, K, out=Xhat, stream=stream)
        e[1].record(stream)
        cdmimo.precode(Hd, S, CS, K, out=Xdl, stream=stream)
        e[2].record(stream)
        flush.fill_(float(i & 7))  # L2 flush between timed steps, outside the brackets
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop() if rank == 0 else None
    t_ul = [ev[i][0].elapsed_time(ev[i][1]) for i in range(args.steps)]
    t_dl = [ev[i][1].elapsed_time(ev[i][2]) for i in range(args.steps)]
    dev_ms = float(np.sum(t_ul) + np.sum(t_dl))
    st = cdmimo.device_status(clear=True)
    if st != 0:
        raise RuntimeError(f"device status {st:#x} after the timed loop")

    if world > 1:
        t = torch.tensor([dev_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_ms = float(t.item())

    # End to end: host (pinned) buffers through the C ABI, copies inside the timed region.
    Hh = torch.from_numpy(wl.as_c64(up["H"])[0]).pin_memory()
    Yh = torch.from_numpy(wl.as_c64(up["Y"])[0]).pin_memory()
    N0h = torch.from_numpy(up["N0"].astype(np.float32)).pin_memory()
    Hdh = torch.from_numpy(wl.as_c64(dl["H"])[0]).pin_memory()
    Sh = torch.from_numpy(wl.as_c64(dl["S"])[0]).pin_memory()
    Xh = torch.empty((N_SC, N_SYM, U), dtype=torch.complex64).pin_memory()
    Xdh = torch.empty((N_SC, N_SYM, B), dtype=torch.complex64).pin_memory()
    ws_ul = torch.empty(cdmimo.host_workspace_size(cdmimo.OP_DETECT, N_SC, N_SYM, B, U, CS, K), dtype=torch.uint8,
                        device=dev)
    ws_dl = torch.empty(cdmimo.host_workspace_size(cdmimo.OP_PRECODE, N_SC, N_SYM, B, U, CS, K), dtype=torch.uint8,
                        device=dev)
    e2e_steps = max(3, min(50, args.steps))
    for _ in range(2):
        cdmimo.detect_host(Hh, Yh, N0h, CS, K, Xh, ws_ul, stream=stream)
        cdmimo.precode_host(Hdh, Sh, CS, K, Xdh, ws_dl, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        cdmimo.detect_host(Hh, Yh, N0h, CS, K, Xh, ws_ul, stream=stream)
        cdmimo.precode_host(Hdh, Sh, CS, K, Xdh, ws_dl, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    h2d = (Hh.numel() * 8 + Yh.numel() * 8 + N0h.numel() * 4) + (Hdh.numel() * 8 + Sh.numel() * 8)
    d2h = Xh.numel() * 8 + Xdh.numel() * 8

    if rank != 0:
        return None
    mse, ber = mse_vs_mmse(up, Xh.numpy().astype(np.complex128))
    hbm_peak, peak_src = load_peaks()
    ms_step = dev_ms / args.steps
    vec_step = N_SC * N_SYM
    value = world * vec_step / (ms_step * 1e-3)
    ul_ms = float(np.mean(t_ul))
    dl_ms = float(np.mean(t_dl))
    dom_ms, dom_name = (ul_ms, "cd_detect_kernel") if ul_ms >= dl_ms else (dl_ms, "cd_precode_kernel")
    achieved_tflops = FLOP_PER_VEC * vec_step / (dom_ms * 1e-3) / 1e12
    dom_bytes = (UL_BYTES_PER_VEC if dom_name == "cd_detect_kernel" else DL_BYTES_PER_VEC) * vec_step
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "vectors/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded i.i.d. Rayleigh, 16-QAM, AWGN)",
        "config": {"workload": WORKLOAD, "n_sc": N_SC, "n_sym": N_SYM, "B": B, "C": C, "B_c": B // C, "U": U, "K": K,
                   "fusion": "colnorm", "qam": M, "l2": "flushed between timed steps (256 MB write, untimed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "gbps": value * BITS / 1e9,
        "ul": {"ms": ul_ms, "vectors_per_s": world * vec_step / (ul_ms * 1e-3),
               "gbps": world * vec_step * BITS / (ul_ms * 1e-3) / 1e9,
               "hbm_frac": UL_BYTES_PER_VEC * vec_step / (ul_ms * 1e-3) / 1e9 / hbm_peak,
               "fp32_frac": FLOP_PER_VEC * vec_step / (ul_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS},
        "dl": {"ms": dl_ms, "vectors_per_s": world * vec_step / (dl_ms * 1e-3),
               "gbps": world * vec_step * BITS / (dl_ms * 1e-3) / 1e9,
               "hbm_frac": DL_BYTES_PER_VEC * vec_step / (dl_ms * 1e-3) / 1e9 / hbm_peak,
               "fp32_frac": FLOP_PER_VEC * vec_step / (dl_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS},
        "roofline": {"bound": "alu", "kernel": dom_name, "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved_tflops / FP32_PEAK_TFLOPS,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                     "hbm": {"achieved_gbs": dom_bytes / (dom_ms * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                             "frac": dom_bytes / (dom_ms * 1e-3) / 1e9 / hbm_peak, "peak_source": peak_src},
                     "traffic": NCU_TRAFFIC.get(dom_name)},
        "mse_vs_mmse": mse,
        "ber": ber,
        "e2e": {"value": world * vec_step / (e2e_ms * 1e-3), "unit": "vectors/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "wall_s": wall,
    }
    line["cpu_baseline"] = cpu_baseline(up, dl) if world == 1 else None
    return line


def cpu_baseline(up, dl, min_seconds=10.0, threads=None):
    """The FP64 oracle as it stands, on the host cores: the whole batch (UL detect + DL precode),
    repeated until about `min_seconds` of wall time have been spent."""
    import oracle

    oracle.build()
    threads = threads or os.cpu_count() or 1
    reps = 0
    t0 = time.perf_counter()
    while True:
        oracle.detect(up["H"], up["Y"], up["N0"], CS, K, threads=threads)
        oracle.precode(dl["H"], dl["S"], CS, K, threads=threads)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds or reps >= 500:
            break
    return {"value": reps * N_SC * N_SYM / dt, "unit": "vectors/s", "cores": threads, "kind": "oracle",
            "sample": f"{reps} x the full batch ({N_SC} subcarriers x {N_SYM} symbols, UL detect + DL precode), "
                      f"{dt:.1f} s wall on {threads} threads"}


def run_reference(args):
    import oracle

    oracle.build()
    up, dl = make_inputs(20190222)
    threads = os.cpu_count() or 1
    n_sub = 120
    for _ in range(args.warmup):
        oracle.detect(up["H"][:8], up["Y"][:8], up["N0"][:8], CS, K, threads=threads)
    times = []
    for i in range(args.steps):
        f0 = (i * n_sub) % N_SC
        sl = slice(f0, f0 + n_sub)
        t0 = time.perf_counter()
        oracle.detect(up["H"][sl], up["Y"][sl], up["N0"][sl], CS, K, threads=threads)
        oracle.precode(dl["H"][sl], dl["S"][sl], CS, K, threads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = n_sub * N_SYM / (ms * 1e-3)
    sample = f"{n_sub} subcarriers x {N_SYM} symbols per step (UL detect + DL precode), FP64 C oracle"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "vectors/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded i.i.d. Rayleigh)",
            "config": {"workload": WORKLOAD, "n_sc": N_SC, "n_sym": N_SYM, "B": B, "C": C, "U": U, "K": K},
            "cpu_baseline": {"value": value, "unit": "vectors/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line = run_cuda(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
