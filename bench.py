#!/usr/bin/env python3
"""Throughput benchmark of the decentralized CD hot path on GB300.

Workload (one "step"): one TDD frame over a batch of 1200 subcarriers x 14 OFDM symbols, B = 256
antennas in C = 8 clusters of 32, U = 16 users, K = 3 sweeps, i.i.d. CN(0,1) channels fixed per
subcarrier, 16-QAM, SNR swept 0..30 dB across subcarriers: uplink CD detection with feedforward
fusion (Algorithm 1, Sec. III) and downlink CD ZF precoding with per-cluster normalization
(Algorithm 2, Sec. IV-B) on the same channel (the downlink channel is the transpose of the uplink
one), through cdmimo_detect_precode.  --step separate times cdmimo_detect and cdmimo_precode on two
independent channels instead.  Inputs are resident in HBM; L2 is flushed (256 MB write) between
timed steps, outside the timed brackets.  value = vectors (subcarrier-symbol pairs, each detected
and precoded) per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference] [--step frame|separate]

--impl reference times the FP64 CPU oracle on the host cores on the same workload, the whole batch
every step (the oracle is the reference implementation of this path).  The default line also
carries a per-pipe roofline of the frame kernel (pipe rates probed on the same GPU) and condensed
runs of configurations 1, 3, 4 and 5 (--no-configs leaves them out).  Under torchrun (N > 1) every
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
# Algorithmic work per vector (8 flop per complex MAC) and direction, by evaluation form:
#   residual (Algorithms 1 and 2 as written): 2 K U B complex MACs;
#   gram: K U^2 per cluster (sweeps) + U B (z = H^H y, or x = H w) + U (U+1)/2 B_c per cluster and
#   subcarrier for the Hermitian G_c, shared by the n_sym symbols (and by both directions of a frame).
GRAM_G = C * (U * (U + 1) // 2) * (B // C) / N_SYM
FLOP_PER_VEC = {"residual": 2 * K * U * B * 8, "gram": 8 * (K * C * U * U + U * B + GRAM_G)}
FLOP_PER_VEC["gram_tc"] = FLOP_PER_VEC["gram_tc_phased"] = FLOP_PER_VEC["gram_tc_umma"] = FLOP_PER_VEC["gram"]  # the same algorithm; its contractions run on the tensor cores
FRAME_FLOP_PER_VEC = {"residual": 2 * FLOP_PER_VEC["residual"], "gram": 8 * (2 * K * C * U * U + 2 * U * B + GRAM_G)}
KERNELS = {"residual": ("cd_detect_pp_kernel", "cd_precode_pp_kernel"),
           "gram": ("cd_detect_gram_kernel", "cd_precode_gram_kernel"),
           "gram_tc": ("cd_frame_ws_kernel<uplink>", "cd_frame_ws_kernel<downlink>"),
           "gram_tc_phased": ("cd_frame_tc_kernel<uplink>", "cd_frame_tc_kernel<downlink>"),
           "gram_tc_umma": ("cd_frame_ws_kernel<uplink>", "cd_frame_ws_kernel<downlink>")}
# One-kernel TDD frames by form: FP32 Gram form, and Gram form with z, G_c and x_c = H_c w on the
# tensor cores (split-TF32 MMAs; the sweeps, K C U^2 of the flops above, stay on the FP32 pipes).
FRAME_KERNELS = {"gram": "cd_frame_gram_kernel", "gram_tc": "cd_frame_ws_kernel",
                 "gram_tc_phased": "cd_frame_tc_kernel", "gram_tc_umma": "cd_frame_ws_kernel"}
# Per-pipe work of the one-kernel frame (Gram form on the tensor cores), per frame vector:
#   FP32 pipes: the Gauss-Seidel sweeps, K U^2 complex MACs per cluster and direction;
#   tensor pipes: z = H_c^H y_c, G_c = H_c^H H_c and x_c = H_c w, algorithmically the rest of
#   FRAME_FLOP_PER_VEC["gram"]; executed as split-TF32 mma.sync m16n8k8 tiles, 288 per cluster and
#   subcarrier at B_c = 32 (phase A: 8 k-steps x 24, phase C: 4 k-steps x 24; 3 MMAs per product,
#   16-row user tiles and 16-column symbol tiles), 2048 flop each.
SWEEP_FLOP_PER_VEC = 2 * 8 * K * C * U * U
CONTRACTION_FLOP_PER_VEC = FRAME_FLOP_PER_VEC["gram"] - SWEEP_FLOP_PER_VEC
MMA_PER_CLUSTER_SUBCARRIER = 288
MMA_FLOP_PER_VEC = C * MMA_PER_CLUSTER_SUBCARRIER * 2048 / N_SYM
# tcgen05 TF32 dense rate implied by the measured cuBLAS bf16 rate and the nominal tf32 / bf16 ratio
TF32_PER_BF16_NOMINAL = 1.1 / 2.25
# Algorithmic HBM bytes per vector: uplink H/14 + y + xhat; downlink H/14 + s + x; frame H/14 once.
UL_BYTES_PER_VEC = U * B * 8 / N_SYM + B * 8 + U * 8
DL_BYTES_PER_VEC = U * B * 8 / N_SYM + U * 8 + B * 8
FRAME_BYTES_PER_VEC = U * B * 8 / N_SYM + B * 8 + U * 8 + U * 8 + B * 8
# DRAM traffic per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum, one capture
# of `python bench.py --profile detect|precode|frame`, see profiles/) for the kernel named in
# the key; a kernel without an entry (or changed since its capture) reports null.  Outputs still in
# L2 when a kernel ends are written back after it, outside the launch.
NCU_TRAFFIC = {"cd_detect_gram_kernel": 73.806592e6 + 0.621568e6,
               "cd_precode_gram_kernel": 41.539072e6 + 0.377088e6,
               "cd_frame_gram_kernel": 76.144896e6 + 4.834560e6,
               "cd_frame_ws_kernel": 75.990016e6 + 5.112064e6}

WORKLOAD = ("TDD frame: UL CD detect + fusion and DL CD ZF precode + normalization on the same channel; "
            "B=256 (C=8 x 32), U=16, K=3, 1200 subcarriers x 14 OFDM symbols, i.i.d. CN(0,1), 16-QAM, "
            "SNR sweep 0-30 dB")
WORKLOAD_SEPARATE = ("UL CD detect + fusion, then DL CD ZF precode + normalization on an independent channel; "
                     "B=256 (C=8 x 32), U=16, K=3, 1200 subcarriers x 14 OFDM symbols, i.i.d. CN(0,1), 16-QAM, "
                     "SNR sweep 0-30 dB")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def measure_pipes(dev, stream):
    """Throughput of the packed-FP32 FMA and TF32 mma.sync pipes on this GPU (cdmimo_pipe_probe:
    eight independent chains per thread or warp on every SM), best of five launches, TFLOP/s."""
    import torch

    from paper_1902_08653_gb300 import cdmimo

    sink = torch.empty(cdmimo.pipe_probe_sink_floats(), dtype=torch.float32, device=dev)
    out = {}
    for name, kind, iters in (("ffma2", cdmimo.PROBE_FFMA2, 4096), ("mma_tf32", cdmimo.PROBE_MMA_TF32, 1024)):
        cdmimo.pipe_probe(kind, 64, sink, stream)
        best = 0.0
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = cdmimo.pipe_probe(kind, iters, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[name] = best
    return out


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


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (each rank's own timing; world 1: x itself)."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(vectors_per_rank, world, max_ms):
    """Weak scaling: every rank processes its own batch; the job's throughput is all ranks' vectors
    over the slowest rank's time."""
    return world * vectors_per_rank / (max_ms * 1e-3)


def rank_seed(rank):
    """Each rank's batch seed (independent synthetic batches, the same shape)."""
    return 20190222 + rank


def bench_config(step, world, scaling="weak"):
    """The line's workload description, the same for the CUDA arm and the reference arm."""
    par = "single GPU"
    if world > 1:
        par = f"subcarrier shards of one batch x{world}" if scaling == "strong" else f"replicas x{world}"
    return {"workload": WORKLOAD if step == "frame" else WORKLOAD_SEPARATE, "step": step, "n_sc": N_SC,
            "n_sym": N_SYM, "B": B, "C": C, "B_c": B // C, "U": U, "K": K, "fusion": "colnorm", "qam": M,
            "l2": "GPU arm: flushed between timed steps (256 MB write, untimed)", "parallelism": par}


def shard_batch(d, lo, hi):
    """The subcarriers [lo, hi) of a workload dict (arrays indexed by subcarrier first)."""
    return {k: (v[lo:hi] if isinstance(v, np.ndarray) and v.ndim >= 1 and v.shape[0] == N_SC else v)
            for k, v in d.items()}


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

    frame = args.step == "frame"
    strong = args.scaling == "strong"
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cdmimo.lib()
    if strong:  # one batch, its subcarriers split over the ranks (no collective on the data path)
        from paper_1902_08653_gb300 import parallel

        lo, hi = parallel.subcarrier_shard(N_SC, world, rank)
        up, dl = (shard_batch(x, lo, hi) for x in make_inputs(rank_seed(0)))
    else:
        up, dl = make_inputs(rank_seed(rank))
    n_loc = up["H"].shape[0]
    t = lambda a: torch.from_numpy(wl.as_c64(a)[0]).to(dev)
    H, Y, S = t(up["H"]), t(up["Y"]), t(dl["S"])
    Hd = H if frame else t(dl["H"])
    N0 = torch.from_numpy(up["N0"].astype(np.float32)).to(dev)
    Xhat = torch.empty((n_loc, N_SYM, U), dtype=torch.complex64, device=dev)
    Xdl = torch.empty((n_loc, N_SYM, B), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def ul():
        cdmimo.detect(H, Y, N0, CS, K, out=Xhat, stream=stream, form=args.form)

    def dl_():
        cdmimo.precode(Hd, S, CS, K, out=Xdl, stream=stream, form=args.form)

    def frm():
        cdmimo.detect_precode(H, Y, N0, S, CS, K, out=Xhat, out_dl=Xdl, stream=stream, form=args.form)

    for _ in range(args.warmup):
        if frame:
            frm()
        else:
            ul()
            dl_()
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
        if frame:
            frm()
            e[1].record(stream)
        else:
            ul()
            e[1].record(stream)
            dl_()
        e[2].record(stream)
        flush.fill_(float(i & 7))  # L2 flush between timed steps, outside the brackets
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop() if rank == 0 else None
    t_a = [ev[i][0].elapsed_time(ev[i][1]) for i in range(args.steps)]
    t_b = [ev[i][1].elapsed_time(ev[i][2]) for i in range(args.steps)]
    dev_ms = float(np.sum(t_a) + np.sum(t_b))
    st = cdmimo.device_status(clear=True)
    if st != 0:
        raise RuntimeError(f"device status {st:#x} after the timed loop")
    dev_ms = max_over_ranks(dev_ms, world, dev)

    # End to end through the public API: every step copies the inputs from pinned host memory to the
    # device and the results back, inside the timed region.  Frame: device buffers + one
    # cdmimo_detect_precode; separate: the host-buffer entry points (copies inside the calls).
    Hh = torch.from_numpy(wl.as_c64(up["H"])[0]).pin_memory()
    Yh = torch.from_numpy(wl.as_c64(up["Y"])[0]).pin_memory()
    N0h = torch.from_numpy(up["N0"].astype(np.float32)).pin_memory()
    Sh = torch.from_numpy(wl.as_c64(dl["S"])[0]).pin_memory()
    Hdh = Hh if frame else torch.from_numpy(wl.as_c64(dl["H"])[0]).pin_memory()
    Xh = torch.empty((n_loc, N_SYM, U), dtype=torch.complex64).pin_memory()
    Xdh = torch.empty((n_loc, N_SYM, B), dtype=torch.complex64).pin_memory()
    if frame:  # cdmimo_detect_precode_host: chunked; uploads, kernels and downloads overlap
        ws_fr = torch.empty(cdmimo.host_workspace_size(cdmimo.OP_FRAME, n_loc, N_SYM, B, U, CS, K), dtype=torch.uint8,
                            device=dev)

        def e2e_step():
            cdmimo.detect_precode_host(Hh, Yh, N0h, Sh, CS, K, Xh, Xdh, ws_fr, n_chunks=args.e2e_chunks,
                                       stream=stream, form=args.form)
    else:
        ws_ul = torch.empty(cdmimo.host_workspace_size(cdmimo.OP_DETECT, n_loc, N_SYM, B, U, CS, K),
                            dtype=torch.uint8, device=dev)
        ws_dl = torch.empty(cdmimo.host_workspace_size(cdmimo.OP_PRECODE, n_loc, N_SYM, B, U, CS, K),
                            dtype=torch.uint8, device=dev)

        def e2e_step():
            cdmimo.detect_host(Hh, Yh, N0h, CS, K, Xh, ws_ul, stream=stream)
            cdmimo.precode_host(Hdh, Sh, CS, K, Xdh, ws_dl, stream=stream)
    e2e_steps = max(3, min(50, args.steps))
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    h2d = Hh.numel() * 8 + Yh.numel() * 8 + N0h.numel() * 4 + Sh.numel() * 8 + (0 if frame else Hdh.numel() * 8)
    d2h = Xh.numel() * 8 + Xdh.numel() * 8

    if rank != 0:
        return None
    mse, ber = mse_vs_mmse(up, Xh.numpy().astype(np.complex128))
    hbm_peak, peak_src = load_peaks()
    ms_step = dev_ms / args.steps
    vec_step = n_loc * N_SYM  # this rank's vectors per step
    value = N_SC * N_SYM / (ms_step * 1e-3) if strong else whole_job_value(vec_step, world, ms_step)
    form_ul = cdmimo.selected_form(cdmimo.OP_DETECT, n_loc, N_SYM, B, U, CS, K, form=args.form, H=H)
    form_dl = cdmimo.selected_form(cdmimo.OP_PRECODE, n_loc, N_SYM, B, U, CS, K, form=args.form, H=Hd)

    def kernel_line(name, form, ms, flop, nbytes):
        return {"kernel": name, "form": form, "ms": ms, "flop_per_vector": flop,
                "fp32_frac": flop * vec_step / (ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                "hbm_frac": nbytes * vec_step / (ms * 1e-3) / 1e9 / hbm_peak}

    if frame:
        form_fr = cdmimo.selected_form(cdmimo.OP_FRAME, n_loc, N_SYM, B, U, CS, K, form=args.form, H=H)
        fused = form_fr in FRAME_KERNELS
        name = FRAME_KERNELS[form_fr] if fused else "+".join(KERNELS[form_ul][:1] + KERNELS[form_dl][1:])
        fl = FRAME_FLOP_PER_VEC["gram"] if fused else FLOP_PER_VEC[form_ul] + FLOP_PER_VEC[form_dl]
        kernels = [kernel_line(name, form_fr if fused else form_ul, float(np.mean(t_a)), fl, FRAME_BYTES_PER_VEC)]
        dom = kernels[0]
        dom_bytes = FRAME_BYTES_PER_VEC * vec_step
    else:
        kernels = [kernel_line(KERNELS[form_ul][0], form_ul, float(np.mean(t_a)), FLOP_PER_VEC[form_ul], UL_BYTES_PER_VEC),
                   kernel_line(KERNELS[form_dl][1], form_dl, float(np.mean(t_b)), FLOP_PER_VEC[form_dl], DL_BYTES_PER_VEC)]
        dom = max(kernels, key=lambda k: k["ms"])
        dom_bytes = (UL_BYTES_PER_VEC if dom is kernels[0] else DL_BYTES_PER_VEC) * vec_step
    achieved = dom["flop_per_vector"] * vec_step / (dom["ms"] * 1e-3) / 1e12
    pipes = measure_pipes(dev, stream)
    roof = {"bound": "alu", "kernel": dom["kernel"], "flop_per_vector": dom["flop_per_vector"],
            "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
            "hbm": {"achieved_gbs": dom_bytes / (dom["ms"] * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                    "frac": dom_bytes / (dom["ms"] * 1e-3) / 1e9 / hbm_peak, "peak_source": peak_src},
            "traffic": NCU_TRAFFIC.get(dom["kernel"]), "pipe_probe_tflops": pipes}
    if frame and dom["kernel"] in ("cd_frame_ws_kernel", "cd_frame_tc_kernel"):
        # The tensor-core frame, pipe by pipe: the sweeps (FP32) bind; contractions and bytes follow.
        t_s = dom["ms"] * 1e-3
        bf16, bf16_src = load_bf16_peak()
        sw = SWEEP_FLOP_PER_VEC * vec_step
        mma = MMA_FLOP_PER_VEC * vec_step
        roof.update({"flop_per_vector": SWEEP_FLOP_PER_VEC, "achieved": sw / t_s / 1e12,
                     "frac": sw / t_s / 1e12 / FP32_PEAK_TFLOPS,
                     "what": "FP32 pipes: the Gauss-Seidel sweeps' flops (K U^2 complex MACs per cluster and "
                             "direction) against the FP32 ALU peak; the other pipes are in 'pipes'"})
        roof["pipes"] = {
            "fp32_sweeps": {"flop_per_vector": SWEEP_FLOP_PER_VEC, "achieved_tflops": sw / t_s / 1e12,
                            "peak_derived_tflops": FP32_PEAK_TFLOPS, "frac_derived": sw / t_s / 1e12 / FP32_PEAK_TFLOPS,
                            "peak_probe_tflops": pipes["ffma2"], "frac_probe": sw / t_s / 1e12 / pipes["ffma2"],
                            "t_min_us": sw / (pipes["ffma2"] * 1e12) * 1e6},
            "tensor_mma_sync_tf32": {"flop_per_vector_algorithmic": CONTRACTION_FLOP_PER_VEC,
                                     "mma_flop_per_vector_executed": MMA_FLOP_PER_VEC,
                                     "achieved_tflops_executed": mma / t_s / 1e12,
                                     "peak_probe_tflops": pipes["mma_tf32"],
                                     "frac_probe": mma / t_s / 1e12 / pipes["mma_tf32"],
                                     "t_min_us": mma / (pipes["mma_tf32"] * 1e12) * 1e6,
                                     "tcgen05_tf32_tflops_from_bf16": bf16 * TF32_PER_BF16_NOMINAL,
                                     "frac_vs_tcgen05_tf32": mma / t_s / 1e12 / (bf16 * TF32_PER_BF16_NOMINAL),
                                     "peak_source": f"probe (mma.sync); tcgen05 figure = {bf16_src} bf16 x 1.1/2.25"},
            "hbm": {"bytes_per_vector": FRAME_BYTES_PER_VEC, "achieved_gbs": dom_bytes / t_s / 1e9,
                    "peak_gbs": hbm_peak, "frac": dom_bytes / t_s / 1e9 / hbm_peak,
                    "t_min_us": dom_bytes / (hbm_peak * 1e9) * 1e6, "peak_source": peak_src},
        }
        roof["l2_writeback_note"] = (
            "the outputs (%.1f MB) can still be in L2 at the end event; their write-back (at most %.1f us of HBM "
            "time) then falls into the untimed L2 flush" % (vec_step * (U + B) * 8 / 1e6,
                                                             vec_step * (U + B) * 8 / (hbm_peak * 1e9) * 1e6))
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "vectors/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "step_ms_percentiles": {q: float(np.percentile(np.add(t_a, t_b), v)) for q, v in
                                (("p10", 10), ("median", 50), ("p90", 90))},
        "higher_is_better": True,
        "scaling": args.scaling,
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded i.i.d. Rayleigh, 16-QAM, AWGN)",
        "config": bench_config(args.step, world, args.scaling),
        "gbps": value * BITS / 1e9,
        "kernels": kernels,
        "roofline": roof,
        "mse_vs_mmse": mse,
        "ber": ber,
        "e2e": {"value": N_SC * N_SYM / (e2e_ms * 1e-3) if strong else whole_job_value(vec_step, world, e2e_ms),
                "unit": "vectors/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "api": "cdmimo_detect_precode_host (chunks: %s)" % (args.e2e_chunks or "default") if frame
                else "cdmimo_detect_host + cdmimo_precode_host"},
        "gpu_launches": (1 if frame and kernels[0]["kernel"] in FRAME_KERNELS.values() else 2) * args.steps,
        "clocks": clocks,
        "wall_s": wall,
    }
    if frame and args.form in ("auto", "gram_tc") and n_loc == N_SC:
        line["precision"] = precision_variants(up, dl, dev, stream, min(args.steps, 200), args.e2e_chunks)
    cb = cpu_baseline(up, dl, frame) if world == 1 else None
    if cb is not None:  # and on one host thread
        st = cpu_baseline(up, dl, frame, min_seconds=3.0, threads=1)
        cb["single_thread"] = {"value": st["value"], "unit": st["unit"], "cores": 1, "sample": st["sample"]}
    line["cpu_baseline"] = cb
    if world == 1 and frame and args.form == "auto" and not args.no_configs:
        line["configs"] = config_summaries(args, dev)
    return line


def precision_variants(up, dl, dev, stream, steps, e2e_chunks):
    """The frame step with H and y stored as fp16 and as bf16 (per-subcarrier scales; every
    arithmetic step FP32): device time (CUDA events, L2 flushed), MSE against the L-MMSE of the
    unquantized data, and the end-to-end rate through cdmimo_detect_precode_host with 16-bit host
    buffers (the uploads of H and y halve)."""
    import torch

    from paper_1902_08653_gb300 import cdmimo
    from paper_1902_08653_gb300 import workload as wl

    N0 = torch.from_numpy(up["N0"].astype(np.float32)).to(dev)
    S = torch.from_numpy(wl.as_c64(dl["S"])[0]).to(dev)
    N0h = torch.from_numpy(up["N0"].astype(np.float32)).pin_memory()
    Sh = torch.from_numpy(wl.as_c64(dl["S"])[0]).pin_memory()
    out = {}
    for kind, tdt, code in (("f16", torch.float16, cdmimo.C16F), ("bf16", torch.bfloat16, cdmimo.C16BF)):
        qH, sH, _ = wl.quantize_c16(up["H"], kind)
        qY, sY, _ = wl.quantize_c16(up["Y"], kind)
        Hq = torch.from_numpy(qH.view(np.int16)).view(tdt)
        Yq = torch.from_numpy(qY.view(np.int16)).view(tdt)
        sHt, sYt = torch.from_numpy(sH), torch.from_numpy(sY)
        H, Y, hs, ys = Hq.to(dev), Yq.to(dev), sHt.to(dev), sYt.to(dev)
        X = torch.empty((N_SC, N_SYM, U), dtype=torch.complex64, device=dev)
        P = torch.empty((N_SC, N_SYM, B), dtype=torch.complex64, device=dev)
        fn = lambda: cdmimo.detect_precode(H, Y, N0, S, CS, K, out=X, out_dl=P, h_scale=hs, y_scale=ys)
        _, ms = time_device(fn, steps, 5, dev)
        fn()
        mse, _ = mse_vs_mmse(up, X.cpu().numpy().astype(np.complex128))
        Hh, Yh = Hq.pin_memory(), Yq.pin_memory()
        Xh = torch.empty((N_SC, N_SYM, U), dtype=torch.complex64).pin_memory()
        Ph = torch.empty((N_SC, N_SYM, B), dtype=torch.complex64).pin_memory()
        ws = torch.empty(cdmimo.host_workspace_size(cdmimo.OP_FRAME, N_SC, N_SYM, B, U, CS, K, in_dtype=code),
                         dtype=torch.uint8, device=dev)
        e2e = lambda: cdmimo.detect_precode_host(Hh, Yh, N0h, Sh, CS, K, Xh, Ph, ws, h_scale=sHt.pin_memory(),
                                                  y_scale=sYt.pin_memory(), n_chunks=e2e_chunks, stream=stream)
        for _ in range(2):
            e2e()
        torch.cuda.synchronize()
        n_e2e = max(3, min(50, steps))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_e2e):
            e2e()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / n_e2e
        out[kind] = {"kernel": FRAME_KERNELS["gram_tc"], "ms": ms, "vectors_per_s": N_SC * N_SYM / (ms * 1e-3),
                     "mse_vs_mmse_mean": float(np.mean(list(mse.values()))),
                     "e2e": {"vectors_per_s": N_SC * N_SYM / (e2e_ms * 1e-3), "ms_per_step": e2e_ms,
                             "h2d_bytes_per_step": int(Hh.numel() * 2 + Yh.numel() * 2 + N0h.numel() * 4 +
                                                       Sh.numel() * 8 + 8 * N_SC),
                             "d2h_bytes_per_step": int(Xh.numel() * 8 + Ph.numel() * 8)}}
    if cdmimo.device_status(clear=True) != 0:
        raise RuntimeError("device status set by the 16-bit frame runs")
    return out


def cpu_baseline(up, dl, frame=True, min_seconds=10.0, threads=None):
    """The FP64 oracle as it stands, on the host cores: the whole batch (UL detect + DL precode),
    repeated until about `min_seconds` of wall time have been spent."""
    import oracle

    oracle.build()
    threads = threads or os.cpu_count() or 1
    reps = 0
    t0 = time.perf_counter()
    while True:
        oracle.detect(up["H"], up["Y"], up["N0"], CS, K, threads=threads)
        oracle.precode(up["H"] if frame else dl["H"], dl["S"], CS, K, threads=threads)
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
    for _ in range(args.warmup):
        oracle.detect(up["H"][:8], up["Y"][:8], up["N0"][:8], CS, K, threads=threads)
    times = []
    for i in range(args.steps):  # every step is the whole batch, as on the GPU
        t0 = time.perf_counter()
        oracle.detect(up["H"], up["Y"], up["N0"], CS, K, threads=threads)
        oracle.precode((up if args.step == "frame" else dl)["H"], dl["S"], CS, K, threads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = N_SC * N_SYM / (ms * 1e-3)
    sample = f"the full batch ({N_SC} subcarriers x {N_SYM} symbols, UL detect + DL precode) per step, FP64 C oracle"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "vectors/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded i.i.d. Rayleigh)",
            "config": bench_config(args.step, 1),
            "cpu_baseline": {"value": value, "unit": "vectors/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------------------------------------
# other configurations (python bench.py --config N): measurement lines for the rest of the path
# ------------------------------------------------------------------------------------------------
def time_device(fn, steps, warmup, dev, flush_mb=256):
    """Median/mean device time of fn() in ms with CUDA events, L2 flushed (untimed) between calls."""
    import torch

    flush = torch.empty(flush_mb * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i & 7))
        ev[i][0].record()
        fn()
        ev[i][1].record()
    torch.cuda.synchronize()
    t = np.array([a.elapsed_time(b) for a, b in ev])
    return float(np.median(t)), float(np.mean(t))


def base_line(name, value, unit, args, config, **kw):
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "config": dict(workload=name, l2="flushed between timed calls (256 MB write, untimed)", **config)}
    line.update(kw)
    return line


def run_config1(args, dev):
    """B = 32 in 2 clusters of 16, U = 4, K = 3, 64 subcarriers x 1 symbol, QPSK at 10 dB, equal fusion."""
    import torch

    from paper_1902_08653_gb300 import cdmimo
    from paper_1902_08653_gb300 import workload as wl

    d = wl.uplink(20190222, 64, 1, 32, 4, snr_db=10.0, M=4)
    H = torch.from_numpy(wl.as_c64(d["H"])[0]).to(dev)
    Y = torch.from_numpy(wl.as_c64(d["Y"])[0]).to(dev)
    N0 = torch.from_numpy(d["N0"].astype(np.float32)).to(dev)
    X = torch.empty((64, 1, 4), dtype=torch.complex64, device=dev)
    med, mean = time_device(lambda: cdmimo.detect(H, Y, N0, [16, 16], 3, fuse="equal", out=X), args.steps, args.warmup, dev)
    return base_line("UL CD detection, B=32 (2 x 16), U=4, K=3, 64 subcarriers x 1 symbol, QPSK 10 dB, equal fusion",
                     64 / (med * 1e-3), "vectors/s", args, {"n_sc": 64, "n_sym": 1, "B": 32, "C": 2, "U": 4, "K": 3},
                     dtype="f32", ms_per_step=med, latency_us=med * 1e3, gpu_launches=1 * args.steps)


def run_config3(args, dev):
    """Config 2's shape at U = 32 with 64-QAM; H and y stored as c64, fp16 or bf16 (+ scale), K = 3 and 5."""
    import torch

    from paper_1902_08653_gb300 import cdmimo
    from paper_1902_08653_gb300 import workload as wl

    Uc, M3 = 32, 64
    up = wl.uplink(20190222, N_SC, N_SYM, B, Uc, snr_db=wl.sweep_snr(N_SC), M=M3)
    N0 = torch.from_numpy(up["N0"].astype(np.float32)).to(dev)
    store = {"c64": (torch.from_numpy(wl.as_c64(up["H"])[0]).to(dev), torch.from_numpy(wl.as_c64(up["Y"])[0]).to(dev),
                     None, None)}
    for kind, tdt in (("f16", torch.float16), ("bf16", torch.bfloat16)):
        qH, sH, _ = wl.quantize_c16(up["H"], kind)
        qY, sY, _ = wl.quantize_c16(up["Y"], kind)
        store[kind] = (torch.from_numpy(qH.view(np.int16)).to(dev).view(tdt),
                       torch.from_numpy(qY.view(np.int16)).to(dev).view(tdt),
                       torch.from_numpy(sH).to(dev), torch.from_numpy(sY).to(dev))
    X = torch.empty((N_SC, N_SYM, Uc), dtype=torch.complex64, device=dev)
    # the FP64 oracle (benchmark-side check only) on the exact values each storage delivers, and on
    # the unquantized channel: the per-vector error of the GPU path against it
    import oracle

    oracle.build()
    exact = {"c64": (wl.as_c64(up["H"])[1], wl.as_c64(up["Y"])[1])}
    for kind in ("f16", "bf16"):
        exact[kind] = (wl.quantize_c16(up["H"], kind)[2], wl.quantize_c16(up["Y"], kind)[2])
    thr = os.cpu_count() or 1
    res, ref, orc_unq = {}, {}, {}
    for K3 in (3, 5):
        orc_unq[K3] = oracle.detect(exact["c64"][0], exact["c64"][1], up["N0"], CS, K3, threads=thr)[0]
        for kind, (Ht, Yt, sH, sY) in store.items():
            fn = lambda: cdmimo.detect(Ht, Yt, N0, CS, K3, h_scale=sH, y_scale=sY, out=X)
            med, _ = time_device(fn, args.steps, args.warmup, dev)
            fn()
            xh = X.cpu().numpy().astype(np.complex128)
            if kind == "c64":
                ref[K3] = xh
            rel = np.linalg.norm(xh - ref[K3], axis=-1) / np.linalg.norm(ref[K3], axis=-1)
            xo = oracle.detect(exact[kind][0], exact[kind][1], up["N0"], CS, K3, threads=thr)[0]
            e_kernel = np.linalg.norm(xh - xo, axis=-1) / np.linalg.norm(xo, axis=-1)
            e_total = np.linalg.norm(xh - orc_unq[K3], axis=-1) / np.linalg.norm(orc_unq[K3], axis=-1)
            mse, ber = mse_vs_mmse_U(up, xh, Uc, M3)
            in_bytes = (Ht.numel() * Ht.element_size() + Yt.numel() * Yt.element_size()) / (N_SC * N_SYM)
            res[f"{kind}_K{K3}"] = {"ms": med, "vectors_per_s": N_SC * N_SYM / (med * 1e-3),
                                    "gbps": N_SC * N_SYM * Uc * 6 / (med * 1e-3) / 1e9,
                                    "input_bytes_per_vector": in_bytes,
                                    "rel_l2_vs_oracle_same_inputs_max": float(e_kernel.max()),
                                    "rel_l2_vs_oracle_unquantized_median": float(np.median(e_total)),
                                    "rel_l2_vs_oracle_unquantized_max": float(e_total.max()),
                                    "rel_l2_vs_c64_median": float(np.median(rel)), "rel_l2_vs_c64_max": float(rel.max()),
                                    "mse_vs_mmse_mean": float(np.mean(list(mse.values()))), "ber": ber}
    best = res["f16_K3"]
    return base_line("UL CD detection, B=256 (8 x 32), U=32, 64-QAM, 1200 x 14, SNR sweep; H, y in c64 / fp16 / bf16",
                     best["vectors_per_s"], "vectors/s", args,
                     {"n_sc": N_SC, "n_sym": N_SYM, "B": B, "C": C, "U": Uc, "K": 3, "qam": M3, "storage": "f16"},
                     dtype="f32 (f16 storage)", ms_per_step=best["ms"], variants=res, gpu_launches=6 * args.steps)


def mse_vs_mmse_U(up, Xhat, Uc, Mq):
    H = up["H"]
    A = np.einsum("fub,fvb->fuv", np.conj(H), H) + up["N0"][:, None, None] * np.eye(Uc)[None]
    Z = np.einsum("fub,fnb->fun", np.conj(H), up["Y"])
    Xm = np.linalg.solve(A, Z).transpose(0, 2, 1)
    err = np.sum(np.abs(Xhat - Xm) ** 2, axis=-1) / Uc
    from paper_1902_08653_gb300 import workload as wl

    mse, ber = {}, {}
    for sv in np.unique(up["snr_db"]):
        sel = up["snr_db"] == sv
        mse[f"{int(sv)}dB"] = float(np.mean(err[sel]))
        lab, _ = wl.hard_decision(Xhat[sel], Mq)
        ber[f"{int(sv)}dB"] = wl.bit_errors(lab, up["labels"][sel]) / (lab.size * int(np.log2(Mq)))
    return mse, ber


def config4_items(dev):
    """The uneven batch's blocks, its detection items (device tensors) and its sweep FLOPs."""
    import torch

    from paper_1902_08653_gb300 import batched
    from paper_1902_08653_gb300 import workload as wl

    blocks = wl.resource_blocks(20190222, n_rb=100, n_sc=12, n_sym=14)
    t = lambda a: torch.from_numpy(wl.as_c64(a)[0]).to(dev)
    items = []
    flops = 0
    for b in blocks:
        n_sc, Ub, Bb = b["H"].shape
        items.append(dict(op=batched.DETECT, H=t(b["H"]), V=t(b["Y"]),
                          N0=torch.from_numpy(b["N0"].astype(np.float32)).to(dev),
                          out=torch.empty((n_sc, 14, Ub), dtype=torch.complex64, device=dev),
                          cluster_size=b["cluster_size"], K=3, fuse="colnorm", Ex=1.0))
        flops += n_sc * 14 * 2 * 3 * Ub * Bb * 8
    return blocks, items, flops


# Tile parameters of the batched kernel under `--profile batched` (the autotuner's usual choice on
# the uneven batch), fixed so that the captured launches do not depend on timing.
BATCH_PROFILE_PLAN = dict(P=16, threads=256, group_bytes=84 * 1024, ctas_per_sm=2)


def run_config4(args, dev):
    """100 resource blocks x 12 subcarriers x 14 symbols, B in {128,256,512}, clusters {16,32,64}, U in [8,64],
    K = 3, 16-QAM at 20 dB: one persistent launch per step, replayed from a CUDA graph, autotuned tiles."""
    from paper_1902_08653_gb300 import batched, cdmimo

    blocks, items, flops = config4_items(dev)
    bt = batched.Batch(items)
    plan, times = batched.autotune(bt, reps=5)
    lb = bt.balance()
    bt.capture()
    med, _ = time_device(bt.replay, args.steps, args.warmup, dev)
    n_vec = sum(b["H"].shape[0] * 14 for b in blocks)
    # the same work as 100 separate single-block calls (one launch per block)
    def separate():
        for it in items:
            cdmimo.detect(it["H"], it["V"], it["N0"], it["cluster_size"], 3, out=it["out"])
    med_sep, _ = time_device(separate, max(3, args.steps // 10), args.warmup, dev)
    tflops = flops / (med * 1e-3) / 1e12
    return base_line("batched uneven UL CD detection, 100 RBs x 12 subcarriers x 14 symbols, B in {128,256,512}, "
                     "clusters {16,32,64}, U in [8,64], K=3, 16-QAM 20 dB, CUDA graph", n_vec / (med * 1e-3),
                     "vectors/s", args, {"n_rb": 100, "n_sc_per_rb": 12, "n_sym": 14, "K": 3},
                     dtype="f32", ms_per_step=med, gpu_launches=1 * args.steps,
                     roofline={"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": tflops / FP32_PEAK_TFLOPS, "traffic": None},
                     autotune={"chosen": {k: getattr(plan, k) for k in ("P", "threads", "group_bytes", "ctas_per_sm")},
                               "candidates_ms": times},
                     load_balance=lb,
                     separate_launches={"ms": med_sep, "vectors_per_s": n_vec / (med_sep * 1e-3),
                                        "speedup_of_one_launch": med_sep / med})


def run_config5(args, dev):
    """Learned deep-unfolded CD, K = 2 (trained here on 1M device-generated channels) against plain CD
    K = 2, 3, 5 on config 2's workload (B = 256, 8 x 32, U = 16, 1200 x 14, SNR sweep)."""
    import torch

    from paper_1902_08653_gb300 import cdmimo, train_learned
    from paper_1902_08653_gb300 import workload as wl

    model, info = train_learned.train(K=2, channels=args.train_channels, device=dev)
    up, _ = make_inputs(20190223)
    H = torch.from_numpy(wl.as_c64(up["H"])[0]).to(dev)
    Y = torch.from_numpy(wl.as_c64(up["Y"])[0]).to(dev)
    N0 = torch.from_numpy(up["N0"].astype(np.float32)).to(dev)
    X = torch.empty((N_SC, N_SYM, U), dtype=torch.complex64, device=dev)
    res = {}
    runs = {"learned_K2": lambda: model.detect(H, Y, N0, CS, out=X, form=args.form),
            "learned_K2_residual_form": lambda: model.detect(H, Y, N0, CS, out=X, form="residual")}
    for Kp in (2, 3, 5):
        runs[f"plain_K{Kp}"] = (lambda Kp=Kp: cdmimo.detect(H, Y, N0, CS, Kp, out=X, form=args.form))
    for name, fn in runs.items():
        med, _ = time_device(fn, args.steps, args.warmup, dev)
        fn()
        mse, ber = mse_vs_mmse(up, X.cpu().numpy().astype(np.complex128))
        res[name] = {"ms": med, "vectors_per_s": N_SC * N_SYM / (med * 1e-3),
                     "mse_vs_mmse": mse, "mse_vs_mmse_mean": float(np.mean(list(mse.values()))), "ber": ber}
    lr = res["learned_K2"]
    return base_line("learned deep-unfolded CD K=2 (tau_t, gamma_t, 17-64-1 MLP fusion) vs plain CD; B=256 (8 x 32), "
                     "U=16, 1200 x 14, 16-QAM, SNR sweep", lr["vectors_per_s"], "vectors/s", args,
                     {"n_sc": N_SC, "n_sym": N_SYM, "B": B, "C": C, "U": U, "K": 2},
                     dtype="f32 (bf16 MLP weights)", ms_per_step=lr["ms"], variants=res,
                     training={k: v for k, v in info.items() if k != "loss"}, gpu_launches=1 * args.steps)


def config_summaries(args, dev):
    """Configurations 1, 3, 4 and 5 on the benchmark's GPU (short runs), condensed for the default
    line: latency (1), storage precision at U = 32 (3), batched uneven blocks (4), learned vs plain
    CD (5)."""
    import copy

    sub = copy.copy(args)
    sub.steps, sub.warmup = max(10, min(args.steps, 30)), 3
    out = {}
    c1 = run_config1(sub, dev)
    out["1"] = {"workload": c1["config"]["workload"], "latency_us": c1["latency_us"], "vectors_per_s": c1["value"]}
    c3 = run_config3(sub, dev)
    v = c3["variants"]
    out["3"] = {"workload": c3["config"]["workload"],
                "variants": {k: {q: x[q] for q in ("ms", "vectors_per_s", "mse_vs_mmse_mean",
                                                    "rel_l2_vs_oracle_same_inputs_max",
                                                    "rel_l2_vs_oracle_unquantized_median")} for k, x in v.items()},
                "reduced_precision_faster_than_c64": {f"K{k}": {kind: v[f"{kind}_K{k}"]["ms"] < v[f"c64_K{k}"]["ms"]
                                                             for kind in ("f16", "bf16")} for k in (3, 5)}}
    c4 = run_config4(sub, dev)
    out["4"] = {"workload": c4["config"]["workload"], "ms": c4["ms_per_step"], "vectors_per_s": c4["value"],
                "fp32_frac": c4["roofline"]["frac"], "autotune_chosen": c4["autotune"]["chosen"],
                "load_balance": c4["load_balance"],
                "speedup_over_separate_launches": c4["separate_launches"]["speedup_of_one_launch"]}
    c5 = run_config5(sub, dev)
    v5 = c5["variants"]
    out["5"] = {"workload": c5["config"]["workload"],
                "variants": {k: {q: x[q] for q in ("ms", "vectors_per_s", "mse_vs_mmse_mean")} for k, x in v5.items()},
                "learned_K2_faster_than_plain_K5": v5["learned_K2"]["ms"] < v5["plain_K5"]["ms"],
                "learned_K2_mse_at_most_plain_K5": v5["learned_K2"]["mse_vs_mmse_mean"] <= v5["plain_K5"]["mse_vs_mmse_mean"],
                "training": c5["training"]}
    return out


def run_profile(args):
    """Three untimed calls of one direction on the step's workload (the launches an ncu capture of
    this command selects with -k / -s / -c)."""
    import torch

    from paper_1902_08653_gb300 import cdmimo
    from paper_1902_08653_gb300 import workload as wl

    dev = torch.device("cuda:0")
    if args.profile == "batched":  # configuration 4's uneven batch, one persistent launch per call
        from paper_1902_08653_gb300 import batched

        _, items, _ = config4_items(dev)
        bt = batched.Batch(items, plan=batched.default_plan(**BATCH_PROFILE_PLAN))
        for _ in range(3):
            bt.run()
        torch.cuda.synchronize()
        assert cdmimo.device_status(clear=True) == 0
        print("ok batched", BATCH_PROFILE_PLAN)
        return
    Up, Mp = (32, 64) if args.profile.startswith("detect_u32") else (U, M)  # configuration 3's users
    up = wl.uplink(20190222, N_SC, N_SYM, B, Up, snr_db=wl.sweep_snr(N_SC), M=Mp)
    t = lambda a: torch.from_numpy(wl.as_c64(a)[0]).to(dev)
    H, Y, S = t(up["H"]), t(up["Y"]), t(up["X"])
    N0 = torch.from_numpy(up["N0"].astype(np.float32)).to(dev)
    sc = {}
    if args.profile in ("frame_f16", "detect_u32_f16"):  # the same batch stored as fp16 with per-subcarrier scales
        qH, sH, _ = wl.quantize_c16(up["H"], "f16")
        qY, sY, _ = wl.quantize_c16(up["Y"], "f16")
        H = torch.from_numpy(qH.view(np.int16)).to(dev).view(torch.float16)
        Y = torch.from_numpy(qY.view(np.int16)).to(dev).view(torch.float16)
        sc = dict(h_scale=torch.from_numpy(sH).to(dev), y_scale=torch.from_numpy(sY).to(dev))
    for _ in range(3):
        if args.profile.startswith("detect"):
            cdmimo.detect(H, Y, N0, CS, K, form=args.form, **sc)
        elif args.profile == "precode":
            cdmimo.precode(H, S, CS, K, form=args.form)
        else:
            cdmimo.detect_precode(H, Y, N0, S, CS, K, form=args.form, **sc)
    torch.cuda.synchronize()
    assert cdmimo.device_status(clear=True) == 0
    print("ok", args.profile, args.form)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5],
                    help="2 (default): UL detect + DL precode bench line; 1, 3, 4, 5: the other configurations")
    ap.add_argument("--train-channels", type=int, default=1_000_000, help="--config 5: training channels")
    ap.add_argument("--profile", choices=["detect", "precode", "frame", "frame_f16", "detect_u32", "detect_u32_f16",
                                          "batched"],
                    default=None,
                    help="untimed: three cdmimo_detect / cdmimo_precode / cdmimo_detect_precode calls, for ncu "
                         "(detect_u32*: configuration 3's U = 32, 64-QAM batch, K = 3; batched: configuration 4's "
                         "uneven batch, three persistent launches)")
    ap.add_argument("--form", choices=["auto", "residual", "gram", "gram_tc", "gram_tc_phased", "gram_tc_umma"],
                    default="auto",
                    help="CD evaluation form")
    ap.add_argument("--e2e-chunks", type=int, default=0,
                    help="chunks of the pipelined host-buffer frame in the e2e leg (0: the library's default)")
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="N > 1: weak (default: every rank its own 1200-subcarrier batch) or strong (one batch, "
                         "its subcarriers split over the ranks); neither has a collective on the data path")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the condensed runs of configurations 1, 3, 4 and 5 from the default line")
    ap.add_argument("--step", choices=["frame", "separate"], default="frame",
                    help="frame (default): UL + DL on one channel, one call; separate: two calls, two channels")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.profile:
        run_profile(args)
        return
    if args.config != 2:
        import torch

        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        fn = {1: run_config1, 3: run_config3, 4: run_config4, 5: run_config5}[args.config]
        if rank == 0:
            print(json.dumps(fn(args, dev)), flush=True)
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
