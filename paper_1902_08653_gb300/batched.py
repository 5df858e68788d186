"""Batched uneven launches: many resource blocks with different shapes in one persistent kernel.

Batch      builds the descriptor table once (cdmimo_batch_build, host only), keeps it and the work
           counter on the device, and enqueues the launch with run(); capture() records run() in a
           CUDA graph and replay() relaunches it.
autotune   the project's tile autotuner: it times cdmimo_detect_batched for candidate tile parameter
           sets (antennas per lane P, threads per CTA, shared-memory budget per cluster group, CTAs
           per SM) on the batch itself and keeps the fastest: a fixed list plus, per register-feasible
           (P, threads, CTAs per SM) shape, the largest group budget that lets those CTAs share an SM
           (found by host-only plan builds); results are cached per batch shape signature (in memory,
           and optionally in a JSON file).
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import cdmimo

DETECT, PRECODE = cdmimo.OP_DETECT, cdmimo.OP_PRECODE

CANDIDATES = [
    dict(P=16, threads=256, group_bytes=64 * 1024, ctas_per_sm=0),
    dict(P=16, threads=512, group_bytes=96 * 1024, ctas_per_sm=0),
    dict(P=16, threads=256, group_bytes=96 * 1024, ctas_per_sm=0),
    dict(P=8, threads=384, group_bytes=96 * 1024, ctas_per_sm=0),
    dict(P=8, threads=384, group_bytes=80 * 1024, ctas_per_sm=0),
    dict(P=8, threads=256, group_bytes=64 * 1024, ctas_per_sm=0),
    dict(P=16, threads=512, group_bytes=64 * 1024, ctas_per_sm=0),
    dict(P=32, threads=256, group_bytes=96 * 1024, ctas_per_sm=0),
    dict(P=16, threads=128, group_bytes=48 * 1024, ctas_per_sm=0),
    dict(P=16, threads=128, group_bytes=44 * 1024, ctas_per_sm=0),
]


def default_plan(**over):
    plan = cdmimo.BatchPlan()
    cdmimo.lib().cdmimo_batch_default_plan(ctypes.byref(plan))
    for k, v in over.items():
        setattr(plan, k, int(v))
    return plan


class Batch:
    """items: list of dicts with keys op (DETECT / PRECODE), H, V (Y or S), out, cluster_size, K,
    and for detection N0, fuse ("equal" / "colnorm"), Ex; for precoding rho.  Tensors are device
    tensors (complex64, float32 for N0) that must stay alive as long as the batch."""

    def __init__(self, items, plan=None, device=None):
        self.items = items
        self.device = device or items[0]["H"].device
        n = len(items)
        self.descs = (cdmimo.BatchDesc * n)()
        self._keep = []
        for i, it in enumerate(items):
            H, V, out = it["H"], it["V"], it["out"]
            n_sc, U, B = H.shape
            cs = (ctypes.c_int * len(it["cluster_size"]))(*[int(v) for v in it["cluster_size"]])
            self._keep.append(cs)
            d = self.descs[i]
            d.op = int(it["op"])
            d.n_sc, d.n_sym, d.B, d.U, d.C, d.K = n_sc, V.shape[1], B, U, len(it["cluster_size"]), int(it["K"])
            d.fuse = cdmimo.FUSE[it.get("fuse", "colnorm")]
            d.Ex = float(it.get("Ex", 1.0))
            d.rho = float(it.get("rho", 1.0))
            d.cluster_size = ctypes.cast(cs, ctypes.POINTER(ctypes.c_int))
            d.H, d.V, d.out = H.data_ptr(), V.data_ptr(), out.data_ptr()
            d.N0 = it["N0"].data_ptr() if it.get("N0") is not None else None
        self.counter = torch.zeros(4, dtype=torch.int32, device=self.device)
        self.graph = None
        self.set_plan(plan or default_plan())

    def set_plan(self, plan):
        L = cdmimo.lib()
        rc = L.cdmimo_batch_build(self.descs, len(self.items), ctypes.byref(plan), None, 0)
        if rc != cdmimo.OK:
            raise cdmimo.CdmimoError("cdmimo_batch_build", rc)
        host = np.zeros((plan.table_bytes + 15) // 16 * 16 + 16, dtype=np.uint8)
        off = (-host.ctypes.data) % 16
        rc = L.cdmimo_batch_build(self.descs, len(self.items), ctypes.byref(plan),
                                  ctypes.c_void_p(host.ctypes.data + off), plan.table_bytes)
        if rc != cdmimo.OK:
            raise cdmimo.CdmimoError("cdmimo_batch_build", rc)
        self.plan = plan
        self.table = torch.from_numpy(host[off:off + plan.table_bytes].copy()).to(self.device)
        self.graph = None

    def run(self, stream=None):
        rc = cdmimo.lib().cdmimo_detect_batched(ctypes.byref(self.plan), ctypes.c_void_p(self.table.data_ptr()),
                                                ctypes.c_void_p(self.counter.data_ptr()), cdmimo._stream(stream))
        if rc != cdmimo.OK:
            raise cdmimo.CdmimoError("cdmimo_detect_batched", rc)

    def balance(self, stream=None):
        """One instrumented run (cdmimo_detect_batched_stats): the fraction of the launch's span that the
        persistent CTAs spent working, the span and the mean CTA lifetime (us), the number of CTAs."""
        stats = torch.zeros(4, dtype=torch.int64, device=self.device)
        rc = cdmimo.lib().cdmimo_detect_batched_stats(
            ctypes.byref(self.plan), ctypes.c_void_p(self.table.data_ptr()), ctypes.c_void_p(self.counter.data_ptr()),
            ctypes.c_void_p(stats.data_ptr()), cdmimo._stream(stream))
        if rc != cdmimo.OK:
            raise cdmimo.CdmimoError("cdmimo_detect_batched_stats", rc)
        t0, t1, busy, n = (int(v) for v in stats.cpu().tolist())
        if n == 0:
            return {"efficiency": None, "span_us": 0.0, "mean_cta_us": 0.0, "ctas": 0}
        span = max(t1 - t0, 1)
        return {"efficiency": busy / (n * span), "span_us": span / 1e3, "mean_cta_us": busy / n / 1e3, "ctas": n}

    def capture(self):
        """Record one run() in a CUDA graph (the first run happens eagerly, outside the capture)."""
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run(stream=s)
        torch.cuda.synchronize()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def signature(self):
        shapes = sorted((int(d.op), int(d.B), int(d.U), int(d.n_sym), tuple(self.items[i]["cluster_size"]))
                        for i, d in enumerate(self.descs))
        return str(hash(tuple(shapes)) & 0xFFFFFFFFFFFF)


def time_plan(batch, plan, reps=10):
    batch.set_plan(plan)
    for _ in range(2):
        batch.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        batch.run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


# Register-feasible (P, threads, CTAs per SM) shapes: the P = 16 and 32 kernels take up to 128 registers
# a thread (one 512-thread CTA per SM), the P = 8 kernel up to 80 (two 384-thread CTAs).
OCCUPANCY_SHAPES = [(16, 512, 1), (16, 256, 2), (16, 128, 4), (8, 384, 2), (8, 256, 3), (8, 128, 6)]
SMEM_PER_SM = 228 * 1024          # shared memory of one SM
SMEM_RESERVED_PER_CTA = 1024      # the runtime's per-CTA reservation


def plan_smem(batch, plan):
    """Host-only build of `plan` for the batch's descriptors: returns the plan's shared memory per CTA, or
    None if the batch does not fit the plan."""
    rc = cdmimo.lib().cdmimo_batch_build(batch.descs, len(batch.items), ctypes.byref(plan), None, 0)
    return int(plan.smem_bytes) if rc == cdmimo.OK else None


def occupancy_candidates(batch, shapes=OCCUPANCY_SHAPES, smem_per_sm=SMEM_PER_SM, step=4096):
    """For each register-feasible shape (P, threads, n), the largest cluster-group budget (in `step`
    bytes) whose plan lets n CTAs share an SM's shared memory: more budget means larger groups (more
    lanes at once), more CTAs mean more warps; the autotuner times both ends of that trade."""
    out = []
    for P, T, n in shapes:
        limit = smem_per_sm // n - SMEM_RESERVED_PER_CTA
        for gb in range(limit // step * step, step - 1, -step):
            sm = plan_smem(batch, default_plan(P=P, threads=T, group_bytes=gb, ctas_per_sm=n))
            if sm is not None and sm <= limit:
                out.append(dict(P=P, threads=T, group_bytes=gb, ctas_per_sm=n))
                break
    return out


_CACHE = {}


def autotune(batch, candidates=None, cache_file=None, reps=10):
    """Pick the fastest tile parameters for this batch; returns (plan, {name: ms}).  The default
    candidates are the fixed list plus the occupancy-derived ones of `occupancy_candidates`."""
    if candidates is None:
        candidates = list(CANDIDATES)
        for c in occupancy_candidates(batch):
            if c not in candidates:
                candidates.append(c)
    key = batch.signature()
    if cache_file and os.path.exists(cache_file):
        with open(cache_file) as f:
            _CACHE.update(json.load(f))
    if key in _CACHE:
        plan = default_plan(**_CACHE[key]["best"])
        batch.set_plan(plan)
        return plan, _CACHE[key]["times"]
    times = {}
    best, best_ms = None, float("inf")
    for cand in candidates:
        plan = default_plan(**cand)
        try:
            ms = time_plan(batch, plan, reps)
        except cdmimo.CdmimoError:
            continue
        name = ",".join(f"{k}={v}" for k, v in cand.items())
        times[name] = ms
        if ms < best_ms:
            best, best_ms = cand, ms
    if best is None:
        raise RuntimeError("no candidate tile configuration supports this batch")
    _CACHE[key] = {"best": best, "times": times}
    if cache_file:
        with open(cache_file, "w") as f:
            json.dump(_CACHE, f, indent=1)
    plan = default_plan(**best)
    batch.set_plan(plan)
    return plan, times
