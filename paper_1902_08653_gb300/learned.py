"""Training and inference driver of the learned deep-unfolded CD detector.

The model (declared with the C ABI in include/cdmimo.h) runs K learned sweeps
    x_u <- x_u + tau_t (h_u^H r - gamma_t alpha x_u) / (||h_u||^2 + gamma_t alpha)
per cluster and fuses the cluster estimates with softmax weights from a two-layer perceptron on
per-cluster column energies and log10(alpha).  This module keeps the FP32 master parameters and
the Adam moments on the GPU, calls the library's gradient, Adam and pack kernels, and saves or
restores a checkpoint.  Every arithmetic step runs in the library's CUDA kernels; torch only holds
device memory.

Initialization: tau = 1, gamma = 1, w2 = 0 (so logits are constant and the fusion is equal):
the untrained model is exactly Algorithm 1 with equal fusion.
"""
from __future__ import annotations

import math
import struct

import numpy as np
import torch

from . import cdmimo

GRAW_ONE = math.log(math.e - 1.0)  # softplus(GRAW_ONE) = 1
CKPT_MAGIC = b"CDMLRN01"


def layout(K, U, hidden):
    """Slices of the master vector: tau, graw, W1, b1, w2, b2."""
    F = U + 1
    o = np.cumsum([0, K, K, hidden * F, hidden, hidden, 1])
    names = ("tau", "graw", "W1", "b1", "w2", "b2")
    return {n: slice(int(o[i]), int(o[i + 1])) for i, n in enumerate(names)}


class LearnedCD:
    def __init__(self, K, U, hidden=64, seed=0, device="cuda", master=None):
        self.K, self.U, self.hidden = int(K), int(U), int(hidden)
        self.device = torch.device(device)
        n = cdmimo.learned_param_count(K, U, hidden)
        if n == 0:
            raise ValueError("unsupported (K, U, hidden)")
        if master is None:
            sl = layout(K, U, hidden)
            g = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), 5])))
            m = np.zeros(n, np.float32)
            m[sl["tau"]] = 1.0
            m[sl["graw"]] = GRAW_ONE
            m[sl["W1"]] = (g.standard_normal(hidden * (U + 1)) / math.sqrt(U + 1)).astype(np.float32)
            master = torch.from_numpy(m)
        self.master = master.to(self.device, torch.float32).contiguous()
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.step = 0
        self.block = torch.zeros(cdmimo.LEARNED_BLOCK_BYTES + 16, dtype=torch.uint8, device=self.device)
        self.pack()

    def pack(self):
        cdmimo.learned_pack(self.master, self.K, self.U, self.hidden, self.block)

    def detect(self, H, Y, N0, cluster_size, **kw):
        """Learned inference through cdmimo_detect (learned sweeps and learned fusion)."""
        return cdmimo.detect(H, Y, N0, cluster_size, self.K, fuse="learned", learned=self.block, **kw)

    def grad(self, H, Y, N0, Xtarget, cluster_size, workspace=None):
        return cdmimo.learned_grad(H, Y, N0, Xtarget, cluster_size, self.K, self.block, self.hidden,
                                   workspace=workspace)

    def train_step(self, H, Y, N0, Xtarget, cluster_size, lr=1e-3, workspace=None):
        loss, g = self.grad(H, Y, N0, Xtarget, cluster_size, workspace=workspace)
        self.step += 1
        cdmimo.adam_step(self.master, g, self.m, self.v, self.step, lr=lr)
        self.pack()
        return loss

    # -- checkpoint -----------------------------------------------------------------------------
    def save(self, path):
        hdr = CKPT_MAGIC + struct.pack("<5i", 1, self.K, self.U, self.hidden, self.step)
        with open(path, "wb") as f:
            f.write(hdr)
            for t in (self.master, self.m, self.v):
                f.write(t.detach().cpu().numpy().astype("<f4").tobytes())

    @classmethod
    def load(cls, path, device="cuda"):
        with open(path, "rb") as f:
            raw = f.read()
        if raw[:8] != CKPT_MAGIC:
            raise ValueError("not a learned-CD checkpoint")
        version, K, U, hidden, step = struct.unpack("<5i", raw[8:28])
        if version != 1:
            raise ValueError(f"unsupported checkpoint version {version}")
        n = cdmimo.learned_param_count(K, U, hidden)
        arr = np.frombuffer(raw[28:], dtype="<f4")
        if arr.size != 3 * n:
            raise ValueError("truncated checkpoint")
        obj = cls(K, U, hidden, device=device, master=torch.from_numpy(arr[:n].copy()))
        obj.m.copy_(torch.from_numpy(arr[n:2 * n].copy()))
        obj.v.copy_(torch.from_numpy(arr[2 * n:].copy()))
        obj.step = step
        return obj
