"""Host-side planning of the batched uneven launch (CPU only: cdmimo_batch_build never touches a
GPU).  Device pointers are stand-in addresses; they are only stored in the table."""
import ctypes

import numpy as np
import pytest

from paper_1902_08653_gb300 import batched, cdmimo
from paper_1902_08653_gb300 import workload as wl


def descs_for(blocks, op=cdmimo.OP_DETECT, n_sc=12, n_sym=14, K=3):
    arr = (cdmimo.BatchDesc * len(blocks))()
    keep = []
    for i, b in enumerate(blocks):
        cs = (ctypes.c_int * len(b["cluster_size"]))(*b["cluster_size"])
        keep.append(cs)
        d = arr[i]
        d.op, d.n_sc, d.n_sym, d.B, d.U, d.C, d.K = op, n_sc, n_sym, b["B"], b["U"], len(b["cluster_size"]), K
        d.fuse, d.Ex, d.rho = 1, 1.0, 1.0
        d.cluster_size = ctypes.cast(cs, ctypes.POINTER(ctypes.c_int))
        d.H, d.V, d.N0, d.out = 0x100000 * (i + 1), 0x200000 * (i + 1), 0x300000 * (i + 1), 0x400000 * (i + 1)
    return arr, keep


def build(arr, n, plan):
    L = cdmimo.lib()
    rc = L.cdmimo_batch_build(arr, n, ctypes.byref(plan), None, 0)
    if rc:
        return rc, None
    buf = np.zeros(plan.table_bytes + 32, np.uint8)
    off = (-buf.ctypes.data) % 16
    rc = L.cdmimo_batch_build(arr, n, ctypes.byref(plan), ctypes.c_void_p(buf.ctypes.data + off), plan.table_bytes)
    return rc, buf[off:off + plan.table_bytes]


def test_config4_shapes_plan():
    g = np.random.default_rng(0)
    blocks = []
    for _ in range(100):
        B = int(g.choice([128, 256, 512]))
        blocks.append({"B": B, "U": int(g.integers(8, 65)), "cluster_size": wl.random_partition(g, B)})
    arr, keep = descs_for(blocks)
    for cand in batched.CANDIDATES:
        plan = batched.default_plan(**cand)
        rc, table = build(arr, len(blocks), plan)
        assert rc == cdmimo.OK, cand
        assert plan.n_items == 100 * 12
        assert plan.n_groups >= 100 and plan.C_max >= 1
        assert plan.smem_bytes <= 227 * 1024
        hdr = np.frombuffer(table[:32].tobytes(), dtype=np.int32)
        assert hdr[0] == 100 and hdr[1] == 1200 and hdr[2] == plan.n_groups
        assert hdr[3] == sum(len(b["cluster_size"]) for b in blocks)


def test_partition_helper():
    g = np.random.default_rng(3)
    for B in (128, 256, 512, 48):
        cs = wl.random_partition(g, B)
        assert sum(cs) == B and set(cs) <= {16, 32, 64}


@pytest.mark.parametrize("bad,code", [
    (dict(cluster_size=[32, 33]), cdmimo.ERR_BAD_PARTITION),
    (dict(U=65), cdmimo.ERR_UNSUPPORTED),
    (dict(K=-1), cdmimo.ERR_INVALID_ARG),
])
def test_invalid_descriptors(bad, code):
    b = {"B": 64, "U": 8, "cluster_size": [32, 32]}
    b.update({k: v for k, v in bad.items() if k in b})
    arr, keep = descs_for([b], K=bad.get("K", 3))
    assert build(arr, 1, batched.default_plan())[0] == code


def test_cluster_too_large_for_budget_is_unsupported():
    arr, keep = descs_for([{"B": 512, "U": 64, "cluster_size": [512]}])
    plan = batched.default_plan(group_bytes=64 * 1024)
    assert build(arr, 1, plan)[0] == cdmimo.ERR_UNSUPPORTED


def test_table_buffer_too_small():
    arr, keep = descs_for([{"B": 64, "U": 8, "cluster_size": [32, 32]}])
    plan = batched.default_plan()
    L = cdmimo.lib()
    assert L.cdmimo_batch_build(arr, 1, ctypes.byref(plan), None, 0) == cdmimo.OK
    buf = np.zeros(plan.table_bytes + 32, np.uint8)
    off = (-buf.ctypes.data) % 16
    assert L.cdmimo_batch_build(arr, 1, ctypes.byref(plan), ctypes.c_void_p(buf.ctypes.data + off),
                                plan.table_bytes - 16) == cdmimo.ERR_WORKSPACE
