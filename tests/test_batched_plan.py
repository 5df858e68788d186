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


DESC_DT = np.dtype([("H", "<u8"), ("V", "<u8"), ("N0", "<u8"), ("out", "<u8"), ("op", "<i4"), ("n_sc", "<i4"),
                    ("n_sym", "<i4"), ("B", "<i4"), ("U", "<i4"), ("C", "<i4"), ("K", "<i4"), ("fuse", "<i4"),
                    ("inv_Ex", "<f4"), ("rho_c", "<f4"), ("item0", "<i4"), ("group0", "<i4"), ("n_groups", "<i4"),
                    ("bulk", "<i4")])
GROUP_DT = np.dtype([(k, "<i4") for k in ("c0", "c1", "cl0", "n_lanes", "h_entries", "padded", "row_bytes",
                                          "packed")])
CLUSTER_DT = np.dtype([(k, "<i4") for k in ("off", "size", "A", "L", "soff", "lane0")])


def parse_table(table):
    hdr = np.frombuffer(table[:32].tobytes(), dtype=np.int32)
    n_desc, n_items, n_groups, n_clusters = hdr[:4]
    off_desc, off_group, off_cluster = hdr[4:7].view(np.uint32)
    descs = np.frombuffer(table[off_desc:off_desc + n_desc * DESC_DT.itemsize].tobytes(), DESC_DT)
    groups = np.frombuffer(table[off_group:off_group + n_groups * GROUP_DT.itemsize].tobytes(), GROUP_DT)
    clus = np.frombuffer(table[off_cluster:off_cluster + n_clusters * CLUSTER_DT.itemsize].tobytes(), CLUSTER_DT)
    return descs, groups, clus


@pytest.mark.parametrize("P,T", [(16, 512), (16, 256), (8, 384), (32, 256)])
def test_table_order_and_packed_lane_layout(P, T):
    """Descriptors enter the table longest item first (K U n_sym B, stable); in packed groups (P = 16
    or 8, every A <= 128 / P) each tile width starts at a warp boundary, lanes of different clusters
    are disjoint and every group's lanes fit the CTA."""
    g = np.random.default_rng(5)
    blocks = []
    for _ in range(40):
        B = int(g.choice([128, 256, 512]))
        cs = wl.random_partition(g, B)
        if g.random() < 0.2:
            cs = [128] + cs[:-1] if sum(cs[:-1]) + 128 == B else cs
        blocks.append({"B": B, "U": int(g.integers(8, 65)), "cluster_size": cs})
    arr, keep = descs_for(blocks)
    rc, table = build(arr, len(blocks), batched.default_plan(P=P, threads=T, group_bytes=96 * 1024))
    assert rc == cdmimo.OK
    descs, groups, clus = parse_table(table)
    work = descs["K"].astype(np.int64) * descs["U"] * descs["n_sym"] * descs["B"]
    assert np.all(np.diff(work) <= 0)
    assert sorted(descs["H"].tolist()) == sorted(arr[i].H for i in range(len(blocks)))
    assert np.all(np.diff(descs["item0"]) == descs["n_sc"][:-1])
    n_packed = 0
    for d in descs:
        for gi in range(d["group0"], d["group0"] + d["n_groups"]):
            gr = groups[gi]
            cl = clus[gr["cl0"]:gr["cl0"] + gr["c1"] - gr["c0"]]
            assert gr["n_lanes"] <= T
            spans = sorted((c["lane0"], c["lane0"] + d["n_sym"] * c["A"], c["A"]) for c in cl)
            assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
            assert max(s[1] for s in spans) == gr["n_lanes"]
            packed = P in (8, 16) and all(c["A"] <= 128 // P for c in cl)
            assert gr["packed"] == int(packed)
            if packed:
                n_packed += 1
                for a, b in zip(spans, spans[1:]):
                    assert a[2] >= b[2]
                    if a[2] != b[2]:
                        assert b[0] % 32 == 0
    assert (n_packed > 0) == (P in (8, 16))


def test_p8_thread_limit():
    arr, keep = descs_for([{"B": 64, "U": 8, "cluster_size": [32, 32]}])
    assert build(arr, 1, batched.default_plan(P=8, threads=512))[0] == cdmimo.ERR_INVALID_ARG
    assert build(arr, 1, batched.default_plan(P=8, threads=384))[0] == cdmimo.OK


def test_occupancy_candidates_fill_the_sm():
    """Each derived candidate's plan fits its CTAs per SM in shared memory, and one budget step more
    would not (or would not build); shapes whose CTAs cannot hold a U = 64, 64-antenna cluster are
    left out."""
    g = np.random.default_rng(9)
    blocks = []
    for _ in range(60):
        B = int(g.choice([128, 256, 512]))
        blocks.append({"B": B, "U": int(g.integers(8, 65)), "cluster_size": wl.random_partition(g, B)})
    arr, keep = descs_for(blocks)

    class Stub:  # what the planner reads of a Batch
        descs, items = arr, blocks

    cands = batched.occupancy_candidates(Stub)
    shapes = {(c["P"], c["threads"], c["ctas_per_sm"]) for c in cands}
    assert shapes <= set(batched.OCCUPANCY_SHAPES) and (16, 512, 1) in shapes and (8, 384, 2) in shapes
    for c in cands:
        limit = batched.SMEM_PER_SM // c["ctas_per_sm"] - batched.SMEM_RESERVED_PER_CTA
        sm = batched.plan_smem(Stub, batched.default_plan(**c))
        assert sm is not None and sm <= limit
        more = batched.plan_smem(Stub, batched.default_plan(**dict(c, group_bytes=c["group_bytes"] + 4096)))
        assert more is None or more > limit or c["group_bytes"] + 4096 > limit
