"""The N > 1 bench path on CPU: two gloo ranks (world_size 2) exercise the host logic of
`bench.py --gpus 2` under torchrun: distinct per-rank batches (weak scaling, no data exchange), the
max-over-ranks timing and the whole-job throughput; and the reference arm prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [1.5, 2.5][rank]
    m = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
    up, _ = bench.make_inputs(bench.rank_seed(rank))
    h = torch.from_numpy(np.ascontiguousarray(up["H"][:2, :2, :4].real)).to(torch.float64)
    hs = [torch.zeros_like(h) for _ in range(world)]
    dist.all_gather(hs, h)
    dist.barrier()
    out[rank] = (m, bench.whole_job_value(16800, world, m), bool(torch.equal(hs[0], hs[1])))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_timing_and_weak_scaling():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        m, value, same_inputs = out[r]
        assert m == 2.5  # both ranks see the slowest rank's time
        assert abs(value - 2 * 16800 / 2.5e-3) < 1e-6  # all ranks' vectors over that time
        assert not same_inputs  # each rank has its own batch


def test_reference_arm_prints_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "vectors/s"


def test_strong_scaling_shards_cover_the_batch():
    """bench.py --scaling strong: every rank loads the same batch and keeps its subcarrier range; the
    ranges partition the batch and each rank's arrays are exactly its rows."""
    import bench
    from paper_1902_08653_gb300 import parallel

    up, dl = bench.make_inputs(bench.rank_seed(0))
    rows = []
    for r in range(3):
        lo, hi = parallel.subcarrier_shard(bench.N_SC, 3, r)
        su, sd = bench.shard_batch(up, lo, hi), bench.shard_batch(dl, lo, hi)
        assert su["H"].shape[0] == su["Y"].shape[0] == su["N0"].shape[0] == sd["S"].shape[0] == hi - lo
        assert np.array_equal(su["H"], up["H"][lo:hi]) and su["M"] == up["M"]
        rows.append(su["N0"])
    assert np.array_equal(np.concatenate(rows), up["N0"])
