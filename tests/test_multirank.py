"""Multi-rank logic of bench.py on the CPU (gloo, world size 2): the step time
is the maximum over ranks, the value is the whole job's rate, each rank
renders its own view, and only rank 0 runs and prints the reference arm."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r's timings: [step, forward]; rank 1 is slower at the step,
        # rank 0 at the forward
        mine = [10.0 + rank * 5.0, 4.0 - rank]
        got = bench.max_over_ranks(mine, world)
        rate = bench.whole_job_rate(world, got[0])
        cam = bench.rank_camera(rank, 64, 48)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.concatenate([got, [rate], cam.w2c.ravel()]).astype(np.float64))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    for r in (r0, r1):
        assert r[0] == 15.0 and r[1] == 4.0          # element-wise max over ranks
        assert r[2] == pytest.approx(2 * 1000.0 / 15.0)  # two views per slowest step
    assert not np.allclose(r0[3:], r1[3:])           # distinct views per rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.5], 1) == [3.0, 1.5]
    assert bench.whole_job_rate(1, 2.0) == 500.0


def test_frame_roofline_takes_the_larger_time():
    sys.path.insert(0, ROOT)
    import bench
    # 6.8 GB at 6800 GB/s = 1 ms; 20 T lane-ops at 40 T/s = 0.5 s
    r = bench.frame_roofline(6.8e9, 6800.0, 20e12, 40.0, 1000.0)
    assert abs(r["ms_bytes"] - 1.0) < 1e-12 and abs(r["ms_ops"] - 500.0) < 1e-9
    assert r["bound"] == "alu" and abs(r["frac"] - 0.5) < 1e-12
    r = bench.frame_roofline(6.8e9, 6800.0, 0.0, 40.0, 4.0)
    assert r["bound"] == "hbm" and abs(r["frac"] - 0.25) < 1e-12


def test_reference_arm_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
