"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): replicas only, so the only
collective is the max over ranks of the timed interval, and the job's value aggregates all ranks.
The reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], world)
        out[rank] = (ms, bench.job_value(world, 10, 1000, ms))
    finally:
        dist.destroy_process_group()


def test_timed_interval_is_the_max_over_ranks_and_value_aggregates_ranks():
    world, times = 2, [12.5, 40.0]
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 40.0
        assert value == pytest.approx(world * 10 * 1000 / 0.040)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_bench_builds_each_instance_drive_for_both_sides():
    """The benchmark hands the library and the oracle the same grid, force and plate speed per
    instance: square cells for the force-driven workloads, the paper's rows for the Couette one."""
    import bench
    import oracle
    rough = bench.instances("rough")[0]
    d = bench.drive(rough)
    assert d == {"ly": 1.0, "force": 1.0, "top_wall_u1": 0.0, "dx1": 0.0, "row_heights": None}
    p = bench.oracle_problem(oracle, rough)
    assert p.dy is None and abs(p.dx - 1.0 / 128) < 1e-15
    cou = bench.instances("couette")
    rough_c, smooth_c = cou[0], cou[3]
    d = bench.drive(rough_c)
    assert d["force"] == 0.0 and d["top_wall_u1"] == 1.0 and abs(d["dx1"] - 1.0 / 300) < 1e-15
    p = bench.oracle_problem(oracle, rough_c)
    assert p.dy.shape == (160,) and abs(p.ly - d["row_heights"].sum()) < 1e-15 and p.top_u == 1.0
    q = bench.couette_q_star(cou, [0.49, 0.48, 0.46, 0.5, 0.5, 0.5])
    assert set(q) == {"0.1", "1", "10"} and abs(q["10"]["Q_star"] - 0.92) < 1e-15
    assert bench.updates_per_step(bench.instances("rough")) == 3 * 14720 * 1024
