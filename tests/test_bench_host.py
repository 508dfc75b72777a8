"""Host-side logic of bench.py that runs without a GPU: the cross-rank rate
(units of all ranks over the slowest rank's time) with two gloo ranks, and the
reference arm (the timed oracle) under a launcher's rank variables."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        # rank r processed (r + 1) * 1000 units in 0.5 + r seconds
        rate = bench.world_rate((rank + 1) * 1000.0, 0.5 + rank, world, "cpu")
        out.put((rank, rate))
    finally:
        dist.destroy_process_group()


def test_world_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    # (1000 + 2000) units / max(0.5, 1.5) s on every rank
    assert got[0] == pytest.approx(2000.0) and got[1] == pytest.approx(2000.0)


def test_world_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.world_rate(300.0, 1.5, 1) == pytest.approx(200.0)


def _run_reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                           "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_reference(1, 2)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_rank0_line():
    r = _run_reference(0, 1)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "DoF-updates/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_profiled_traffic_matches_shape_and_order(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    # the committed summary has lines for the orders the autotuner picks
    path = os.path.join(ROOT, "profiles", bench.TRAFFIC_PROFILE)
    for groups in (6, 12):
        t = bench.profiled_traffic(path, 0, groups, 196608, "bulk")
        assert t is not None and 0.9 < t / 374341632 < 1.3
    f = tmp_path / "p.md"
    f.write_text("traffic_bytes_per_element_stage variant=0 tile_groups=6 loads=bulk: 1922\n"
                 "traffic_bytes_per_element_stage variant=0 tile_groups=6 loads=per_thread: 1950\n"
                 "traffic_bytes_per_element_stage variant=1 tile_groups=6 loads=bulk: 2000\n")
    assert bench.profiled_traffic(str(f), 0, 6, 10) == 19220
    assert bench.profiled_traffic(str(f), 0, 6, 10, "per_thread") == 19500
    assert bench.profiled_traffic(str(f), 1, 6, 10) == 20000
    assert bench.profiled_traffic(str(f), 1, 6, 10, "per_thread") is None
    assert bench.profiled_traffic(str(f), 0, 3, 10) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.md"), 0, 6, 10) is None
