"""Host-side pieces of bench.py on CPU: the whole-job aggregation over replicas (world size
2, gloo), and the reference arm (the CPU oracle), including the ranks that do no work."""
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


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: 1e9 (r + 1) point updates in 2 + r seconds
    value, t_max = bench.whole_job(1e9 * (rank + 1), 2.0 + rank, world)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"value": value, "t_max": t_max}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_is_sum_over_max_time_gloo(tmp_path):
    """value = all ranks' updates / the slowest rank's time, identical on every rank."""
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["t_max"] == pytest.approx(3.0)
        assert got["value"] == pytest.approx(3e9 / 3.0 / 1e9)


def test_whole_job_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(4e9, 2.0, 1) == (2.0, 2.0)


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl",
                           "reference", "--steps", "1", "--warmup", "0"], env=env,
                          capture_output=True, text=True, timeout=600, cwd=ROOT)


def test_reference_arm_other_ranks_do_no_work():
    p = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_reference_arm_prints_one_json_line():
    """The oracle on the host cores: one line with the base contract's keys."""
    p = _run_reference({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GLUP/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_recorded_traffic_matches_the_profiled_kernel_source():
    """The roofline's measured DRAM traffic is reported only while the march kernel's
    source is the one the ncu counters were taken from (profiles/traffic.txt keys it by
    the source hash); this fails as soon as that source changes without a new capture."""
    import bench
    assert bench.recorded_traffic("march_kernel") is not None, bench.kernel_sha()
