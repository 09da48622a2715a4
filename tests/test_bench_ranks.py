"""Host logic of bench.py for N > 1 ranks, on CPU: two gloo ranks agree on
the slowest rank's time and on the whole-job rate; under the reference arm
only rank 0 prints its line and the others exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 3.0 * rank, dist, "cpu")
        out[rank] = (ms, bench.whole_job_mlups(world, 1_000_000, 50, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(rank_main, args=(world, free_port(), out), nprocs=world, join=True)
        got = dict(out)
    assert got[0] == got[1]
    ms, value = got[0]
    assert ms == 13.0
    assert value == pytest.approx(2 * 1_000_000 * 50 / 0.013 / 1e6)


def test_without_a_group_the_local_time_stands():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.whole_job_mlups(1, 2_000_000, 10, 20.0) == pytest.approx(1000.0)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if rank:
        assert lines == []
    else:
        assert len(lines) == 1
        d = json.loads(lines[0])
        assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
        assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_step_kernel_traffic_record_matches_the_kernel_sources():
    """The DRAM traffic the bench reports comes from an ncu record keyed by
    the step kernels' source hash; a kernel edit without a new capture
    would silently drop it (the bench then reports null), so the committed
    record must belong to the committed sources."""
    import json
    import bench
    with open(bench.PROFILE_JSON) as fh:
        rec = json.load(fh)
    assert rec["source_sha256"] == bench.kernel_source_hash()
    assert bench.traffic_per_launch(rec["precision"], rec["workload"], rec["kernel"].split("<")[0]) == \
        rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]
