"""The bench's multi-rank host logic on CPU (gloo, world size 2): the step
time is the slowest rank's, the job value sums every replica's bytes, and the
reference arm prints from rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = 100.0 + 50.0 * rank          # rank 1 is the slow one
    t = bench.max_over_ranks(elapsed)
    v = bench.job_throughput(world, 1e9, 10, t)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "v": v}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo(tmp_path):
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["t"] == 150.0
        assert abs(d["v"] - 2 * 1e9 * 10 / 0.150 / 1e9) < 1e-9


def test_single_rank_helpers_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 2e9, 5, 1000.0) == 10.0


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_on_rank0_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-qubits", "8", "--gpus", "2"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    if rank == 0:
        d = json.loads(lines[-1])
        assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["n_gpus"] == 2
        assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
        import bench
        # the reference arm reports the GPU arm's workload; the bounded sample is stated beside it
        assert d["config"]["workload"] == bench.sweep_workload(30) and "8-qubit" in d["config"]["sample"]
        assert d["metric"] == bench.METRIC and d["higher_is_better"] is True
    else:
        assert lines == []
