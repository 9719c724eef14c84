"""The multi-GPU path: independent replicas, one scan per GPU, no collective
on the data path.  Its host logic is the step time's maximum over ranks (the
slowest replica sets the step) and the whole-job throughput (the units of
all ranks over that time).  Exercised here with two gloo ranks on the CPU.
Under torchrun the reference arm runs on rank 0 alone; the other ranks exit
0 without output."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world_size, port, ms, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    sys.path.insert(0, ROOT)
    import bench
    step_ms = bench.max_over_ranks(ms[rank], "cpu")
    value = bench.replica_value(5.12e10, world_size, step_ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, step_ms, value))


def test_two_gloo_ranks_take_the_slowest_step_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms = [118.7, 131.9]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in got] == [0, 1]
    for _, step_ms, value in got:
        assert step_ms == pytest.approx(131.9)
        # both replicas' station-samples over the slower replica's step
        assert value == pytest.approx(2 * 5.12e10 / 0.1319)


def test_one_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(118.7, "cpu") == 118.7
    assert bench.replica_value(5.12e10, 1, 118.7) == pytest.approx(5.12e10 / 0.1187)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_line_with_the_contract_keys():
    """rank 0 (no torchrun): the FP64 oracle timed on a bounded sample, with
    the same metric and unit as the GPU arm and a zero-copy e2e."""
    import json
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "station-samples/s" and d["unit"] == d["metric"]
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
