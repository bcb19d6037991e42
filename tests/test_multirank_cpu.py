"""The N > 1 host path of the benchmark on CPU (gloo, world size 2): every
rank runs its own replica (no data-path collective); the only cross-rank
operations are the barrier around the timed region and the max over ranks of
the elapsed time, from which rank 0 forms the whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        elapsed_ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
        ms_max = bench.max_over_ranks(ws, elapsed_ms)
        rate = bench.aggregate_rate(ws, 4, 1 << 20, ms_max)
        bench.barrier(ws)
        q.put((rank, ms_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, rate in res:
        assert ms_max == 15.0                           # the slowest rank's time
        assert rate == pytest.approx(2 * 4 * (1 << 20) / 15e-3 / 1e6)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, ref_frames = 1, 0, 16
    bench.run_reference(A, 2, 1)
    assert capsys.readouterr().out == ""


def test_reference_arm_rank0_prints_the_contract_line():
    """`bench.py --impl reference` on one process: the oracle timed on a host
    core, one JSON line with the contract's keys (runs without a GPU)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--ref-frames", "16"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3   # W >= 3 enforced
    for k in ("metric", "value", "unit", "n_gpus", "ms_per_step", "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
