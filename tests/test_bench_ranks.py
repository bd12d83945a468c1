"""bench.py's host logic at world size 2 (CPU, gloo): replicas only -- every rank runs its own
seeded query, the job's time is the slowest rank's (max over ranks), the value counts every
rank's rows, and the reference arm runs on rank 0 alone."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        t = bench.max_over_ranks(10.0 + 5.0 * rank, w, "cpu")   # rank 1 is the slower one
        spec, _ = bench.spec_for("plain_1M", r)
        from paper_2508_04701_gb300 import datagen as dg
        head = dg.gen_fact_host(spec, 0, 64)["fk"].tolist()
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            bench.run_reference(bench.parse(["--impl", "reference", "--steps", "1",
                                                           "--warmup", "0", "--workload", "plain_1M"]))
        dist.barrier()
        q.put((r, w, t, spec.seed, head, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_replicas_max_time_and_reference_on_rank_zero():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, w, t, seed, head, printed = q.get(timeout=240)
        res[r] = (w, t, seed, head, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 2
    assert res[0][1] == res[1][1] == 15.0              # both ranks see the slowest rank's time
    assert (res[0][2], res[1][2]) == (0, 1)            # each rank its own seeded tables
    assert res[0][3] != res[1][3]
    assert '"impl": "reference"' in res[0][4] and res[1][4] == ""


def test_job_value_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rows_per_s(1, 600_000_000, 5.0e-3) == pytest.approx(1.2e11)
    assert bench.job_rows_per_s(4, 600_000_000, 5.0e-3) == pytest.approx(4.8e11)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference runs the CPU oracle and prints one JSON line with the keys the
    bench contract asks of the reference arm (no host<->device bytes: it never touches a GPU)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "plain_1M"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "rows/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "plain_1M"
