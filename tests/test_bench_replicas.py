"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks run
independent replicas; the job time is the maximum over ranks and the value
counts the units of all ranks.  The reference arm prints on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [120.0, 200.0][rank]               # rank 1 is the slow one
    t = bench.job_time_ms(local, dist, "cpu")
    v = bench.job_value(1000, 4, world, t)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_value_counts_all_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 200.0
        assert v == pytest.approx(1000 * 4 * 2 / 0.2)


def test_reference_arm_prints_once_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(30000 + os.getpid() % 1000),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "1"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_bench_recount_matches_the_oracle():
    """bench.py's host-side recount of cost and feasibility (used for the
    learned order's results) against the oracle's own partition."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth
    g = synth.random_snn(700, 14, 2, size_max=30)
    r = oracle.partition(g, 24, 160)
    assert bench.recount(g, r.part_ids, 24, 160) == (r.cost, True)
    assert bench.recount(g, r.part_ids, int(r.part_weight.max()) - 1, 160)[1] is False
    assert bench.recount(g, r.part_ids, 24, int(r.part_inbound.max()) - 1)[1] is False
