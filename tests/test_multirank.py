"""The multi-process paths of bench.py on CPU, as gloo ranks (world size 2).

Every rank of a multi-GPU run is an independent replica of the workload (the
path is not sharded), so the only collectives are the timing ones: a barrier
around the timed region and the max over ranks of the elapsed time."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out: str) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    w, r, local, pg = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(pg)
    m = bench.max_over_ranks(pg, 1.5 + rank)
    with open(f"{out}.{rank}", "w") as f:
        f.write(repr(m))
    pg.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    out = str(tmp_path / "m")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    for rank in range(2):
        assert float(open(f"{out}.{rank}").read()) == 2.5


def test_reference_arm_under_torchrun_prints_one_line():
    # the driver's launch line for N = 2, on CPU: rank 0 times the oracle and
    # prints one JSON line; rank 1 exits without work
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "cavity64"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
