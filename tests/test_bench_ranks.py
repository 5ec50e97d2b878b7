"""The N > 1 path of bench.py on CPU: two gloo ranks combine their timed
regions (time = the slowest rank's, edges = the sum over ranks), and the
reference arm does its work on rank 0 only."""
import json
import os
import socket
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
r = dist.get_rank()
t, u = bench.combine_ranks(10.0 + 5.0 * r, 1000 + 7 * r, dist, "cpu")
print(json.dumps({"rank": r, "t": t, "u": u}))
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_combine_ranks_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, BENCH_ROOT=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=180)
            assert p.returncode == 0, err[-2000:]
            outs.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["t"] == 15.0            # the slower rank's time
        assert o["u"] == 1000 + 1007     # every rank's edges


def test_combine_ranks_without_process_group():
    import bench
    assert bench.combine_ranks(12.5, 99, None) == (12.5, 99)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = types.SimpleNamespace(ref_queries=10, warmup=1, steps=1)
    assert bench.run_reference(args, {"kind": "gmm", "n": 10, "dim": 4, "seed": 0}) == 0
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("env,expect", [({}, (0, 1, 0)),
                                        ({"RANK": "3", "WORLD_SIZE": "4", "LOCAL_RANK": "1"}, (3, 4, 1))])
def test_dist_env(monkeypatch, env, expect):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    assert bench.dist_env() == expect
