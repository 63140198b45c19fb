"""Host logic of bench.py's N > 1 path on CPU: two gloo ranks (world size 2,
rendezvous on 127.0.0.1).  Each rank reports a different step time; both must
see the slowest one, and the whole-job value counts the units of every rank
over that time.  The replicas share no data, so these reductions are the only
collectives of the path."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank, world = dist.get_rank(), dist.get_world_size()
ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
value = bench.whole_job_value(1000.0, ms * 1e-3, world)
dist.barrier()
print(json.dumps({"rank": rank, "world": world, "ms": ms, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("gloo ranks did not finish")
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2
        assert o["ms"] == 15.0                       # the slower rank's time, on both ranks
        assert o["value"] == pytest.approx(2 * 1000.0 / 15e-3)


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_value(100.0, 0.5, 1) == 200.0


@pytest.mark.parametrize("which", ["c1", "c5"])
def test_config_oracle_baselines_report_their_sample(which):
    # the cpu_baseline leg of `bench.py --config` (no GPU): a bounded oracle
    # sample with its throughput (c1) or seconds per gradient (c5)
    sys.path.insert(0, ROOT)
    import bench
    r = bench.oracle_config_baseline(which)
    assert r["value"] > 0 and r["s"] > 0 and r["sample"]
    assert r["unit"] == ("RHS*unknowns/s" if which == "c1" else "s per gradient")
