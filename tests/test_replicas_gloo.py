"""The multi-process side of bench.py on CPU: two gloo ranks run the
barrier and the reductions that turn per-rank replica timings into the
whole-job value (iterations summed over ranks, time = slowest rank), and
the reference arm prints only on rank 0.  The method has no data-path
exchange (replicas only), so this is all the multi-GPU path there is."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")

CHILD = r"""
import io, json, os, sys, contextlib
sys.path.insert(0, %(root)r)
import bench
d = bench.Dist()
d.init("gloo")
d.barrier()
rank = d.rank
iters = 100 + rank            # per-rank iterations of the timed steps
ms = 10.0 + 5.0 * rank         # per-rank device time
total = d.reduce(iters, "sum")
slowest = d.reduce(ms, "max")
value = total / (slowest / 1e3)
# the reference arm under torchrun: only rank 0 may print a line
buf = io.StringIO()
if rank != 0:
    with contextlib.redirect_stdout(buf):
        class A: pass
        a = A(); a.workload = "grid4_T20"; a.steps = 1; a.warmup = 0; a.gpus = 2; a.tol = 1e-8
        bench.run_reference(a, d)
d.barrier()
d.close()
print(json.dumps({"rank": rank, "total": total, "slowest": slowest, "value": value,
                  "ref_output": buf.getvalue()}))
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_aggregate_replica_timings():
    port = free_port()
    code = CHILD % {"root": ROOT}
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["total"] == 201.0
        assert o["slowest"] == 15.0
        assert abs(o["value"] - 201.0 / 0.015) < 1e-6
    # rank 1 of the reference arm does no work and prints nothing
    assert outs[1]["ref_output"] == ""
