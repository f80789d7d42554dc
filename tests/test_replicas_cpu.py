"""Multi-process host logic of replica runs (world size 2, gloo, CPU): the benchmark's barrier and
max-over-ranks timing, and the reference arm printing on rank 0 only."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import os, sys, io, contextlib, argparse
sys.path.insert(0, {root!r})
import bench
rank, world, _ = bench._dist()
bar = bench._Barrier(world, None, backend="gloo")
bar.barrier()
assert bar.max(float(rank + 1)) == float(world)
assert bar.max(-float(rank)) == 0.0
args = argparse.Namespace(workload="qv30", steps=1, warmup=0, ref_gates_per_step=1)
out = io.StringIO()
if rank != 0:
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(args) == 0
    assert out.getvalue() == ""
bar.barrier()
bar.close()
print("rank", rank, "ok")
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_barrier_max_and_rank0_output():
    port = _free_port()
    code = _CHILD.format(root=ROOT)
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    for rank, (rc, o, e) in enumerate(outs):
        assert rc == 0, e[-2000:]
        assert f"rank {rank} ok" in o
