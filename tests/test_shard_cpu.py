"""A state partitioned over 2, 4 or 8 pieces on its top qubits (the paper's scheme, Sec. II.B and
IV.C, Fig. 10), on the host with no GPU: the exchange schedule of paper_2102_02957_gb300.shard
drives pieces whose local work is the oracle's (sections on physical bits, local bit swaps), and
the gathered pieces must equal the oracle's simulation of the whole circuit (complex128, 1e-12).
Once in one process (all pieces in lock step), once as world-size-2 and -4 gloo process groups
exchanging through torch.distributed."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import circuitgen as cg
from oracle import gates as og
from oracle import planner, sim
from paper_2102_02957_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class HostPiece:
    """One piece as a numpy array; plan ops by the oracle (the plan's gates on their physical
    bits, bit swaps inside the piece)."""

    def __init__(self, state, n_local, desc, plan_ops, as_torch=False):
        self.a = np.ascontiguousarray(state, dtype=np.complex128)
        self.n = n_local
        self.desc = desc
        self.ops = plan_ops
        self.as_torch = as_torch

    def apply_ops(self, a, b):
        for kind, body in self.ops[a:b]:
            if kind in ("swap", "unpermute"):
                for p, q in body:
                    if max(p, q) < self.n:
                        sim.swap_bits(self.a, self.n, p, q)
            else:
                phys = []
                for gi, pq in body:
                    k, qubits, params = self.desc[gi]
                    order, u = og.matrix_of(k, qubits, params)
                    where = {q: p for q, p in zip(sorted(qubits), pq)}
                    phys.append(("unitary", tuple(where[q] for q in order), (u,)))
                sim.apply(self.a, self.n, phys)

    def _index(self, bit, value):
        idx = np.arange(1 << self.n, dtype=np.int64)
        return idx if bit < 0 else idx[((idx >> bit) & 1) == value]

    def pack(self, bit, value):
        out = self.a[self._index(bit, value)].copy()
        if self.as_torch:
            import torch
            return torch.from_numpy(out.view(np.float64).copy())
        return out

    def unpack(self, bit, value, buf):
        if self.as_torch:
            buf = buf.numpy().view(np.complex128)
        self.a[self._index(bit, value)] = buf


def _circuits(n, seed):
    return [("qv", cg.quantum_volume(n, 6, seed)), ("rl", cg.random_layers(n, 5, seed)), ("qft", cg.qft(n)),
            ("mirror", cg.mirror(cg.quantum_volume(n, 3, seed + 1)))]


def _run_lockstep(n, g, desc, c, basis):
    plan = planner.plan_blocking(n, desc, c)
    ops = shard.parse_ops(plan.serialize())
    n_local = n - g
    full = sim.basis_state(n, basis)
    pieces = [HostPiece(full[r << n_local:(r + 1) << n_local], n_local, desc, plan.ops) for r in range(1 << g)]
    steps = [shard.schedule(ops, n_local, r) for r in range(1 << g)]
    shard.run_lockstep(pieces, steps)
    return np.concatenate([p.a for p in pieces]), steps


@pytest.mark.parametrize("n,g,c", [(10, 1, 5), (11, 2, 6), (12, 3, 6), (9, 2, 4)])
def test_partitioned_plan_matches_oracle_lockstep(n, g, c):
    for name, desc in _circuits(n, 7 * n + g):
        basis = cg.basis_index(n, g + 3)
        got, steps = _run_lockstep(n, g, desc, c, basis)
        ref = sim.simulate(n, desc, basis)
        assert np.abs(got - ref).max() < 1e-12, name


def test_schedule_exchanges_only_where_the_partition_is_crossed():
    n, g, c = 12, 2, 6
    desc = cg.quantum_volume(n, 6, 3)
    plan = planner.plan_blocking(n, desc, c)
    ops = shard.parse_ops(plan.serialize())
    n_local = n - g
    crossing = sum(1 for _k, pairs in ops for p, q in pairs if max(p, q) >= n_local)
    for r in range(1 << g):
        steps = shard.schedule(ops, n_local, r)
        exch = [s for s in steps if s.kind != "ops"]
        assert len(exch) == crossing
        for s in exch:
            assert 0 <= s.partner < (1 << g)
            if s.kind == "half":
                # the partner differs in exactly one partition bit, and sends the complementary half
                d = s.partner ^ r
                assert d and d & (d - 1) == 0
                peer = [t for t in shard.schedule(ops, n_local, s.partner) if t.kind != "ops"][exch.index(s)]
                assert peer.partner == r and peer.a == s.a and peer.b == 1 - s.b
        covered = [False] * len(ops)
        for s in steps:
            if s.kind == "ops":
                for k in range(s.a, s.b):
                    assert not covered[k]
                    covered[k] = True
        assert all(covered)


def test_reordering_of_partition_qubits_moves_whole_pieces():
    """A SWAP relabel between two partition qubits ends as a reordering pair of two partition bits
    (Fig. 10 case (b)): pieces trade places whole."""
    n, g, c = 8, 2, 4
    # qubits 6 and 7 are never brought into a chunk, so the relabel stays a reordering of them
    desc = [("h", (q,), ()) for q in range(6)] + [("cx", (0, 5), ()), ("swap", (6, 7), ()), ("h", (1,), ())]
    got, steps = _run_lockstep(n, g, desc, c, basis=0b01110001)
    assert np.abs(got - sim.simulate(n, desc, 0b01110001)).max() < 1e-12
    assert any(s.kind == "whole" for s in steps[0])


_CHILD = r"""
import os, sys
sys.path.insert(0, {root!r})
sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np
import torch
import torch.distributed as dist
import circuitgen as cg
from oracle import planner, sim
from paper_2102_02957_gb300 import shard
from test_shard_cpu import HostPiece
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
g = world.bit_length() - 1
n, c = {n}, {c}
for desc in (cg.quantum_volume(n, 6, 5), cg.random_layers(n, 5, 6), cg.qft(n)):
    basis = cg.basis_index(n, 4)
    plan = planner.plan_blocking(n, desc, c)
    ops = shard.parse_ops(plan.serialize())
    n_local = n - g
    full = sim.basis_state(n, basis)
    piece = HostPiece(full[rank << n_local:(rank + 1) << n_local], n_local, desc, plan.ops, as_torch=True)
    shard.run(piece, shard.TorchTransport(), shard.schedule(ops, n_local, rank))
    mine = torch.from_numpy(piece.a.view(np.float64).copy())
    parts = [torch.empty_like(mine) for _ in range(world)] if rank == 0 else None
    dist.gather(mine, parts, dst=0)
    if rank == 0:
        got = np.concatenate([p.numpy().view(np.complex128) for p in parts])
        err = float(np.abs(got - sim.simulate(n, desc, basis)).max())
        assert err < 1e-12, err
dist.barrier()
dist.destroy_process_group()
print("rank", rank, "ok")
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,n,c", [(2, 11, 6), (4, 12, 6)])
def test_partitioned_plan_over_gloo_processes(world, n, c):
    port = _free_port()
    code = _CHILD.format(root=ROOT, n=n, c=c)
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OMP_NUM_THREADS="2")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    for rank, (rc, o, e) in enumerate(outs):
        assert rc == 0, e[-3000:]
        assert f"rank {rank} ok" in o
