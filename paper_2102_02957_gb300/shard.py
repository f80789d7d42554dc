"""One state partitioned over several GPUs (one process each) on its top qubits.

Sec. II.B of Doi & Horii divides the state vector into pieces, one per process, on the highest
qubits; Sec. IV.C runs the cache-blocking plan on every piece and exchanges data only where a
chunk_swap crosses the partition (Fig. 10: case (a), a chunk qubit with a partition qubit; case
(b), two partition qubits, in the output reordering).  With G = 2^g pieces, rank r holds the
2^(n-g) amplitudes whose index is (r << n_l) | k, n_l = n - g.

Per plan op (the paper's layout: contiguous chunks of c <= n_l bits and chunk_swap rounds):

* a blocking section runs on every piece alone (sv_apply_plan_ops);
* a round's pairs with both bits below n_l are a local permutation (sv_apply_plan_ops again);
* a pair (s, h) with s < n_l <= h swaps state bits s and h.  Let b = bit h - n_l of the rank:
  amplitudes with local bit s equal to b stay, the others move to the partner rank
  r ^ 2^(h - n_l) at the same local index with bit s flipped -- exactly the places the
  partner's outgoing half comes back to.  So each rank sends its half with bit s = 1 - b and
  receives the partner's half into those places (half a piece each way);
* a pair (a, h) with both bits at or above n_l relabels pieces: ranks whose bits a - n_l and
  h - n_l differ trade their whole piece with r ^ (2^(a - n_l) | 2^(h - n_l)); the others keep it.

The pairs of one round are disjoint transpositions, so they commute and run one after another.
The data exchange itself is a pair of point-to-point transfers (torch.distributed: NCCL between
GPUs, gloo between CPU processes); every other step is the library's own kernels."""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Step:
    kind: str           # "ops": plan ops [a, b); "half": exchange half; "whole": exchange the piece
    a: int = 0          # ops: first op; half: local bit s
    b: int = 0          # ops: end op; half: value of bit s that is sent (and received)
    partner: int = -1   # half / whole: the other rank (== own rank: nothing to do)


def parse_ops(stream):
    """(kind, pairs) of every op of a serialised plan (sv_plan_serialize): kind 1 = chunk_swap
    round, 2 = blocking section, 3 = reordering round; pairs are empty for sections."""
    it = iter(stream)
    _n, _c, _reserve, _restore, nops = (next(it) for _ in range(5))
    ops = []
    for _ in range(nops):
        kind = next(it)
        if kind in (1, 3):
            cnt = next(it)
            ops.append((kind, [(next(it), next(it)) for _ in range(cnt)]))
        else:
            if kind == 4:
                raise ValueError("gathered-chunk plans are not partitioned (use gather_pinned = 0)")
            cnt = next(it)
            for _ in range(4 * cnt):
                next(it)
            ops.append((kind, []))
    return ops


def schedule(ops, n_local: int, rank: int):
    """The steps of one rank.  Every rank gets the same sequence of step kinds (ranks that keep
    their piece in a "whole" step get partner == rank), so ranks that run in lock step pair up."""
    steps = []
    begin = 0
    for oi, (kind, pairs) in enumerate(ops):
        crossing = [(p, q) for p, q in pairs if max(p, q) >= n_local]
        if not crossing:
            continue
        # local work up to and including this round (its local pairs), then its exchanges
        steps.append(Step("ops", begin, oi + 1))
        begin = oi + 1
        for p, q in crossing:
            lo, hi = min(p, q), max(p, q)
            if lo < n_local:
                bit = (rank >> (hi - n_local)) & 1
                steps.append(Step("half", lo, 1 - bit, rank ^ (1 << (hi - n_local))))
            else:
                ba = (rank >> (lo - n_local)) & 1
                bb = (rank >> (hi - n_local)) & 1
                other = rank ^ ((1 << (lo - n_local)) | (1 << (hi - n_local))) if ba != bb else rank
                steps.append(Step("whole", partner=other))
    if begin < len(ops):
        steps.append(Step("ops", begin, len(ops)))
    return steps


def run(piece, transport, steps):
    """Run one rank's steps.  piece: apply_ops(a, b), pack(bit, value) -> buffer,
    unpack(bit, value, buffer) (bit = -1: the whole piece); transport: exchange(partner, buffer)
    -> the partner's buffer."""
    for st in steps:
        if st.kind == "ops":
            if st.b > st.a:
                piece.apply_ops(st.a, st.b)
        elif st.kind == "half":
            piece.unpack(st.a, st.b, transport.exchange(st.partner, piece.pack(st.a, st.b)))
        elif st.partner != transport.rank:
            piece.unpack(-1, 0, transport.exchange(st.partner, piece.pack(-1, 0)))


def run_lockstep(pieces, steps_per_rank):
    """All ranks' steps in one process (an emulation of G GPUs on one: each exchange is a swap of
    the packed buffers)."""
    nsteps = len(steps_per_rank[0])
    assert all(len(s) == nsteps for s in steps_per_rank)
    for i in range(nsteps):
        kinds = {steps[i].kind for steps in steps_per_rank}
        assert len(kinds) == 1, kinds
        kind = kinds.pop()
        if kind == "ops":
            for piece, steps in zip(pieces, steps_per_rank):
                if steps[i].b > steps[i].a:
                    piece.apply_ops(steps[i].a, steps[i].b)
            continue
        half = kind == "half"
        sent = [piece.pack(steps[i].a, steps[i].b) if half else piece.pack(-1, 0)
                for piece, steps in zip(pieces, steps_per_rank)]
        for r, (piece, steps) in enumerate(zip(pieces, steps_per_rank)):
            p = steps[i].partner
            assert steps_per_rank[p][i].partner == r, "exchange partners must pair up"
            if half:
                piece.unpack(steps[i].a, steps[i].b, sent[p])
            elif p != r:
                piece.unpack(-1, 0, sent[p])


class TorchTransport:
    """Pairwise exchange of equal-size tensors through torch.distributed point-to-point
    transfers (NCCL between GPUs, gloo between CPU processes)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)

    def exchange(self, partner: int, buf):
        import torch
        out = torch.empty_like(buf)
        ops = [self.dist.P2POp(self.dist.isend, buf, partner, self.group),
               self.dist.P2POp(self.dist.irecv, out, partner, self.group)]
        for req in self.dist.batch_isend_irecv(ops):
            req.wait()
        return out


class GpuPiece:
    """One piece on this process's GPU: a StateVector of n_l qubits, driven through the library
    (sv_apply_plan_ops, sv_shard_pack / sv_shard_unpack); exchange buffers are CUDA tensors on
    the current torch stream, which the state uses too."""

    def __init__(self, state, gates, plan):
        self.state, self.gates, self.plan = state, gates, plan

    def apply_ops(self, a: int, b: int):
        self.state.apply_ops(self.gates, self.plan, a, b)

    def _buffer(self, amps: int):
        import torch
        dt = torch.complex64 if self.state.amp_bytes == 8 else torch.complex128
        return torch.empty(amps, dtype=dt, device="cuda")

    def pack(self, bit: int, value: int):
        buf = self._buffer((1 << self.state.n) if bit < 0 else (1 << (self.state.n - 1)))
        self.state.pack(bit, value, buf.data_ptr())
        return buf

    def unpack(self, bit: int, value: int, buf):
        self.state.unpack(bit, value, buf.data_ptr())
