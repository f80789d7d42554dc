"""CPU oracle for the cache-blocked state-vector simulator -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct restatement of what the method computes, in
complex128, written from the paper (Doi & Horii, "Cache Blocking Technique to Large Scale
Quantum Computing Simulation on Supercomputers"):

* ``gates``    -- gate matrices: u3 (Sec. II.A, Eq. 1), CNOT (Eq. 2) and the standard gates
                  the workloads use.
* ``sim``      -- the per-gate state-vector update of Sec. II.A (pairs ``i`` and
                  ``i XOR 2^k``) in C with OpenMP (``sv_oracle.c``), a dense 2^n x 2^n
                  Kronecker-embedding brute force for n <= 10, probabilities (Sec. II.A), inverse-CDF
                  sampling and Pauli expectation values.
* ``planner``  -- the cache-blocking transpiler of Sec. IV.A (Listing 3) and the final output
                  reordering of Sec. IV.C (Fig. 10 case (b)), as an independent Python
                  implementation whose swap schedule is the result the library's planner must
                  match bit-exactly.
* ``mlp``      -- a numpy reference of the planner cost-model network (forward, backward, Adam)
                  used to check the library's GPU training kernels.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import, call, link or execute anything here.  The CUDA library never does: it shares no
code, header, table or helper with this package, and it fails loudly rather than falling
back to it.

Pins (checked by ``tests/test_oracle_*.py`` without a GPU): literal Eq. 1/Eq. 2 values,
unitarity, Bell/GHZ amplitudes, the QFT closed form, the dense brute force at n <= 10,
unit norm, mirror circuits, the Listing 2 index-map bijection, and planner validity and
equivalence; for ``mlp``: central finite differences, a hand-computed case, the closed form of
Adam's first step and dead relu units.  The paper's own worked transpiler example (Fig. 9, its count of added swap gates) is an
image that is not available, so the planner's swap *count* is parity unpinned; its schedule
is pinned by validity + simulation equivalence and by agreement with the library's planner.
"""
