"""FP64 CPU oracle for the pilot-wave exact sampler (arXiv 2510.24218).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it. It shares no code, tables
or helpers with the CUDA path; both sides read their inputs from the seeded
generators in ``workloads.py`` and build everything else on their own.

Modules (each function cites the passage of the paper it follows):

* ``philox``      Philox4x32-10 counter-based generator (Salmon et al., SC'11)
                  and the 53-bit uniform draw used by both samplers.
* ``circuit``     gate and Kraus-channel semantics, the QAOA circuit of
                  App. D, gate classification and BlockDecompose (Alg. 1).
* ``statevector`` dense state-vector and density-matrix simulation.
* ``tn``          amplitudes <x|C_t|0^n> by plain variable elimination over
                  the circuit's tensor network with diagonal legs identified
                  (App. A).
* ``sampler``     Alg. 1 (Sample/UpdateState) and Alg. 2 (NoisySample/AddGate/
                  PropagateX) written out step by step, plus exact enumeration
                  of the Markov chain's output distribution for tiny circuits.
* ``closed_form`` the p=1 QAOA expectation <Z_u Z_v> in closed form.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; none is marked "parity unpinned".
"""
