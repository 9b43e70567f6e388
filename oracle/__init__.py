"""Plain FP64 CPU oracle for the Gutzwiller-projection PQMC sweep.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is written for a reader who checks it against the paper by eye: plain numpy,
no blocking, no fusion, no reordering beyond what the algorithm states.  It
shares no code with the CUDA path (``paper_2303_13403_gb300``) and never
imports it.

Modules
-------
philox    Philox4x32-10 counter-based generator (Salmon et al., SC'11).
lattice   Hopping matrices of the honeycomb model, Eq. (2), and of the square
          t-t' lattice used for the doped workload.
hs        Hubbard-Stratonovich couplings: Eq. (1) (Gutzwiller factor) and the
          same identity for the Trotterised U term (Method section).
trial     Neel mean-field trial Slater determinant |psi_N> (honeycomb Hubbard
          section, H_N).
pqmc      The PQMC sweep: ratios, Metropolis, Sherman-Morrison / delayed
          updates, slice wrapping, QR-stabilised stacks, measurement.
ed        Fock-space exact diagonalisation and the exact Trotterised
          projection of small clusters.
hs_enum   Brute-force enumeration of all auxiliary fields on tiny systems.

Parity pins (tests/test_oracle_*.py) tie every function here to something
other than itself: Philox known-answer vectors, closed forms at U=0, Fock-space
ED, exact enumeration of the HS sum, invariants of G, and the g=0 reduction.
"""
