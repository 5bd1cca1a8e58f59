"""Plain, slow, obviously-correct CPU oracle for the state-vector simulator of
arXiv:1805.04708 (JUQCS).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
leg / ``--impl reference`` arm of ``bench.py`` use it.  It shares no code with
the CUDA path: its gate table is retyped from the paper's instruction set
(Appendix A), its arithmetic is numpy complex128 (FP64), and its reductions are
compensated FP64 sums.

Modules
-------
gates     : the 2x2 / 4x4 / 8x8 matrices of Appendix A.
statevec  : |0..0>, the pair update of Eq. (NUM2) for any U(2) with 0..2
            controls, dense k-qubit gates, index permutations, SHORBOX, the
            projections CLEAR/SET, and the reductions (norm Eq. (STAT1),
            single-qubit probabilities of Sec. 2, BEGIN MEASUREMENT, register
            marginals).
adapt2    : the 2-byte adaptive polar encoding of Sec. 4.1, step by step.
shor      : the classical side of Shor's algorithm (Sec. 5.4) and the
            closed-form x-register distribution after SHORBOX + QFT.
circuit   : runs a gate list (mnemonic records) through statevec / adapt2.
measure   : M, CLEAR, SET, GENERATE EVENTS and the DEPOLARIZING CHANNEL of
            Appendix A, with the SplitMix64 counter-based generator for
            seeded draws.
aux       : the auxiliary-variable method of Sec. 4.2 (discrete
            Hubbard-Stratonovich rewrite of controlled phases, amplitudes as a
            sum over 2^P sign configurations of single-qubit products).
program   : parses and runs a program in the instruction language of
            Appendix A (the front-end), on the complex128 oracle or the
            adaptive encoding's emulation.

Parity pins: every function here is pinned in ``tests/test_oracle_*.py``
against brute force, closed forms or the paper's printed tables.  Functions
without such a pin are listed as "parity unpinned" in their docstring (none at
present).
"""
