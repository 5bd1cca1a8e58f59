"""Run a gate list (mnemonic records) through the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A gate record is (name, qubits, params) with the mnemonics of Appendix A
(H, X, Y, Z, S, S+, T, T+, U1, U2, U3, +X, -X, +Y, -Y, R, CNOT, U, TOFFOLI,
I), plus RZ (z rotation) and MAT / CMAT (an explicit 2x2 matrix, params =
8 floats row-major (re, im), with 0..2 leading control qubits).
"""
import math
import numpy as np

from . import gates, statevec as sv
from .adapt2 import AState


def run(v, N, records):
    """Apply every record to the complex128 state v, in order."""
    for rec in records:
        if rec[0].upper() == "I":
            continue
        controls, target, U = gates.as_controlled(rec)
        sv.apply_controlled_u2(v, N, controls, target, U)
    return v


def _phase_m(f):
    """m if the unit-modulus factor f equals e^{i pi m/128} (m integer), else None."""
    if abs(abs(f) - 1.0) > 1e-15:
        return None
    m = math.atan2(f.imag, f.real) * 128.0 / math.pi
    mr = round(m)
    return int(mr) if abs(m - mr) <= 1e-9 else None


def _is_permutation(U):
    return U[0, 0] == 0 and U[1, 1] == 0 and U[0, 1] == 1 and U[1, 0] == 1


def _subspace(N, controls, target, bit):
    i = np.arange(1 << N, dtype=np.int64)
    on = ((i >> target) & 1) == bit
    for c in controls:
        on &= ((i >> c) & 1) == 1
    return on


def run_adapt2(a, records):
    """Apply records to an adaptive-encoded state (Sec. 4.1).

    X-type gates (X, CNOT, TOFFOLI) only move codes.  Diagonal and
    anti-diagonal unitaries (Z, S, T, R, U(k), Y, RZ, ...) leave every |z|
    unchanged, so r0 and r1 are kept: with phases e^{i pi m/128} the codes
    move and b1 gains m; with other phases the state is decoded, multiplied
    and re-encoded with the same (r0, r1).  Every other gate is
    decode -> exact gate -> retune (r0, r1) -> encode."""
    N = a.N
    for rec in records:
        if rec[0].upper() == "I":
            continue
        controls, target, U = gates.as_controlled(rec)

        def gate(x, controls=controls, target=target, U=U):
            sv.apply_controlled_u2(x, N, controls, target, U)

        if _is_permutation(U):
            a.permute(gate)
            continue
        diag = U[0, 1] == 0 and U[1, 0] == 0
        anti = U[0, 0] == 0 and U[1, 1] == 0
        if diag or anti:
            f0, f1 = (U[0, 0], U[1, 1]) if diag else (U[0, 1], U[1, 0])
            m0, m1 = _phase_m(f0), _phase_m(f1)
            if m0 is not None and m1 is not None:
                if anti:
                    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
                    a.permute(lambda x: sv.apply_controlled_u2(x, N, controls, target, X))
                steps = np.where(_subspace(N, controls, target, 0), m0, 0) + \
                    np.where(_subspace(N, controls, target, 1), m1, 0)
                a.phase_steps(steps)
            else:
                a.arithmetic(gate, retune_range=False)
            continue
        a.arithmetic(gate)
    return a
