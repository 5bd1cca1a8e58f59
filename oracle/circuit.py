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


def _pi128_steps(U):
    """If U = diag(1, e^{i pi m/128}) exactly in angle (|u11| == 1 to 1e-15),
    return m; else None."""
    if U[0, 1] != 0 or U[1, 0] != 0 or U[0, 0] != 1:
        return None
    if abs(abs(U[1, 1]) - 1.0) > 1e-15:
        return None
    m = math.atan2(U[1, 1].imag, U[1, 1].real) * 128.0 / math.pi
    mr = round(m)
    if abs(m - mr) > 1e-9:
        return None
    return int(mr)


def _is_permutation(U):
    return U[0, 0] == 0 and U[1, 1] == 0 and U[0, 1] == 1 and U[1, 0] == 1


def run_adapt2(a, records):
    """Apply records to an adaptive-encoded state (Sec. 4.1).  X-type gates
    (X, CNOT, TOFFOLI) move codes; diag(1, e^{i pi m/128}) phases (Z, S, T,
    R(k<=8), U(k<=8), ...) add m to b1 where the controls and target are 1;
    every other gate is decode -> exact gate -> retune -> encode."""
    N = a.N
    for rec in records:
        if rec[0].upper() == "I":
            continue
        controls, target, U = gates.as_controlled(rec)
        if _is_permutation(U):
            a.permute(lambda x: sv.apply_controlled_u2(x, N, controls, target, U))
            continue
        m = _pi128_steps(U)
        if m is not None:
            i = np.arange(1 << N, dtype=np.int64)
            on = ((i >> target) & 1) == 1
            for c in controls:
                on &= ((i >> c) & 1) == 1
            a.phase_steps(np.where(on, m, 0))
            continue
        a.arithmetic(lambda z: sv.apply_controlled_u2(z, N, controls, target, U))
    return a
