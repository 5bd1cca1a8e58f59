"""Gate matrices of the JUQCS instruction set (Appendix A), retyped for the
oracle.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every matrix acts on (psi_0, psi_1) of Eq. (AQS0); controlled gates act on the
target's pair only when every control bit is 1 (the matrices printed for CNOT,
U(k) and TOFFOLI in the basis |control, target>, Appendix A).

RZ is not in Appendix A; it is the standard z rotation diag(e^{-i t/2}, e^{+i t/2})
used by the random-gate workload.  MAT is an explicit 2x2 matrix supplied by the
caller (row-major (re, im) pairs), used for Haar-random U(2) layers.
"""
import math
import numpy as np

_S2 = 1.0 / math.sqrt(2.0)


def one_qubit(name, params=()):
    """Return the 2x2 complex128 matrix of a single-qubit mnemonic (Appendix A)."""
    n = name.upper()
    if n == "I":
        return np.array([[1, 0], [0, 1]], dtype=np.complex128)
    if n == "H":
        return _S2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)
    if n == "X":
        return np.array([[0, 1], [1, 0]], dtype=np.complex128)
    if n == "Y":
        return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    if n == "Z":
        return np.array([[1, 0], [0, -1]], dtype=np.complex128)
    if n == "S":
        return np.array([[1, 0], [0, 1j]], dtype=np.complex128)
    if n == "S+":
        return np.array([[1, 0], [0, -1j]], dtype=np.complex128)
    if n == "T":
        return np.array([[1, 0], [0, (1 + 1j) * _S2]], dtype=np.complex128)
    if n == "T+":
        return np.array([[1, 0], [0, (1 - 1j) * _S2]], dtype=np.complex128)
    if n == "U1":
        (lam,) = params
        return np.array([[1, 0], [0, np.exp(1j * lam)]], dtype=np.complex128)
    if n == "U2":
        phi, lam = params
        return _S2 * np.array([[1, -np.exp(1j * lam)],
                               [np.exp(1j * phi), np.exp(1j * (phi + lam))]],
                              dtype=np.complex128)
    if n == "U3":
        th, phi, lam = params
        c, s = math.cos(th / 2), math.sin(th / 2)
        return np.array([[c, -np.exp(1j * lam) * s],
                         [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]],
                        dtype=np.complex128)
    if n == "+X":
        return _S2 * np.array([[1, 1j], [1j, 1]], dtype=np.complex128)
    if n == "-X":
        return _S2 * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128)
    if n == "+Y":
        return _S2 * np.array([[1, 1], [-1, 1]], dtype=np.complex128)
    if n == "-Y":
        return _S2 * np.array([[1, -1], [1, 1]], dtype=np.complex128)
    if n == "R":
        # R(k): phase 2*pi/2^k on |1>;  "R n -k" is the inverse R^dagger(k).
        (k,) = params
        k = int(k)
        ang = 2.0 * math.pi / (2.0 ** abs(k))
        if k < 0:
            ang = -ang
        return np.array([[1, 0], [0, np.exp(1j * ang)]], dtype=np.complex128)
    if n == "RZ":
        (th,) = params
        return np.array([[np.exp(-0.5j * th), 0], [0, np.exp(0.5j * th)]],
                        dtype=np.complex128)
    if n == "MAT":
        p = np.asarray(params, dtype=np.float64)
        return (p[0::2] + 1j * p[1::2]).reshape(2, 2).astype(np.complex128)
    raise ValueError("unknown single-qubit mnemonic %r" % name)


def controlled_phase(k):
    """U(k) of Appendix A: diag(1,1,1,e^{2 pi i/2^k}) on |control,target>;
    negative k gives U^dagger(k).  Returned as the 2x2 applied to the target
    when the control is 1."""
    k = int(k)
    ang = 2.0 * math.pi / (2.0 ** abs(k))
    if k < 0:
        ang = -ang
    return np.array([[1, 0], [0, np.exp(1j * ang)]], dtype=np.complex128)


def as_controlled(record):
    """Map a gate record (name, qubits, params) to (controls, target, U2x2).

    CNOT c t, U c t k and TOFFOLI c1 c2 t are controlled forms (Appendix A);
    every other mnemonic is a single-qubit gate on qubits[0].
    """
    name, qubits, params = record
    n = name.upper()
    qubits = [int(q) for q in qubits]
    if n == "CNOT":
        return qubits[:1], qubits[1], one_qubit("X")
    if n == "U":
        return qubits[:1], qubits[1], controlled_phase(params[0])
    if n in ("TOFFOLI", "CCX"):
        return qubits[:2], qubits[2], one_qubit("X")
    if n in ("CMAT",):
        nc = len(qubits) - 1
        return qubits[:nc], qubits[nc], one_qubit("MAT", params)
    return [], qubits[0], one_qubit(n, params)
