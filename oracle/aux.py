"""The auxiliary-variable method of Sec. 4.2, step by step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every entangling gate is rewritten in terms of controlled phase shifts
U_ct(a) = diag(1, 1, 1, e^{ia}) (Eq. (appa4)); each of those becomes, by the
discrete Hubbard-Stratonovich transformation (Eqs. (appa5), (appa6)),
  U_ct(a) = (1/2) sum_{s = +-1} exp(i (sigma^z_c + sigma^z_t)(x s - a/4)),
  cos 2x = e^{ia/2},
i.e. a sum over one two-valued auxiliary variable s of products of two
single-qubit diagonal operators diag(e^{i theta}, e^{-i theta}) with
theta = x s - a/4 (sigma^z = +1 on |0>, -1 on |1>).  With P such variables
the output state is 2^{-P} sum_s prod_j W_j(s) |0>_j (Eq. (appa7)), where
W_j(s) is the ordered product of the single-qubit operators on qubit j.
An amplitude <z|psi> is then 2^{-P} sum_s prod_j (W_j(s)|0>)(z_j): O(N) per
term, O(N M 2^P) for M amplitudes.

Rewrites (the paper states the first two; the others follow from them):
  * CNOT c t = H_t U_ct(pi) H_t;
  * U c t k (controlled R(k)) = U_ct(+-2 pi / 2^|k|);
  * a controlled diagonal unitary diag(d0, d1) on target t with control c is
    diag(1, d0) on c followed by U_ct(arg(d1 / d0));
  * TOFFOLI c1 c2 t: the standard decomposition into H, T, T^dagger and six
    CNOTs (Nielsen and Chuang, Quantum Computation and Quantum Information,
    Fig. 4.9), each CNOT rewritten as above.
Other controlled (non-diagonal, non-X) gates are not covered by the method as
the paper states it and raise ValueError.
"""
import cmath
import math

import numpy as np

from . import gates as og

_H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
_T = np.diag([1.0, np.exp(1j * math.pi / 4)]).astype(np.complex128)
_TD = np.diag([1.0, np.exp(-1j * math.pi / 4)]).astype(np.complex128)


def hs_x(a):
    """x with cos 2x = e^{ia/2} (principal branch of the complex arccos)."""
    return 0.5 * cmath.acos(cmath.exp(0.5j * a))


def hs_factor(a, s):
    """diag(e^{i theta}, e^{-i theta}), theta = x s - a/4: one qubit's factor
    of the term s of Eq. (appa6)."""
    th = hs_x(a) * s - a / 4.0
    return np.array([cmath.exp(1j * th), cmath.exp(-1j * th)], dtype=np.complex128)


def _toffoli_ops(c1, c2, t):
    one = lambda q, U: ("1q", q, U)
    cx = lambda c, tt: ("cx", c, tt)
    return [one(t, _H), cx(c2, t), one(t, _TD), cx(c1, t), one(t, _T), cx(c2, t), one(t, _TD), cx(c1, t),
            one(c2, _T), one(t, _T), one(t, _H), cx(c1, c2), one(c1, _T), one(c2, _TD), cx(c1, c2)]


def rewrite(records):
    """Gate records -> ops ("1q", q, U) and ("cp", c, t, a) in circuit order."""
    ops = []
    for rec in records:
        name = rec[0].upper()
        if name == "I":
            continue
        if name == "TOFFOLI":
            pre = _toffoli_ops(*rec[1])
        elif name == "CNOT":
            pre = [("cx",) + tuple(rec[1])]
        else:
            controls, target, U = og.as_controlled(rec)
            if not controls:
                pre = [("1q", target, U)]
            elif len(controls) == 1 and U[0, 1] == 0 and U[1, 0] == 0:
                d0, d1 = U[0, 0], U[1, 1]
                c = controls[0]
                pre = [("1q", c, np.diag([1.0, d0]).astype(np.complex128)),
                       ("cp", c, target, cmath.phase(d1 / d0))]
            elif len(controls) == 1 and U[0, 0] == 0 and U[1, 1] == 0 and U[0, 1] == 1 and U[1, 0] == 1:
                pre = [("cx", controls[0], target)]
            else:
                raise ValueError("the auxiliary-variable method covers single-qubit gates, controlled "
                                 "phases, CNOT and TOFFOLI")
        for op in pre:
            if op[0] == "cx":
                ops += [("1q", op[2], _H), ("cp", op[1], op[2], math.pi), ("1q", op[2], _H)]
            else:
                ops.append(op)
    return ops


def amplitudes(records, N, basis):
    """<z|C|0..0> for every basis index z in `basis` (bit q of z = qubit q),
    by the sum over all 2^P auxiliary configurations of Eq. (appa7)."""
    ops = rewrite(records)
    cps = [op for op in ops if op[0] == "cp"]
    P = len(cps)
    basis = [int(z) for z in basis]
    out = np.zeros(len(basis), dtype=np.complex128)
    for cfg in range(1 << P):
        s = [1 - 2 * ((cfg >> p) & 1) for p in range(P)]
        w = [np.array([1.0, 0.0], dtype=np.complex128) for _ in range(N)]
        p = 0
        for op in ops:
            if op[0] == "1q":
                w[op[1]] = op[2] @ w[op[1]]
            else:
                f = hs_factor(op[3], s[p])
                w[op[1]] = f * w[op[1]]
                w[op[2]] = f * w[op[2]]
                p += 1
        for m, z in enumerate(basis):
            term = 1.0 + 0.0j
            for j in range(N):
                term *= w[j][(z >> j) & 1]
            out[m] += term
    return out / float(1 << P), P


def count_aux(records):
    """P, the number of auxiliary variables of a circuit."""
    return sum(1 for op in rewrite(records) if op[0] == "cp")
