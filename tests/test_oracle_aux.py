"""Pins of the auxiliary-variable method (Sec. 4.2, oracle/aux.py): the
discrete Hubbard-Stratonovich identity of Eqs. (appa5)-(appa6) as 4x4
matrices, the CNOT and TOFFOLI rewrites against their matrices, and the
amplitudes of Eq. (appa7) against the state-vector oracle (brute force)."""
import cmath
import math

import numpy as np
import pytest

from oracle import aux, circuit, statevec as sv
from paper_1805_04708_gb300 import workloads as wl


@pytest.mark.parametrize("a", [math.pi, math.pi / 2, -math.pi / 4, 2 * math.pi / 2 ** 7, 0.3, -2.9])
def test_hs_identity(a):
    # U_01(a) = (1/2) sum_s exp(i (sz_0 + sz_1)(x s - a/4)) as 4x4 matrices in
    # the basis |q0 q1> = |00>, |01>, |10>, |11> (sigma^z = +1 on |0>)
    x = aux.hs_x(a)
    assert abs(cmath.cos(2 * x) - cmath.exp(0.5j * a)) < 1e-14
    sig = [1, 1, -1, -1], [1, -1, 1, -1]
    M = np.zeros(4, dtype=np.complex128)
    for s in (1, -1):
        th = x * s - a / 4
        M += np.array([cmath.exp(1j * (sig[0][k] + sig[1][k]) * th) for k in range(4)])
    M /= 2
    assert np.max(np.abs(M - np.array([1, 1, 1, cmath.exp(1j * a)]))) < 1e-14
    # Eq. (appa5) itself: e^{ia s0 s1 / 4} for the four sign pairs
    for s0 in (1, -1):
        for s1 in (1, -1):
            rhs = cmath.exp(-0.25j * a) / 2 * sum(cmath.exp(1j * x * (s0 + s1) * s) for s in (1, -1))
            assert abs(rhs - cmath.exp(0.25j * a * s0 * s1)) < 1e-14


@pytest.mark.parametrize("gate", [("CNOT", (0, 1), ()), ("CNOT", (2, 0), ()), ("TOFFOLI", (0, 1, 2), ()),
                                  ("TOFFOLI", (2, 0, 1), ()), ("U", (1, 2), (3,)), ("U", (2, 0), (-2,)),
                                  ("CMAT", (0, 2), (0.6, 0.8, 0, 0, 0, 0, 0, 1))])
def test_rewrites_reproduce_gates(gate):
    # every basis input of 3 qubits through the rewritten ops (as plain
    # matrices, no auxiliary sum) equals the gate's matrix
    N = 3
    ops = aux.rewrite([gate])
    for z in range(8):
        v = np.zeros(8, dtype=np.complex128)
        v[z] = 1
        want = circuit.run(v.copy(), N, [gate])
        for op in ops:
            if op[0] == "1q":
                sv.apply_controlled_u2(v, N, [], op[1], op[2])
            else:
                sv.apply_controlled_u2(v, N, [op[1]], op[2], np.diag([1, cmath.exp(1j * op[3])]))
        assert np.max(np.abs(v - want)) < 1e-14


@pytest.mark.parametrize("N,ne,ns,toff,seed", [(3, 8, 10, 0, 1), (5, 10, 12, 0, 2), (7, 12, 14, 0, 3),
                                               (3, 2, 4, 1, 4), (4, 0, 6, 2, 5)])
def test_amplitudes_against_state_vector(N, ne, ns, toff, seed):
    recs = wl.aux_circuit(N, ne, ns, seed, toffoli=toff)
    g = np.random.default_rng(seed)
    P = aux.count_aux(recs)
    assert P == ne + 6 * toff
    ref = circuit.run(sv.zero_state(N), N, recs)
    basis = list(range(1 << N)) if N <= 4 else [int(x) for x in g.integers(0, 1 << N, 8)]
    got, P2 = aux.amplitudes(recs, N, basis)
    assert P2 == P
    assert np.max(np.abs(got - ref[basis])) < 1e-12


def test_product_circuit_has_no_aux_variables():
    N = 5
    recs = wl.layered_circuit(N, 1, seed=1)
    recs = [r for r in recs if r[0] == "MAT"]
    got, P = aux.amplitudes(recs, N, range(32))
    assert P == 0
    assert np.max(np.abs(got - circuit.run(sv.zero_state(N), N, recs))) < 1e-14


def test_qft_controlled_phases():
    # the QFT of a basis state: controlled phases only (plus H), closed form
    n = 4
    j = 5
    recs = [("X", (0,), ()), ("X", (2,), ())] + wl.qft(list(range(n)))
    got, P = aux.amplitudes(recs, n, range(16))
    assert P == n * (n - 1) // 2
    # output k is read bit-reversed (wl.qft leaves the reversal to the reader)
    rev = lambda k: int(format(k, "0%db" % n)[::-1], 2)
    want = np.array([np.exp(2j * math.pi * j * rev(k) / 16) / 4 for k in range(16)])
    assert np.max(np.abs(got - want)) < 1e-13


def test_unsupported_gate():
    with pytest.raises(ValueError):
        h = 1 / math.sqrt(2)
        aux.rewrite([("CMAT", (0, 1), (h, 0, h, 0, h, 0, -h, 0))])   # controlled Hadamard
