"""Pins of the oracle's gate arithmetic against brute force (dense 2^N x 2^N
matrices built entry by entry), algebraic identities of the Appendix A gate
table, unitarity round trips and norm invariance."""
import math

import numpy as np
import pytest

from oracle import gates, statevec as sv, circuit
from paper_1805_04708_gb300 import workloads as wl


def rand_state(N, seed):
    g = np.random.default_rng(seed)
    v = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    return v / np.linalg.norm(v)


def brute_controlled(N, controls, target, U):
    """Dense matrix of a controlled U(2), entry by entry: column i maps to rows
    i with bit `target` set to 0/1 when every control bit of i is 1, else to
    itself."""
    D = 1 << N
    M = np.zeros((D, D), dtype=np.complex128)
    for i in range(D):
        if all((i >> c) & 1 for c in controls):
            bt = (i >> target) & 1
            for r in (0, 1):
                row = (i & ~(1 << target)) | (r << target)
                M[row, i] = U[r, bt]
        else:
            M[i, i] = 1.0
    return M


def brute_dense(N, qubits, U):
    D = 1 << N
    k = len(qubits)
    M = np.zeros((D, D), dtype=np.complex128)
    mask = sum(1 << q for q in qubits)
    for i in range(D):
        col = sum(((i >> q) & 1) << m for m, q in enumerate(qubits))
        for row_l in range(1 << k):
            row = i & ~mask
            for m, q in enumerate(qubits):
                row |= ((row_l >> m) & 1) << q
            M[row, i] = U[row_l, col]
    return M


def haar(seed, n=2):
    g = np.random.default_rng(seed)
    Z = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


@pytest.mark.parametrize("N", [1, 2, 3, 5, 6])
def test_single_qubit_vs_kronecker(N):
    for t in range(N):
        U = haar(100 + t)
        v = rand_state(N, N * 7 + t)
        # Kronecker form of the Sec. 2 operator 1 x .. x U_t x .. x 1, qubit
        # N-1 leftmost (qubit 0 is the rightmost bit).
        K = np.kron(np.kron(np.eye(1 << (N - 1 - t)), U), np.eye(1 << t))
        ref = K @ v
        got = sv.apply_controlled_u2(v.copy(), N, [], t, U)
        assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_controlled_vs_brute_force(N):
    g = np.random.default_rng(N)
    for trial in range(12):
        nc = int(g.integers(1, min(2, N - 1) + 1))
        q = g.choice(N, nc + 1, replace=False)
        controls, target = [int(x) for x in q[:nc]], int(q[nc])
        U = haar(trial + 50 * N)
        v = rand_state(N, trial)
        ref = brute_controlled(N, controls, target, U) @ v
        got = sv.apply_controlled_u2(v.copy(), N, controls, target, U)
        assert np.max(np.abs(got - ref)) < 1e-14


def test_cnot_toffoli_matrices_in_control_target_basis():
    # Appendix A prints CNOT / TOFFOLI in the basis |control,target>; build the
    # 4x4 / 8x8 from the oracle on qubits (control=1, target=0) and compare.
    CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]])
    M = np.zeros((4, 4), dtype=np.complex128)
    for i in range(4):
        e = np.zeros(4, dtype=np.complex128)
        e[i] = 1
        M[:, i] = circuit.run(e, 2, [("CNOT", (1, 0), ())])
    assert np.array_equal(M.real, CNOT) and not M.imag.any()
    TOF = np.eye(8)
    TOF[[6, 7]] = TOF[[7, 6]]
    M = np.zeros((8, 8), dtype=np.complex128)
    for i in range(8):
        e = np.zeros(8, dtype=np.complex128)
        e[i] = 1
        M[:, i] = circuit.run(e, 3, [("TOFFOLI", (2, 1, 0), ())])
    assert np.array_equal(M.real, TOF)
    UK = np.diag([1, 1, 1, np.exp(2j * math.pi / 8)])
    M = np.zeros((4, 4), dtype=np.complex128)
    for i in range(4):
        e = np.zeros(4, dtype=np.complex128)
        e[i] = 1
        M[:, i] = circuit.run(e, 2, [("U", (1, 0), (3,))])
    assert np.max(np.abs(M - UK)) < 1e-15


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_dense_vs_brute_force(k):
    N = 6
    g = np.random.default_rng(k)
    for trial in range(4):
        qubits = [int(x) for x in g.choice(N, k, replace=False)]
        U = haar(1000 + trial, 1 << k)
        v = rand_state(N, 40 + trial)
        ref = brute_dense(N, qubits, U) @ v
        got = sv.apply_dense(v.copy(), N, qubits, U)
        assert np.max(np.abs(got - ref)) < 1e-13


def test_dense_of_kron_equals_sequential():
    # A 2-qubit dense gate U_b (x) U_a on (qa, qb) equals U_a on qa then U_b on qb.
    N = 5
    Ua, Ub = haar(1), haar(2)
    v = rand_state(N, 3)
    ref = sv.apply_controlled_u2(sv.apply_controlled_u2(v.copy(), N, [], 1, Ua), N, [], 3, Ub)
    got = sv.apply_dense(v.copy(), N, [1, 3], np.kron(Ub, Ua))
    assert np.max(np.abs(got - ref)) < 1e-14


def test_permutation_vs_loop():
    N, reg_lo, w = 7, 3, 3
    g = np.random.default_rng(5)
    table = g.permutation(1 << w)
    v = rand_state(N, 9)
    got = sv.apply_permutation(v.copy(), N, [0, 6], reg_lo, w, table)
    ref = np.empty_like(v)
    for i in range(1 << N):
        if (i & 1) and (i >> 6) & 1:
            f = (i >> reg_lo) & 7
            j = (i & ~(7 << reg_lo)) | (int(table[f]) << reg_lo)
        else:
            j = i
        ref[j] = v[i]
    assert np.array_equal(got, ref)
    with pytest.raises(ValueError):
        sv.apply_permutation(v.copy(), N, [], 0, 2, [0, 1, 1, 3])


def test_appendix_a_identities():
    G = gates.one_qubit
    I = np.eye(2)
    names = ["I", "H", "X", "Y", "Z", "S", "S+", "T", "T+", "+X", "-X", "+Y", "-Y"]
    for n in names:
        U = G(n)
        assert np.max(np.abs(U.conj().T @ U - I)) < 1e-15, n
    assert np.max(np.abs(G("H") @ G("H") - I)) < 1e-15
    assert np.max(np.abs(G("T") @ G("T") - G("S"))) < 1e-15
    assert np.max(np.abs(G("S") @ G("S") - G("Z"))) < 1e-15
    assert np.max(np.abs(G("S") @ G("S+") - I)) < 1e-15
    assert np.max(np.abs(G("T") @ G("T+") - I)) < 1e-15
    assert np.max(np.abs(G("H") @ G("Z") @ G("H") - G("X"))) < 1e-15
    assert np.max(np.abs(1j * G("X") @ G("Z") - G("Y"))) < 1e-15
    assert np.max(np.abs(G("+X") @ G("-X") - I)) < 1e-15
    assert np.max(np.abs(G("+Y") @ G("-Y") - I)) < 1e-15
    # +X is the rotation by -pi/2 about x: exp(+i pi/4 X) = (1 + iX)/sqrt 2
    assert np.max(np.abs(G("+X") - (I + 1j * G("X")) / math.sqrt(2))) < 1e-15
    assert np.max(np.abs(G("+Y") - (I + 1j * G("Y")) / math.sqrt(2))) < 1e-15
    for th, phi, lam in [(0.3, 1.1, -0.7), (2.0, -2.5, 0.4)]:
        U3 = G("U3", (th, phi, lam))
        assert np.max(np.abs(U3.conj().T @ U3 - I)) < 1e-15
        assert np.max(np.abs(G("U3", (math.pi / 2, phi, lam)) - G("U2", (phi, lam)))) < 1e-15
        assert np.max(np.abs(G("U3", (0.0, 0.0, lam)) - G("U1", (lam,)))) < 1e-15
    for k in range(0, 10):
        assert np.max(np.abs(G("R", (k,)) - G("U1", (2 * math.pi / 2 ** k,)))) < 1e-15
        assert np.max(np.abs(G("R", (-k,)) @ G("R", (k,)) - I)) < 1e-15
    assert np.max(np.abs(G("R", (1,)) - G("Z"))) < 1e-15
    assert np.max(np.abs(G("R", (2,)) - G("S"))) < 1e-15
    assert np.max(np.abs(G("R", (3,)) - G("T"))) < 1e-15
    th = 0.77
    rz = G("RZ", (th,))
    assert np.max(np.abs(rz - np.exp(-0.5j * th) * G("U1", (th,)))) < 1e-15


def inverse_records(recs):
    out = []
    for rec in reversed(recs):
        controls, target, U = gates.as_controlled(rec)
        Ud = U.conj().T
        p = []
        for x in Ud.ravel():
            p += [x.real, x.imag]
        out.append(("CMAT" if controls else "MAT", tuple(controls) + (target,), tuple(p)))
    return out


@pytest.mark.parametrize("N", [3, 7, 10])
def test_round_trip_and_norm(N):
    recs = wl.random_mixed_circuit(N, 60, seed=N)
    v0 = rand_state(N, 77)
    v = circuit.run(v0.copy(), N, recs)
    assert abs(sv.norm(v) - 1.0) < 1e-13
    back = circuit.run(v, N, inverse_records(recs))
    assert np.max(np.abs(back - v0)) < 1e-13


def test_random_circuit_vs_dense_product():
    # A whole random circuit equals the product of its brute-force matrices.
    N = 5
    recs = wl.random_mixed_circuit(N, 25, seed=11)
    M = np.eye(1 << N, dtype=np.complex128)
    for rec in recs:
        if rec[0] == "I":
            continue
        c, t, U = gates.as_controlled(rec)
        M = brute_controlled(N, c, t, U) @ M
    v0 = rand_state(N, 5)
    got = circuit.run(v0.copy(), N, recs)
    assert np.max(np.abs(got - M @ v0)) < 1e-13
