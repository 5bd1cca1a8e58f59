"""Pins of the adaptive 2-byte encoding (Sec. 4.1) in the oracle: the code
definitions, the quantisation bound, exactness on the all-Hadamard and GHZ
circuits (Tables 2 and 3), the accuracy scale on Shor's algorithm (Table 5),
and the equivalence of code moves with decode -> gate -> encode."""
import math

import numpy as np
import pytest

from oracle import adapt2 as a2, circuit, statevec as sv, shor, gates
from paper_1805_04708_gb300 import workloads as wl


def test_special_codes():
    r0, r1 = 0.1, 0.6
    z = np.array([0.0, 1.0, 1.0 + 1e-9, -1.0j, r0, r1, r0 * np.exp(0.3j), -r1, 0.35 * np.exp(-0.5j * math.pi)])
    b0, b1 = a2.encode(z, r0, r1)
    assert (b0[0], b1[0]) == (-128, 0)          # r = 0 exactly
    assert b0[1] == 127 and b0[2] == 127 and b0[3] == 127   # |z| >= 1 -> r = 1
    assert b1[3] == -64                          # -pi/2
    assert b0[4] == -127 and b1[4] == 0          # r0 -> -127
    assert b0[5] == 126                          # r1 -> 126
    assert b0[6] == -127 and b1[6] == round(0.3 * 128 / math.pi)
    assert b0[7] == 126 and b1[7] == -128        # theta = pi wraps to -128
    assert b1[8] == -64
    d = a2.decode(b0, b1, r0, r1)
    assert d[0] == 0 and abs(d[1] - 1) < 1e-15 and abs(abs(d[4]) - r0) < 1e-15
    assert abs(abs(d[5]) - r1) < 1e-15 and abs(d[7] + r1) < 1e-15
    # the magnitude grid is r = (b0 + 127)(r1 - r0)/253 + r0
    for b in (-127, -1, 0, 63, 126):
        assert abs(a2.decode(np.int8(b), np.int8(0), r0, r1) - ((b + 127) * (r1 - r0) / 253 + r0)) < 1e-15
    # degenerate range r1 == r0: every 0 < |z| < 1 gets -127
    b0, _ = a2.encode(np.array([0.3, 0.3j]), 0.3, 0.3)
    assert list(b0) == [-127, -127]


def test_retune():
    assert a2.retune(np.array([0, 1, -1j])) == (0.0, 0.0)
    assert a2.retune(np.array([0, 0.2, 0.5j, 1.0, 0.9])) == (0.2, 0.9)


def test_quantisation_bound():
    g = np.random.default_rng(1)
    z = (g.standard_normal(20000) + 1j * g.standard_normal(20000)) * 0.2
    z = z[np.abs(z) < 1]
    r0, r1 = a2.retune(z)
    b0, b1 = a2.encode(z, r0, r1)
    d = a2.decode(b0, b1, r0, r1)
    bound = (r1 - r0) / 506 + np.abs(z) * math.pi / 256 + 1e-15
    err = np.abs(d - z)
    assert np.all(err <= bound)
    # and it is attained to within a few percent (the bound is not loose)
    assert err.max() > 0.5 * bound.max()


@pytest.mark.parametrize("N", [2, 6, 12])
def test_all_hadamard_exact(N):
    a = circuit.run_adapt2(a2.AState.zero(N), wl.all_hadamard(N))
    z = a.to_complex()
    assert a.r0 == a.r1 and np.all(a.b0 == -127) and np.all(a.b1 == 0)
    assert np.max(np.abs(z - 2.0 ** (-N / 2))) < 1e-15
    qx, qy, qz = sv.expect_xyz(z, N)
    assert np.max(np.abs(qx)) < 1e-14 and np.max(np.abs(qy - 0.5)) < 1e-14 and np.max(np.abs(qz - 0.5)) < 1e-14


@pytest.mark.parametrize("N", [2, 7, 13])
def test_ghz_exact(N):
    a = circuit.run_adapt2(a2.AState.zero(N), wl.ghz(N))
    z = a.to_complex()
    ref = np.zeros(1 << N)
    ref[0] = ref[-1] = 2 ** -0.5
    assert np.max(np.abs(z - ref)) < 1e-15
    qx, qy, qz = sv.expect_xyz(z, N)
    for arr in (qx, qy, qz):
        assert np.max(np.abs(arr - 0.5)) < 1e-15


def test_code_moves_equal_arithmetic():
    # X / CNOT / TOFFOLI move codes, pi/128-multiple phases add to b1: the
    # same codes as decode -> exact gate -> encode with the range kept
    N = 7
    g = np.random.default_rng(3)
    z = (g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N))
    z /= np.linalg.norm(z)
    a = a2.AState.from_complex(N, z)
    for rec in [("X", (3,), ()), ("CNOT", (0, 5), ()), ("TOFFOLI", (6, 1, 2), ()), ("Z", (4,), ()),
                ("S", (0,), ()), ("T+", (6,), ()), ("R", (2, ), (7,)), ("U", (1, 3), (5,)), ("Y", (2,), ()),
                ("RZ", (4,), (0.123,)), ("U1", (5,), (2.0,))]:
        b = circuit.run_adapt2(a.copy(), [rec])
        c, t, U = gates.as_controlled(rec)
        zz = a.to_complex()
        sv.apply_controlled_u2(zz, N, c, t, U)
        e0, e1 = a2.encode(zz, a.r0, a.r1)
        assert np.array_equal(b.b0, e0) and np.array_equal(b.b1, e1), rec
        assert (b.r0, b.r1) == (a.r0, a.r1)


def test_shor_accuracy_scale():
    # Sec. 5.4: JUQCS-A reproduces single-qubit expectations to about three
    # digits (Table 5 deviates by at most 0.006); the same holds for the
    # oracle's encoding on a smaller instance of the same circuit.
    G, y = 33, 5
    X, F = shor.qubit_budget(G)
    N = X + F
    r = shor.order(y, G)
    a = a2.AState.zero(N)
    z = sv.shorbox(N, X, G, y)
    a = a2.AState.from_complex(N, z)
    assert a.r0 == a.r1 == 2.0 ** (-X / 2)
    a = circuit.run_adapt2(a, wl.qft(list(range(X))))
    P = sv.marginal(a.to_complex(), N, list(range(X - 1, -1, -1)))
    qz = shor.qz_from_distribution(P / P.sum(), X)
    qz_ref = shor.qz_from_distribution(shor.closed_form_distribution(X, r), X)
    assert np.max(np.abs(qz - qz_ref)) < 0.01
    assert np.max(np.abs(qz - qz_ref)) > 0.0   # the encoding is not exact here


def test_pack_unpack():
    b0 = np.array([-128, -127, 0, 126, 127], dtype=np.int8)
    b1 = np.array([0, -128, 5, 127, -1], dtype=np.int8)
    w = a2.pack(b0, b1)
    assert w.dtype == np.uint16 and w[0] == 0x0080 and w[4] == 0xFF7F
    c0, c1 = a2.unpack(w)
    assert np.array_equal(c0, b0) and np.array_equal(c1, b1)
