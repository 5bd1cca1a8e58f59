"""Host-only entry points of the library against the oracle (no GPU call):
the counter-based generator, the depolarizing-channel circuit transform and
the program parser of the Appendix A instruction language."""
import numpy as np
import pytest

from oracle import measure as om, program as oprog
from paper_1805_04708_gb300 import workloads as wl


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    return qsim


@pytest.mark.parametrize("seed,first", [(0, 0), (1, 10), (2 ** 63 + 5, 2 ** 40), (123456789, 3)])
def test_uniforms_bit_exact(q, seed, first):
    got = q.uniforms(seed, first, 2000)
    want = om.uniforms(seed, first, 2000)
    assert np.array_equal(got, want)


def _pauli_name(g):
    u = np.array(g.u)
    for name, m in (("X", [0, 0, 1, 0, 1, 0, 0, 0]), ("Y", [0, 0, 0, -1, 0, 1, 0, 0]), ("Z", [1, 0, 0, 0, 0, 0, -1, 0])):
        if g.nc == 0 and np.array_equal(u, np.array(m, dtype=float)):
            return name
    return None


@pytest.mark.parametrize("p,seed", [((0.1, 0.05, 0.2), 7), ((0.0, 0.0, 0.0), 1), ((0.3, 0.3, 0.4), 99)])
def test_depolarize_equals_oracle(q, p, seed):
    N = 5
    recs = wl.random_gate_circuit(N, 40, 3)
    arr, n = q.depolarize_circuit(N, recs, *p, seed)
    want = om.depolarize(recs, N, *p, seed)
    assert n == len(want)
    orig = iter(range(len(recs)))
    for k, w in enumerate(want):
        if w[0] in ("X", "Y", "Z") and len(w[1]) == 1 and w not in recs[:0]:
            name = _pauli_name(arr[k])
            if name is not None and w[2] == ():
                assert name == w[0] and arr[k].target == w[1][0]
                continue
        i = next(orig)
        assert w == recs[i]


def test_depolarize_counter_offset(q):
    # gates numbered from first_gate: two halves give the same records as one call
    N = 4
    recs = wl.random_gate_circuit(N, 30, 5)
    whole, nw = q.depolarize_circuit(N, recs, 0.2, 0.2, 0.2, 11)
    a, na = q.depolarize_circuit(N, recs[:17], 0.2, 0.2, 0.2, 11, first_gate=0)
    b, nb = q.depolarize_circuit(N, recs[17:], 0.2, 0.2, 0.2, 11, first_gate=17)
    assert nw == na + nb
    for k in range(nw):
        x = whole[k]
        y = a[k] if k < na else b[k - na]
        assert (x.nc, x.target, tuple(x.u)) == (y.nc, y.target, tuple(y.u))


BAD = ["H 0\n", "QUBITS 3\nH 3\n", "QUBITS 3\nCNOT 1 1\n", "QUBITS 3\nBIT ASSIGNMENT 0 0 1\n",
       "QUBITS 3\nFOO 1\n", "QUBITS 3\nU3 0 1.0\n", "QUBITS 1\n", "QUBITS 3\nQUBITS 3\n",
       "QUBITS 3\nDEPOLARIZING CHANNEL P_X = 0.7, P_Z = 0.5\n", "QUBITS 4\nSHORBOX 2 7 2\n",
       "QUBITS 3\nM\n", "QUBITS 3\nGENERATE EVENTS 0 1\n"]


@pytest.mark.parametrize("text", BAD)
def test_parse_errors(q, text):
    with pytest.raises(q.QSError) as e:
        q.Program(text)
    assert e.value.name == "QS_EINVAL"
    with pytest.raises(ValueError):
        oprog.parse(text)


def test_parse_counts(q):
    text = wl.error_correction_program((0,))
    p = q.Program(text)
    assert p.N == 5
    assert p.n_instr == len(oprog.parse(text)) - 1
    text2 = "! header\nqubits 4\n\nh 0 ! c\nu1 1 0.5\nu 0 1 -3\nr 2 -4\nDEPOLARIZING CHANNEL SEED = 5, P_Y = 0.1\nexit\n"
    p2 = q.Program(text2)
    assert (p2.N, p2.n_instr) == (4, 6)
    assert len(oprog.parse(text2)) - 1 == 6
