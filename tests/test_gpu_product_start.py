"""GPU parity of the product start: a tile run from a pending |0..0>
composes the single-qubit gates that precede every multi-qubit gate on their
qubit and writes their product state in the first pass.  Checked against the
oracle's gate-by-gate run from |0..0> (complex64 max-abs 1e-5, complex128
max-abs 1e-12 with double-float tile passes and with FP64 units), with the
product start on and off, in every tile mode, and on circuits whose gates all
go into the product start."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import circuit, statevec as sv  # noqa: E402
from paper_1805_04708_gb300 import workloads as wl  # noqa: E402

TOL = {"c64": 1e-5, "c128": 1e-12}
# (encoding, complex128 arithmetic: 1 double-float everywhere, 2 double-float
# sweeps with FP64 tile passes, 0 FP64 units)
ENCS = [("c64", 1), ("c128", 1), ("c128", 0), ("c128", 2)]


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    return qsim


def maxerr(a, b):
    return float(np.max(np.abs(np.asarray(a, np.complex128) - np.asarray(b, np.complex128))))


def new_sim(q, N, enc, df):
    s = q.Sim(N, enc)
    if enc == "c128":
        s.set_fp64_emulation(df)
    return s


def modes(q):
    return (1, 2, 3) if q.tile_compiler_info()[0] else (1,)


@pytest.mark.parametrize("N,kind", [(13, "mixed"), (16, "layered"), (21, "gates")])
@pytest.mark.parametrize("product", [True, False])
@pytest.mark.parametrize("enc,df", ENCS)
def test_random_circuits_from_zero(q, N, kind, product, enc, df):
    recs = {"gates": wl.random_gate_circuit(N, 120, seed=N),
            "mixed": wl.random_mixed_circuit(N, 120, seed=N + 1),
            "layered": wl.layered_circuit(N, 3, seed=N + 2)}[kind]
    ref = circuit.run(sv.zero_state(N), N, recs)
    ref2 = circuit.run(ref.copy(), N, recs)
    for mode in modes(q)[:2]:
        with new_sim(q, N, enc, df) as s:
            s.set_product_start(product)
            s.circuit_run(recs, mode=mode)
            assert maxerr(s.copy_out(), ref) <= TOL[enc]
            # a second run on the written state: no product start
            s.circuit_run(recs, mode=mode)
            assert maxerr(s.copy_out(), ref2) <= TOL[enc]


@pytest.mark.parametrize("N", [13, 15, 20])
@pytest.mark.parametrize("enc,df", ENCS)
def test_whole_circuit_is_product(q, N, enc, df):
    # only single-qubit gates: the run is one pass that writes the product
    g = np.random.default_rng(N)
    recs = wl.all_hadamard(N) + [("U3", (int(x),), tuple(g.uniform(0, 6.3, 3))) for x in g.integers(0, N, 3 * N)]
    ref = circuit.run(sv.zero_state(N), N, recs)
    for mode in modes(q):
        with new_sim(q, N, enc, df) as s:
            npass = s.circuit_run(recs, mode=mode)
            assert npass == 1
            assert maxerr(s.copy_out(), ref) <= TOL[enc]
            assert abs(s.norm() - 1.0) < (1e-12 if enc == "c128" else 1e-5)


@pytest.mark.parametrize("enc,df", ENCS)
def test_prefix_order_cases(q, enc, df):
    # H 2 folds (qubit 2 untouched by the CNOT); H 1 after CNOT 0 1 does not;
    # gates after the first run see a written state
    N = 14
    recs = [("H", (0,), ()), ("CNOT", (0, 1), ()), ("H", (1,), ()), ("H", (2,), ()), ("T", (2,), ()),
            ("TOFFOLI", (1, 2, 13), ()), ("H", (13,), ()), ("RZ", (5,), (0.7,)), ("H", (5,), ()),
            ("CNOT", (5, 0), ()), ("U3", (7,), (0.3, 0.2, 0.1))]
    ref = circuit.run(sv.zero_state(N), N, recs)
    for mode in modes(q):
        with new_sim(q, N, enc, df) as s:
            s.circuit_run(recs, mode=mode)
            assert maxerr(s.copy_out(), ref) <= TOL[enc]


@pytest.mark.parametrize("enc,df", ENCS)
def test_not_from_zero(q, enc, df):
    # a state that was copied in, or reset with lazy reset off, runs every gate
    N = 15
    recs = wl.random_gate_circuit(N, 60, seed=7)
    g = np.random.default_rng(1)
    v0 = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    v0 /= np.linalg.norm(v0)
    vin = v0.astype(np.complex64).astype(np.complex128) if enc == "c64" else v0.copy()
    ref = circuit.run(vin, N, recs)
    with new_sim(q, N, enc, df) as s:
        s.copy_in(v0)
        s.circuit_run(recs, mode=1)
        assert maxerr(s.copy_out(), ref) <= TOL[enc]
        s.reset()
        s.copy_out()                     # writes the pending |0..0>
        s.circuit_run(recs, mode=1)
        assert maxerr(s.copy_out(), circuit.run(sv.zero_state(N), N, recs)) <= TOL[enc]


@pytest.mark.parametrize("tail", ["U0", "CMAT_I", "I"])
@pytest.mark.parametrize("enc,df", ENCS)
def test_prefix_then_only_identities(q, tail, enc, df):
    # every gate after the product start is an identity (U(k = 0) is the
    # controlled phase e^{2 pi i} = 1; an explicit controlled identity; I):
    # the planner drops them all, and the product state must still be written
    N = 14
    ident = {"U0": ("U", (0, 1), (0,)),
             "CMAT_I": ("CMAT", (3, 5), (1, 0, 0, 0, 0, 0, 1, 0)),
             "I": ("I", (2,), ())}[tail]
    recs = [("H", (0,), ()), ("H", (1,), ()), ("U3", (9,), (0.4, 1.1, 2.0)), ident]
    ref = circuit.run(sv.zero_state(N), N, recs)
    for mode in modes(q):
        with new_sim(q, N, enc, df) as s:
            npass = s.circuit_run(recs, mode=mode)
            assert npass == 1
            assert maxerr(s.copy_out(), ref) <= TOL[enc]
