"""Host-side pin of the product start (no GPU): from |0..0>, every
single-qubit gate that comes before all multi-qubit gates on its qubit can be
composed per qubit into a product state, and running the remaining gates in
order on that product state gives the circuit's state.  The library's complex64
tile runs rely on this (the first pass writes the product state); checked here
with the oracle alone, against the circuit run gate by gate from |0..0>.  A
rule that also folds gates after their qubit is entangled must fail.  The
library's own extraction (circuit_product_start, host only) must take the same
gates and give the same per-qubit factors."""
import numpy as np
import pytest

from oracle import circuit, gates, statevec as sv
from paper_1805_04708_gb300 import workloads as wl


def split(recs, fold_after_entangling=False):
    """(per-qubit 2x2 products, remaining records) under the prefix rule."""
    entangled, U, rest = set(), {}, []
    for r in recs:
        qs = r[1]
        if len(qs) == 1 and (fold_after_entangling or qs[0] not in entangled):
            _, t, M = gates.as_controlled(r)
            U[t] = M @ U.get(t, np.eye(2, dtype=np.complex128))
            continue
        if len(qs) > 1:
            entangled.update(qs)
        rest.append(r)
    return U, rest


def product_state(N, U):
    """prod_q (U_q |0>)(bit q of i), qubit 0 the lowest index bit."""
    v = np.ones(1, dtype=np.complex128)
    for q in range(N):
        f = U[q][:, 0] if q in U else np.array([1.0, 0.0], dtype=np.complex128)
        v = np.kron(f, v)
    return v


@pytest.mark.parametrize("N,kind,seed", [(8, "gate", 1), (10, "mixed", 2), (12, "layered", 3), (11, "gate", 4)])
def test_product_start_gives_the_circuit_state(N, kind, seed):
    recs = {"gate": wl.random_gate_circuit(N, 80, seed=seed),
            "mixed": wl.random_mixed_circuit(N, 80, seed=seed),
            "layered": wl.layered_circuit(N, 3, seed=seed)}[kind]
    U, rest = split(recs)
    assert len(U) > 0 and len(rest) < len(recs)
    ref = circuit.run(sv.zero_state(N), N, recs)
    got = circuit.run(product_state(N, U), N, rest)
    assert np.max(np.abs(got - ref)) <= 1e-12


def test_whole_circuit_product():
    N = 9
    recs = wl.all_hadamard(N) + [("T", (3,), ()), ("RZ", (5,), (0.4,)), ("H", (3,), ())]
    U, rest = split(recs)
    assert rest == []
    ref = circuit.run(sv.zero_state(N), N, recs)
    assert np.max(np.abs(product_state(N, U) - ref)) <= 1e-14


@pytest.mark.parametrize("N,kind,seed", [(13, "gate", 1), (16, "mixed", 2), (14, "layered", 3)])
def test_library_product_start_matches_the_rule(N, kind, seed):
    # the library's host-side extraction (no GPU work) against the rule above
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    recs = {"gate": wl.random_gate_circuit(N, 80, seed=seed),
            "mixed": wl.random_mixed_circuit(N, 80, seed=seed),
            "layered": wl.layered_circuit(N, 3, seed=seed)}[kind]
    U, rest = split(recs)
    npre, f = qsim.circuit_product_start(N, recs)
    assert npre == len(recs) - len(rest)
    for q in range(N):
        want = U[q][:, 0] if q in U else np.array([1.0, 0.0])
        assert np.max(np.abs(f[q] - want)) <= 1e-14


def test_folding_after_entangling_is_wrong():
    # the planted mistake: single-qubit gates folded after their qubit took
    # part in a multi-qubit gate
    N = 10
    recs = wl.random_gate_circuit(N, 80, seed=5)
    U, rest = split(recs, fold_after_entangling=True)
    ref = circuit.run(sv.zero_state(N), N, recs)
    got = circuit.run(product_state(N, U), N, rest)
    assert np.max(np.abs(got - ref)) > 1e-3
