"""Host-side check of the tile planner's gate order (no GPU): circuit_plan
returns the order in which the passes take the gates; running the oracle in
that order must give the state of the circuit order, since a pass only takes a
gate ahead of gates left for later passes when it commutes with all of them
(complex128 passes keep circuit order)."""
import numpy as np
import pytest

from oracle import circuit, statevec as sv
from paper_1805_04708_gb300 import workloads as wl


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    return qsim


def rand_state(N, seed):
    g = np.random.default_rng(seed)
    v = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("enc", ["c64", "c128"])
@pytest.mark.parametrize("N,kind,seed", [(13, "mixed", 1), (14, "mixed", 2), (14, "gate", 3), (16, "gate", 4)])
def test_planned_order_gives_the_same_state(q, N, kind, seed, enc):
    # both encodings' planners move commuting gates ahead into earlier passes
    recs = (wl.random_mixed_circuit(N, 150, seed=seed) if kind == "mixed"
            else wl.random_gate_circuit(N, 150, seed=seed, hadamard_layer=False))
    passes = q.circuit_plan(N, recs, enc)
    order = [i for p in passes for i in p]
    assert sorted(order) == sorted(set(order))            # each gate at most once
    dropped = set(range(len(recs))) - set(order)          # only identities may be dropped
    for i in dropped:
        name, qs, params = recs[i]
        u = np.array(q.gate_std(name, qs, params).u[:])
        assert np.allclose(u, [1, 0, 0, 0, 0, 0, 1, 0], atol=1e-15), recs[i]
    assert len(passes) > 1
    assert order != sorted(order)                          # something was moved ahead
    v0 = rand_state(N, seed)
    ref = circuit.run(v0.copy(), N, recs)
    got = circuit.run(v0.copy(), N, [recs[i] for i in order])
    assert np.max(np.abs(got - ref)) <= 1e-12


def test_plan_rejects(q):
    with pytest.raises(q.QSError):
        q.circuit_plan(8, [("H", (0,), ())], "c64")      # below the tile size
    with pytest.raises(q.QSError):
        q.circuit_plan(16, [("H", (0,), ())], "adapt2")
