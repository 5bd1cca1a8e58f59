"""GPU parity of the auxiliary-variable amplitudes (Sec. 4.2) through the C
ABI: against the oracle's step-by-step sum over configurations, against the
state-vector oracle at N = 16..20, and at N = 45 (no state vector fits)
against the product of block states of a circuit whose gates stay inside
blocks of three qubits.  Tolerance: 1e-12 max-abs (FP64 throughout)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from blockref import block_amplitudes, block_states  # noqa: E402
from oracle import aux, circuit, statevec as sv  # noqa: E402
from paper_1805_04708_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    return qsim


@pytest.mark.parametrize("N,ne,ns,toff,seed", [(3, 8, 10, 0, 1), (5, 10, 12, 0, 2), (7, 12, 14, 0, 3),
                                               (3, 2, 4, 1, 4), (4, 0, 6, 2, 5)])
def test_aux_matches_oracle_sum(q, N, ne, ns, toff, seed):
    recs = wl.aux_circuit(N, ne, ns, seed, toffoli=toff)
    basis = list(range(1 << N)) if N <= 5 else [int(x) for x in np.random.default_rng(seed).integers(0, 1 << N, 20)]
    want, P = aux.amplitudes(recs, N, basis)
    got, P2 = q.aux_amplitudes(N, recs, basis)
    assert P2 == P
    assert np.max(np.abs(got - want)) <= 1e-12


@pytest.mark.parametrize("N,ne,seed", [(16, 14, 7), (20, 18, 8), (18, 22, 9)])
def test_aux_matches_state_vector(q, N, ne, seed):
    recs = wl.aux_circuit(N, ne, 3 * N, seed)
    ref = circuit.run(sv.zero_state(N), N, recs)
    g = np.random.default_rng(seed)
    basis = np.concatenate([np.argsort(-np.abs(ref))[:40], g.integers(0, 1 << N, 60)])
    got, P = q.aux_amplitudes(N, recs, basis)
    assert P <= ne   # U(k = 0) is the identity and needs no variable
    assert np.max(np.abs(got - ref[basis])) <= 1e-12
    # deterministic: a second call gives the same bits
    got2, _ = q.aux_amplitudes(N, recs, basis)
    assert np.array_equal(got, got2)


def test_aux_beyond_state_vector_n45(q):
    # 15 blocks of 3 qubits, entangling gates inside blocks only: the exact
    # amplitude is the product of the blocks' oracle amplitudes
    N = 45
    blocks = wl.block_partition(N, 3, seed=21)
    g = np.random.default_rng(22)
    recs = [("H", (qq,), ()) for qq in range(N)]
    for b in blocks:
        c, t = (int(x) for x in g.choice(b, 2, replace=False))
        recs.append(("CNOT", (c, t), ()))
        recs.append(("U3", (int(g.choice(b)),), tuple(float(x) for x in g.uniform(0, 6.28, 3))))
        if g.integers(2):
            c, t = (int(x) for x in g.choice(b, 2, replace=False))
            recs.append(("U", (c, t), (int(g.integers(1, 5)),)))
    states = block_states(blocks, recs)
    basis = np.concatenate([g.integers(0, 1 << N, 30, dtype=np.int64), [0, (1 << N) - 1]])
    want = block_amplitudes(blocks, states, basis)
    got, P = q.aux_amplitudes(N, recs, basis.astype(np.uint64))
    assert 15 <= P <= 30
    assert np.max(np.abs(got - want)) <= 1e-12


def test_aux_product_and_errors(q):
    N = 6
    recs = [("H", (k,), ()) for k in range(N)] + [("T", (2,), ())]
    got, P = q.aux_amplitudes(N, recs, range(1 << N))
    assert P == 0
    assert np.max(np.abs(got - circuit.run(sv.zero_state(N), N, recs))) <= 1e-15
    h = 2 ** -0.5
    with pytest.raises(q.QSError) as e:
        q.aux_amplitudes(N, [("CMAT", (0, 1), (h, 0, h, 0, h, 0, -h, 0))], [0])
    assert e.value.name == "QS_EUNSUPPORTED"
    with pytest.raises(q.QSError) as e:
        q.aux_amplitudes(N, [("CNOT", (0, 1), ())] * 41, [0])
    assert e.value.name == "QS_EINVAL"
    with pytest.raises(q.QSError):
        q.aux_amplitudes(N, recs, [1 << N])
