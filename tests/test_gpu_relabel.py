"""GPU parity of the relabelled swaps in complex64 tile passes: X, CNOT and
TOFFOLI whose controls lie outside the register slots and the lanes become
relabellings of their target bit (no data moves), and later ops read the
relabelling: gates on the relabelled slot (roles exchanged), lane gates and
conditions on relabelled lane or warp bits, factor tables and register-slot
controls that need the slot back in place (exchanges inserted), transposes
of merged last passes and the store.  Swap-heavy circuits in the
interpreter (mode 1) and the compiled passes (modes 2, 3), with and without
the product start, against the oracle (complex64 max-abs 1e-5)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import circuit, statevec as sv  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    return qsim


def swap_heavy(N, ngates, seed):
    """Half swaps (X, CNOT, TOFFOLI on random qubits, so their controls fall
    inside and outside the tiles), a quarter Hadamard / U3 (dense, also on
    qubits 0..3), a quarter diagonals (T, S, Z, RZ, controlled phases) that
    become factor tables or per-thread factors."""
    g = np.random.default_rng(seed)
    recs = [("H", (k,), ()) for k in range(N)]
    for _ in range(ngates):
        r = g.random()
        qs = [int(x) for x in g.choice(N, 3, replace=False)]
        if r < 0.5:
            k = int(g.integers(3))
            recs.append((("X", "CNOT", "TOFFOLI")[k], tuple(qs[:k + 1][::-1]) if k else (qs[0],), ()))
        elif r < 0.75:
            if g.random() < 0.5:
                recs.append(("H", (qs[0] if g.random() < 0.6 else int(g.integers(min(4, N))),), ()))
            else:
                recs.append(("U3", (qs[0],), tuple(float(x) for x in g.uniform(0, 2 * math.pi, 3))))
        else:
            k = ("T", "S", "Z", "RZ", "CU")[int(g.integers(5))]
            if k == "RZ":
                recs.append(("RZ", (qs[0],), (float(g.uniform(0, 2 * math.pi)),)))
            elif k == "CU":
                recs.append(("U", (qs[1], qs[0]), (int(g.integers(1, 6)),)))
            else:
                recs.append((k, (qs[0],), ()))
    return recs


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("N,seed", [(14, 1), (18, 2), (21, 3)])
@pytest.mark.parametrize("product_start", [True, False])
def test_swap_heavy_circuits(q, N, seed, mode, product_start):
    recs = swap_heavy(N, 160, seed)
    ref = circuit.run(sv.zero_state(N), N, recs)
    if mode in (2, 3):
        q.circuit_compile(N, recs, mode=mode)
    with q.Sim(N, "c64") as s:
        s.set_product_start(product_start)
        for _ in range(9 if mode == 2 else 1):   # mode 2 tries its kernel candidates
            s.reset()
            s.circuit_run(recs, mode=mode)
        got = s.copy_out().astype(np.complex128)
    assert float(np.max(np.abs(got - ref))) <= TOL


def test_swaps_only_are_exact_permutations(q):
    # a circuit of X / CNOT / TOFFOLI on a random state is a permutation of
    # the amplitudes: relabelled or moved, every value comes through unchanged
    N = 17
    g = np.random.default_rng(9)
    v0 = (g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)).astype(np.complex64)
    recs = [r for r in swap_heavy(N, 300, 4)[N:] if r[0] in ("X", "CNOT", "TOFFOLI")]
    ref = circuit.run(v0.astype(np.complex128), N, recs)
    with q.Sim(N, "c64") as s:
        s.copy_in(v0)
        s.circuit_run(recs, mode=1)
        got = s.copy_out()
    assert np.array_equal(got.astype(np.complex128), ref)
