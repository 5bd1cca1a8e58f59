"""GPU parity of the tile passes compiled at run time (circuit_run modes 2 and
3) against the oracle and the op interpreter (mode 1); complex64 max-abs
tolerance 1e-5 as for every complex64 path."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import circuit, statevec as sv  # noqa: E402
from paper_1805_04708_gb300 import workloads as wl  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    if not qsim.tile_compiler_info()[0]:
        pytest.fail("NVRTC cannot be loaded on the GPU machine")
    return qsim


def run(q, N, recs, mode, enc="c64"):
    if mode in (2, 3) and enc == "c64":
        q.circuit_compile(N, recs, mode=mode)
    with q.Sim(N, enc) as s:
        npass = s.circuit_run(recs, mode=mode)
        return s.copy_out().astype(np.complex128), npass


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("N", [14, 17])
def test_compiled_passes_mixed_circuit(q, N, mode):
    # every gate kind with 0..2 controls: dense, real, diagonal, anti-diagonal
    # ops on register slots, lanes and warp bits, folded diagonals, transposes.
    # Mode 2 tries one kernel candidate per run of a structure: four runs
    # cover the interpreter and the three compiled variants of every pass
    recs = wl.random_mixed_circuit(N, 160, seed=200 + N)
    ref = circuit.run(sv.zero_state(N), N, recs)
    interp, npass1 = run(q, N, recs, 1)
    for _ in range(4 if mode == 2 else 1):
        got, npass = run(q, N, recs, mode)
        assert npass == npass1
        assert np.max(np.abs(got - ref)) <= TOL
        assert np.max(np.abs(got - interp)) <= TOL


@pytest.mark.parametrize("mode", [2, 3])
def test_compiled_passes_random_gate_circuit(q, mode):
    N = 21
    recs = wl.random_gate_circuit(N, 240, seed=9)
    ref = circuit.run(sv.zero_state(N), N, recs)
    for _ in range(5 if mode == 2 else 1):
        got, _ = run(q, N, recs, mode)
        assert np.max(np.abs(got - ref)) <= TOL


def test_compiled_pass_cache_and_c128(q):
    N = 15
    recs = wl.random_mixed_circuit(N, 80, seed=77)
    run(q, N, recs, 3)
    _, c0 = q.tile_compiler_info()
    got, _ = run(q, N, recs, 3)
    assert q.tile_compiler_info()[1] == c0          # every structure cached
    ref = circuit.run(sv.zero_state(N), N, recs)
    assert np.max(np.abs(got - ref)) <= TOL
    # complex128 states run the interpreter in every tile mode
    got128, _ = run(q, N, recs, 3, enc="c128")
    assert np.max(np.abs(got128 - ref)) <= 1e-12
