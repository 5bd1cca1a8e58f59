"""Full-size checks at the sizes of the benchmark configurations, through the
same entry points and launch configurations the benchmark uses, via
properties that hold at any size: the paper's Tables 2 and 3 (uniform
superposition, GHZ) at N = 33 (complex128, 128 GiB) and N = 36 (adaptive
2-byte, 128 GiB); a unitarity round trip of the N = 30 random-gate circuit;
agreement of the tile planner with the per-gate sweeps at N = 30."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1805_04708_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    return qsim


def inverse(recs):
    """Inverse circuit: reversed order, every gate's conjugate transpose
    (as explicit matrices from the library's own gate table)."""
    from paper_1805_04708_gb300 import qsim
    out = []
    for name, qs, p in reversed(recs):
        g = qsim.gate_std(name, qs, p)
        U = (np.array(g.u[0::2]) + 1j * np.array(g.u[1::2])).reshape(2, 2)
        Ud = U.conj().T
        flat = []
        for x in Ud.ravel():
            flat += [float(x.real), float(x.imag)]
        ctrl = tuple(g.controls[:g.nc])
        out.append(("CMAT" if g.nc else "MAT", ctrl + (g.target,), tuple(flat)))
    return out


def free(s):
    s.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("enc,tol", [("c64", 2e-6), ("c128", 1e-12)])
def test_random_gate_circuit_n30_round_trip(q, enc, tol):
    N = 30
    recs = wl.random_gate_circuit(N, 200, 1)
    body = recs[N:]          # after the Hadamard layer the state is uniform
    s = q.Sim(N, enc)
    s.circuit_run(recs[:N], mode=1)
    s.circuit_run(body, mode=1)
    assert abs(s.norm() - 1.0) < (1e-4 if enc == "c64" else 1e-12)
    s.circuit_run(inverse(body), mode=1)
    # back to the uniform state: every amplitude 2^-15, checked on samples and
    # through the marginal of 16 qubits (uniform = 2^-16 everywhere)
    P = s.measure_probs(list(range(0, 30, 2)) + [1])
    assert np.max(np.abs(P - 2.0 ** -16)) < (1e-9 if enc == "c64" else 1e-15)
    qx, qy, qz = s.expect_xyz()
    assert np.max(np.abs(qx)) < 50 * tol and np.max(np.abs(qz - 0.5)) < 50 * tol
    free(s)


def test_tile_planner_equals_per_gate_n30(q):
    N = 30
    recs = wl.random_gate_circuit(N, 200, 2)
    s = q.Sim(N, "c64")
    s.circuit_run(recs, mode=1)
    P1 = s.measure_probs(list(range(14)))
    _, _, z1 = s.expect_xyz()
    s.reset()
    s.circuit_run(recs, mode=0)
    P0 = s.measure_probs(list(range(14)))
    _, _, z0 = s.expect_xyz()
    assert np.max(np.abs(P1 - P0)) < 1e-9
    assert np.max(np.abs(z1 - z0)) < 1e-5
    free(s)


@pytest.mark.parametrize("enc,N,tol", [("c128", 33, 1e-12), ("adapt2", 36, 1e-6)])
def test_tables_2_and_3_full_size(q, enc, N, tol):
    s = q.Sim(N, enc)
    s.circuit_run(wl.all_hadamard(N), mode=0 if enc == "adapt2" else 1)
    qx, qy, qz = s.expect_xyz()
    assert abs(s.norm() - 1.0) < tol
    assert np.max(np.abs(qx)) < tol and np.max(np.abs(qy - 0.5)) < tol and np.max(np.abs(qz - 0.5)) < tol
    s.reset()
    s.circuit_run(wl.ghz(N), mode=0 if enc == "adapt2" else 1)
    qx, qy, qz = s.expect_xyz()
    for arr in (qx, qy, qz):
        assert np.max(np.abs(arr - 0.5)) < tol
    P = s.measure_probs([0, N - 1])   # only |0..0> and |1..1>
    assert abs(P[0] - 0.5) < tol and abs(P[3] - 0.5) < tol and P[1] < tol and P[2] < tol
    free(s)
