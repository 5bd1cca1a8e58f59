"""GPU parity of the batched small-state path and of the dense fused k-qubit
gate against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import circuit, statevec as sv  # noqa: E402
from paper_1805_04708_gb300 import workloads as wl  # noqa: E402

TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    return qsim


def haar(n, seed):
    g = np.random.default_rng(seed)
    Z = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


@pytest.mark.parametrize("enc,N", [("c64", 4), ("c64", 9), ("c64", 12), ("c64", 14),
                                   ("c128", 5), ("c128", 9), ("c128", 13)])
def test_batch_matches_oracle(q, enc, N):
    ns = 37 if N <= 12 else 9
    circs = [wl.random_mixed_circuit(N, 5 + 7 * (s % 5), seed=1000 * N + s) for s in range(ns)]
    with q.Batch(N, enc, ns) as b:
        b.set_circuits(circs)
        b.run()
        got = b.copy_out()
        nrm = b.norms()
    for s in range(ns):
        ref = circuit.run(sv.zero_state(N), N, circs[s])
        assert np.max(np.abs(got[s] - ref)) <= TOL[enc], s
        assert abs(nrm[s] - sv.norm(got[s].astype(np.complex128))) <= 1e-12


@pytest.mark.parametrize("enc,N", [("c64", 7), ("c64", 11), ("c128", 10)])
def test_batch_graph_and_autotune(q, enc, N):
    ns = 64
    circs = [wl.layered_circuit(N, 2, seed=s) for s in range(ns)]
    with q.Batch(N, enc, ns) as b:
        b.set_circuits(circs)
        layout, threads, ms = b.autotune()
        assert layout in (0, 1, 2) and threads in (64, 128, 256, 512, 1024) and ms > 0
        fk, tb, th = b.tuning()
        assert th == threads and (fk > 0) == (layout == 2)
        if layout < 2:
            assert b.info()[:2] == (layout, threads)
        b.capture()
        b.run()          # graph replay: one pass of every circuit
        b.run()          # and a second one
        got = b.copy_out()
    for s in range(0, ns, 7):
        ref = circuit.run(sv.zero_state(N), N, circs[s] + circs[s])
        assert np.max(np.abs(got[s] - ref)) <= TOL[enc] * 2


@pytest.mark.parametrize("enc,N", [("c64", 5), ("c64", 10), ("c64", 14), ("c128", 6), ("c128", 12)])
def test_batch_fused_configurations(q, enc, N):
    # every fusion width and several states-per-CTA tilings against the
    # oracle, gate lists of different lengths per state (with TOFFOLI and
    # controlled gates, so blocks of 3 and 4 qubits occur), and a graph replay
    ns = 19
    circs = [wl.random_mixed_circuit(N, 4 + 9 * (s % 4), seed=77 * N + s) for s in range(ns)]
    refs = [circuit.run(sv.zero_state(N), N, c) for c in circs]
    with q.Batch(N, enc, ns) as b:
        b.set_circuits(circs)
        tried = 0
        for k in (1, 2, 3, 4):
            for tb, th in ((N, 128), (N + 1, 256), (N + 2, 512), (N + 3, 512)):
                try:
                    b.set_tuning(k, tb, th)
                except q.QSError:
                    continue   # more shared memory or fewer threads per state than allowed
                tried += 1
                b.reset()
                b.run()
                got = b.copy_out()
                for st in range(ns):
                    assert np.max(np.abs(got[st] - refs[st])) <= TOL[enc] * 4, (k, tb, th, st)
        assert tried >= 4
        b.set_tuning(3, N, 256)
        b.capture()
        b.reset()
        b.run()
        got = b.copy_out()
        for st in range(ns):
            assert np.max(np.abs(got[st] - refs[st])) <= TOL[enc] * 4


def test_batch_errors(q):
    with pytest.raises(q.QSError):
        q.Batch(15, "c64", 4)
    with q.Batch(4, "c64", 2) as b:
        with pytest.raises(q.QSError):
            b.set_circuits([[("H", (4,), ())], []])
        with pytest.raises(q.QSError):
            b.set_circuits([[("CNOT", (1, 1), ())], []])


# complex128 in double-float (mode 1, the default) and on the FP64 units (0)
@pytest.mark.parametrize("enc,df", [("c128", 1), ("c128", 0), ("c64", 1)])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("N", [11, 16])
def test_apply_fused_dense(q, enc, df, k, N):
    g = np.random.default_rng(k)
    v0 = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    v0 /= np.linalg.norm(v0)
    with q.Sim(N, enc) as s:
        if enc == "c128":
            s.set_fp64_emulation(df)
        s.copy_in(v0)
        ref = v0.astype(np.complex64).astype(np.complex128) if enc == "c64" else v0.copy()
        for trial in range(3):
            qubits = [int(x) for x in g.choice(N, k, replace=False)]
            U = haar(1 << k, 10 * k + trial)
            s.apply_fused(qubits, U)
            sv.apply_dense(ref, N, qubits, U)
        got = s.copy_out()
    assert np.max(np.abs(got - ref)) <= TOL[enc] * (4 if enc == "c64" and k == 5 else 1)


@pytest.mark.parametrize("N", [12, 14, 21])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
@pytest.mark.parametrize("engine", ["auto", "mma_sync"])
def test_apply_fused_tensor_cores(q, engine, k, N):
    # complex64, gate on the k lowest qubits (any order): "auto" runs the
    # tcgen05 kernel for k >= 3 (N >= 12: one CTA at N = 12, several stages
    # per CTA at N = 21), "mma_sync" the warp-level tensor-core kernel
    g = np.random.default_rng(100 + k + N)
    v0 = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    v0 /= np.linalg.norm(v0)
    ref = v0.astype(np.complex64).astype(np.complex128)
    with q.Sim(N, "c64") as s:
        s.set_fused_engine(engine)
        s.copy_in(v0)
        for trial in range(3):
            qubits = [int(x) for x in g.permutation(k)]
            U = haar(1 << k, 7 * k + trial)
            s.apply_fused(qubits, U)
            sv.apply_dense(ref, N, qubits, U)
        got = s.copy_out()
    # 3xTF32 keeps each product near FP32 rounding: after three gates the
    # deviation is a few FP32 ulps of the unit-norm state
    assert np.max(np.abs(got - ref)) <= 1e-5
    assert np.linalg.norm(got - ref) <= 2e-6


def test_fused_engines_agree(q):
    # the three kernel families on one k = 5 gate (lowest qubits, N = 16)
    N, k = 16, 5
    g = np.random.default_rng(5)
    v0 = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    v0 /= np.linalg.norm(v0)
    U = haar(1 << k, 99)
    outs = {}
    for engine in ("auto", "mma_sync", "cuda_cores"):
        with q.Sim(N, "c64") as s:
            s.set_fused_engine(engine)
            s.copy_in(v0)
            s.apply_fused(list(range(k)), U)
            outs[engine] = s.copy_out()
    for e in ("mma_sync", "cuda_cores"):
        assert np.linalg.norm(outs["auto"] - outs[e]) <= 1e-6
    with q.Sim(4, "c64") as s, pytest.raises(KeyError):
        s.set_fused_engine("tcgen06")


def test_fused_engine_rejects_unknown(q):
    with q.Sim(4, "c64") as s:
        assert q._lib.sim_set_fused_engine(s._h, 7) == 1     # QS_EINVAL


def test_apply_fused_rejects(q):
    with q.Sim(6, "c128") as s:
        with pytest.raises(q.QSError) as e:
            s.apply_fused([0, 1], np.ones((4, 4)))
        assert e.value.name == "QS_ENOTUNITARY"
        with pytest.raises(q.QSError):
            s.apply_fused([0, 0], np.eye(4))


@pytest.mark.parametrize("N,qubits", [(14, [9, 2, 13]), (14, [0, 5, 1, 12]), (21, [3, 9, 17, 20, 11]),
                                      (21, [4, 0, 2, 1, 3]), (16, [15, 7]), (22, [21, 0, 1, 2, 3]),
                                      (12, [11, 5, 0]), (12, [0, 2, 4, 6, 8]), (13, [12, 11, 10, 9, 8]),
                                      (13, [7, 8, 9, 10, 11]), (15, [1, 3, 5, 7]), (20, [19, 18, 17, 0]),
                                      (18, [0, 1, 2, 3, 17]), (17, [6, 7, 8])])
def test_apply_fused_any_qubits_on_tensor_cores(q, N, qubits):
    # complex64, "auto": for k >= 3 on qubits other than 0..k-1 the tcgen05
    # kernel gathers whole groups (one CTA at N = 12; a stage of one
    # contiguous run when the qubits lie in bits 0..11; runs of 2^(12-k)
    # amplitudes when they lie high); k = 2 runs on the CUDA cores
    g = np.random.default_rng(N + len(qubits))
    v0 = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    v0 /= np.linalg.norm(v0)
    U = haar(1 << len(qubits), N)
    with q.Sim(N, "c64") as s:
        s.copy_in(v0)
        s.apply_fused(qubits, U)
        got = s.copy_out()
    ref = v0.astype(np.complex64).astype(np.complex128)
    sv.apply_dense(ref, N, qubits, U)
    assert np.max(np.abs(got - ref)) <= 4e-5
