"""GPU parity: the CUDA path (through the C ABI) against the oracle on the same
seeded inputs.  Tolerances: complex128 max-abs 1e-12, complex64 max-abs 1e-5
(amplitudes); permutations and SHORBOX bit-exact; reductions of a state
against the oracle's compensated sums of the same stored values."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import circuit, gates as ogates, statevec as sv, shor  # noqa: E402
from paper_1805_04708_gb300 import workloads as wl  # noqa: E402

TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    return qsim


def rand_state(N, seed):
    g = np.random.default_rng(seed)
    v = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    return v / np.linalg.norm(v)


def stored(v, enc):
    """The values the device holds after copy_in (complex64 rounds)."""
    return v.astype(np.complex64).astype(np.complex128) if enc == "c64" else v


def maxerr(a, b):
    return float(np.max(np.abs(np.asarray(a, np.complex128) - np.asarray(b, np.complex128))))


@pytest.mark.parametrize("enc", ["c128", "c64"])
@pytest.mark.parametrize("N", [2, 3, 5, 8, 11, 14, 17])
@pytest.mark.parametrize("mode", [0, 1])
def test_random_mixed_circuit(q, enc, N, mode):
    # N >= 14 exceeds one tile: several passes, with commuting gates moved
    # ahead of the gates left for later passes
    recs = wl.random_mixed_circuit(N, 50 if N < 14 else 160, seed=100 + N)
    v0 = rand_state(N, N)
    ref = circuit.run(stored(v0, enc).copy(), N, recs)
    with q.Sim(N, enc) as s:
        s.copy_in(v0)
        s.circuit_run(recs, mode=mode)
        got = s.copy_out()
    assert maxerr(got, ref) <= TOL[enc]


@pytest.mark.parametrize("enc", ["c128", "c64"])
@pytest.mark.parametrize("N", [16, 21])
def test_tile_pass_packing(q, enc, N):
    # H / T / RZ / CNOT / TOFFOLI on random qubits: most gates commute with
    # some of their neighbours, so the passes take gates out of circuit order;
    # the state must equal the per-gate sweeps' and the oracle's
    recs = wl.random_gate_circuit(N, 300, seed=40 + N)
    ref = circuit.run(sv.zero_state(N), N, recs)
    with q.Sim(N, enc) as s:
        npass = s.circuit_run(recs, mode=1)
        got = s.copy_out()
    with q.Sim(N, enc) as s:
        s.circuit_run(recs, mode=0)
        per_gate = s.copy_out()
    assert maxerr(got, ref) <= TOL[enc]
    assert maxerr(got, per_gate) <= TOL[enc]
    assert 1 < npass < len(recs) // 4


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_reset_then_every_access(q, enc):
    # a reset state is |0..0> whichever call reads or writes it first: the
    # first tile pass makes its tiles, every other call writes the state first
    N = 14
    recs = wl.random_gate_circuit(N, 60, seed=4)
    ref = circuit.run(sv.zero_state(N), N, recs)
    e0 = sv.zero_state(N)
    with q.Sim(N, enc) as s:
        s.circuit_run(recs, mode=1)
        s.reset()
        s.circuit_run(recs, mode=1)               # first pass starts from |0..0>
        assert maxerr(s.copy_out(), ref) <= TOL[enc]
        s.reset()
        assert maxerr(s.copy_out(), e0) == 0.0
        s.circuit_run(recs, mode=1)
        s.reset()
        assert abs(s.norm() - 1.0) == 0.0
        s.reset()
        p = s.measure_probs([0, 1, 2])
        assert p[0] == 1.0 and np.all(p[1:] == 0.0)
        s.reset()
        qx, qy, qz = s.expect_xyz()
        assert np.allclose(qz, 0.0, atol=0) and np.allclose(qx, 0.5, atol=1e-15)
        s.reset()
        s.apply_gate(3, np.array([[1, 1], [1, -1]]) / np.sqrt(2))
        want = np.zeros(1 << N, complex)
        want[0] = want[8] = 2 ** -0.5
        assert maxerr(s.copy_out(), want) <= TOL[enc]
        s.reset()
        # the device pointer: the caller may read the memory directly
        ptr = s.device_ptr()
        s.sync()
        p = q.measure_probs_static(ptr, N, enc, [0, 5, 13])
        assert p[0] == 1.0 and np.all(p[1:] == 0.0)


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_every_gate_every_position(q, enc):
    N = 6
    names = ["H", "X", "Y", "Z", "S", "S+", "T", "T+", "+X", "-X", "+Y", "-Y"]
    with q.Sim(N, enc) as s:
        for t in range(N):
            for name in names + ["U1", "U3", "RZ", "MAT", "R"]:
                p = {"U1": (0.37,), "U3": (0.4, 1.3, -2.2), "RZ": (2.9,), "R": (5,),
                     "MAT": wl.haar_u2(wl.rng(t))}.get(name, ())
                v0 = rand_state(N, t * 31 + len(name))
                s.copy_in(v0)
                s.circuit_run([(name, (t,), p)], mode=0)
                ref = circuit.run(stored(v0, enc).copy(), N, [(name, (t,), p)])
                assert maxerr(s.copy_out(), ref) <= TOL[enc], (name, t)
        # controlled forms at every (control, target) and (c1, c2, target)
        for c in range(N):
            for t in range(N):
                if c == t:
                    continue
                for rec in [("CNOT", (c, t), ()), ("U", (c, t), (3,)), ("U", (c, t), (-7,)),
                            ("CMAT", (c, t), wl.haar_u2(wl.rng(c * 8 + t)))]:
                    v0 = rand_state(N, c * 7 + t)
                    s.copy_in(v0)
                    s.circuit_run([rec], mode=0)
                    ref = circuit.run(stored(v0, enc).copy(), N, [rec])
                    assert maxerr(s.copy_out(), ref) <= TOL[enc], rec
        for c1 in range(N):
            for c2 in range(N):
                for t in range(N):
                    if len({c1, c2, t}) < 3:
                        continue
                    rec = ("TOFFOLI", (c1, c2, t), ())
                    v0 = rand_state(N, c1 + 8 * c2 + 64 * t)
                    s.copy_in(v0)
                    s.circuit_run([rec], mode=0)
                    ref = circuit.run(stored(v0, enc).copy(), N, [rec])
                    # a pure swap: bit-exact
                    assert np.array_equal(s.copy_out(), ref.astype(s.copy_out().dtype)), rec


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_layered_circuit_n20(q, enc):
    # the 16 MiB complex128 configuration: N = 20, depth 20, Haar U(2) layers +
    # CNOTs on random matchings
    N = 20
    recs = wl.layered_circuit(N, 20, seed=1)
    ref = circuit.run(sv.zero_state(N), N, recs)
    for mode in (0, 1):
        with q.Sim(N, enc) as s:
            s.circuit_run(recs, mode=mode)
            assert maxerr(s.copy_out(), ref) <= TOL[enc]


@pytest.mark.parametrize("enc", ["c128", "c64"])
@pytest.mark.parametrize("N", [2, 4, 9, 12, 13, 14, 17, 22, 23])
def test_reductions(q, enc, N):
    v0 = rand_state(N, 5 * N) * 0.97
    with q.Sim(N, enc) as s:
        s.copy_in(v0)
        v = stored(v0, enc)
        assert abs(s.norm() - sv.norm(v)) <= 1e-13
        qx, qy, qz = s.expect_xyz()
        rx, ry, rz = sv.expect_xyz(v, N)
        # complex64 BEGIN MEASUREMENT: FP32 products and <= 32-term FP32 leaf
        # sums folded into float-float / FP64 accumulators; complex128: FP64
        tol = 1e-8 if (enc == "c64" and N >= 13) else 1e-13
        assert np.max(np.abs(qx - rx)) <= tol
        assert np.max(np.abs(qy - ry)) <= tol
        assert np.max(np.abs(qz - rz)) <= tol
        # both in one call (complex64, N >= 23: one pass also sums |a|^2)
        qx2, qy2, qz2, nrm2 = s.expect_xyz_norm()
        assert abs(nrm2 - sv.norm(v)) <= 1e-13
        for a, b in ((qx2, qx), (qy2, qy), (qz2, qz)):
            assert np.max(np.abs(a - b)) <= 1e-15
        g = np.random.default_rng(N)
        for nq in sorted({1, min(3, N), min(N, 7)}):
            qs = [int(x) for x in g.choice(N, nq, replace=False)]
            P = s.measure_probs(qs)
            assert np.max(np.abs(P - sv.marginal(v, N, qs))) <= 1e-13


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_permutation_bit_exact(q, enc):
    g = np.random.default_rng(3)
    for N, lo, w, ctrls in [(8, 3, 3, [0]), (10, 0, 4, [9, 5]), (12, 6, 6, [1, 2]), (9, 2, 5, []),
                            (14, 10, 4, [0, 1, 2])]:
        table = g.permutation(1 << w).astype(np.uint32)
        v0 = rand_state(N, N + w)
        with q.Sim(N, enc) as s:
            s.copy_in(v0)
            s.apply_permutation(ctrls, lo, w, table)
            got = s.copy_out()
        ref = sv.apply_permutation(stored(v0, enc).copy(), N, ctrls, lo, w, table)
        assert np.array_equal(got, ref.astype(got.dtype))


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_shorbox_bit_exact(q, enc):
    for N, nx, G, y in [(12, 8, 15, 7), (14, 9, 21, 2), (18, 12, 55, 7)]:
        with q.Sim(N, enc) as s:
            s.shorbox_init(nx, G, y)
            got = s.copy_out()
        ref = sv.shorbox(N, nx, G, y)
        assert np.array_equal(got, ref.astype(got.dtype))


def test_errors(q):
    with q.Sim(4, "c128") as s:
        with pytest.raises(q.QSError) as e:
            s.apply_gate(4, np.eye(2))
        assert e.value.name == "QS_EINVAL"
        with pytest.raises(q.QSError) as e:
            s.apply_gate(0, [[1, 1], [0, 1]])
        assert e.value.name == "QS_ENOTUNITARY"
        with pytest.raises(q.QSError) as e:
            s.apply_controlled([1], 1, np.eye(2))
        assert e.value.name == "QS_EINVAL"
        with pytest.raises(q.QSError) as e:
            s.apply_permutation([], 0, 2, [0, 1, 1, 3])
        assert e.value.name == "QS_ENOTBIJECTIVE"
        with pytest.raises(q.QSError):
            s.apply_permutation([1], 0, 2, [0, 1, 2, 3])  # control inside register
        # the state is untouched by the rejected calls
        a = s.copy_out()
        assert a[0] == 1 and not np.any(a[1:])
    with pytest.raises(q.QSError):
        q.Sim(1, "c128")


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_shor_config_n30(q, enc):
    """Shor period finding for G = 899 = 29 x 31 with a seeded base, X = 20,
    F = 10, N = 30: X on qubit 20, H layer, 20 controlled modular
    multiplications as bit-exact permutations, inverse QFT; the x-register
    distribution against the closed form, and the factors recovered."""
    G = 899
    X, F = shor.qubit_budget(G)
    assert (X, F) == (20, 10)
    y = wl.coprime_base(G, 1)
    r = shor.order(y, G)
    P_ref = shor.closed_form_distribution(X, r)
    with q.Sim(X + F, enc) as s:
        s.run_records(wl.shor_modmul(G, y, X, F), mode=1)
        P = s.measure_probs(list(range(X - 1, -1, -1)))
        nrm = s.norm()
    tol = 1e-9 if enc == "c128" else 2e-6
    assert abs(nrm - 1.0) <= (1e-12 if enc == "c128" else 1e-5)
    assert np.max(np.abs(P - P_ref)) <= tol
    ks = np.argsort(P)[::-1][:8]
    periods = {shor.period_from_sample(int(k), X, G) for k in ks if k}
    assert any(p and r % p == 0 for p in periods)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("df", [1, 0, 2])
@pytest.mark.parametrize("N,kind", [(9, "mixed"), (14, "mixed"), (17, "layered"), (20, "gates")])
def test_c128_tile_passes_fp64_and_double_float(q, df, N, kind, mode):
    # complex128 tile passes computed on FP32 pairs (double-float), on the
    # FP64 units, and in the default mode: all within 1e-12 of the oracle
    recs = {"mixed": wl.random_mixed_circuit(N, 120, seed=300 + N),
            "layered": wl.layered_circuit(N, 4, seed=N),
            "gates": wl.random_gate_circuit(N, 150, seed=N)}[kind]
    v0 = rand_state(N, 500 + N)
    ref = circuit.run(v0.copy(), N, recs)
    with q.Sim(N, "c128") as s:
        s.set_fp64_emulation(df)
        s.copy_in(v0)
        s.circuit_run(recs, mode=mode)
        assert maxerr(s.copy_out(), ref) <= 1e-12
