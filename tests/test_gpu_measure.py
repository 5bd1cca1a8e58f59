"""GPU parity of the stochastic instructions (Appendix A: M, CLEAR, SET,
GENERATE EVENTS, DEPOLARIZING CHANNEL), the bit permutation and the program
front-end, through the C ABI, against the oracle on the same draws.

Tolerances: complex128 1e-12, complex64 1e-5 max-abs for states and
probabilities; M outcomes and events are integers decided by comparing a
draw with FP64 sums, so they must agree exactly except where the draw's
target lies within the two sides' summation error of a boundary (then the
device's event must be a neighbouring index whose interval reaches the
target); permutations bit-exact."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import circuit, measure as om, program as oprog, statevec as sv  # noqa: E402
from oracle.adapt2 import AState  # noqa: E402
from paper_1805_04708_gb300 import workloads as wl  # noqa: E402

TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    return qsim


def rand_state(N, seed, zeros=0):
    g = np.random.default_rng(seed)
    v = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    if zeros:
        v[g.choice(1 << N, zeros, replace=False)] = 0
    return v / np.linalg.norm(v)


def stored(v, enc):
    return v.astype(np.complex64).astype(np.complex128) if enc == "c64" else v.copy()


def maxerr(a, b):
    return float(np.max(np.abs(np.asarray(a, np.complex128) - np.asarray(b, np.complex128))))


# ---------------------------------------------------------------------------
# M, CLEAR, SET
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("enc", ["c128", "c64"])
@pytest.mark.parametrize("N", [3, 9, 17])
def test_measure_matches_oracle(q, enc, N):
    v0 = rand_state(N, N)
    u = om.uniforms(N, 0, 2 * N)
    with q.Sim(N, enc) as s:
        ref = stored(v0, enc)
        s.copy_in(ref)
        for k, qq in enumerate(list(range(N)) + list(range(N - 1, -1, -1))):
            o, p0, p1 = s.measure(qq, u[k])
            wo, wp0, wp1 = om.measure(ref, N, qq, u[k])
            assert abs(p0 - wp0) <= 1e-12 and abs(p1 - wp1) <= 1e-12
            # a draw within rounding of the boundary may go either way
            if abs(u[k] * (wp0 + wp1) - wp0) > 1e-12:
                assert o == wo
            got = s.copy_out()
            if o == wo:
                assert maxerr(got, ref) <= TOL[enc]
            ref = np.asarray(got, np.complex128)   # continue from the device state


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_clear_set_match_oracle(q, enc):
    N = 12
    v0 = rand_state(N, 4)
    with q.Sim(N, enc) as s:
        for qq, bit in ((0, 0), (5, 1), (11, 0), (3, 1)):
            s.copy_in(v0)
            ref = stored(v0, enc)
            pw = om.probs_of_qubit(ref, N, qq)[bit]
            p = s.project(qq, bit)
            assert abs(p - pw) <= 1e-12
            (om.clear if bit == 0 else om.set_)(ref, N, qq)
            assert maxerr(s.copy_out(), ref) <= TOL[enc]
            assert abs(s.norm() - 1.0) <= (1e-12 if enc == "c128" else 1e-6)


@pytest.mark.parametrize("enc", ["c128", "c64", "adapt2"])
def test_zero_projection_fails_and_keeps_state(q, enc):
    N = 6
    with q.Sim(N, enc) as s:
        s.circuit_run([("X", (2,), ()), ("H", (4,), ())], mode=0)
        before = s.copy_out()
        with pytest.raises(q.QSError) as e:
            s.project(2, 0)
        assert e.value.name == "QS_EZEROPROJ"
        after = s.copy_out()
        if enc == "adapt2":
            assert np.array_equal(before[0], after[0])
        else:
            assert np.array_equal(before, after)
        # SET on the same qubit keeps everything: its probability is the
        # stored state's whole norm (complex64 rounds 1/sqrt(2))
        if enc == "adapt2":
            assert abs(s.project(2, 1) - 1.0) <= 1e-6
        else:
            assert abs(s.project(2, 1) - sv.norm(np.asarray(before, np.complex128))) <= 1e-12


def test_measure_adapt2_against_emulation(q):
    # the adaptive encoding re-encodes after the projection (decode, project,
    # re-tune, encode); compare the decoded state with the oracle's emulation
    N = 8
    recs = wl.layered_circuit(N, 2, seed=3)
    a = circuit.run_adapt2(AState.zero(N), recs)
    u = om.uniforms(77, 0, 4)
    with q.Sim(N, "adapt2") as s:
        s.circuit_run(recs, mode=0)
        for k, qq in enumerate((1, 6, 3, 0)):
            z = a.to_complex()
            wo, _, _ = om.measure(z, N, qq, u[k])
            from oracle.adapt2 import retune, encode
            a.r0, a.r1 = retune(z)
            a.b0, a.b1 = encode(z, a.r0, a.r1)
            o, _, _ = s.measure(qq, u[k])
            assert o == wo
            words, (r0, r1) = s.copy_out()
            from oracle.adapt2 import unpack, decode
            b0, b1 = unpack(words)
            got = decode(b0, b1, r0, r1)
            # both sides quantise: within a few code steps of the magnitude
            # range plus the angle step
            step = (a.r1 - a.r0) / 253 + np.max(np.abs(z)) * math.pi / 128
            assert maxerr(got, a.to_complex()) <= 4 * step


# ---------------------------------------------------------------------------
# GENERATE EVENTS
# ---------------------------------------------------------------------------
def check_events(got, v, u, eps_rel):
    """Equal to the oracle's inverse CDF except within eps of a boundary, where
    the device's index must still be a valid one for the target."""
    want = om.sample_events(v, u)
    p = sv.probabilities(v)
    C = np.cumsum(p)
    T = C[-1]
    assert np.all(p[got] > 0)
    bad = np.nonzero(got != want)[0]
    for k in bad:
        t = u[k] * T
        lo = C[got[k] - 1] if got[k] > 0 else 0.0
        assert lo - eps_rel * T <= t <= C[got[k]] + eps_rel * T
    return len(bad)


@pytest.mark.parametrize("enc", ["c128", "c64"])
@pytest.mark.parametrize("N,zeros", [(3, 2), (5, 0), (10, 100), (11, 500), (16, 3000), (21, 0)])
def test_events_match_oracle(q, enc, N, zeros):
    v0 = rand_state(N, 100 + N, zeros)
    ref = stored(v0, enc)
    g = np.random.default_rng(N)
    C = np.cumsum(sv.probabilities(ref))
    u = np.concatenate([g.random(20000), [0.0, np.nextafter(1.0, 0)], C[:-1:max(1, len(C) // 500)] / C[-1]])
    with q.Sim(N, enc) as s:
        s.copy_in(v0)
        got = s.generate_events(u)
        nbad = check_events(got, ref, u, 1e-10)
        assert nbad <= 10 + len(u) - 20002
        # the state is unchanged
        assert maxerr(s.copy_out(), ref) == 0.0


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_events_seeded_equal_explicit_draws(q, enc):
    N = 14
    v0 = rand_state(N, 5, 1000)
    with q.Sim(N, enc) as s:
        s.copy_in(v0)
        a = s.generate_events(n=5000, seed=99)
        b = s.generate_events(u=q.uniforms(99, 0, 5000))
        assert np.array_equal(a, b)


def test_events_ghz_and_basis(q):
    N = 20
    with q.Sim(N, "c64") as s:
        s.circuit_run(wl.ghz(N), mode=1)
        ev = s.generate_events(n=20000, seed=3)
        assert set(np.unique(ev)) <= {0, (1 << N) - 1}
        frac = float(np.mean(ev == 0))
        assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / 20000)
        s.reset()
        s.circuit_run([("X", (3,), ()), ("X", (19,), ())], mode=0)
        assert np.all(s.generate_events(n=1000, seed=4) == (1 << 3) + (1 << 19))


def test_events_adapt2(q):
    N = 12
    recs = wl.layered_circuit(N, 1, seed=8)
    with q.Sim(N, "adapt2") as s:
        s.circuit_run(recs, mode=0)
        words, (r0, r1) = s.copy_out()
        from oracle.adapt2 import unpack, decode
        b0, b1 = unpack(words)
        z = decode(b0, b1, r0, r1)
        u = om.uniforms(1, 0, 10000)
        got = s.generate_events(u)
        # the device decodes magnitudes from an FP32 table: boundaries agree
        # to about 1e-6 of the total
        nbad = check_events(got, z, u, 1e-6)
        assert nbad <= 20


def test_events_n26_c64(q):
    N = 26
    recs = wl.random_gate_circuit(N, 60, 2)
    with q.Sim(N, "c64") as s:
        s.circuit_run(recs, mode=1)
        v = np.asarray(s.copy_out(), np.complex128)
        u = om.uniforms(26, 0, 50000)
        got = s.generate_events(u)
    nbad = check_events(got, v, u, 1e-9)
    assert nbad <= 5


def test_events_reject_bad_draws(q):
    with q.Sim(5, "c64") as s:
        for bad in ([1.0], [-0.1], [float("nan")]):
            with pytest.raises(q.QSError):
                s.generate_events(np.array(bad))


# ---------------------------------------------------------------------------
# DEPOLARIZING CHANNEL, bit permutation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_depolarized_circuit_matches_oracle(q, enc):
    N = 9
    recs = wl.random_gate_circuit(N, 60, 4)
    noisy = om.depolarize(recs, N, 0.02, 0.03, 0.05, 1234)
    ref = circuit.run(sv.zero_state(N), N, noisy)
    arr = q.depolarize_circuit(N, recs, 0.02, 0.03, 0.05, 1234)
    with q.Sim(N, enc) as s:
        s.circuit_run(arr, mode=1)
        assert maxerr(s.copy_out(), ref) <= TOL[enc]


@pytest.mark.parametrize("enc", ["c128", "c64", "adapt2"])
@pytest.mark.parametrize("N", [5, 14, 20])
def test_permute_qubits_exact(q, enc, N):
    g = np.random.default_rng(N)
    perm = [int(x) for x in g.permutation(N)]
    with q.Sim(N, enc) as s:
        if enc == "adapt2":
            s.circuit_run(wl.layered_circuit(N, 1, seed=2), mode=0)
            before = s.copy_out()[0]
        else:
            s.copy_in(rand_state(N, 7))
            before = s.copy_out()
        s.permute_qubits(perm)
        after = s.copy_out()[0] if enc == "adapt2" else s.copy_out()
    i = np.arange(1 << N, dtype=np.int64)
    j = np.zeros_like(i)
    for k in range(N):
        j |= ((i >> k) & 1) << perm[k]
    want = np.empty_like(before)
    want[j] = before
    assert np.array_equal(after, want)


# ---------------------------------------------------------------------------
# programs
# ---------------------------------------------------------------------------
def _golden():
    import os
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "appB_error_correction.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        case, stage, qq, x, y, z = line.split()
        rows[(case, int(stage), int(qq))] = (float(x), float(y), float(z))
    return rows


@pytest.mark.parametrize("enc", ["c128", "c64", "adapt2"])
@pytest.mark.parametrize("case,errors", [("i", ()), ("ii", (0,)), ("iii", (0, 1))])
def test_appendix_b_program_on_gpu(q, enc, case, errors):
    rows = _golden()
    text = wl.error_correction_program(errors)
    want = oprog.run(text, run_seed=3, enc="adapt2" if enc == "adapt2" else "c128")
    prog = q.Program(text)
    with q.Sim(5, enc) as s:
        res = prog.run(s, run_seed=3, mode=1)
    assert len(res["measurements"]) == 2
    wm = [o for o in want["out"] if o[0] == "BEGIN MEASUREMENT"]
    tol = {"c128": 1e-12, "c64": 1e-5, "adapt2": 2e-3}[enc]
    for stage, (got, w) in enumerate(zip(res["measurements"], wm), 1):
        for a, b in zip(got, w[1:]):
            assert float(np.max(np.abs(a - b))) <= tol
        for qq in range(5):   # the paper's printed digits
            for a, b in zip((got[0][qq], got[1][qq], got[2][qq]), rows[(case, stage, qq)]):
                assert abs(a - b) <= 5e-4 + (2e-3 if enc == "adapt2" else 0)
    wM = [o for o in want["out"] if o[0] == "M"]
    assert [(m[0], m[1]) for m in res["m"]] == [(o[1], o[2]) for o in wM]
    wev = [o for o in want["out"] if o[0] == "GENERATE EVENTS"][0][1]
    assert len(res["events"]) == 8192
    assert np.array_equal(res["events"], wev)


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_random_program_with_bit_assignment(q, enc):
    # gates, measurements, projections, noise and events, with qubits renumbered
    # before the first gate and again in the middle: every result per logical
    # qubit equals the oracle's run of the program without any renumbering
    N = 10
    g = np.random.default_rng(5)
    recs = wl.random_gate_circuit(N, 40, 9)
    half = len(recs) // 2
    p1 = [int(x) for x in g.permutation(N)]
    p2 = [int(x) for x in g.permutation(N)]
    body = wl.program_text(N, recs[:half], bit_assignment=p1, noise=(0.01, 0.01, 0.02, 17)).splitlines()
    body += ["BEGIN MEASUREMENT", "M 3", "BIT ASSIGNMENT " + " ".join(map(str, p2))]
    body += wl.program_text(N, recs[half:]).splitlines()[1:]
    body += ["M 7", "CLEAR 0", "BEGIN MEASUREMENT", "GENERATE EVENTS 4000 5"]
    text = "\n".join(body) + "\n"
    plain = text.replace("BIT ASSIGNMENT " + " ".join(map(str, p1)), "").replace(
        "BIT ASSIGNMENT " + " ".join(map(str, p2)), "")
    want = oprog.run(plain, run_seed=11)
    with q.Sim(N, enc) as s:
        res = q.Program(text).run(s, run_seed=11, mode=1)
        res0 = q.Program(plain).run(s, run_seed=11, mode=1)
    wm = [o for o in want["out"] if o[0] == "BEGIN MEASUREMENT"]
    for r in (res, res0):
        for got, w in zip(r["measurements"], wm):
            for a, b in zip(got, w[1:]):
                assert float(np.max(np.abs(a - b))) <= TOL[enc]
        assert [(m[0], m[1]) for m in r["m"]] == [(o[1], o[2]) for o in want["out"] if o[0] == "M"]
    wev = [o for o in want["out"] if o[0] == "GENERATE EVENTS"][0][1]
    # events: both runs agree exactly; against the oracle up to boundary rounding
    assert np.array_equal(res["events"], res0["events"])
    assert np.count_nonzero(res["events"] != wev) <= 4


def test_program_shorbox_and_exit(q):
    # SHORBOX then EXIT (one BEGIN MEASUREMENT, nothing after it runs)
    text = "QUBITS 12\nSHORBOX 8 15 7\nEXIT\nH 0\nBEGIN MEASUREMENT\n"
    want = oprog.run(text)
    with q.Sim(12, "c128") as s:
        res = q.Program(text).run(s)
    assert len(res["measurements"]) == 1
    for a, b in zip(res["measurements"][0], want["out"][0][1:]):
        assert float(np.max(np.abs(a - b))) <= 1e-12


def test_program_clear_zero_fails(q):
    text = "QUBITS 4\nX 1\nCLEAR 1\n"
    with q.Sim(4, "c64") as s:
        with pytest.raises(q.QSError) as e:
            q.Program(text).run(s)
        assert e.value.name == "QS_EZEROPROJ"
