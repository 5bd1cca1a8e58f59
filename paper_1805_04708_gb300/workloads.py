"""Seeded synthetic workloads (inputs only).

This module draws random numbers and writes gate lists; it contains none of
the simulator's arithmetic (no gate is applied here) and is shared by the
tests, the benchmark and both implementations as their common input.

Gate records are tuples (name, qubits, params) using the mnemonics of the
paper's instruction set (Appendix A): H, X, Y, Z, S, S+, T, T+, U1, U2, U3,
+X, -X, +Y, -Y, R, CNOT, U, TOFFOLI, plus RZ(theta) and MAT / CMAT (an
explicit 2x2 complex matrix given as 8 floats, row-major (re, im), after 0..2
control qubits), and MODMUL (controlled f -> a*f mod G on a register):
("MODMUL", (control,), (a, G, reg_lo, reg_w)).
"""
import math
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_u2(g):
    """A Haar-distributed U(2): QR of a complex Ginibre 2x2 matrix with the
    phases of R's diagonal moved into Q (Mezzadri, Notices AMS 54 (2007))."""
    Z = (g.standard_normal((2, 2)) + 1j * g.standard_normal((2, 2))) / math.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    Q = Q * (d / np.abs(d))
    out = np.empty(8)
    out[0::2] = Q.ravel().real
    out[1::2] = Q.ravel().imag
    return tuple(float(x) for x in out)


def layered_circuit(N, depth, seed):
    """Depth-`depth` random circuit: each layer applies a Haar-random U(2) to
    every qubit, then CNOTs on a random perfect matching of the qubits with a
    random orientation (one qubit idles when N is odd)."""
    g = rng(seed)
    recs = []
    for _ in range(depth):
        for q in range(N):
            recs.append(("MAT", (q,), haar_u2(g)))
        perm = g.permutation(N)
        for j in range(0, N - 1, 2):
            a, b = int(perm[j]), int(perm[j + 1])
            if g.integers(2):
                a, b = b, a
            recs.append(("CNOT", (a, b), ()))
    return recs


def random_gate_circuit(N, ngates, seed, hadamard_layer=True):
    """An all-Hadamard layer (optional) followed by `ngates` gates drawn
    uniformly from {H, T, RZ(theta ~ U[0, 2 pi)), CNOT, TOFFOLI}, on distinct
    qubits drawn uniformly from 0..N-1."""
    g = rng(seed)
    recs = [("H", (q,), ()) for q in range(N)] if hadamard_layer else []
    kinds = ("H", "T", "RZ", "CNOT", "TOFFOLI")
    for _ in range(ngates):
        k = kinds[int(g.integers(len(kinds)))]
        if k in ("H", "T"):
            recs.append((k, (int(g.integers(N)),), ()))
        elif k == "RZ":
            q = int(g.integers(N))
            recs.append(("RZ", (q,), (float(g.uniform(0.0, 2.0 * math.pi)),)))
        elif k == "CNOT":
            q = g.choice(N, 2, replace=False)
            recs.append(("CNOT", (int(q[0]), int(q[1])), ()))
        else:
            q = g.choice(N, 3, replace=False)
            recs.append(("TOFFOLI", (int(q[0]), int(q[1]), int(q[2])), ()))
    return recs


def block_partition(N, m, seed):
    """A seeded random partition of the qubits 0..N-1 into blocks of m (the
    last block takes the remainder), each block's qubits in increasing order."""
    perm = [int(x) for x in rng(seed).permutation(N)]
    return [sorted(perm[i:i + m]) for i in range(0, N, m)]


def block_gate_circuit(blocks, ngates, seed):
    """The random-gate family restricted to blocks of qubits: an
    all-Hadamard layer, then `ngates` gates drawn uniformly from {H, T,
    RZ(theta), U3 (random angles), CNOT, TOFFOLI}, each on distinct qubits of
    one uniformly chosen block (blocks too small for a gate redraw).  Every
    gate stays inside its block, so the final state is a tensor product of
    one state per block."""
    g = rng(seed)
    N = sum(len(b) for b in blocks)
    recs = [("H", (q,), ()) for q in range(N)]
    kinds = ("H", "T", "RZ", "U3", "CNOT", "TOFFOLI")
    while len(recs) < N + ngates:
        k = kinds[int(g.integers(len(kinds)))]
        b = blocks[int(g.integers(len(blocks)))]
        need = {"CNOT": 2, "TOFFOLI": 3}.get(k, 1)
        if len(b) < need:
            continue
        q = tuple(int(b[i]) for i in g.choice(len(b), need, replace=False))
        if k == "RZ":
            p = (float(g.uniform(0.0, 2.0 * math.pi)),)
        elif k == "U3":
            p = tuple(float(x) for x in g.uniform(0.0, 2.0 * math.pi, 3))
        else:
            p = ()
        recs.append((k, q, p))
    return recs


def aux_circuit(N, n_entangling, n_single, seed, toffoli=0):
    """A circuit for the auxiliary-variable method (Sec. 4.2): an
    all-Hadamard layer, then n_single single-qubit gates (H, T, RZ, U3) and
    n_entangling CNOT or controlled-phase U(k) gates (plus `toffoli` TOFFOLI
    gates) in random order on random distinct qubits."""
    g = rng(seed)
    kinds = ["1"] * n_single + ["2"] * n_entangling + ["3"] * toffoli
    order = g.permutation(len(kinds))
    recs = [("H", (q,), ()) for q in range(N)]
    for i in order:
        k = kinds[int(i)]
        if k == "1":
            name = ("H", "T", "RZ", "U3")[int(g.integers(4))]
            q = (int(g.integers(N)),)
            p = {"RZ": (float(g.uniform(0, 2 * math.pi)),),
                 "U3": tuple(float(x) for x in g.uniform(0, 2 * math.pi, 3))}.get(name, ())
            recs.append((name, q, p))
        elif k == "2":
            q = tuple(int(x) for x in g.choice(N, 2, replace=False))
            if g.integers(2):
                recs.append(("CNOT", q, ()))
            else:
                recs.append(("U", q, (int(g.integers(-6, 7)),)))
        else:
            recs.append(("TOFFOLI", tuple(int(x) for x in g.choice(N, 3, replace=False)), ()))
    return recs


def random_mixed_circuit(N, ngates, seed, max_controls=2):
    """Gates of every kind the instruction set has (random angles, random
    Haar matrices, 0..max_controls controls) on random distinct qubits; used
    for parity tests."""
    g = rng(seed)
    one_q = ("H", "X", "Y", "Z", "S", "S+", "T", "T+", "U1", "U2", "U3",
             "+X", "-X", "+Y", "-Y", "R", "RZ", "MAT", "I")
    recs = []
    for _ in range(ngates):
        u = int(g.integers(4))
        if u <= 1 or N < 2:
            k = one_q[int(g.integers(len(one_q)))]
            q = (int(g.integers(N)),)
            if k in ("U1", "RZ"):
                p = (float(g.uniform(0, 2 * math.pi)),)
            elif k == "U2":
                p = tuple(float(x) for x in g.uniform(0, 2 * math.pi, 2))
            elif k == "U3":
                p = tuple(float(x) for x in g.uniform(0, 2 * math.pi, 3))
            elif k == "R":
                p = (int(g.integers(-12, 13)),)
            elif k == "MAT":
                p = haar_u2(g)
            else:
                p = ()
            recs.append((k, q, p))
        elif u == 2:
            q = g.choice(N, 2, replace=False)
            if g.integers(2):
                recs.append(("CNOT", (int(q[0]), int(q[1])), ()))
            else:
                recs.append(("U", (int(q[0]), int(q[1])), (int(g.integers(-12, 13)),)))
        else:
            nc = min(int(g.integers(1, max_controls + 1)), N - 1)
            q = g.choice(N, nc + 1, replace=False)
            if N >= 3 and nc == 2 and g.integers(2):
                recs.append(("TOFFOLI", tuple(int(x) for x in q), ()))
            else:
                recs.append(("CMAT", tuple(int(x) for x in q), haar_u2(g)))
    return recs


def all_hadamard(N):
    """H on every qubit (Sec. 5.1, Table 2)."""
    return [("H", (q,), ()) for q in range(N)]


def ghz(N):
    """(H 0), (CNOT 0 1), ..., (CNOT N-2 N-1) (Sec. 5.2, Table 3)."""
    return [("H", (0,), ())] + [("CNOT", (q, q + 1), ()) for q in range(N - 1)]


def qft(qubits, inverse=False):
    """Textbook quantum Fourier transform on the register `qubits` (qubits[0]
    least significant) built from H and controlled phases U(k); the final bit
    reversal is left to the reader of the register (the output value k has
    bit m on qubit qubits[n-1-m]).  inverse=True conjugates every phase
    (U(-k) in the same order), which gives the inverse transform with the same
    bit-reversed output."""
    n = len(qubits)
    s = -1 if inverse else 1
    recs = []
    for j in range(n - 1, -1, -1):
        recs.append(("H", (qubits[j],), ()))
        for m in range(j - 1, -1, -1):
            recs.append(("U", (qubits[m], qubits[j]), (s * (j - m + 1),)))
    return recs


def shor_modmul(G, y, X, F):
    """Shor's circuit with the modular exponentiation written as controlled
    register permutations: X on qubit X (f = 1), H on x-register qubits
    0..X-1, then for j = 0..X-1 the multiplication f -> a_j f mod G
    (a_j = y^{2^j} mod G) controlled by x-bit j, and finally the inverse QFT of
    the x-register."""
    recs = [("X", (X,), ())]
    recs += [("H", (q,), ()) for q in range(X)]
    a = y % G
    for j in range(X):
        recs.append(("MODMUL", (j,), (a, G, X, F)))
        a = (a * a) % G
    recs += qft(list(range(X)), inverse=True)
    return recs


def coprime_base(G, seed):
    """A seeded random base 1 < y < G with gcd(y, G) = 1."""
    g = rng(seed)
    while True:
        y = int(g.integers(2, G))
        if math.gcd(y, G) == 1:
            return y


def error_correction_example(errors=(0,)):
    """The five-qubit error-correction example (Appendix B) up to the
    projective measurements: state preparation H T H on qubit 0, encoding,
    bit-flip errors on `errors`, syndrome extraction and correction.  The
    mid-circuit measurements M 3 and M 4 are deterministic in the three
    printed cases and are omitted."""
    recs = [("H", (0,), ()), ("T", (0,), ()), ("H", (0,), ()),
            ("CNOT", (0, 1), ()), ("CNOT", (0, 2), ())]
    stage1 = len(recs)
    recs += [("X", (q,), ()) for q in errors]
    recs += [("CNOT", (0, 3), ()), ("CNOT", (1, 3), ()),
             ("CNOT", (0, 4), ()), ("CNOT", (2, 4), ()),
             ("TOFFOLI", (3, 4, 0), ()), ("X", (4,), ()),
             ("TOFFOLI", (3, 4, 1), ()), ("X", (3,), ()), ("X", (4,), ()),
             ("TOFFOLI", (3, 4, 2), ()), ("X", (3,), ())]
    return recs, stage1


def program_text(N, records, bit_assignment=None, noise=None):
    """Program text in the instruction language of Appendix A for gate
    records; further instruction lines may be appended by the caller.
    noise: (p_x, p_y, p_z, seed) for a DEPOLARIZING CHANNEL line."""
    lines = ["QUBITS %d" % N]
    if bit_assignment is not None:
        lines.append("BIT ASSIGNMENT " + " ".join(str(int(x)) for x in bit_assignment))
    if noise is not None:
        lines.append("DEPOLARIZING CHANNEL P_X = %r, P_Y = %r, P_Z = %r, SEED = %d" % tuple(noise))
    for name, qs, ps in records:
        lines.append(" ".join([name] + [str(int(q)) for q in qs] + [repr(p) for p in ps]))
    return "\n".join(lines) + "\n"


def error_correction_program(errors=(0,), events=8192, seed=-1):
    """The Appendix B error-correction example as a program: preparation and
    encoding, BEGIN MEASUREMENT, bit-flip errors on `errors`, syndrome
    extraction with projective measurements M 3 and M 4 before the
    correction, re-preparation of qubit 3 (H, CLEAR) and qubit 4 (H, SET),
    BEGIN MEASUREMENT, and GENERATE EVENTS."""
    recs, stage1 = error_correction_example(errors)
    nerr = len(errors)
    syndrome = recs[stage1 + nerr: stage1 + nerr + 4]
    correct = recs[stage1 + nerr + 4:]
    body = program_text(5, recs[:stage1]).splitlines()
    body.append("BEGIN MEASUREMENT")
    body += program_text(5, recs[stage1: stage1 + nerr] + syndrome).splitlines()[1:]
    body += ["M 3", "M 4"]
    body += program_text(5, correct).splitlines()[1:]
    body += ["H 3", "CLEAR 3", "H 4", "SET 4", "BEGIN MEASUREMENT", "GENERATE EVENTS %d %d" % (events, seed)]
    return "\n".join(body) + "\n"


def serving_stream(n, rate, seed, nmin=12, nmax=28, dmin=10, dmax=100):
    """Requests for the serving loop: Poisson arrivals at `rate` per second,
    N ~ U{nmin..nmax}, depth ~ U{dmin..dmax}, each with its own circuit seed."""
    g = rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, n))
    Ns = g.integers(nmin, nmax + 1, n)
    ds = g.integers(dmin, dmax + 1, n)
    seeds = g.integers(1, 2 ** 31, n)
    return [dict(arrival=float(t[i]), N=int(Ns[i]), depth=int(ds[i]), seed=int(seeds[i]))
            for i in range(n)]
