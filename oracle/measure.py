"""The stochastic instructions of Appendix A: M, GENERATE EVENTS, CLEAR, SET
and DEPOLARIZING CHANNEL, plus the counter-based generator that turns a
program's seeds into uniform draws.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every random number is an input: the functions take uniform draws u in
[0, 1), and ``uniform(seed, counter)`` makes them from a seed with SplitMix64
(G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), written here from its published definition.

Readings (the appendix gives no formula for the draws):
  * M n picks outcome 0 when u * (p0 + p1) < p0, else 1 (inverse CDF over the
    outcomes in the order 0, 1), then projects like CLEAR / SET;
  * GENERATE EVENTS draws basis state i for a uniform u as the smallest i with
    C_i > u * C_last, C the cumulative sum of |a_i|^2 (inverse CDF in index
    order); it leaves the state unchanged;
  * DEPOLARIZING CHANNEL: after every gate, for every qubit q, one draw r
    decides X (r < p_x), Y (p_x <= r < p_x + p_y), Z (p_x + p_y <= r <
    p_x + p_y + p_z) or nothing; the draw for gate g (0-based) and qubit q is
    uniform(seed, g * N + q).
"""
import math
from fractions import Fraction

import numpy as np

from . import statevec as sv

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed, counter):
    """Output number `counter` (0-based) of the SplitMix64 sequence started at
    `seed`: the state advances by the golden-ratio increment before each
    output, and the output is the state passed through the two
    xor-shift-multiply rounds and a final xor-shift of the published mixer."""
    z = (int(seed) + (int(counter) + 1) * _GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform(seed, counter):
    """A uniform double in [0, 1): the top 53 bits of the SplitMix64 output."""
    return (splitmix64(seed, counter) >> 11) * (1.0 / (1 << 53))


def uniforms(seed, first, n):
    return np.array([uniform(seed, first + k) for k in range(n)], dtype=np.float64)


def probs_of_qubit(v, N, q):
    """(p0, p1): probabilities of outcomes 0 and 1 of qubit q (Sec. 2)."""
    p1 = sv.prob_one(v, N, q)
    P = sv.probabilities(v).reshape((2,) * N)
    sel = [slice(None)] * N
    sel[N - 1 - q] = 0
    p0 = sv.csum(P[tuple(sel)])
    return p0, p1


def measure(v, N, q, u):
    """M q (Appendix A): outcome 0 if u (p0 + p1) < p0 else 1, then the state
    is projected onto that outcome and renormalised (in place).  Returns
    (outcome, p0, p1)."""
    p0, p1 = probs_of_qubit(v, N, q)
    outcome = 0 if u * (p0 + p1) < p0 else 1
    sv.project(v, N, q, outcome)
    return outcome, p0, p1


def clear(v, N, q):
    """CLEAR q: |0><0| on qubit q, renormalised; ValueError on a zero state."""
    return sv.project(v, N, q, 0)


def set_(v, N, q):
    """SET q: |1><1| on qubit q, renormalised; ValueError on a zero state."""
    return sv.project(v, N, q, 1)


def cumulative(v):
    """C_i = sum_{j <= i} |a_j|^2 (FP64 running sum in index order)."""
    return np.cumsum(sv.probabilities(v))


def sample_events(v, u):
    """GENERATE EVENTS: for every draw u, the smallest index i with
    C_i > u * C_last; a draw at or beyond the last boundary takes the last
    index with nonzero probability.  The state is not changed."""
    C = cumulative(v)
    T = C[-1]
    u = np.asarray(u, dtype=np.float64)
    idx = np.searchsorted(C, u * T, side="right")
    nz = np.nonzero(sv.probabilities(v) > 0)[0]
    last = nz[-1] if nz.size else len(C) - 1
    return np.minimum(idx, last).astype(np.int64)


def sample_events_exact(probs, u):
    """The same inverse CDF in exact rational arithmetic on the FP64 values
    of |a_i|^2 (pure Python; small cases only)."""
    p = [Fraction(float(x)) for x in probs]
    C, s = [], Fraction(0)
    for x in p:
        s += x
        C.append(s)
    T = C[-1]
    last = max(i for i, x in enumerate(p) if x > 0)
    out = []
    for uu in u:
        t = Fraction(float(uu)) * T
        i = next((k for k, c in enumerate(C) if c > t), last)
        out.append(min(i, last))
    return np.array(out, dtype=np.int64)


def depolarize(records, N, px, py, pz, seed):
    """DEPOLARIZING CHANNEL P_X = px, P_Y = py, P_Z = pz, SEED = seed: the
    circuit with X, Y or Z inserted after every gate on every qubit where the
    draw falls in the respective interval."""
    if min(px, py, pz) < 0 or px + py + pz > 1:
        raise ValueError("probabilities out of range")
    out = []
    for g, rec in enumerate(records):
        out.append(rec)
        for q in range(N):
            r = uniform(seed, g * N + q)
            if r < px:
                out.append(("X", (q,), ()))
            elif r < px + py:
                out.append(("Y", (q,), ()))
            elif r < px + py + pz:
                out.append(("Z", (q,), ()))
    return out


def brute_projector(N, q, bit):
    """The 2^N x 2^N matrix of |bit><bit| on qubit q (a dense diagonal), for
    pins at small N."""
    i = np.arange(1 << N)
    return np.diag((((i >> q) & 1) == bit).astype(np.float64)).astype(np.complex128)


def chi_square(counts, probs):
    """Pearson's statistic of observed counts against expected probabilities
    (bins with expectation 0 must have count 0)."""
    counts = np.asarray(counts, dtype=np.float64)
    n = counts.sum()
    e = n * np.asarray(probs, dtype=np.float64)
    m = e > 0
    if np.any(counts[~m] > 0):
        return math.inf
    return float(np.sum((counts[m] - e[m]) ** 2 / e[m]))
