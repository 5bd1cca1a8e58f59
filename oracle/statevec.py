"""Complex128 state-vector oracle (Secs. 2 and 3 of arXiv:1805.04708).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (Sec. 2, Eq. (STAT2) and the paragraph after it): the state of N
qubits is a vector v of 2^N complex amplitudes; qubit q is bit q of the basis
index, qubit 0 the rightmost (least significant) bit.  In the numpy view
``v.reshape((2,)*N)`` qubit q is axis N-1-q.
"""
import math
import numpy as np


# --------------------------------------------------------------------------
# state preparation
# --------------------------------------------------------------------------
def zero_state(N):
    """|0...0> (Eq. (appa0)): a(0) = 1, all other amplitudes 0."""
    v = np.zeros(1 << N, dtype=np.complex128)
    v[0] = 1.0
    return v


def _view(v, N):
    return v.reshape((2,) * N)


def _axis(N, q):
    return N - 1 - q


# --------------------------------------------------------------------------
# gates
# --------------------------------------------------------------------------
def apply_controlled_u2(v, N, controls, target, U):
    """Apply the 2x2 matrix U to qubit ``target`` on the subspace where every
    qubit in ``controls`` is 1, in place.

    This is the update rule of Eq. (NUM2) with H replaced by a general U
    (Eq. (AQS0)): for every basis index whose bit ``target`` is 0 (and whose
    control bits are 1) the pair (a(*0_t*), a(*1_t*)) is replaced by
    U (a(*0_t*), a(*1_t*))^T.  With no controls this is the single-qubit gate of
    Sec. 2; with one (two) controls it is the group-of-four (group-of-eight)
    update of CNOT / U(k) (TOFFOLI) described after Eq. (NUM2).
    """
    U = np.asarray(U, dtype=np.complex128)
    qs = list(controls) + [target]
    if len(set(qs)) != len(qs) or min(qs) < 0 or max(qs) >= N:
        raise ValueError("qubits out of range or not distinct")
    T = _view(v, N)
    sel0 = [slice(None)] * N
    for c in controls:
        sel0[_axis(N, c)] = 1
    sel1 = list(sel0)
    sel0[_axis(N, target)] = 0
    sel1[_axis(N, target)] = 1
    sel0, sel1 = tuple(sel0), tuple(sel1)
    a0 = T[sel0].copy()
    a1 = T[sel1].copy()
    T[sel0] = U[0, 0] * a0 + U[0, 1] * a1
    T[sel1] = U[1, 0] * a0 + U[1, 1] * a1
    return v


def apply_dense(v, N, qubits, U):
    """Apply a dense 2^k x 2^k matrix U to the qubits ``qubits`` (k of them), in
    place.  Local index convention: bit m of the row/column index of U is the
    value of qubit ``qubits[m]``.

    This is the multi-qubit gate of Eq. (AQS0): an n-qubit gate is a unitary
    matrix of size 2^n acting on the n qubits' part of the index; the end of
    Sec. 5.2 proposes fusing several gates into one such matrix.
    """
    U = np.asarray(U, dtype=np.complex128)
    k = len(qubits)
    if U.shape != (1 << k, 1 << k):
        raise ValueError("U has the wrong shape")
    if len(set(qubits)) != k or min(qubits) < 0 or max(qubits) >= N:
        raise ValueError("qubits out of range or not distinct")
    T = _view(v, N)
    # last axis = qubits[0] (least significant local bit), ...
    src = [_axis(N, q) for q in reversed(qubits)]
    dst = list(range(N - k, N))
    Tm = np.moveaxis(T, src, dst)
    shape = Tm.shape
    M = Tm.reshape(-1, 1 << k)
    M2 = M @ U.T
    T[...] = np.moveaxis(M2.reshape(shape), dst, src)
    return v


def apply_permutation(v, N, controls, reg_lo, reg_w, table):
    """Controlled register permutation, in place: on every basis index whose
    control bits are all 1, the value f of the register (bits reg_lo ..
    reg_lo+reg_w-1) is replaced by table[f].  ``table`` must be a bijection of
    [0, 2^reg_w).

    Used for the controlled modular multiplication f -> a*f mod G that
    computes f(x) = y^x mod G "conditional on the qubits in the x-register"
    (Sec. 5.4 and the SHORBOX entry of Appendix A).
    """
    table = np.asarray(table, dtype=np.int64)
    if table.shape != (1 << reg_w,) or not np.array_equal(np.sort(table), np.arange(1 << reg_w)):
        raise ValueError("table is not a bijection on the register")
    i = np.arange(1 << N, dtype=np.int64)
    on = np.ones(i.shape, dtype=bool)
    for c in controls:
        on &= ((i >> c) & 1) == 1
    mask = ((1 << reg_w) - 1) << reg_lo
    f = (i >> reg_lo) & ((1 << reg_w) - 1)
    j = np.where(on, (i & ~mask) | (table[f] << reg_lo), i)
    out = np.empty_like(v)
    out[j] = v[i]
    v[...] = out
    return v


def modmul_table(a, G, width):
    """Table of f -> a*f mod G for f < G, identity for G <= f < 2^width."""
    f = np.arange(1 << width, dtype=np.int64)
    return np.where(f < G, (a * f) % G, f)


def shorbox(N, nx, G, y):
    """SHORBOX n_x G y (Appendix A; Sec. 5.4): the state
    2^{-n_x/2} sum_{x=0}^{2^{n_x}-1} |x> |y^x mod G>, with the x-register on
    qubits 0..n_x-1 and f(x) = y^x mod G on qubits n_x..N-1."""
    if not (0 < nx < N) or G >= (1 << (N - nx)):
        raise ValueError("bad SHORBOX arguments")
    v = np.zeros(1 << N, dtype=np.complex128)
    amp = 2.0 ** (-nx / 2.0)
    f = 1 % G
    for x in range(1 << nx):
        v[x + (f << nx)] = amp
        f = (f * y) % G
    return v


def project(v, N, q, bit):
    """CLEAR (bit=0) / SET (bit=1) of Appendix A: apply |b><b| on qubit q and
    renormalise; fails (ValueError) when the projected state has zero norm."""
    T = _view(v, N)
    sel = [slice(None)] * N
    sel[_axis(N, q)] = 1 - bit
    T[tuple(sel)] = 0
    nrm = norm(v)
    if nrm == 0.0:
        raise ValueError("projection gives a zero state")
    v /= math.sqrt(nrm)
    return v


# --------------------------------------------------------------------------
# reductions (compensated FP64)
# --------------------------------------------------------------------------
def csum(x):
    """Compensated sum of a 1-D float64 array: the correctly rounded sum for
    small arrays (math.fsum), else a Neumaier sum down the rows of a 2-D
    reshaping (vectorised across columns) whose running sums and
    compensation terms are then added exactly (fsum of both, so a large
    column total that cancels against another keeps its compensation)."""
    x = np.asarray(x, dtype=np.float64).ravel()
    if x.size <= (1 << 20):
        return math.fsum(x.tolist())
    rows = 1 << 10
    cols = x.size // rows
    M = x[: rows * cols].reshape(rows, cols)
    s = np.zeros(cols)
    c = np.zeros(cols)
    for r in range(rows):
        t = s + M[r]
        big = np.abs(s) >= np.abs(M[r])
        c += np.where(big, (s - t) + M[r], (M[r] - t) + s)
        s = t
    return math.fsum(s.tolist() + c.tolist() + x[rows * cols:].tolist())


def csum_rows(M):
    """Neumaier sum of a 2-D array down axis 0 (one compensated sum per column)."""
    M = np.asarray(M, dtype=np.float64)
    s = np.zeros(M.shape[1:])
    c = np.zeros(M.shape[1:])
    for r in range(M.shape[0]):
        t = s + M[r]
        big = np.abs(s) >= np.abs(M[r])
        c += np.where(big, (s - t) + M[r], (M[r] - t) + s)
        s = t
    return s + c


def probabilities(v):
    """|a_i|^2 for every basis state."""
    return v.real * v.real + v.imag * v.imag


def norm(v):
    """<Phi|Phi> = sum_i |a_i|^2 (Eq. (STAT1); the bound 2^L there reads 2^N)."""
    return csum(probabilities(v))


def prob_one(v, N, q):
    """Probability that measuring qubit q gives 1: sum over |a(*1_q*)|^2 (Sec. 2)."""
    T = _view(probabilities(v), N)
    sel = [slice(None)] * N
    sel[_axis(N, q)] = 1
    return csum(T[tuple(sel)])


def pair_overlap(v, N, q):
    """w_q = sum over indices with bit q = 0 of conj(a(*0_q*)) * a(*1_q*)."""
    T = _view(v, N)
    s0 = [slice(None)] * N
    s1 = [slice(None)] * N
    s0[_axis(N, q)] = 0
    s1[_axis(N, q)] = 1
    prod = np.conj(T[tuple(s0)]) * T[tuple(s1)]
    return complex(csum(prod.real), csum(prod.imag))


def expect_xyz(v, N):
    """BEGIN MEASUREMENT (Appendix A): for every qubit n,
    <Qx(n)> = <Psi|(1 - sigma^x_n)|Psi>/2, and likewise for y and z.

    With w_n = sum conj(a(*0_n*)) a(*1_n*):  <sigma^x_n> = 2 Re w_n,
    <sigma^y_n> = 2 Im w_n, <sigma^z_n> = P0 - P1 and <1> = <Psi|Psi>, so
    Qx = <Psi|Psi>/2 - Re w_n, Qy = <Psi|Psi>/2 - Im w_n and
    Qz = (<Psi|Psi> - P0 + P1)/2 = P1.
    """
    nrm = norm(v)
    qx = np.empty(N)
    qy = np.empty(N)
    qz = np.empty(N)
    for n in range(N):
        w = pair_overlap(v, N, n)
        qx[n] = 0.5 * nrm - w.real
        qy[n] = 0.5 * nrm - w.imag
        qz[n] = prob_one(v, N, n)
    return qx, qy, qz


def marginal(v, N, qubits):
    """Probability of each value k of the qubits ``qubits`` (bit m of k is the
    value of qubits[m]): P(k) = sum over the other bits of |a|^2 (Sec. 2)."""
    k = len(qubits)
    T = _view(probabilities(v), N)
    src = [_axis(N, q) for q in reversed(qubits)]
    dst = list(range(N - k, N))
    M = np.moveaxis(T, src, dst).reshape(-1, 1 << k)
    return csum_rows(M)
