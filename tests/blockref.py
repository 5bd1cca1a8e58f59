"""Reference values of a tensor product of small blocks of qubits, from the
oracle run on each block alone: a circuit whose gates never cross blocks
leaves the state prod_b |psi_b>, so an amplitude is the product of the
blocks' amplitudes at the index's bits, a qubit's BEGIN MEASUREMENT values are
those of its block, and a register marginal is the product of the blocks'
marginals.  Used for parity at sizes where the whole oracle state is too
large to form; pinned against the full oracle in test_blockref.py."""
import numpy as np

from oracle import circuit, statevec as sv


def block_states(blocks, recs):
    """The oracle's state of every block (its qubits renumbered 0..m-1 in
    the block's order) after the records that act on it."""
    states = []
    for b in blocks:
        loc = {qq: p for p, qq in enumerate(b)}
        mine = [r for r in recs if r[1][0] in loc]
        if not all(all(x in loc for x in r[1]) for r in mine):
            raise ValueError("a gate crosses blocks")
        lrecs = [(r[0], tuple(loc[x] for x in r[1]), r[2]) for r in mine]
        states.append(circuit.run(sv.zero_state(len(b)), len(b), lrecs))
    return states


def sample_indices(N, seed):
    g = np.random.default_rng(seed)
    full = (1 << N) - 1
    one_hot = [1 << k for k in range(N)]
    idx = np.concatenate([g.integers(0, 1 << N, 1 << 20, dtype=np.int64),
                          np.array([0, full] + one_hot + [full ^ x for x in one_hot], dtype=np.int64)])
    return idx


def block_amplitudes(blocks, states, idx):
    amp = np.ones(idx.shape, dtype=np.complex128)
    for b, v in zip(blocks, states):
        loc = np.zeros(idx.shape, dtype=np.int64)
        for p, qq in enumerate(b):
            loc |= ((idx >> qq) & 1) << p
        amp *= v[loc]
    return amp


def block_expectations(blocks, states, N):
    qx, qy, qz = np.empty(N), np.empty(N), np.empty(N)
    for b, v in zip(blocks, states):
        x, y, z = sv.expect_xyz(v, len(b))
        for p, qq in enumerate(b):
            qx[qq], qy[qq], qz[qq] = x[p], y[p], z[p]
    return qx, qy, qz


def block_marginal(blocks, states, qubits):
    """P(k) of the register `qubits` (bit m of k = qubits[m]) of the product
    state: the product of each block's marginal of its share of the register."""
    P = np.ones(1 << len(qubits))
    k = np.arange(1 << len(qubits))
    for b, v in zip(blocks, states):
        mine = [m for m, qq in enumerate(qubits) if qq in b]
        if not mine:
            continue
        marg = sv.marginal(v, len(b), [b.index(qubits[m]) for m in mine])
        loc = np.zeros_like(k)
        for j, m in enumerate(mine):
            loc |= ((k >> m) & 1) << j
        P *= marg[loc]
    return P
