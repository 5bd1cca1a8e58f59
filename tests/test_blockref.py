"""The block-product reference (tests/blockref.py) against the whole oracle
state at N = 9 and 10: amplitudes, BEGIN MEASUREMENT values and register
marginals of a circuit whose gates stay inside blocks of three qubits."""
import numpy as np
import pytest

from blockref import block_amplitudes, block_expectations, block_marginal, block_states
from oracle import circuit, statevec as sv
from paper_1805_04708_gb300 import workloads as wl


@pytest.mark.parametrize("N,seed", [(9, 3), (10, 4)])
def test_block_reference_equals_oracle(N, seed):
    blocks = wl.block_partition(N, 3, seed=seed)
    recs = wl.block_gate_circuit(blocks, 80, seed=seed + 1)
    states = block_states(blocks, recs)
    full = circuit.run(sv.zero_state(N), N, recs)
    assert np.max(np.abs(block_amplitudes(blocks, states, np.arange(1 << N)) - full)) < 1e-14
    for a, b in zip(block_expectations(blocks, states, N), sv.expect_xyz(full, N)):
        assert np.max(np.abs(a - b)) < 1e-13
    for reg in ([blocks[0][1], blocks[1][0], blocks[2][2]], list(range(3, N)), list(blocks[1])):
        assert np.max(np.abs(block_marginal(blocks, states, reg) - sv.marginal(full, N, reg))) < 1e-14


def test_block_reference_rejects_crossing_gates():
    blocks = [[0, 1], [2, 3]]
    with pytest.raises(ValueError):
        block_states(blocks, [("CNOT", (1, 2), ())])
