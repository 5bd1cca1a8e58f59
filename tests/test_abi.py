"""Host-side checks of the C-ABI library (no GPU work): it builds for sm_103a,
loads, and exports every function include/qsim.h declares; the binding knows
each of them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_04708_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared_functions()
    assert "sim_create" in names and "apply_gate" in names and "sim_norm" in names
    assert len(names) >= 20


def test_every_declared_symbol_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header(lib):
    from paper_1805_04708_gb300 import qsim
    missing = set(declared_functions()) - set(qsim.EXPORTED)
    assert not missing, missing


def test_host_only_calls(lib):
    # calls that need no device: version, the gate table, modmul tables,
    # argument rejection before any CUDA work
    from paper_1805_04708_gb300 import qsim
    assert "sm_103a" in qsim.version()
    g = qsim.gate_std("TOFFOLI", (3, 4, 0))
    assert g.nc == 2 and list(g.controls) == [3, 4] and g.target == 0
    assert list(g.u) == [0, 0, 1, 0, 1, 0, 0, 0]
    h = qsim.gate_std("H", (5,))
    assert h.nc == 0 and abs(h.u[0] - 2 ** -0.5) < 2.3e-16 and h.u[6] == -h.u[0]
    with pytest.raises(qsim.QSError):
        qsim.gate_std("NOPE", (0,))
    with pytest.raises(qsim.QSError):
        qsim.gate_std("CNOT", (0,))
    t = qsim.modmul_table(7, 15, 4)
    assert sorted(t.tolist()) == list(range(16))
    assert [int(t[f]) for f in range(15)] == [(7 * f) % 15 for f in range(15)]
    with pytest.raises(qsim.QSError):
        qsim.modmul_table(5, 15, 4)  # not coprime
    out = ctypes.c_void_p()
    assert lib.sim_create(1, 0, None, ctypes.byref(out)) == 1  # QS_EINVAL: N must be > 1
    assert lib.sim_create(64, 0, None, ctypes.byref(out)) == 1


def test_gate_table_matches_oracle_matrices():
    # the library's instruction-set table and the oracle's are typed
    # independently; they must agree entry by entry
    import numpy as np
    from paper_1805_04708_gb300 import qsim
    from oracle import gates
    cases = [("H", ()), ("X", ()), ("Y", ()), ("Z", ()), ("S", ()), ("S+", ()), ("T", ()), ("T+", ()),
             ("+X", ()), ("-X", ()), ("+Y", ()), ("-Y", ()), ("U1", (0.7,)), ("U2", (0.3, -1.1)),
             ("U3", (1.9, 0.2, 2.5)), ("R", (0,)), ("R", (1,)), ("R", (2,)), ("R", (3,)), ("R", (9,)),
             ("R", (-4,)), ("RZ", (1.234,)), ("I", ())]
    for name, p in cases:
        g = qsim.gate_std(name, (0,), p)
        U = np.array(g.u[0::2]) + 1j * np.array(g.u[1::2])
        ref = gates.one_qubit(name, p).ravel()
        assert np.max(np.abs(U - ref)) < 1e-15, name
    for k in (0, 1, 2, 3, 5, -3, -8):
        g = qsim.gate_std("U", (1, 0), (k,))
        U = np.array(g.u[0::2]) + 1j * np.array(g.u[1::2])
        assert np.max(np.abs(U - gates.controlled_phase(k).ravel())) < 1e-15
