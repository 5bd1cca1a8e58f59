"""Host-side checks of the tile passes compiled at run time (no GPU work):
the planner's passes of a circuit compile for sm_103a with NVRTC, compiled
structures are cached, and bad arguments are rejected before compiling."""
import pytest

from paper_1805_04708_gb300 import workloads as wl


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    if not qsim.tile_compiler_info()[0]:
        pytest.skip("NVRTC cannot be loaded on this machine")
    return qsim


def after_product_start(recs):
    """The gates a run from |0..0> keeps in its passes: every single-qubit
    gate before the first multi-qubit gate on its qubit goes into the
    product start."""
    entangled, rest = set(), []
    for r in recs:
        qs = r[1]
        if len(qs) == 1 and qs[0] not in entangled:
            continue
        if len(qs) > 1:
            entangled.update(qs)
        rest.append(r)
    return rest


def test_circuit_compiles_and_is_cached(q):
    recs = wl.random_mixed_circuit(16, 60, seed=3)
    _, before = q.tile_compiler_info()
    npass = q.circuit_compile(16, recs, mode=3)
    _, after = q.tile_compiler_info()
    assert npass >= 2
    # the passes of the circuit and of its runs from |0..0>
    rest = after_product_start(recs)
    assert len(rest) < len(recs)
    npass_z = len(q.circuit_plan(16, rest, "c64"))
    assert 1 <= after - before <= npass + npass_z
    # the same structures again: nothing new to compile
    assert q.circuit_compile(16, recs, mode=3) == npass
    assert q.tile_compiler_info()[1] == after


def test_mode2_compiles_every_candidate(q):
    # mode 3 compiles one kernel per structure; mode 2 adds the two variants
    # with CTA barriers (the variant without barriers is shared)
    recs = wl.random_gate_circuit(22, 120, seed=5)
    _, c0 = q.tile_compiler_info()
    n3 = q.circuit_compile(22, recs, mode=3)
    _, c1 = q.tile_compiler_info()
    n2 = q.circuit_compile(22, recs, mode=2)
    _, c2 = q.tile_compiler_info()
    assert n2 == n3
    npass_z = len(q.circuit_plan(22, after_product_start(recs), "c64"))
    assert 1 <= c1 - c0 <= n3 + npass_z
    assert c2 - c1 == 2 * (c1 - c0)


def test_compile_rejects(q):
    recs = [("H", (0,), ())]
    with pytest.raises(q.QSError):
        q.circuit_compile(16, recs, mode=1)
    with pytest.raises(q.QSError):
        q.circuit_compile(8, recs, mode=3)           # below the tile size
    with pytest.raises(q.QSError):
        q.circuit_compile(16, [("H", (16,), ())], mode=3)
