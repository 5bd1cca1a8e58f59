"""The bounded-wait exits of the tensor-core fused gate (tcgen05 pipeline)
and of the complex64 BEGIN MEASUREMENT kernel (TMA ring), made to run out on
purpose through the test-only pipeline wait limit: limit 0 gives up at the
first test of every wait (nothing in flight), a few microseconds gives up
while tensor loads are in flight (the exit waits for them).  Each call must
return QS_ETIMEOUT (or, for the racy limit, finish correctly), and the next
call with the normal limit must be oracle-correct."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import statevec as sv  # noqa: E402


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    yield qsim
    qsim.set_pipeline_wait_limit(-1)


def rand_state(N, seed):
    g = np.random.default_rng(seed)
    v = g.standard_normal(1 << N) + 1j * g.standard_normal(1 << N)
    return v / np.linalg.norm(v)


def haar(n, seed):
    g = np.random.default_rng(seed)
    Z = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


@pytest.mark.parametrize("limit", [0, 3])
def test_fused_tcgen05_wait_runs_out(q, limit):
    N = 16
    v0 = rand_state(N, 1)
    U = haar(32, 2)
    ref = v0.astype(np.complex64).astype(np.complex128)
    sv.apply_dense(ref, N, [0, 1, 2, 3, 4], U)
    with q.Sim(N, "c64") as s:
        s.copy_in(v0)
        q.set_pipeline_wait_limit(limit)
        try:
            s.apply_fused([0, 1, 2, 3, 4], U)
            timed_out = False
        except q.QSError as e:
            assert e.name == "QS_ETIMEOUT"
            timed_out = True
        finally:
            q.set_pipeline_wait_limit(-1)
        if limit == 0:
            assert timed_out
        if not timed_out:
            assert np.max(np.abs(s.copy_out() - ref)) <= 4e-5
        # the state is undefined after a timeout: start again with the normal limit
        s.copy_in(v0)
        s.apply_fused([0, 1, 2, 3, 4], U)
        assert np.max(np.abs(s.copy_out() - ref)) <= 4e-5


@pytest.mark.parametrize("limit", [0, 3])
def test_expect_tma_wait_runs_out(q, limit):
    N = 24
    v0 = rand_state(N, 3)
    stored = v0.astype(np.complex64).astype(np.complex128)
    rx, ry, rz = sv.expect_xyz(stored, N)
    with q.Sim(N, "c64") as s:
        s.copy_in(v0)
        q.set_pipeline_wait_limit(limit)
        try:
            out = s.expect_xyz()
            timed_out = False
        except q.QSError as e:
            assert e.name == "QS_ETIMEOUT"
            timed_out = True
        finally:
            q.set_pipeline_wait_limit(-1)
        if limit == 0:
            assert timed_out
        if not timed_out:
            for a, b in zip(out, (rx, ry, rz)):
                assert np.max(np.abs(a - b)) <= 1e-6
        # BEGIN MEASUREMENT leaves the state unchanged, timeout or not
        assert np.array_equal(s.copy_out(), v0.astype(np.complex64))
        qx, qy, qz = s.expect_xyz()
        for a, b in zip((qx, qy, qz), (rx, ry, rz)):
            assert np.max(np.abs(a - b)) <= 1e-6
