"""measure_probs_static: the register marginal for callers that cannot
allocate device memory (a framework's pool owns it, or a loop must not enter
the allocator).  It must agree with measure_probs, call after call, while
using only the library's fixed scratch array.  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


@pytest.mark.parametrize("enc", ["c128", "c64"])
def test_static_matches_measure_probs(q, enc):
    N = 18
    with q.Sim(N, enc) as s:
        s.copy_in(rand_state(N, 11))
        for qubits in ([0, 5, 17], [17, 3], list(range(16)), [9]):
            ref = s.measure_probs(qubits)
            for _ in range(2):   # two calls in a row share the scratch
                got = q.measure_probs_static(s.device_ptr(), N, enc, qubits, stream=s.stream_handle)
                assert np.max(np.abs(got - ref)) <= 1e-13


def test_static_many_complement_indices_per_thread(q):
    # N = 22: the complement of a small register has more indices than the
    # fixed 2^18 partial sums, so every partial covers several of them
    N = 22
    with q.Sim(N, "c64") as s:
        s.copy_in(rand_state(N, 12))
        for qubits in ([7], [21], list(range(16)), list(range(6, 22)), [0, 11, 21]):
            ref = s.measure_probs(qubits)
            for _ in range(2):
                got = q.measure_probs_static(s.device_ptr(), N, "c64", qubits, stream=s.stream_handle)
                assert np.max(np.abs(got - ref)) <= 1e-13


def test_static_rejects_beyond_limit(q):
    N = 18
    with q.Sim(N, "c64") as s:
        with pytest.raises(q.QSError) as e:
            q.measure_probs_static(s.device_ptr(), N, "c64", list(range(17)), stream=s.stream_handle)
        assert e.value.name == "QS_EINVAL"
    with q.Sim(12, "adapt2") as s:
        with pytest.raises(q.QSError) as e:
            q.measure_probs_static(s.device_ptr(), 12, "adapt2", [0], stream=s.stream_handle)
        assert e.value.name == "QS_EUNSUPPORTED"
