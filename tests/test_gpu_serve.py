"""The serving loop: continuous batching of requests with mixed qubit counts.
Each request's result in the mix equals the same circuit run alone (within
the complex64 tolerance), requests overlap on the device, admission respects
the memory budget, and the small-state path agrees with the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import circuit, statevec as sv  # noqa: E402
from paper_1805_04708_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def q():
    from paper_1805_04708_gb300 import build
    build.build()
    from paper_1805_04708_gb300 import qsim
    torch.cuda.set_device(0)
    return qsim


def stream(n, seed, nmin, nmax, dmin, dmax, rate):
    reqs = wl.serving_stream(n, rate, seed, nmin=nmin, nmax=nmax, dmin=dmin, dmax=dmax)
    for r in reqs:
        r["records"] = wl.layered_circuit(r["N"], r["depth"], r["seed"])
    return reqs


def test_serve_mixed_equals_alone(q):
    reqs = stream(40, 3, 4, 18, 2, 6, rate=4000.0)
    budget = 12 << 20          # room for a few 2 MiB (N = 18) states at a time
    res, st = q.serve(reqs, budget, quantum=16, nstreams=3)
    assert st["completed"] == len(reqs)
    assert st["max_active"] > 1                    # requests were in flight together
    assert st["peak_bytes"] <= budget
    for r, out in zip(reqs, res):
        assert out["admit_s"] >= r["arrival"] - 1e-9
        assert out["finish_s"] >= out["admit_s"]
        with q.Sim(r["N"], "c64") as s:
            s.circuit_run(r["records"], mode=1)
            _, _, qz = s.expect_xyz()
            nrm = s.norm()
        assert np.max(np.abs(out["qz"] - qz)) <= 1e-5
        assert abs(out["norm"] - nrm) <= 1e-5
    # and against the oracle for the small ones
    for r, out in list(zip(reqs, res))[:10]:
        if r["N"] > 12:
            continue
        v = circuit.run(sv.zero_state(r["N"]), r["N"], r["records"])
        _, _, rz = sv.expect_xyz(v, r["N"])
        assert np.max(np.abs(out["qz"] - rz)) <= 1e-5


def test_serve_rejects(q):
    reqs = stream(2, 1, 10, 10, 1, 1, rate=10.0)
    with pytest.raises(q.QSError) as e:
        q.serve(reqs, 1 << 10)
    assert e.value.name == "QS_ENOMEM"
    bad = [dict(arrival=0.0, N=5, records=[("H", (7,), ())])]
    with pytest.raises(q.QSError):
        q.serve(bad, 1 << 20)
