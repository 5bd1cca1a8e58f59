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


@pytest.mark.parametrize("persistent", [False, True])
def test_serve_mixed_equals_alone(q, persistent):
    reqs = stream(40, 3, 4, 18, 2, 6, rate=4000.0)
    budget = 12 << 20          # room for a few 2 MiB (N = 18) states at a time
    res, st = q.serve(reqs, budget, quantum=16, nstreams=3, persistent=persistent, persistent_ctas=8)
    assert st["completed"] == len(reqs)
    if persistent:
        nsmall = sum(1 for r in reqs if r["N"] <= 14)
        assert st["work_items"] >= nsmall and st["relaunches"] >= 1
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


def test_persistent_bounded_waits_run_out(q):
    # sparse arrivals and a 2 ms device wait: the persistent CTAs run out of
    # work between requests, end their bounded waits (counted), and the host
    # launches the kernel again for the next request; every result still
    # equals the circuit run alone
    reqs = stream(6, 5, 6, 12, 3, 5, rate=20.0)      # about 50 ms apart
    res, st = q.serve(reqs, 64 << 20, quantum=8, persistent=True, persistent_ctas=4, device_wait_ms=2.0)
    assert st["completed"] == len(reqs)
    assert st["idle_exits"] >= 4 and st["relaunches"] >= 2
    for r, out in zip(reqs, res):
        v = circuit.run(sv.zero_state(r["N"]), r["N"], r["records"])
        _, _, rz = sv.expect_xyz(v, r["N"])
        assert np.max(np.abs(out["qz"] - rz)) <= 1e-5
        assert abs(out["norm"] - 1.0) <= 1e-5


def test_persistent_large_and_small_overlap(q):
    # states of 8..22 qubits together: small ones in the persistent kernel,
    # larger ones in chunks on their own streams, all against running alone
    reqs = stream(24, 9, 8, 22, 2, 4, rate=2000.0)
    res, st = q.serve(reqs, 1 << 30, quantum=12, large_quantum=20, persistent=True, nstreams=4)
    assert st["completed"] == len(reqs) and st["max_active"] > 1
    for r, out in zip(reqs, res):
        with q.Sim(r["N"], "c64") as s:
            s.circuit_run(r["records"], mode=1)
            _, _, qz = s.expect_xyz()
        assert np.max(np.abs(out["qz"] - qz)) <= 1e-5
