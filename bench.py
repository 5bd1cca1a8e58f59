"""Benchmark: gate-amplitude updates/s of the random-gate workload at N = 30.

Workload (one step): a 30-qubit complex64 state (8 GiB, larger than L2, so no
L2 flush is needed between steps) is reset to |0..0>, an all-Hadamard layer
and 200 seeded random gates from {H, T, RZ(theta), CNOT, TOFFOLI} on qubits
0..29 are applied through the native tile-pass planner, then the FP64
compensated norm and BEGIN MEASUREMENT (<Qx>, <Qy>, <Qz> of every qubit) are
computed.  Gate-amplitude updates = (logical gates) x 2^N per step.

The same line reports, measured in the same run: the per-gate sweep path, the
complex128 state (16 GiB), the HBM roofline of the dominant kernel (the
complex64 tile pass), the end-to-end number through the public API with host
buffers, the SM clocks seen during the timed region, and the oracle timed on
the host cores on a bounded sample (cpu_baseline).

Multi-GPU (torchrun, one process per GPU): replicas only -- every rank runs
the same workload on its own GPU, no collective on the data path; value is
the sum over ranks divided by the slowest rank's time ("scaling": "weak").

--impl reference times the oracle (the plain complex128 CPU simulator) on the
host cores instead, on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_QUBITS = 30
N_GATES = 200
SEED = 1
METRIC = "gate-amplitude updates/s"
UNIT = "updates/s"
# algorithmic bytes of one tile pass: read + write of the whole state
# (2 * 2^N * 8 B for complex64)
TILE_TRAFFIC_PER_PASS = None  # dram bytes per tile-pass launch from ncu; None until captured for this kernel


def workload_records(N=N_QUBITS, ngates=N_GATES, seed=SEED):
    from paper_1805_04708_gb300 import workloads as wl
    return wl.random_gate_circuit(N, ngates, seed)


def config_dict(N, enc):
    return {
        "workload": "random-gate circuit N=%d: %d H + %d gates from {H,T,RZ,CNOT,TOFFOLI}, seed %d, "
                    "%s state + FP64 norm and <Qx,Qy,Qz>" % (N, N, N_GATES, SEED, enc),
        "N": N, "encoding": enc, "gates_per_step": N + N_GATES,
        "state_bytes": (8 if enc == "c64" else 16) << N,
        "l2": "inputs larger than L2 (no flush)",
        "path": "tile-pass planner (circuit_run mode 1)",
    }


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
CPU_SAMPLE_N = 20


def oracle_step(N=CPU_SAMPLE_N):
    from oracle import circuit, statevec as sv
    recs = workload_records(N)
    t0 = time.perf_counter()
    v = circuit.run(sv.zero_state(N), N, recs)
    sv.norm(v)
    sv.expect_xyz(v, N)
    dt = time.perf_counter() - t0
    return len(recs) * float(1 << N) / dt, dt


def cpu_baseline(budget_s=20.0):
    vals, spent = [], 0.0
    while spent < budget_s:
        v, dt = oracle_step()
        vals.append(v)
        spent += dt
        if len(vals) >= 3 and spent > budget_s / 2:
            break
    return {"value": statistics.median(vals), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "same circuit family at N=%d (%d H + %d gates) + norm + <Qx,Qy,Qz>, "
                      "numpy complex128, %d runs, median" % (CPU_SAMPLE_N, CPU_SAMPLE_N, N_GATES, len(vals))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_step()
    vals, tot = [], 0.0
    for _ in range(args.steps):
        v, dt = oracle_step()
        vals.append(v)
        tot += dt
    value = sum(vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)",
        "data": "synthetic", "config": config_dict(N_QUBITS, "c64"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "each step: the circuit family at N=%d (%d H + %d gates) + norm + "
                                   "<Qx,Qy,Qz> on numpy complex128" % (CPU_SAMPLE_N, CPU_SAMPLE_N, N_GATES)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    from paper_1805_04708_gb300 import build
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1805_04708_gb300 import qsim

    N = N_QUBITS
    recs = workload_records(N)
    gates = qsim.gate_array(recs)
    ngates = len(recs)
    upd_per_step = ngates * float(1 << N)
    stream = torch.cuda.current_stream()
    sim = qsim.Sim(N, "c64", stream=stream)

    def step(timed_passes=None):
        sim.reset()
        ms = sim.circuit_run_timed(gates, mode=1)
        if timed_passes is not None:
            timed_passes.extend(ms)
        sim.norm()
        sim.expect_xyz()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    pass_ms = []
    launches0 = qsim.kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(pass_ms)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launches = qsim.kernel_launches() - launches0
    clocks = sampler.stop()
    if world > 1:
        t = torch.tensor([elapsed_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = float(t.item())

    value = world * upd_per_step * args.steps / (elapsed_ms / 1e3)
    ms_per_step = elapsed_ms / args.steps

    # roofline of the dominant kernel: the complex64 tile pass
    peak, peak_kind = load_peaks()
    alg_bytes = 2.0 * (8 << N)
    mean_pass = sum(pass_ms) / len(pass_ms)
    achieved = alg_bytes / (mean_pass / 1e3) / 1e9
    passes_per_step = len(pass_ms) // args.steps
    roofline = {"kernel": "k_tile<float,float2> (complex64 tile pass)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "traffic": TILE_TRAFFIC_PER_PASS, "algorithmic_bytes_per_launch": alg_bytes,
                "mean_launch_ms": mean_pass, "launches_per_step": passes_per_step,
                "share_of_step": sum(pass_ms) / elapsed_ms}

    # end to end through the public API: gate records from host memory each
    # step, results (norm, 3N expectation values) read back to the host
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.reset()
        sim.circuit_run(recs, mode=1)
        sim.norm()
        sim.expect_xyz()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": world * upd_per_step / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": ngates * qsim.ctypes.sizeof(qsim.qs_gate),
           "d2h_bytes_per_step": 8 * (3 * N + 1)}

    # variants measured in the same run (one step each)
    variants = {}
    if not args.no_variants:
        def timed(fn):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b)

        def per_gate_c64():
            sim.reset()
            sim.circuit_run(gates, mode=0)
        ms = timed(per_gate_c64)
        variants["c64_per_gate_sweeps"] = {"value": upd_per_step / (ms / 1e3), "ms_per_circuit": ms}
        sim.close()
        del sim
        torch.cuda.empty_cache()
        s128 = qsim.Sim(N, "c128", stream=stream)
        for mode, key in ((1, "c128_tile_passes"), (0, "c128_per_gate_sweeps")):
            def run128(mode=mode):
                s128.reset()
                s128.circuit_run(gates, mode=mode)
            run128()
            ms = timed(run128)
            variants[key] = {"value": upd_per_step / (ms / 1e3), "ms_per_circuit": ms}
        s128.close()
    else:
        sim.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32 arithmetic, f64 reductions)",
        "data": "synthetic", "config": dict(config_dict(N, "c64"), parallelism="replicas" if world > 1 else "single"),
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "variants": variants,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
