"""Runs a program in the instruction language of Appendix A on the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A program is text, one instruction per line; '!' starts a comment and case
does not matter.  Instructions: QUBITS N (first), BIT ASSIGNMENT p_0 ..
p_{N-1}, the gate mnemonics with their qubits then their numeric arguments
(H n, U1 n lambda, U2 n phi lambda, U3 n theta phi lambda, R n k, CNOT c t,
U c t k, TOFFOLI c1 c2 t, ...), BEGIN MEASUREMENT, M n, CLEAR n, SET n,
SHORBOX n_x G y, DEPOLARIZING CHANNEL P_X = p, P_Y = p, P_Z = p, SEED = k
(any order, any subset, commas optional), GENERATE EVENTS events seed, EXIT.

Readings (where Appendix A leaves a choice open):
  * BIT ASSIGNMENT only renumbers where qubits are stored; the circuit is
    unchanged (Appendix A), so every result here is per logical qubit and the
    oracle ignores it after checking that it is a permutation;
  * a seed <= 0 means "the system's value" in the paper; here it is replaced
    by the run's seed, so that runs repeat: M number m draws
    uniform(run_seed, m), GENERATE EVENTS draws uniform(s, k) for event k with
    s = seed if seed > 0 else run_seed + 1, and the depolarizing channel draws
    uniform(s, g N + q) for gate operation g and qubit q with s = SEED if
    SEED > 0 else run_seed + 2 (uniform: SplitMix64, oracle/measure.py);
  * the depolarizing channel acts after every gate instruction that follows
    it (not after M, CLEAR, SET, SHORBOX or a measurement);
  * EXIT and GENERATE EVENTS end the run; EXIT records one BEGIN MEASUREMENT
    ("measure all qubits").
"""
import re

import numpy as np

from . import circuit, gates as og, measure as om, statevec as sv
from .adapt2 import AState, encode, retune

GATES_1Q = {"I", "H", "X", "Y", "Z", "S", "S+", "T", "T+", "U1", "U2", "U3", "+X", "-X", "+Y", "-Y", "R", "RZ"}
NPARAM = {"U1": 1, "U2": 2, "U3": 3, "R": 1, "RZ": 1, "U": 1}
NQUBIT = {"CNOT": 2, "U": 2, "TOFFOLI": 3}


def _num(tok):
    return float(tok) if any(c in tok for c in ".eE") else int(tok)


def parse(text):
    """List of (name, args) in program order; raises ValueError on bad input."""
    prog = []
    N = None
    for lineno, raw in enumerate(text.splitlines(), 1):
        line = raw.split("!", 1)[0].strip()
        if not line:
            continue
        up = line.upper()
        toks = up.split()
        try:
            if toks[0] == "QUBITS":
                if N is not None or prog:
                    raise ValueError("QUBITS must come first, once")
                N = int(toks[1])
                if not 1 < N < 64:
                    raise ValueError("N out of range")
                prog.append(("QUBITS", (N,)))
                continue
            if N is None:
                raise ValueError("QUBITS must come first")
            if up.startswith("BIT ASSIGNMENT"):
                perm = [int(x) for x in toks[2:]]
                if sorted(perm) != list(range(N)):
                    raise ValueError("BIT ASSIGNMENT is not a permutation of 0..N-1")
                prog.append(("BIT ASSIGNMENT", tuple(perm)))
            elif up.startswith("BEGIN MEASUREMENT"):
                prog.append(("BEGIN MEASUREMENT", ()))
            elif up.startswith("GENERATE EVENTS"):
                nev = int(toks[2])
                if not 1 <= nev <= 2 ** 31:
                    raise ValueError("events out of range")
                prog.append(("GENERATE EVENTS", (nev, int(toks[3]) if len(toks) > 3 else 0)))
            elif up.startswith("DEPOLARIZING CHANNEL"):
                kv = dict(P_X=0.0, P_Y=0.0, P_Z=0.0, SEED=0)
                for key, val in re.findall(r"(P_X|P_Y|P_Z|SEED)\s*=\s*([-+0-9.eE]+)", up):
                    kv[key] = _num(val)
                px, py, pz = float(kv["P_X"]), float(kv["P_Y"]), float(kv["P_Z"])
                if min(px, py, pz) < 0 or px + py + pz > 1:
                    raise ValueError("depolarizing probabilities out of range")
                prog.append(("DEPOLARIZING CHANNEL", (px, py, pz, int(kv["SEED"]))))
            elif toks[0] in ("M", "CLEAR", "SET"):
                q = int(toks[1])
                if not 0 <= q < N:
                    raise ValueError("qubit out of range")
                prog.append((toks[0], (q,)))
            elif toks[0] == "SHORBOX":
                nx, G, y = int(toks[1]), int(toks[2]), int(toks[3])
                if not (1 <= nx < N and G >= 2 and 1 <= y < G and G <= 2 ** (N - nx)):
                    raise ValueError("SHORBOX arguments out of range")
                prog.append(("SHORBOX", (nx, G, y)))
            elif toks[0] == "EXIT":
                prog.append(("EXIT", ()))
            elif toks[0] in GATES_1Q or toks[0] in NQUBIT:
                nq = NQUBIT.get(toks[0], 1)
                qs = tuple(int(x) for x in toks[1:1 + nq])
                ps = tuple(_num(x) for x in toks[1 + nq:])
                if len(qs) != nq or len(ps) != NPARAM.get(toks[0], 0):
                    raise ValueError("wrong operand count")
                if len(set(qs)) != nq or min(qs) < 0 or max(qs) >= N:
                    raise ValueError("qubits out of range or repeated")
                prog.append(("GATE", (toks[0], qs, ps)))
            else:
                raise ValueError("unknown instruction")
        except (IndexError, ValueError) as e:
            raise ValueError("line %d: %s (%s)" % (lineno, raw.strip(), e))
    if N is None:
        raise ValueError("no QUBITS instruction")
    return prog


def run(text, run_seed=1, enc="c128"):
    """Execute a program; returns a dict with N and the list `out` of results
    in order: ("BEGIN MEASUREMENT", qx, qy, qz), ("M", q, outcome, p0, p1),
    ("CLEAR" / "SET", q, p), ("GENERATE EVENTS", events array).  enc
    "c128" runs the complex128 oracle, "adapt2" the adaptive encoding's
    step-by-step emulation (Sec. 4.1)."""
    prog = parse(text)
    N = prog[0][1][0]
    if enc == "adapt2":
        st = AState.zero(N)
    else:
        st = sv.zero_state(N)
    out = []
    noise = None
    ngate = 0
    nmeas = 0

    def state():
        return st.to_complex() if enc == "adapt2" else st

    def gate_records(rec):
        if noise is None:
            return [rec]
        px, py, pz, s = noise
        recs = [rec]
        for q in range(N):
            r = om.uniform(s, ngate * N + q)
            if r < px:
                recs.append(("X", (q,), ()))
            elif r < px + py:
                recs.append(("Y", (q,), ()))
            elif r < px + py + pz:
                recs.append(("Z", (q,), ()))
        return recs

    def project(q, bit):
        nonlocal st
        if enc == "adapt2":
            # an arithmetic operation of the encoding: decode, exact
            # projection and renormalisation, re-tune (r0, r1), encode
            z = st.to_complex()
            sv.project(z, N, q, bit)
            st.r0, st.r1 = retune(z)
            st.b0, st.b1 = encode(z, st.r0, st.r1)
        else:
            sv.project(st, N, q, bit)

    for name, args in prog[1:]:
        if name == "GATE":
            recs = gate_records(args)
            if enc == "adapt2":
                circuit.run_adapt2(st, recs)
            else:
                circuit.run(st, N, recs)
            ngate += 1
        elif name == "BIT ASSIGNMENT":
            continue
        elif name == "DEPOLARIZING CHANNEL":
            px, py, pz, k = args
            noise = (px, py, pz, k if k > 0 else run_seed + 2)
        elif name == "BEGIN MEASUREMENT":
            qx, qy, qz = sv.expect_xyz(state(), N)
            out.append(("BEGIN MEASUREMENT", qx, qy, qz))
        elif name == "M":
            q = args[0]
            v = state()
            p0, p1 = om.probs_of_qubit(v, N, q)
            u = om.uniform(run_seed, nmeas)
            nmeas += 1
            outcome = 0 if u * (p0 + p1) < p0 else 1
            project(q, outcome)
            out.append(("M", q, outcome, p0, p1))
        elif name in ("CLEAR", "SET"):
            q = args[0]
            bit = 0 if name == "CLEAR" else 1
            p0, p1 = om.probs_of_qubit(state(), N, q)
            p = p1 if bit else p0
            if p == 0.0:
                raise ValueError("%s %d: the projection gives a zero state" % (name, q))
            project(q, bit)
            out.append((name, q, p))
        elif name == "SHORBOX":
            nx, G, y = args
            v = sv.shorbox(N, nx, G, y)
            if enc == "adapt2":
                st = AState.from_complex(N, v)
            else:
                st = v
        elif name == "GENERATE EVENTS":
            n, seed = args
            s = seed if seed > 0 else run_seed + 1
            u = om.uniforms(s, 0, n)
            out.append(("GENERATE EVENTS", om.sample_events(state(), u)))
            break
        elif name == "EXIT":
            qx, qy, qz = sv.expect_xyz(state(), N)
            out.append(("BEGIN MEASUREMENT", qx, qy, qz))
            break
    return {"N": N, "out": out, "gates": ngate}
