"""ctypes binding of libqsim.so (include/qsim.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels.  PyTorch supplies device memory (a state can live in a torch
tensor's storage) and the CUDA stream.  Importing this module loads the
compiled library and raises ImportError when it is missing: there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsim.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libqsim.so is not built (run paper_1805_04708_gb300.build.build() or "
        "__graft_entry__.build()); the simulator has no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

C128, C64, ADAPT2 = 0, 1, 2
ENCODINGS = {"c128": C128, "c64": C64, "adapt2": ADAPT2}
AMP_BYTES = {C128: 16, C64: 8, ADAPT2: 2}

STATUS = {0: "QS_OK", 1: "QS_EINVAL", 2: "QS_ENOMEM", 3: "QS_ENOTBIJECTIVE",
          4: "QS_ECUDA", 5: "QS_ETIMEOUT", 6: "QS_EZEROPROJ", 7: "QS_ENOTUNITARY",
          8: "QS_EUNSUPPORTED"}


class QSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status
        self.name = STATUS.get(status, str(status))


class qs_gate(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int32), ("controls", ctypes.c_int32 * 2),
                ("target", ctypes.c_int32), ("u", ctypes.c_double * 8)]


class qs_request(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("N", ctypes.c_int), ("ngates", ctypes.c_int),
                ("gates", ctypes.POINTER(qs_gate)), ("qz", ctypes.POINTER(ctypes.c_double)),
                ("norm", ctypes.c_double), ("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double)]


class qs_serve_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("quantum", ctypes.c_int), ("max_small", ctypes.c_int),
                ("nstreams", ctypes.c_int), ("small_max_n", ctypes.c_int), ("persistent", ctypes.c_int),
                ("persistent_ctas", ctypes.c_int), ("device_wait_ms", ctypes.c_double),
                ("large_quantum", ctypes.c_int)]


class qs_serve_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int), ("ticks", ctypes.c_int), ("max_active", ctypes.c_int),
                ("wall_s", ctypes.c_double), ("busy_s", ctypes.c_double), ("launches", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_size_t), ("work_items", ctypes.c_uint64), ("idle_exits", ctypes.c_int),
                ("relaunches", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "qs_last_error_string": (ctypes.c_char_p, []),
    "qs_version": (ctypes.c_char_p, []),
    "qs_kernel_launches": (ctypes.c_uint64, []),
    "qs_set_pipeline_wait_limit": (_I, [ctypes.c_int64]),
    "sim_create": (_I, [_I, _I, _P, ctypes.POINTER(_P)]),
    "sim_create_in": (_I, [_I, _I, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "sim_destroy": (_I, [_P]),
    "sim_info": (_I, [_P, _IP, _IP, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t)]),
    "sim_reset": (_I, [_P]),
    "sim_set_lazy_reset": (_I, [_P, _I]),
    "sim_set_product_start": (_I, [_P, _I]),
    "sim_set_fp64_emulation": (_I, [_P, _I]),
    "apply_gate": (_I, [_P, _I, _D]),
    "apply_controlled": (_I, [_P, _IP, _I, _I, _D]),
    "apply_fused": (_I, [_P, _IP, _I, _D]),
    "sim_set_fused_engine": (_I, [_P, _I]),
    "apply_permutation": (_I, [_P, _IP, _I, _I, _I, ctypes.POINTER(ctypes.c_uint32)]),
    "modmul_table": (_I, [ctypes.c_uint64, ctypes.c_uint64, _I, ctypes.POINTER(ctypes.c_uint32)]),
    "shorbox_init": (_I, [_P, _I, ctypes.c_uint64, ctypes.c_uint64]),
    "circuit_run": (_I, [_P, ctypes.POINTER(qs_gate), _I, _I, _IP]),
    "circuit_compile": (_I, [_I, ctypes.POINTER(qs_gate), _I, _I, _IP]),
    "tile_compiler_info": (_I, [_IP, ctypes.POINTER(ctypes.c_long)]),
    "circuit_plan": (_I, [_I, _I, ctypes.POINTER(qs_gate), _I, _IP, _IP, _IP]),
    "circuit_product_start": (_I, [_I, ctypes.POINTER(qs_gate), _I, _IP, _D]),
    "circuit_run_timed": (_I, [_P, ctypes.POINTER(qs_gate), _I, _I, _IP, ctypes.POINTER(ctypes.c_float), _I]),
    "gate_std": (_I, [ctypes.c_char_p, _IP, _I, _D, _I, ctypes.POINTER(qs_gate)]),
    "sim_norm": (_I, [_P, _D]),
    "expect_xyz": (_I, [_P, _D, _D, _D]),
    "expect_xyz_norm": (_I, [_P, _D, _D, _D, _D]),
    "measure_probs": (_I, [_P, _IP, _I, _D]),
    "measure_probs_static": (_I, [_P, _I, _I, _IP, _I, _D, _P]),
    "sim_overlap": (_I, [_P, _P, _D, _D]),
    "qs_uniforms": (_I, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, _D]),
    "measure_qubit": (_I, [_P, _I, ctypes.c_double, _IP, _D]),
    "project_qubit": (_I, [_P, _I, _I, _D]),
    "generate_events": (_I, [_P, _D, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]),
    "generate_events_seeded": (_I, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]),
    "program_parse": (_I, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "program_destroy": (_I, [_P]),
    "program_info": (_I, [_P, _IP, _IP]),
    "program_run": (_I, [_P, _P, ctypes.c_uint64, _I]),
    "program_results": (_I, [_P, _IP, _IP, _IP, ctypes.POINTER(ctypes.c_int64)]),
    "program_expectations": (_I, [_P, _I, _D, _D, _D]),
    "program_outcomes": (_I, [_P, _IP, _IP, _D, _D]),
    "program_events": (_I, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "permute_qubits": (_I, [_P, _IP]),
    "aux_amplitudes": (_I, [_I, ctypes.POINTER(qs_gate), _I, ctypes.POINTER(ctypes.c_uint64), _I, _D, _IP, _P]),
    "aux_count": (_I, [_I, ctypes.POINTER(qs_gate), _I, _IP]),
    "depolarize_circuit": (_I, [_I, ctypes.POINTER(qs_gate), _I, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(qs_gate), _I, _IP]),
    "sim_copy_out": (_I, [_P, _P, ctypes.c_size_t, _D]),
    "sim_copy_in": (_I, [_P, _P, ctypes.c_size_t, _D]),
    "sim_sync": (_I, [_P]),
    "batch_create": (_I, [_I, _I, _I, _P, ctypes.POINTER(_P)]),
    "batch_destroy": (_I, [_P]),
    "batch_reset": (_I, [_P]),
    "batch_set_circuits": (_I, [_P, ctypes.POINTER(qs_gate), _IP]),
    "batch_run": (_I, [_P]),
    "batch_capture": (_I, [_P]),
    "batch_autotune": (_I, [_P, _IP, _IP, ctypes.POINTER(ctypes.c_float)]),
    "batch_norms": (_I, [_P, _D]),
    "batch_copy_out": (_I, [_P, _P, ctypes.c_size_t]),
    "batch_copy_in": (_I, [_P, _P, ctypes.c_size_t]),
    "batch_info": (_I, [_P, _IP, _IP, ctypes.POINTER(_P)]),
    "batch_set_tuning": (_I, [_P, _I, _I, _I]),
    "batch_get_tuning": (_I, [_P, _IP, _IP, _IP]),
    "serve_run": (_I, [ctypes.POINTER(qs_request), _I, ctypes.POINTER(qs_serve_config), ctypes.POINTER(qs_serve_stats)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _check(status):
    if status != 0:
        raise QSError(status, _lib.qs_last_error_string().decode())


def _ints(xs):
    xs = [int(x) for x in xs]
    return (ctypes.c_int * max(1, len(xs)))(*xs), len(xs)


def _dbl(xs):
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.float64).ravel())
    return a, a.ctypes.data_as(_D)


def version():
    return _lib.qs_version().decode()


def lib_path():
    return LIB_PATH


def set_pipeline_wait_limit(us):
    """Limit (microseconds; -1 = default) of the pipeline waits of the
    tensor-core fused gate and BEGIN MEASUREMENT (see include/qsim.h)."""
    _check(_lib.qs_set_pipeline_wait_limit(int(us)))


def kernel_launches():
    """Number of CUDA kernels the library has launched in this process."""
    return int(_lib.qs_kernel_launches())


# ---------------------------------------------------------------------------
# gate records
# ---------------------------------------------------------------------------
def gate_std(name, qubits, params=()):
    """Mnemonic record (name, qubits, params) -> qs_gate via the library's
    instruction-set table."""
    g = qs_gate()
    q, nq = _ints(qubits)
    p, pp = _dbl(params if len(params) else [0.0])
    _check(_lib.gate_std(name.encode(), q, nq, pp, len(params), ctypes.byref(g)))
    return g


def gate_array(records):
    """Convert a list of gate records (no MODMUL) to a ctypes qs_gate array."""
    arr = (qs_gate * max(1, len(records)))()
    for i, (name, q, p) in enumerate(records):
        arr[i] = gate_std(name, q, p)
    return arr, len(records)


def modmul_table(a, G, width):
    t = np.empty(1 << width, dtype=np.uint32)
    _check(_lib.modmul_table(int(a), int(G), int(width), t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return t


def circuit_compile(N, gates, mode=2):
    """Plan the complex64 tile passes of a circuit on N qubits and compile the
    kernels that circuit_run in `mode` (2 or 3) would launch compiled (host
    only).  Returns the number of passes planned."""
    if isinstance(gates, tuple):
        arr, n = gates
    else:
        arr, n = gate_array(gates)
    npass = ctypes.c_int(0)
    _check(_lib.circuit_compile(int(N), arr, n, int(mode), ctypes.byref(npass)))
    return npass.value


def circuit_plan(N, gates, enc="c64"):
    """The tile passes' gate order (host only): a list of passes, each the
    list of gate indices (into `gates`) in the order the pass takes them
    (identity gates are dropped)."""
    if isinstance(gates, tuple):
        arr, n = gates
    else:
        arr, n = gate_array(gates)
    order = np.full(max(1, n), -1, dtype=np.int32)
    start = np.zeros(max(1, n), dtype=np.int32)
    npass = ctypes.c_int(0)
    e = ENCODINGS[enc] if isinstance(enc, str) else int(enc)
    _check(_lib.circuit_plan(int(N), e, arr, n, order.ctypes.data_as(_IP), start.ctypes.data_as(_IP),
                             ctypes.byref(npass)))
    used = int(np.count_nonzero(order[:n] >= 0))
    bounds = [int(x) for x in start[:npass.value]] + [used]
    return [[int(x) for x in order[bounds[i]:bounds[i + 1]]] for i in range(npass.value)]


def circuit_product_start(N, gates):
    """The product start of a run from |0..0> (host only): (number of gates it
    takes, (N, 2) complex array of the factors f_q(0), f_q(1))."""
    if isinstance(gates, tuple):
        arr, n = gates
    else:
        arr, n = gate_array(gates)
    f = np.zeros(4 * int(N), dtype=np.float64)
    npre = ctypes.c_int(0)
    _check(_lib.circuit_product_start(int(N), arr, n, ctypes.byref(npre), f.ctypes.data_as(_D)))
    return npre.value, (f[0::2] + 1j * f[1::2]).reshape(int(N), 2)


def tile_compiler_info():
    """(NVRTC available, number of pass kernels compiled in this process)."""
    a = ctypes.c_int(0)
    c = ctypes.c_long(0)
    _check(_lib.tile_compiler_info(ctypes.byref(a), ctypes.byref(c)))
    return bool(a.value), int(c.value)


def uniforms(seed, first, n):
    """Draws first .. first + n - 1 of the library's counter-based generator."""
    out = np.empty(int(n))
    _check(_lib.qs_uniforms(int(seed) & (2 ** 64 - 1), int(first), int(n), out.ctypes.data_as(_D)))
    return out


def depolarize_circuit(N, gates, px, py, pz, seed, first_gate=0):
    """The circuit with the depolarizing channel's Pauli gates inserted (a
    ctypes qs_gate array and its length)."""
    if isinstance(gates, tuple):
        arr, n = gates
    else:
        arr, n = gate_array(gates)
    need = ctypes.c_int(0)
    _check(_lib.depolarize_circuit(int(N), arr, n, float(px), float(py), float(pz), int(seed) & (2 ** 64 - 1),
                                   int(first_gate), None, 0, ctypes.byref(need)))
    out = (qs_gate * max(1, need.value))()
    _check(_lib.depolarize_circuit(int(N), arr, n, float(px), float(py), float(pz), int(seed) & (2 ** 64 - 1),
                                   int(first_gate), out, need.value, ctypes.byref(need)))
    return out, need.value


def aux_amplitudes(N, gates, basis, stream=0):
    """Amplitudes <z|C|0..0> for the basis indices z by the auxiliary-variable
    method (Sec. 4.2): (complex array, number of auxiliary variables)."""
    if isinstance(gates, tuple):
        arr, n = gates
    else:
        arr, n = gate_array(gates)
    b = np.ascontiguousarray(np.asarray(basis, dtype=np.uint64))
    out = np.empty(2 * b.size)
    P = ctypes.c_int(0)
    _check(_lib.aux_amplitudes(int(N), arr, n, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), b.size,
                               out.ctypes.data_as(_D), ctypes.byref(P), _P(int(stream))))
    return out[0::2] + 1j * out[1::2], P.value


def aux_count(N, gates):
    arr, n = gates if isinstance(gates, tuple) else gate_array(gates)
    P = ctypes.c_int(0)
    _check(_lib.aux_count(int(N), arr, n, ctypes.byref(P)))
    return P.value


class Program:
    """A parsed program in the instruction language of Appendix A."""

    def __init__(self, text):
        h = _P()
        _check(_lib.program_parse(text.encode(), ctypes.byref(h)))
        self._h = h
        n, ni = ctypes.c_int(0), ctypes.c_int(0)
        _check(_lib.program_info(h, ctypes.byref(n), ctypes.byref(ni)))
        self.N, self.n_instr = n.value, ni.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.program_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, sim, run_seed=1, mode=1):
        """Run on a Sim of N qubits; returns dict(measurements=[(qx, qy,
        qz), ...], m=[(qubit, outcome, p0, p1), ...], proj=[p, ...],
        events=array)."""
        _check(_lib.program_run(self._h, sim._h, int(run_seed) & (2 ** 64 - 1), int(mode)))
        nm, nmm, npj = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        nev = ctypes.c_int64(0)
        _check(_lib.program_results(self._h, ctypes.byref(nm), ctypes.byref(nmm), ctypes.byref(npj),
                                    ctypes.byref(nev)))
        meas = []
        for k in range(nm.value):
            x, y, z = np.empty(self.N), np.empty(self.N), np.empty(self.N)
            _check(_lib.program_expectations(self._h, k, x.ctypes.data_as(_D), y.ctypes.data_as(_D),
                                             z.ctypes.data_as(_D)))
            meas.append((x, y, z))
        qs = np.zeros(max(1, nmm.value), dtype=np.int32)
        os_ = np.zeros(max(1, nmm.value), dtype=np.int32)
        pr = np.zeros(2 * max(1, nmm.value))
        pj = np.zeros(max(1, npj.value))
        _check(_lib.program_outcomes(self._h, qs.ctypes.data_as(_IP), os_.ctypes.data_as(_IP),
                                     pr.ctypes.data_as(_D), pj.ctypes.data_as(_D)))
        ev = np.zeros(max(1, nev.value), dtype=np.uint64)
        _check(_lib.program_events(self._h, ev.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        m = [(int(qs[i]), int(os_[i]), float(pr[2 * i]), float(pr[2 * i + 1])) for i in range(nmm.value)]
        return dict(measurements=meas, m=m, proj=[float(x) for x in pj[:npj.value]],
                    events=ev[:nev.value].astype(np.int64))


# ---------------------------------------------------------------------------
# simulator handle
# ---------------------------------------------------------------------------
class Sim:
    """An N-qubit state on the current CUDA device.

    enc: "c128", "c64" or "adapt2".  stream: a torch.cuda.Stream, a raw
    cudaStream_t integer, or None for torch's current stream.  buffer: an
    optional torch CUDA tensor whose storage holds the state (the library then
    borrows it); by default torch allocates one.
    """

    def __init__(self, N, enc="c128", stream=None, buffer=None):
        import torch
        self.N = int(N)
        self.enc = ENCODINGS[enc] if isinstance(enc, str) else int(enc)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream_handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        nbytes = AMP_BYTES[self.enc] << self.N
        own = buffer is None
        if own:
            buffer = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        self._buf = buffer
        ptr = buffer.data_ptr()
        ptr_al = (ptr + 255) & ~255
        avail = buffer.numel() * buffer.element_size() - (ptr_al - ptr)
        h = _P()
        _check(_lib.sim_create_in(self.N, self.enc, _P(ptr_al), avail, _P(self.stream_handle), ctypes.byref(h)))
        self._h = h
        self.nbytes = nbytes
        if own:   # the buffer is private: resets may stay pending, from the start
            _check(_lib.sim_set_lazy_reset(h, 1))
            _check(_lib.sim_reset(h))

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            _check(_lib.sim_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self):
        _check(_lib.sim_reset(self._h))

    def sync(self):
        _check(_lib.sim_sync(self._h))

    def device_ptr(self):
        p = _P()
        _check(_lib.sim_info(self._h, None, None, ctypes.byref(p), None))
        return p.value

    # -- gates --
    def apply_gate(self, target, U):
        u, up = _dbl(_mat8(U))
        _check(_lib.apply_gate(self._h, int(target), up))

    def apply_controlled(self, controls, target, U):
        c, nc = _ints(controls)
        u, up = _dbl(_mat8(U))
        _check(_lib.apply_controlled(self._h, c, nc, int(target), up))

    def apply_fused(self, qubits, U):
        q, k = _ints(qubits)
        U = np.asarray(U, dtype=np.complex128)
        flat = np.empty(2 * U.size)
        flat[0::2] = U.ravel().real
        flat[1::2] = U.ravel().imag
        f, fp = _dbl(flat)
        _check(_lib.apply_fused(self._h, q, k, fp))

    FUSED_ENGINES = {"auto": 0, "cuda_cores": 1, "mma_sync": 2}

    def set_fused_engine(self, engine):
        """Kernel family for apply_fused on complex64 states: "auto" (tcgen05
        where the gate qualifies), "cuda_cores" or "mma_sync"."""
        _check(_lib.sim_set_fused_engine(self._h, self.FUSED_ENGINES[engine]))

    def set_product_start(self, on=True):
        """Product start of tile runs from a pending |0..0> (complex64 and
        complex128; see sim_set_product_start); on by default."""
        _check(_lib.sim_set_product_start(self._h, 1 if on else 0))

    def set_fp64_emulation(self, on=1):
        """complex128 gate arithmetic: True / 1 (default) double-float
        everywhere, False / 0 FP64 units everywhere, 2 double-float in the
        per-gate sweeps and FP64 units in the tile passes."""
        _check(_lib.sim_set_fp64_emulation(self._h, int(on)))

    def apply_permutation(self, controls, reg_lo, reg_w, table):
        c, nc = _ints(controls)
        t = np.ascontiguousarray(np.asarray(table, dtype=np.uint32))
        _check(_lib.apply_permutation(self._h, c, nc, int(reg_lo), int(reg_w),
                                      t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))

    def shorbox_init(self, nx, G, y):
        _check(_lib.shorbox_init(self._h, int(nx), int(G), int(y)))

    def circuit_run(self, gates, mode=1):
        """gates: a ctypes qs_gate array (from gate_array) plus count, or a list
        of records.  Returns the number of state sweeps launched."""
        if isinstance(gates, tuple):
            arr, n = gates
        else:
            arr, n = gate_array(gates)
        npass = ctypes.c_int(0)
        _check(_lib.circuit_run(self._h, arr, n, int(mode), ctypes.byref(npass)))
        return npass.value

    def circuit_run_timed(self, gates, mode=1, max_passes=256):
        """As circuit_run; returns the device time (ms) of every sweep."""
        if isinstance(gates, tuple):
            arr, n = gates
        else:
            arr, n = gate_array(gates)
        npass = ctypes.c_int(0)
        ms = (ctypes.c_float * max_passes)()
        _check(_lib.circuit_run_timed(self._h, arr, n, int(mode), ctypes.byref(npass), ms, max_passes))
        return [ms[i] for i in range(min(npass.value, max_passes))]

    def run_records(self, records, mode=1):
        """Run records in order; MODMUL records become a modmul table plus a
        controlled permutation, runs of other records one circuit_run."""
        run = []
        passes = 0
        for rec in records:
            if rec[0] == "MODMUL":
                if run:
                    passes += self.circuit_run(run, mode)
                    run = []
                a, G, lo, w = rec[2]
                self.apply_permutation(rec[1], lo, w, modmul_table(a, G, w))
                passes += 1
            else:
                run.append(rec)
        if run:
            passes += self.circuit_run(run, mode)
        return passes

    # -- reductions --
    def norm(self):
        out = ctypes.c_double(0.0)
        _check(_lib.sim_norm(self._h, ctypes.byref(out)))
        return out.value

    def expect_xyz(self):
        qx = np.empty(self.N)
        qy = np.empty(self.N)
        qz = np.empty(self.N)
        _check(_lib.expect_xyz(self._h, qx.ctypes.data_as(_D), qy.ctypes.data_as(_D), qz.ctypes.data_as(_D)))
        return qx, qy, qz

    def expect_xyz_norm(self):
        """(qx, qy, qz, norm): expect_xyz and norm from one call."""
        qx = np.empty(self.N)
        qy = np.empty(self.N)
        qz = np.empty(self.N)
        nrm = ctypes.c_double(0.0)
        _check(_lib.expect_xyz_norm(self._h, qx.ctypes.data_as(_D), qy.ctypes.data_as(_D), qz.ctypes.data_as(_D),
                                    ctypes.byref(nrm)))
        return qx, qy, qz, nrm.value

    def overlap(self, other):
        """(<self|other>, ||self - other||^2) in FP64 (any encodings)."""
        ov = np.zeros(2)
        d2 = ctypes.c_double(0.0)
        _check(_lib.sim_overlap(self._h, other._h, ov.ctypes.data_as(_D), ctypes.byref(d2)))
        return complex(ov[0], ov[1]), d2.value

    def measure_probs(self, qubits):
        q, nq = _ints(qubits)
        out = np.empty(1 << nq)
        _check(_lib.measure_probs(self._h, q, nq, out.ctypes.data_as(_D)))
        return out

    def permute_qubits(self, perm):
        """The content of index bit k moves to index bit perm[k]."""
        p, n = _ints(perm)
        _check(_lib.permute_qubits(self._h, p))

    # -- stochastic instructions --
    def measure(self, q, u):
        """M q with the draw u: (outcome, p0, p1); the state is projected."""
        o = ctypes.c_int(0)
        pr = np.zeros(2)
        _check(_lib.measure_qubit(self._h, int(q), float(u), ctypes.byref(o), pr.ctypes.data_as(_D)))
        return o.value, float(pr[0]), float(pr[1])

    def project(self, q, bit):
        """CLEAR q (bit 0) / SET q (bit 1); returns the probability of `bit`."""
        p = ctypes.c_double(0.0)
        _check(_lib.project_qubit(self._h, int(q), int(bit), ctypes.byref(p)))
        return p.value

    def generate_events(self, u=None, n=None, seed=None):
        """Basis-state events from the draws u, or n events from `seed`."""
        if u is not None:
            u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
            out = np.empty(u.size, dtype=np.uint64)
            _check(_lib.generate_events(self._h, u.ctypes.data_as(_D), u.size,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        else:
            out = np.empty(int(n), dtype=np.uint64)
            _check(_lib.generate_events_seeded(self._h, int(seed) & (2 ** 64 - 1), int(n),
                                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out.astype(np.int64)

    # -- raw access --
    def copy_out(self):
        """Raw amplitudes as numpy: complex128 / complex64 arrays, or
        (uint16 words, (r0, r1)) for ADAPT2."""
        r = np.zeros(2)
        if self.enc == C128:
            a = np.empty(1 << self.N, dtype=np.complex128)
        elif self.enc == C64:
            a = np.empty(1 << self.N, dtype=np.complex64)
        else:
            a = np.empty(1 << self.N, dtype=np.uint16)
        _check(_lib.sim_copy_out(self._h, _P(a.ctypes.data), self.nbytes, r.ctypes.data_as(_D)))
        return (a, (float(r[0]), float(r[1]))) if self.enc == ADAPT2 else a

    def copy_in(self, a, r0r1=None):
        if self.enc == C128:
            a = np.ascontiguousarray(a, dtype=np.complex128)
        elif self.enc == C64:
            a = np.ascontiguousarray(a, dtype=np.complex64)
        else:
            a = np.ascontiguousarray(a, dtype=np.uint16)
        if a.nbytes != self.nbytes:
            raise ValueError("need %d bytes" % self.nbytes)
        r = np.asarray(r0r1 if r0r1 is not None else (0.0, 0.0), dtype=np.float64)
        _check(_lib.sim_copy_in(self._h, _P(a.ctypes.data), self.nbytes, r.ctypes.data_as(_D)))


class Batch:
    """nstates independent N-qubit states advanced in one launch (see
    include/qsim.h, batched small states)."""

    def __init__(self, N, enc, nstates, stream=None):
        import torch
        self.N, self.nstates = int(N), int(nstates)
        self.enc = ENCODINGS[enc] if isinstance(enc, str) else int(enc)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream_handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        h = _P()
        _check(_lib.batch_create(self.N, self.enc, self.nstates, _P(self.stream_handle), ctypes.byref(h)))
        self._h = h
        self.nbytes = (self.nstates << self.N) * AMP_BYTES[self.enc]

    def close(self):
        if getattr(self, "_h", None):
            _check(_lib.batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self):
        _check(_lib.batch_reset(self._h))

    def set_circuits(self, circuits):
        """circuits: one list of gate records per state."""
        recs = [r for c in circuits for r in c]
        arr, n = gate_array(recs)
        offs = np.zeros(self.nstates + 1, dtype=np.int32)
        offs[1:] = np.cumsum([len(c) for c in circuits])
        o = (ctypes.c_int * (self.nstates + 1))(*offs.tolist())
        _check(_lib.batch_set_circuits(self._h, arr, o))

    def run(self):
        _check(_lib.batch_run(self._h))

    def capture(self):
        _check(_lib.batch_capture(self._h))

    def autotune(self):
        lay, th, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_float(0)
        _check(_lib.batch_autotune(self._h, ctypes.byref(lay), ctypes.byref(th), ctypes.byref(ms)))
        return lay.value, th.value, ms.value

    def set_tuning(self, fuse_k, tile_bits, threads):
        """Kernel configuration (see batch_set_tuning)."""
        _check(_lib.batch_set_tuning(self._h, int(fuse_k), int(tile_bits), int(threads)))

    def tuning(self):
        """(fuse_k, tile_bits, threads) of the current configuration."""
        k, b, t = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(_lib.batch_get_tuning(self._h, ctypes.byref(k), ctypes.byref(b), ctypes.byref(t)))
        return k.value, b.value, t.value

    def info(self):
        lay, th, p = ctypes.c_int(0), ctypes.c_int(0), _P()
        _check(_lib.batch_info(self._h, ctypes.byref(lay), ctypes.byref(th), ctypes.byref(p)))
        return lay.value, th.value, p.value

    def norms(self):
        out = np.empty(self.nstates)
        _check(_lib.batch_norms(self._h, out.ctypes.data_as(_D)))
        return out

    def copy_out(self):
        dt = np.complex128 if self.enc == C128 else np.complex64
        a = np.empty(self.nstates << self.N, dtype=dt)
        _check(_lib.batch_copy_out(self._h, _P(a.ctypes.data), self.nbytes))
        return a.reshape(self.nstates, 1 << self.N)

    def copy_in(self, a):
        dt = np.complex128 if self.enc == C128 else np.complex64
        a = np.ascontiguousarray(a, dtype=dt)
        _check(_lib.batch_copy_in(self._h, _P(a.ctypes.data), self.nbytes))


def serve(requests, mem_budget, quantum=64, nstreams=4, small_max_n=14, max_small=4096, persistent=False,
          persistent_ctas=0, device_wait_ms=0.0, large_quantum=0):
    """Run the serving loop.  requests: list of dicts with arrival (s), N and
    records (gate records).  persistent: the persistent-kernel mode (device
    work queue, bounded device waits).  Returns (results, stats): per request
    a dict with qz, norm, admit_s, finish_s, latency_s."""
    n = len(requests)
    reqs = (qs_request * max(1, n))()
    keep = []
    for i, r in enumerate(requests):
        arr, ng = gate_array(r["records"])
        qz = np.zeros(r["N"])
        keep.append((arr, qz))
        reqs[i].arrival_s = float(r["arrival"])
        reqs[i].N = int(r["N"])
        reqs[i].ngates = ng
        reqs[i].gates = ctypes.cast(arr, ctypes.POINTER(qs_gate))
        reqs[i].qz = qz.ctypes.data_as(_D)
    cfg = qs_serve_config(int(mem_budget), int(quantum), int(max_small), int(nstreams), int(small_max_n),
                          1 if persistent else 0, int(persistent_ctas), float(device_wait_ms), int(large_quantum))
    st = qs_serve_stats()
    _check(_lib.serve_run(reqs, n, ctypes.byref(cfg), ctypes.byref(st)))
    out = []
    for i in range(n):
        out.append(dict(qz=keep[i][1].copy(), norm=reqs[i].norm, admit_s=reqs[i].admit_s,
                        finish_s=reqs[i].finish_s, latency_s=reqs[i].finish_s - reqs[i].arrival_s))
    stats = dict(completed=st.completed, ticks=st.ticks, max_active=st.max_active, wall_s=st.wall_s,
                 busy_s=st.busy_s, launches=st.launches, peak_bytes=st.peak_bytes, work_items=st.work_items,
                 idle_exits=st.idle_exits, relaunches=st.relaunches)
    return out, stats


def measure_probs_static(state_ptr, N, enc, qubits, stream=0):
    """measure_probs on a caller-held device state without any allocation
    (the library's fixed scratch; see include/qsim.h)."""
    q, nq = _ints(qubits)
    out = np.empty(1 << nq)
    e = ENCODINGS[enc] if isinstance(enc, str) else int(enc)
    _check(_lib.measure_probs_static(_P(state_ptr), int(N), e, q, nq, out.ctypes.data_as(_D), _P(int(stream))))
    return out


def _mat8(U):
    U = np.asarray(U)
    if U.shape == (8,):
        return U.astype(np.float64)
    U = U.astype(np.complex128).reshape(2, 2)
    out = np.empty(8)
    out[0::2] = U.ravel().real
    out[1::2] = U.ravel().imag
    return out
