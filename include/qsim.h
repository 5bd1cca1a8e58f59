/*
 * qsim.h -- C ABI of the GB300 state-vector engine (libqsim.so).
 *
 * The engine holds the 2^N complex amplitudes of an N-qubit quantum computer
 * (Sec. 2, Eq. (STAT2) of arXiv:1805.04708) in device memory and updates them
 * in place with hand-written sm_103a CUDA kernels.  Qubit q is bit q of the
 * basis index, qubit 0 the least significant ("rightmost") bit (Sec. 2, the
 * paragraph after Eq. (STAT1)).
 *
 * Conventions for every entry point
 *  - Plain C types only; device pointers are marked "device", host pointers
 *    "host".  The caller owns every host array it passes, and allocates every
 *    output array.
 *  - Calls are ordered on the stream given at creation (NULL = the legacy
 *    default stream).  Gate calls return once the work is enqueued; calls that
 *    return numbers to the host (norm, expect_xyz, measure_probs, copy_out)
 *    synchronise that stream before returning.
 *  - Invalid arguments are rejected before anything is launched, with
 *    QS_EINVAL (qubit out of range, repeated qubit, N out of range, bad
 *    sizes), QS_ENOTUNITARY (a matrix further than the stated tolerance from
 *    unitary) or QS_ENOTBIJECTIVE (a permutation table that is not a
 *    bijection).  CUDA failures return QS_ECUDA; qs_last_error_string() then
 *    describes the error.  Nothing aborts the process.
 *  - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

/* Storage encodings of one amplitude.
 *  QS_C128  : complex128, interleaved (re, im) FP64, 16 B per amplitude (the
 *             double-precision form of JUQCS-E, Sec. 4.1).
 *  QS_C64   : complex64, interleaved (re, im) FP32, 8 B per amplitude.
 *  QS_ADAPT2: the 2-byte adaptive polar code of JUQCS-A (Sec. 4.1): one
 *             little-endian 16-bit word per amplitude, low byte b0 (magnitude
 *             code), high byte b1 (angle code), both two's-complement int8,
 *             plus the state-wide pair (r0, r1) kept by the handle. */
typedef enum { QS_C128 = 0, QS_C64 = 1, QS_ADAPT2 = 2 } qs_encoding;

typedef enum {
  QS_OK = 0,
  QS_EINVAL = 1,
  QS_ENOMEM = 2,
  QS_ENOTBIJECTIVE = 3,
  QS_ECUDA = 4,
  QS_ETIMEOUT = 5,
  QS_EZEROPROJ = 6,
  QS_ENOTUNITARY = 7,
  QS_EUNSUPPORTED = 8
} qs_status;

typedef struct qs_sim qs_sim; /* opaque; owns or borrows its device state */

/* A gate record: a 2x2 complex matrix u applied to qubit `target` on the
 * subspace where the nc qubits controls[0..nc-1] are all 1 (nc = 0, 1, 2).
 * This covers every gate of the instruction set (Appendix A): single-qubit
 * gates (nc = 0), CNOT and U(k) (nc = 1), TOFFOLI (nc = 2); the update is the
 * pair rule of Eq. (NUM2) with H replaced by u (Eq. (AQS0)).
 * u is row-major with interleaved (re, im): u00, u01, u10, u11. */
typedef struct {
  int32_t nc;
  int32_t controls[2];
  int32_t target;
  double u[8];
} qs_gate;

/* ---- errors ------------------------------------------------------------- */
/* Text of the last error on this thread (static storage, never NULL). */
const char* qs_last_error_string(void);
/* Library version string, e.g. "qsim 0.1 sm_103a". */
const char* qs_version(void);
/* Number of CUDA kernels this library has launched in this process. */
uint64_t qs_kernel_launches(void);

/* Limit, process-wide, of the pipeline waits inside the tensor-core fused
 * gate and the complex64 BEGIN MEASUREMENT kernels (waits for a tensor load,
 * a conversion, an MMA or a free buffer): about `us` microseconds (0: give up
 * at the first test; -1: the default, about one second).  A wait that runs
 * out ends the kernel cleanly (the copies in flight are waited for with the
 * full limit, the tensor memory is freed) and the call returns QS_ETIMEOUT;
 * the next call with a normal limit runs as usual.  For tests of those exit
 * paths; the paper has no counterpart. */
qs_status qs_set_pipeline_wait_limit(int64_t us);

/* ---- lifetime (QUBITS N, Appendix A; |0..0> of Eq. (appa0)) -------------- */
/* Create an N-qubit state |0...0> (a_0 = 1, every other amplitude 0) in
 * encoding `enc`, in device memory the handle allocates and owns.
 * 1 < N < 64 (Appendix A, QUBITS); N must also fit the device memory
 * (2^N * 16, 8 or 2 bytes), else QS_ENOMEM.  cuda_stream is a cudaStream_t
 * (NULL = default stream) used by every later call on the handle. */
qs_status sim_create(int N, qs_encoding enc, void* cuda_stream, qs_sim** out);

/* As sim_create, but the state lives in a caller-owned device buffer
 * (dev_ptr, `bytes` >= 2^N * bytes-per-amplitude, 256-byte aligned), e.g. a
 * torch tensor's storage.  The caller keeps ownership and must keep the
 * buffer alive until sim_destroy.  The buffer is overwritten with |0..0>. */
qs_status sim_create_in(int N, qs_encoding enc, void* dev_ptr, size_t bytes,
                        void* cuda_stream, qs_sim** out);

/* Release the handle and the device memory it owns (never a borrowed
 * buffer).  Synchronises the handle's stream first. */
qs_status sim_destroy(qs_sim* sim);

/* Number of qubits, encoding, device pointer of the amplitudes and their size
 * in bytes. */
qs_status sim_info(const qs_sim* sim, int* N, int* enc, void** dev_ptr, size_t* bytes);

/* Reset to |0..0> (a_0 = 1).  With lazy reset (the default for sim_create,
 * see sim_set_lazy_reset) nothing is written yet: the first tile pass of a
 * following circuit_run makes its tiles from |0..0> instead of reading them,
 * and every other call that reads or writes the amplitudes (including
 * sim_info asking for the device pointer) writes |0..0> first. */
qs_status sim_reset(qs_sim* sim);

/* Turn lazy reset on or off (on: nonzero).  Default on for sim_create, off
 * for sim_create_in, whose buffer its owner may read without a call of this
 * library; a caller that only reaches the amplitudes through this library
 * may turn it on.  Turning it off writes a pending |0..0>.  The paper has no
 * counterpart. */
qs_status sim_set_lazy_reset(qs_sim* sim, int on);

/* Product start (on: nonzero; default on).  When circuit_run (modes 1-3) of a
 * complex64 or complex128 state starts from a pending |0..0>, every
 * single-qubit gate that
 * comes before all multi-qubit gates on its qubit acts on an unentangled
 * qubit and commutes with every earlier gate on other qubits; these gates are
 * composed per qubit (FP64) and the first tile pass writes the product state
 * prod_q (U_q |0>)(bit q) instead of applying them one by one.  The result
 * equals the gate-by-gate one up to rounding.  Off: every gate runs in the
 * passes.  The paper has no counterpart (its runs start from a written
 * state). */
qs_status sim_set_product_start(qs_sim* sim, int on);

/* Arithmetic of the complex128 gate kernels (apply_gate, apply_controlled,
 * circuit_run): 1 (the default) holds each FP64 value as a double-float pair
 * of FP32 numbers (about 48 significant bits; products by an error-free
 * transformation, sums with an exact sum of the high parts) and computes on
 * the FP32 pipes, which this GPU runs at about 52 times its FP64 rate, in the
 * per-gate sweeps and the tile passes; 0 computes on the FP64 units
 * everywhere; 2 takes double-float in the per-gate sweeps and the FP64 units
 * in the tile passes.  The dense fused gate (apply_fused) computes in
 * double-float in modes 1 and 2 and on the FP64 units in mode 0.  Gates that
 * only move amplitudes or multiply them by +-1, +-i run in FP64 in every mode
 * (exact).  Amplitudes stay FP64 in memory, and every mode agrees with the
 * FP64 oracle to 1e-12.  Reductions stay FP64.  Other values give QS_EINVAL.
 * The paper's double-precision simulator (Sec. 4.1) computes in FP64. */
qs_status sim_set_fp64_emulation(qs_sim* sim, int on);

/* ---- gates (Sec. 2, Eq. (NUM2); Appendix A) ------------------------------ */
/* Single-qubit gate: for every basis index i with bit `target` = 0,
 * (a_i, a_{i+2^target}) <- U (a_i, a_{i+2^target}) (Eq. (NUM2), Eq. (AQS0)).
 * U: host, 8 doubles, row-major (re, im) of u00, u01, u10, u11; it must be
 * unitary to 1e-10 (max-abs of U U^dagger - 1), else QS_ENOTUNITARY.
 * Diagonal, anti-diagonal and Hadamard-shaped matrices run specialised
 * kernels that give the same result. */
qs_status apply_gate(qs_sim* sim, int target, const double U[8]);

/* Controlled gate: the same update restricted to the indices whose nc
 * control bits are all 1 (nc in {0,1,2}; CNOT, U(k), TOFFOLI of Appendix A;
 * the groups of four and eight amplitudes described after Eq. (NUM2)).
 * controls: host, nc distinct qubits, none equal to target. */
qs_status apply_controlled(qs_sim* sim, const int* controls, int nc, int target,
                           const double U[8]);

/* Dense k-qubit gate (1 <= k <= 5): a 2^k x 2^k complex matrix applied to the
 * amplitudes of each group of 2^k basis states that differ only in the
 * qubits `qubits` (Eq. (AQS0) for n-qubit gates; the fused multi-qubit gates
 * proposed at the end of Sec. 5.2).  Bit m of the local row/column index is
 * the value of qubits[m].  U: host, 2*4^k doubles, row-major (re, im).
 * The matrix must be unitary to 1e-10. */
qs_status apply_fused(qs_sim* sim, const int* qubits, int k, const double* U);

/* Kernel family for apply_fused on QS_C64 states (every choice computes the
 * same product; the tensor-core paths round each operand as x = hi + lo in
 * TF32 and keep the three largest partial products, error near FP32
 * rounding).  The paper has no counterpart: it applies gates one at a time.
 *  QS_FUSED_AUTO       : tcgen05 tensor cores (TMEM accumulators) when
 *                        3 <= k <= 5 and N >= 12, on any k distinct qubits:
 *                        the qubits 0..k-1 (any order) stream whole groups
 *                        with TMA tensor copies, other sets gather each
 *                        group's runs with bulk copies and store from the
 *                        accumulators; else the mma.sync tensor-core kernel
 *                        when 2 <= k, the qubits are 0..k-1 and N >= k+4;
 *                        everything else runs the CUDA-core kernel.
 *  QS_FUSED_CUDA_CORES : the CUDA-core kernel for every gate.
 *  QS_FUSED_MMA_SYNC   : as AUTO without the tcgen05 kernel.
 * QS_C128 states always take the CUDA-core kernel (see
 * sim_set_fp64_emulation for its arithmetic).
 * The default is QS_FUSED_AUTO.  Unknown values give QS_EINVAL.  A wait
 * inside the tcgen05 kernel that runs out (about a second) makes
 * apply_fused return QS_ETIMEOUT with the state undefined. */
typedef enum { QS_FUSED_AUTO = 0, QS_FUSED_CUDA_CORES = 1, QS_FUSED_MMA_SYNC = 2 } qs_fused_engine;
qs_status sim_set_fused_engine(qs_sim* sim, int engine);

/* Controlled register permutation (SHORBOX's f(x) = y^x mod G built from
 * controlled modular multiplications, Sec. 5.4): on every basis index whose
 * nc control bits are all 1, the value f of the register bits
 * reg_lo .. reg_lo+reg_w-1 is replaced by table[f].  table: host, 2^reg_w
 * uint32 entries forming a bijection of [0, 2^reg_w), else QS_ENOTBIJECTIVE.
 * Amplitudes (or ADAPT2 codes) move bit-exactly.  1 <= reg_w <= 12; controls
 * must lie outside the register. */
qs_status apply_permutation(qs_sim* sim, const int* controls, int nc, int reg_lo,
                            int reg_w, const uint32_t* table);

/* Fill `table` (host, 2^width uint32) with f -> a*f mod G for f < G and the
 * identity for G <= f < 2^width (the controlled multiplication of Sec. 5.4).
 * Requires gcd(a, G) = 1 and G <= 2^width. */
qs_status modmul_table(uint64_t a, uint64_t G, int width, uint32_t* table);

/* SHORBOX nx G y (Appendix A): overwrite the state with
 * 2^{-nx/2} sum_{x=0}^{2^nx - 1} |x>|y^x mod G>: x-register on qubits
 * 0..nx-1, f-register on qubits nx..N-1 (G <= 2^{N-nx}, 1 <= y < G).
 * One write sweep, no gate is applied. */
qs_status shorbox_init(qs_sim* sim, int nx, uint64_t G, uint64_t y);

/* ---- circuits ----------------------------------------------------------- */
/* Run a gate list.  mode 0: one kernel per gate, in order (the per-gate sweep
 * of Sec. 3).  Modes 1-3: the native planner groups gates into shared-memory
 * tile passes (several gates per read and write of the state; the fusion
 * strategy suggested at the end of Sec. 5.2) and runs each pass as one
 * kernel.  A pass may take a gate ahead of earlier gates only when it
 * commutes with all of them (they share no qubit on which either acts
 * non-diagonally), so the circuit's product is unchanged.  The pass kernel:
 *   mode 1: the op interpreter compiled into the library;
 *   mode 2: for QS_C64 states, per pass structure (the pass's op types,
 *           qubits and control masks; not its coefficients) the fastest of
 *           the interpreter and three kernels compiled at run time for that
 *           structure (NVRTC, sm_103a; without barriers, and with a CTA
 *           barrier every 2 or every 8 ops).  The first eight launches of
 *           a structure try each candidate twice, timed with CUDA events on
 *           the handle's stream; later launches use the candidate with the
 *           fastest launch.  Compiled
 *           kernels are cached; a new structure pays its compile time unless
 *           circuit_compile ran first; a variant that fails to compile is
 *           never picked.  Compiled kernels (a few hundred KB each) stay
 *           loaded until the process ends;
 *   mode 3: the compiled kernel without barriers for every QS_C64 pass.
 * Modes 2 and 3 give QS_EUNSUPPORTED on a QS_C64 state when NVRTC cannot be
 * loaded; QS_C128 states use the interpreter in every tile mode.  For
 * QS_C64, a last pass of at most 4 gates joins the previous pass when their
 * targets fit its tile; for QS_C64 and QS_C128 a run from a pending |0..0>
 * starts from the product state of its leading single-qubit gates
 * (sim_set_product_start).
 * Results equal mode 0 up to floating-point rounding order.  gates: host
 * array of n records.  n_passes (may be NULL) receives the number of state
 * sweeps launched.  The paper has no counterpart for modes 1-3. */
qs_status circuit_run(qs_sim* sim, const qs_gate* gates, int n, int mode, int* n_passes);

/* Plan the tile passes of a QS_C64 circuit on N qubits (13 <= N <= 63) and
 * compile the kernels of each new pass structure that circuit_run in `mode`
 * may launch (mode 2: its three compiled candidates; mode 3: the one kernel)
 * on up to 16 host threads (host only: no device call; NVRTC must be
 * loadable, else QS_EUNSUPPORTED), for runs on a written state and for runs
 * from a pending |0..0> (the passes after the product start).  A later
 * circuit_run of the same circuit in that mode then launches without
 * compiling.  n_passes (may be NULL) receives the number of passes planned
 * for a written state.  Gate validation as in circuit_run. */
qs_status circuit_compile(int N, const qs_gate* gates, int n, int mode, int* n_passes);

/* The order in which circuit_run's tile passes take the gates (host only, no
 * device call): for a QS_C64 or QS_C128 circuit on N >= 13 (QS_C64) / 12
 * (QS_C128) qubits, order (host, n ints) receives the indices of the
 * non-identity gates in run order and pass_start (host, n ints) the position
 * in order where each pass begins; *n_passes the number of passes.  Inside a
 * pass the op rewriting (delayed diagonals, composed neighbours, factor
 * tables) is not shown, and the plan is that of a run on a written state (no
 * product start).  The paper has no counterpart. */
qs_status circuit_plan(int N, int enc, const qs_gate* gates, int n, int* order, int* pass_start, int* n_passes);

/* The product start of a run of this circuit from a pending |0..0> (host
 * only, no device call; see sim_set_product_start): *n_prefix receives the
 * number of gates it takes (the single-qubit gates that come before every
 * multi-qubit gate on their qubit), factors (host, 4N doubles, or NULL) the
 * product-state factors f_q(0), f_q(1) of every qubit q as (re, im) pairs,
 * f_q = U_q |0> with U_q the product of qubit q's gates in order (FP64).
 * N in 1..63; gate validation as in circuit_run.  The paper has no
 * counterpart. */
qs_status circuit_product_start(int N, const qs_gate* gates, int n, int* n_prefix, double* factors);

/* Whether NVRTC could be loaded (available: 1 or 0) and how many pass
 * kernels this process has compiled so far (compiles).  Outputs may be NULL. */
qs_status tile_compiler_info(int* available, long* compiles);

/* As circuit_run, and records a CUDA event pair around every sweep on the
 * handle's stream: pass_ms (host, room for max_passes floats, may be NULL)
 * receives the device time of each sweep in order.  Synchronises the stream
 * before returning. */
qs_status circuit_run_timed(qs_sim* sim, const qs_gate* gates, int n, int mode, int* n_passes,
                            float* pass_ms, int max_passes);

/* Build a gate record from an instruction-set mnemonic (Appendix A):
 * "I","H","X","Y","Z","S","S+","T","T+","U1","U2","U3","+X","-X","+Y","-Y",
 * "R" (params[0] = k, negative for R^dagger), "CNOT", "U" (params[0] = k),
 * "TOFFOLI", plus "RZ" (params[0] = theta: diag(e^{-i theta/2}, e^{i theta/2}))
 * and "MAT"/"CMAT" (params = 8 doubles of an explicit U).  qubits: host, the
 * mnemonic's qubit operands in the paper's order (controls first). */
qs_status gate_std(const char* mnemonic, const int* qubits, int nqubits,
                   const double* params, int nparams, qs_gate* out);

/* ---- reductions (Sec. 2 probabilities; BEGIN MEASUREMENT, Appendix A) ----- */
/* The "norm" call: <Phi|Phi> = sum_i |a_i|^2 (Eq. (STAT1)), accumulated in
 * FP64 with compensation, in a fixed order (bit-stable run to run).  Named
 * sim_norm because the CUDA math library already exports a C function norm. */
qs_status sim_norm(qs_sim* sim, double* out);

/* BEGIN MEASUREMENT (Appendix A): for every qubit n = 0..N-1,
 * qx[n] = <(1 - sigma^x_n)>/2, qy[n] = <(1 - sigma^y_n)>/2,
 * qz[n] = <(1 - sigma^z_n)>/2, i.e. with w_n = sum_{bit n = 0} conj(a_i) a_{i+2^n}:
 * qx = <Phi|Phi>/2 - Re w_n, qy = <Phi|Phi>/2 - Im w_n, qz = P(qubit n = 1).
 * qx, qy, qz: host arrays of N doubles.  The state is unchanged.  Sums are
 * FP64 in a fixed order (FP32 leaf sums of at most 16 pairs per thread and
 * tile for complex64 and the adaptive words).  Returns QS_ETIMEOUT (outputs
 * undefined, the state unchanged) if a bounded wait of the complex64 kernel
 * for its tensor loads ran out. */
qs_status expect_xyz(qs_sim* sim, double* qx, double* qy, double* qz);

/* expect_xyz and sim_norm in one call: the same values (norm: sim_norm's
 * exact-product, compensated sum), from fewer sweeps of the state where the
 * kernels allow (complex64, N >= 23: one BEGIN MEASUREMENT pass also sums
 * |a|^2).  norm: host, one double.  Errors as expect_xyz. */
qs_status expect_xyz_norm(qs_sim* sim, double* qx, double* qy, double* qz, double* norm);

/* Overlap of two states of the same N on the same device, any encodings:
 * ov (host, 2 doubles) = <a|b> = sum_i conj(a_i) b_i as (re, im), and
 * *dist2 = ||a - b||^2 = sum_i |a_i - b_i|^2, both FP64 in a fixed order
 * (adaptive words decoded with their own (r0, r1)).  The fidelity of the two
 * states is |<a|b>|^2 / (<a|a> <b|b>).  The paper compares its two
 * simulators, double precision and the 2-byte encoding, on the same circuits
 * (Sec. 4.1, Tables 4-6); this is the device form of that comparison.  Runs on
 * a's stream after b's pending work; synchronises a's stream. */
qs_status sim_overlap(qs_sim* a, qs_sim* b, double* ov, double* dist2);

/* Marginal distribution of the nq qubits `qubits` (Sec. 2: the probability
 * of outcome 0/1 for a single qubit, generalised to a register):
 * out[k] = sum over basis states whose qubit qubits[m] equals bit m of k of
 * |a|^2, for k = 0..2^nq - 1 (1 <= nq <= 24).  out: host, 2^nq doubles. */
qs_status measure_probs(qs_sim* sim, const int* qubits, int nq, double* out);

/* As measure_probs, for a caller that cannot allocate device memory (its
 * memory is owned by another framework's pool, or it runs in a loop that must
 * not enter the driver's allocator).  The paper has no counterpart: this is a
 * calling convention of this library, not a step of the method.
 * state: device, the caller's 2^N amplitudes (QS_C128 or QS_C64 layout; other
 * encodings give QS_EUNSUPPORTED); qubits, out: host, as in measure_probs;
 * cuda_stream: the stream the work is ordered on (NULL = default stream).
 * Allocates nothing: the scratch is a fixed array of 2^18 + 2^16 doubles
 * (2.5 MiB) in the library's device memory, held by every GPU that loads the
 * library until the process exits, so nq is limited to 16 (larger gives
 * QS_EINVAL).  The first call on a device looks the array's address up on
 * that device; make it before any stream capture.  Every call shares the one
 * array, which keeps the last call's contents (each call writes every entry
 * it reads): calls that overlap on the GPU, on any streams, race and give
 * wrong results.  Synchronises cuda_stream before returning. */
qs_status measure_probs_static(const void* state, int N, qs_encoding enc, const int* qubits, int nq,
                               double* out, void* cuda_stream);

/* ---- stochastic instructions (Appendix A: M, CLEAR, SET, GENERATE EVENTS,
 *      DEPOLARIZING CHANNEL) ----------------------------------------------- */
/* Every random number is an argument: a uniform draw in [0, 1).  A caller
 * with a seed instead gets the draws from qs_uniforms (SplitMix64 of Steele,
 * Lea and Flood, OOPSLA 2014, evaluated at (seed, counter)), the generator
 * that generate_events_seeded and depolarize_circuit use. */

/* out[k] = uniform draw number first + k of `seed`: the top 53 bits of
 * SplitMix64's output for counter first + k, times 2^-53 (host only). */
qs_status qs_uniforms(uint64_t seed, uint64_t first, int64_t n, double* out);

/* M q (Appendix A): p0, p1 = probabilities of outcomes 0, 1 of qubit q (FP64
 * sums of |a|^2 over the two halves, Sec. 2); outcome = 0 if u (p0 + p1) <
 * p0, else 1 (inverse CDF over the outcomes); then the state is projected
 * onto the outcome and renormalised (multiplied by 1/sqrt(p_outcome)).
 * outcome (host int) and probs (host, 2 doubles: p0, p1) may be NULL.  u must
 * lie in [0, 1).  QS_EZEROPROJ for a state of zero norm.  QS_ADAPT2 states
 * re-encode with a re-tuned (r0, r1) (an arithmetic operation, Sec. 4.1).
 * Synchronises the stream (the outcome comes back to the host). */
qs_status measure_qubit(qs_sim* sim, int q, double u, int* outcome, double* probs);

/* CLEAR q (bit = 0) / SET q (bit = 1) (Appendix A): the projection
 * |bit><bit| on qubit q, renormalised.  prob (host, may be NULL) receives the
 * probability of `bit` before the projection.  If that probability is
 * exactly zero the projection would give a zero state: QS_EZEROPROJ, the
 * state unchanged (the failure the appendix prescribes).  Synchronises. */
qs_status project_qubit(qs_sim* sim, int q, int bit, double* prob);

/* GENERATE EVENTS (Appendix A): n basis states sampled from the
 * probabilities |a_i|^2 of the current state.  Event k is the smallest index
 * i with C_i > u[k] C_last, C_i = sum_{j <= i} |a_j|^2 (inverse CDF in index
 * order, FP64 sums in a fixed order); where rounding moves a target across a
 * boundary the event is the neighbouring index, and an index whose
 * amplitude is exactly zero is never drawn.  u: host, n draws in [0, 1);
 * events: host, n uint64 indices (bit q = qubit q).  1 <= n <= 2^31.  The
 * state is left unchanged (the appendix lets the simulator stop here).
 * Device scratch: about 2^(N-10) * 16 bytes plus 16 bytes per event.
 * Synchronises. */
qs_status generate_events(qs_sim* sim, const double* u, int64_t n, uint64_t* events);
/* The same with u[k] = qs_uniforms(seed, k) drawn on the device. */
qs_status generate_events_seeded(qs_sim* sim, uint64_t seed, int64_t n, uint64_t* events);

/* DEPOLARIZING CHANNEL P_X = px, P_Y = py, P_Z = pz, SEED = seed (Appendix
 * A), as a circuit transformation on the host: after gate g of `gates` and
 * for every qubit q, the draw r = qs_uniforms(seed, (first_gate + g) N + q)
 * inserts X (r < px), Y (px <= r < px + py), Z (px + py <= r < px + py + pz)
 * or nothing.  (first_gate numbers gates across successive calls.)  out:
 * host, room for cap records; *n_out receives the number of records the
 * noisy circuit has.  With out == NULL only *n_out is computed (QS_OK); with
 * a cap too small, QS_EINVAL.  Requires 0 <= px, py, pz and px + py + pz <= 1. */
qs_status depolarize_circuit(int N, const qs_gate* gates, int n, double px, double py, double pz,
                             uint64_t seed, int64_t first_gate, qs_gate* out, int cap, int* n_out);

/* ---- the instruction language of Appendix A (front-end) --------------------- */
/* A program is text, one instruction per line, '!' starting a comment, case
 * ignored: QUBITS N (first), BIT ASSIGNMENT p_0 .. p_{N-1}, the gate
 * mnemonics with their qubits then their numbers (the operand order of
 * gate_std: "U1 n lambda", "U c t k", "TOFFOLI c1 c2 t", ...; also RZ),
 * BEGIN MEASUREMENT, M n, CLEAR n, SET n, SHORBOX n_x G y, DEPOLARIZING
 * CHANNEL P_X = p, P_Y = p, P_Z = p, SEED = k (any order, any subset),
 * GENERATE EVENTS events [seed], EXIT.  The paper has no C interface; these
 * calls run its instruction list on a state handle. */
typedef struct qs_program qs_program;

/* Parse program text (host).  Errors: QS_EINVAL with the line number and the
 * reason in qs_last_error_string (unknown mnemonic, qubit out of range or
 * repeated, wrong operand count, QUBITS missing or not first, BIT ASSIGNMENT
 * not a permutation, probabilities out of range). */
qs_status program_parse(const char* text, qs_program** out);
qs_status program_destroy(qs_program* prog);
/* Number of qubits and of instructions after QUBITS. */
qs_status program_info(const qs_program* prog, int* N, int* n_instr);

/* Run the program on `sim` (same N; reset to |0..0> first).  Consecutive
 * gates run as one circuit_run in `mode` (QS_ADAPT2 states always per gate).
 * BIT ASSIGNMENT p: logical qubit k is stored in index bit p[k] from then on
 * (before any gate nothing moves; later the stored qubits are moved with
 * permute_qubits); every result is per logical qubit.  GENERATE EVENTS
 * first moves the qubits back to their own bits (the run ends there), so the
 * inverse CDF walks the logical index order and the events do not depend on
 * the renumbering.  Draws: M number m uses qs_uniforms(run_seed, m); GENERATE EVENTS n
 * s uses seed s, or run_seed + 1 when s <= 0 (the paper's "system value");
 * the depolarizing channel draws qs_uniforms(seed, g N + q) for gate
 * operation g of the program and logical qubit q, seed = SEED, or run_seed +
 * 2 when SEED <= 0.  GENERATE EVENTS and EXIT end the run (EXIT records one
 * BEGIN MEASUREMENT).  A CLEAR / SET with a zero projection returns
 * QS_EZEROPROJ.  Results stay in `prog` until the next run. */
qs_status program_run(qs_program* prog, qs_sim* sim, uint64_t run_seed, int mode);
/* Counts of the last run's results: BEGIN MEASUREMENT tables, M outcomes,
 * CLEAR / SET projections, events.  Outputs may be NULL. */
qs_status program_results(const qs_program* prog, int* n_measurements, int* n_m, int* n_proj, int64_t* n_events);
/* Table k (0-based) of BEGIN MEASUREMENT: qx, qy, qz (host, N doubles each). */
qs_status program_expectations(const qs_program* prog, int k, double* qx, double* qy, double* qz);
/* Per M in order: logical qubit, outcome, (p0, p1) before the projection;
 * per CLEAR / SET: the probability of the kept outcome.  Host arrays sized
 * by program_results; any may be NULL. */
qs_status program_outcomes(const qs_program* prog, int* qubits, int* outcomes, double* probs, double* proj_probs);
/* The events of GENERATE EVENTS (host, n_events uint64). */
qs_status program_events(const qs_program* prog, uint64_t* events);

/* Move the stored qubits: the content of index bit k goes to index bit
 * perm[k] (perm: host, a permutation of 0..N-1), i.e. amplitude i moves to
 * the index whose bit perm[k] is bit k of i.  In place, as transpositions of
 * bits (three CNOTs each, through the tile passes; bit-exact moves).  The
 * BIT ASSIGNMENT of Appendix A renumbers qubits this way (Sec. 3.2 motivates
 * it by the communication it saves). */
qs_status permute_qubits(qs_sim* sim, const int* perm);

/* ---- auxiliary-variable amplitudes (Sec. 4.2) ------------------------------- */
/* M amplitudes <z_m| C |0..0> of the circuit C without the 2^N state: every
 * CNOT, controlled phase U(k), controlled diagonal unitary and TOFFOLI is
 * rewritten into single-qubit gates and controlled phase shifts U_ct(a)
 * (Eq. (appa4); CNOT = H U(pi) H, TOFFOLI by the standard H / T / CNOT
 * decomposition), each U_ct(a) into a sum over one auxiliary variable
 * s = +-1 of single-qubit factors diag(e^{i th}, e^{-i th}) on c and t with
 * th = x s - a/4, cos 2x = e^{ia/2} (Eqs. (appa5), (appa6)); the amplitude is
 * 2^-P times the sum over all 2^P configurations of the product over qubits
 * of (W_j(s)|0>)(bit j of z) (Eq. (appa7)).  One device thread per
 * configuration, FP64, fixed-order sums (deterministic).  gates: host, n
 * records (single-qubit gates, or nc = 1 with an X or a diagonal unitary, or
 * nc = 2 with an X; others give QS_EUNSUPPORTED); basis: host, M indices
 * < 2^N (bit q = qubit q), 1 <= M <= 4096; out: host, 2M doubles (re, im);
 * *P_out (may be NULL) the number of auxiliary variables, at most 40 (more
 * gives QS_EINVAL).  N <= 63: the state is never formed.  Work grows as 2^P;
 * device memory: a few KB, allocated and freed on cuda_stream (NULL =
 * default stream).  Synchronises the stream. */
qs_status aux_amplitudes(int N, const qs_gate* gates, int n, const uint64_t* basis, int M, double* out,
                         int* P_out, void* cuda_stream);
/* The number P of auxiliary variables of a circuit (host only). */
qs_status aux_count(int N, const qs_gate* gates, int n, int* P);

/* ---- batched small states ------------------------------------------------- */
/* Many independent N-qubit states advanced through their own gate lists in
 * one launch (each gate is the pair update of Eq. (NUM2) / Eq. (AQS0); the
 * batching itself has no counterpart in the paper).  Every state is held in
 * on-chip shared memory for its whole gate list, so one launch reads and
 * writes each state once.  QS_C64 (2 <= N <= 14) or QS_C128 (2 <= N <= 13);
 * the states live in one device allocation owned by the handle, state s at
 * element offset s * 2^N, each starting as |0..0>. */
typedef struct qs_batch qs_batch;
qs_status batch_create(int N, qs_encoding enc, int nstates, void* cuda_stream, qs_batch** out);
qs_status batch_destroy(qs_batch* b);
/* Every state back to |0..0>. */
qs_status batch_reset(qs_batch* b);
/* Gate lists: state s runs gates[offsets[s] .. offsets[s+1]-1] (host arrays;
 * offsets has nstates + 1 non-decreasing entries starting at 0).  Validated
 * like circuit_run; copied to the device (the host arrays may be freed). */
qs_status batch_set_circuits(qs_batch* b, const qs_gate* gates, const int* offsets);
/* Advance every state through its gate list: one kernel launch, or the
 * captured CUDA graph when batch_capture was called. */
qs_status batch_run(qs_batch* b);
/* Capture one batch_run into a CUDA graph that later batch_run calls replay. */
qs_status batch_capture(qs_batch* b);
/* Time the launch layouts (one CTA per state, one warp per state for N <= 9)
 * and CTA sizes of the per-gate kernels, and the fused configurations of
 * batch_set_tuning (fusion width 1..4, 2^0..2^5 states per CTA, 128 / 256 /
 * 512 threads), on the current gate lists, and keep the fastest; the states
 * are restored afterwards.  layout (0 / 1 for the per-gate kernels, 2 for
 * the fused kernel), threads and the best time may be NULL;
 * batch_get_tuning reports the whole choice. */
qs_status batch_autotune(qs_batch* b, int* layout, int* threads, float* best_ms);
/* Kernel configuration of batch_run (the batching has no counterpart in the
 * paper).  fuse_k = 0: one shared-memory step per gate (the kernels of
 * batch_autotune's layouts: tile_bits = N gives one CTA per state, tile_bits
 * > N one warp per state); fuse_k = 1..4: each state's consecutive gates are
 * composed on the host in FP64 into dense blocks on at most fuse_k qubits (a
 * gate wider than fuse_k is its own block; the block's matrix is rounded
 * once to the state's precision, so results equal the gate-by-gate product
 * up to rounding) and applied as 2^m x 2^m products in shared memory, with
 * 2^(tile_bits - N) states per CTA (tile_bits from N to N + 5, every state
 * getting at least 32 threads, shared memory within 200 KB).  threads: the
 * CTA size.  Invalid combinations give QS_EINVAL.  batch_autotune times
 * these configurations as well and keeps the fastest. */
qs_status batch_set_tuning(qs_batch* b, int fuse_k, int tile_bits, int threads);
qs_status batch_get_tuning(const qs_batch* b, int* fuse_k, int* tile_bits, int* threads);
/* <Phi|Phi> of every state (host, nstates doubles), FP64. */
qs_status batch_norms(qs_batch* b, double* out);
/* Raw amplitudes of all states (nstates * 2^N * 8 or 16 bytes), host. */
qs_status batch_copy_out(qs_batch* b, void* host, size_t bytes);
qs_status batch_copy_in(qs_batch* b, const void* host, size_t bytes);
/* Current layout (0: CTA per state, 1: warp per state), CTA size and the
 * device address of the states. */
qs_status batch_info(const qs_batch* b, int* layout, int* threads, void** dev_states);

/* ---- serving loop ---------------------------------------------------------- */
/* A stream of requests (circuits of mixed qubit counts, complex64 storage,
 * FP64 results) served with continuous batching: the oldest waiting request
 * is admitted as soon as its state fits the device-memory budget (admission
 * by HBM footprint); every admitted request advances by up to `quantum` gates
 * per scheduling tick -- all small states (N <= small_max_n <= 14) together in
 * one launch that keeps each state on chip for its gate chunk, larger states
 * through the tile planner on their own streams, overlapping on the device;
 * finished requests are retired and their memory reused.  Each gate is the
 * pair update of Eq. (NUM2); serving has no counterpart in the paper. */
typedef struct {
  double arrival_s;       /* in: arrival, seconds after serve_run starts (non-decreasing) */
  int N;                  /* in: qubits, 2..34 */
  int ngates;             /* in */
  const qs_gate* gates;   /* in: host, ngates records, must stay valid during serve_run */
  double* qz;             /* out: host, N doubles: P(qubit n = 1) of the final state */
  double norm;            /* out: <Phi|Phi> of the final state (FP64) */
  double admit_s;         /* out: admission time (seconds after start) */
  double finish_s;        /* out: completion time (seconds after start) */
} qs_request;
typedef struct {
  size_t mem_budget;      /* bytes of device memory for resident states and gate lists */
  int quantum;            /* gates per request per tick / work item (<= 0: 64) */
  int max_small;          /* small states per batched launch (<= 0: 4096) */
  int nstreams;           /* streams for larger states (<= 0: 4, at most 16) */
  int small_max_n;        /* largest N of the batched path (<= 0: 14) */
  int persistent;         /* 1: persistent kernel and device work queue (below); 0: ticks */
  int persistent_ctas;    /* CTAs of the persistent kernel (<= 0: half the SMs) */
  double device_wait_ms;  /* longest wait of a persistent CTA for work (<= 0: 200 ms) */
  int large_quantum;      /* gates per chunk of a larger state (<= 0: quantum) */
} qs_serve_config;
typedef struct {
  int completed, ticks, max_active;
  double wall_s;          /* from start to the last completion */
  double busy_s;          /* time with at least one request active */
  uint64_t launches;      /* kernels launched */
  size_t peak_bytes;      /* peak pool usage */
  uint64_t work_items;    /* persistent mode: work items the device took from the queue */
  int idle_exits;         /* persistent mode: CTAs that ended a bounded wait without work */
  int relaunches;         /* persistent mode: launches of the persistent kernel */
} qs_serve_stats;
/* Serve n requests (sorted by arrival) in real time on the current device.
 * Rejects malformed requests and requests that cannot fit the budget before
 * anything runs.  Allocates the budget once (plus small staging buffers).
 *
 * Persistent mode (cfg->persistent = 1): the small states run in a
 * persistent kernel whose CTAs take work items (one state, its next chunk of
 * up to `quantum` gates) from a queue in host-mapped memory as the host
 * publishes them, each state held in shared memory for its chunk; every wait
 * of a CTA for work is bounded by device_wait_ms (%globaltimer), after which
 * the CTA ends (counted in idle_exits) and the host launches the kernel
 * again when new work arrives.  Larger states run their chunks of
 * large_quantum gates through the tile planner on their own streams, each
 * advanced as soon as its previous chunk completes (no global tick), so all
 * of this overlaps on the device.  The host gives up with QS_ETIMEOUT when
 * nothing completes for 60 s. */
qs_status serve_run(qs_request* reqs, int n, const qs_serve_config* cfg, qs_serve_stats* stats);

/* ---- raw state access (parity dumps) ------------------------------------- */
/* Copy the raw amplitudes (2^N * bytes-per-amplitude bytes, layout as in
 * qs_encoding) to / from host memory.  For QS_ADAPT2, r0r1 (host, 2 doubles,
 * may be NULL on copy_out) carries (r0, r1). */
qs_status sim_copy_out(qs_sim* sim, void* host, size_t bytes, double* r0r1);
qs_status sim_copy_in(qs_sim* sim, const void* host, size_t bytes, const double* r0r1);

/* Wait for every call enqueued on the handle's stream. */
qs_status sim_sync(qs_sim* sim);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
