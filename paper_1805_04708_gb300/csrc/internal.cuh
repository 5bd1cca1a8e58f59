// Internal declarations shared by the translation units of libqsim.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include "qsim.h"

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct qs_sim {
  int N;
  qs_encoding enc;
  cudaStream_t stream;
  void* state;        // device amplitudes
  size_t bytes;       // 2^N * bytes per amplitude
  bool owns;          // state allocated by the handle
  void* a2dev;        // ADAPT2: device A2Dev block (current and next magnitude range)
  void* scratch;      // device scratch for reductions and ADAPT2 range passes
  cudaEvent_t* evpool = nullptr;   // circuit_run_timed's per-pass events, kept between calls
  int evpool_n = 0;
  size_t scratch_bytes;
  void* hbuf;         // pinned host staging for results
  size_t hbuf_bytes;
  int device;
  int num_sms;
  int fused_engine;   // qs_fused_engine for apply_fused on complex64 states
  bool lazy_reset;    // reset leaves |0..0> pending (library-owned states, or
                      // borrowed ones whose owner asked for it)
  bool zero_pending;  // the state is |0..0> but not written yet: the first
                      // tile pass makes its tiles instead of loading them,
                      // every other call that touches the amplitudes writes
                      // them first
  bool product_start; // tile runs from a pending |0..0> start from
                      // the product state of their leading single-qubit gates
  int c128_df;        // 0: FP64 units; 1: double-float (FP32 pairs) in every gate kernel;
                      // 2: double-float in the per-gate sweeps, FP64 units in the tile passes
};
// Write a pending |0..0> (no-op otherwise).
qs_status materialize_state(qs_sim* s);

// error reporting ------------------------------------------------------------
void qs_set_error(const char* fmt, ...);
#define QS_CUDA(call)                                                         \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      qs_set_error("%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                 \
      return QS_ECUDA;                                                        \
    }                                                                         \
  } while (0)
void qs_count_launch(void);
#define QS_LAUNCH_CHECK()          \
  do {                             \
    qs_count_launch();             \
    QS_CUDA(cudaGetLastError());   \
  } while (0)
#define QS_TRY(x)                      \
  do {                                 \
    qs_status s_ = (x);                \
    if (s_ != QS_OK) return s_;        \
  } while (0)

static inline size_t qs_amp_bytes(qs_encoding e) {
  return e == QS_C128 ? 16 : (e == QS_C64 ? 8 : 2);
}

// ---------------------------------------------------------------------------
// gate classification (host)
// ---------------------------------------------------------------------------
#include "gatekind.h"
// Unit factors multiply exactly: 0 = 1, 1 = i, 2 = -1, 3 = -i, 4 = general.
struct GateClass {
  int kind;
  int c0, c1;        // unit codes of the two factors (diag: d0, d1; anti: f01, f10)
};
GateClass classify_u2(const double u[8]);
int unit_code(double re, double im);

// Unitarity check: max-abs of U U^dagger - 1 over a d x d matrix (row-major
// interleaved re, im).
double unitarity_defect(const double* U, int d);

// ---------------------------------------------------------------------------
// kernel launchers (each returns QS_OK or QS_ECUDA)
// ---------------------------------------------------------------------------
// Controlled 2x2 update on the dense encodings (C128 / C64).
qs_status launch_u2(qs_sim* s, const int* controls, int nc, int target, const double u[8]);
// Dense k-qubit gate (C128 / C64).
qs_status launch_fused_dense(qs_sim* s, const int* qubits, int k, const double* U);
// Dense k-qubit gate on the k lowest qubits of a complex64 state, on tensor
// cores (qubits: a permutation of 0..k-1, 2 <= k <= 5).
qs_status launch_fused_tc(qs_sim* s, const int* qubits, int k, const double* U);
// The same on tcgen05 tensor cores (3 <= k <= 5, N >= 12); eligibility test.
bool fused_tc05_eligible(const qs_sim* s, const int* qubits, int k);
qs_status launch_fused_tc05(qs_sim* s, const int* qubits, int k, const double* U);
// Real block form B (KR x KR, KR = 2^(k+1)) of U^T for the lowest-k-qubit
// tensor-core kernels.
void fused_block_matrix(const int* qubits, int k, const double* U, float* B);
// Register permutation (all encodings).
qs_status launch_permutation(qs_sim* s, const int* controls, int nc, int reg_lo, int reg_w,
                             const uint32_t* table);
qs_status launch_shorbox(qs_sim* s, int nx, uint64_t G, uint64_t y);
qs_status launch_reset(qs_sim* s);
// Reductions (all encodings); results on the host.
qs_status launch_norm(qs_sim* s, double* out);
qs_status launch_expect(qs_sim* s, double* qx, double* qy, double* qz);
qs_status launch_expect_norm(qs_sim* s, double* qx, double* qy, double* qz, double* norm);
qs_status launch_marginal(qs_sim* s, const int* qubits, int nq, double* out);
// P(qubit q = 0) and P(qubit q = 1) in one coalesced sweep (any encoding)
qs_status launch_qubit_probs(qs_sim* s, int q, double* p0, double* p1);

// Tile passes --------------------------------------------------------------------
// Optional per-launch timing: events ev[2i], ev[2i+1] around launch i.
struct PassTimer {
  cudaEvent_t* ev;
  int max_ev;
  int n;
};
// Number of tile bits used by the tile passes for an encoding.
int tile_bits(qs_encoding enc);
// Plan a gate list into tile passes and launch them (the product of the
// circuit is preserved).  jit: 0 the op interpreter; 1 per complex64 pass
// structure the fastest of the interpreter and the kernels compiled at run
// time (each timed once); 2 the compiled kernel (no barriers) for every
// complex64 pass.  jit 1 and 2 give QS_EUNSUPPORTED on a complex64 state when
// NVRTC cannot be loaded.
qs_status run_tile_passes(qs_sim* s, const qs_gate* gates, int n, int* n_passes, PassTimer* timer, int jit);
// Plan the complex64 passes of an N-qubit circuit and compile each (host
// only; the compiled kernels are cached for later launches): the kernel
// circuit_run mode 3 launches (all_passes) or every compiled candidate of
// mode 2.
qs_status compile_tile_passes(int N, const qs_gate* gates, int n, int* n_passes, bool all_passes);
// Product start of a run from |0..0>: number of gates it takes; factors (or
// null): 4 doubles per qubit, (U_q |0>)(0) and (U_q |0>)(1) as (re, im).
int product_start_factors(int N, const qs_gate* gates, int n, double* factors);
// The planner's pass order (host only): order gets the non-identity gate
// indices in the order the passes take them, pass_start the first position
// of each pass (both sized n by the caller).
qs_status plan_tile_pass_order(int N, qs_encoding enc, const qs_gate* gates, int n, int* order, int* pass_start,
                               int* n_passes);

// ADAPT2 --------------------------------------------------------------------------
// Device-resident range of the adaptive encoding (Sec. 4.1): the current
// (r0, r1) used to decode, and the min / max of |z| over 0 < |z| < 1 of the
// post-gate values, gathered by the range pass (float bit patterns, atomics).
struct A2Dev {
  double r0, r1;
  unsigned int mn, mx;
  unsigned int pad[2];
};
qs_status a2_set_range(qs_sim* s, double r0, double r1);
qs_status a2_get_range(qs_sim* s, double* r0, double* r1);
qs_status a2_apply_u2(qs_sim* s, const int* controls, int nc, int target, const double u[8]);
// The same update always through the arithmetic path (decode, apply, re-tune
// (r0, r1), encode), for non-unitary updates such as a scaled projection.
qs_status a2_apply_arith(qs_sim* s, const int* controls, int nc, int target, const double u[8]);
qs_status a2_norm(qs_sim* s, double* out);
qs_status a2_shorbox(qs_sim* s, int nx, uint64_t G, uint64_t y);
qs_status a2_reset(qs_sim* s);

// Spin limit of the pipeline waits of the tensor-core fused gate and of
// BEGIN MEASUREMENT (each spin suspends for at most about a microsecond); the
// drain waits of their exit paths keep the full limit.
uint32_t pipeline_wait_spins(void);

// Fixed-order compensated sum of n device doubles into *out (device).
qs_status sum_partials(qs_sim* s, const double* part, int n, double* out);

// scratch management
qs_status ensure_scratch(qs_sim* s, size_t bytes);
qs_status ensure_hbuf(qs_sim* s, size_t bytes);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
// Insert a zero bit at position b of x.
__device__ __forceinline__ uint64_t ins0(uint64_t x, int b) {
  uint64_t lo = x & ((1ull << b) - 1);
  return ((x >> b) << (b + 1)) | lo;
}
#endif
