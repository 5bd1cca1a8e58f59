// C ABI entry points (include/qsim.h): argument validation, handle
// management and dispatch to the kernels.  Every argument is checked on the
// host before anything is launched.
#include "internal.cuh"
#include "tile_jit.h"
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <new>

static thread_local char g_err[512] = "no error";

void qs_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

extern "C" const char* qs_last_error_string(void) { return g_err; }
extern "C" const char* qs_version(void) { return "qsim 0.1 sm_103a"; }

#include <atomic>
static std::atomic<uint64_t> g_launches{0};
void qs_count_launch(void) { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" uint64_t qs_kernel_launches(void) { return g_launches.load(); }

#define CHECK_ARG(cond, ...)            \
  do {                                  \
    if (!(cond)) {                      \
      qs_set_error(__VA_ARGS__);        \
      return QS_EINVAL;                 \
    }                                   \
  } while (0)

static qs_status check_sim(const qs_sim* s) {
  CHECK_ARG(s != nullptr, "null handle");
  return QS_OK;
}

static qs_status check_qubits(const qs_sim* s, const int* q, int n, const char* what) {
  CHECK_ARG(n == 0 || q != nullptr, "%s: null qubit list", what);
  for (int i = 0; i < n; ++i) {
    CHECK_ARG(q[i] >= 0 && q[i] < s->N, "%s: qubit %d out of range [0, %d)", what, q[i], s->N);
    for (int j = 0; j < i; ++j) CHECK_ARG(q[i] != q[j], "%s: qubit %d repeated", what, q[i]);
  }
  return QS_OK;
}

static qs_status init_handle(qs_sim* s, int N, qs_encoding enc, void* stream) {
  s->N = N;
  s->enc = enc;
  s->stream = (cudaStream_t)stream;
  s->a2dev = nullptr;
  s->scratch = nullptr;
  s->scratch_bytes = 0;
  s->hbuf = nullptr;
  s->hbuf_bytes = 0;
  s->fused_engine = QS_FUSED_AUTO;
  s->zero_pending = false;
  s->lazy_reset = false;
  s->product_start = true;
  s->c128_df = 1;
  QS_CUDA(cudaGetDevice(&s->device));
  QS_CUDA(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device));
  if (enc == QS_ADAPT2) QS_CUDA(cudaMalloc(&s->a2dev, sizeof(A2Dev)));
  return QS_OK;
}

// A lazy dense state is reset without a write: |0..0> is left to the first
// tile pass (which makes the tiles instead of loading them) or to
// materialize_state.  Other states are written at once (a caller's buffer
// may be read by its owner directly).
static qs_status do_reset(qs_sim* s) {
  if (s->enc == QS_ADAPT2) return a2_reset(s);
  if (s->lazy_reset) {
    s->zero_pending = true;
    return QS_OK;
  }
  s->zero_pending = false;
  return launch_reset(s);
}

qs_status materialize_state(qs_sim* s) {
  if (!s->zero_pending) return QS_OK;
  QS_TRY(launch_reset(s));
  s->zero_pending = false;
  return QS_OK;
}

extern "C" qs_status sim_create(int N, qs_encoding enc, void* cuda_stream, qs_sim** out) {
  CHECK_ARG(out != nullptr, "sim_create: null out");
  *out = nullptr;
  CHECK_ARG(N > 1 && N < 64, "sim_create: N = %d must satisfy 1 < N < 64", N);
  CHECK_ARG(enc == QS_C128 || enc == QS_C64 || enc == QS_ADAPT2, "sim_create: bad encoding %d", (int)enc);
  const size_t ab = qs_amp_bytes(enc);
  if (N > 44) { qs_set_error("sim_create: 2^%d amplitudes do not fit one GPU", N); return QS_ENOMEM; }
  const size_t bytes = ab << N;
  size_t freeb = 0, totalb = 0;
  QS_CUDA(cudaMemGetInfo(&freeb, &totalb));
  if (bytes + (64u << 20) > freeb) {
    qs_set_error("sim_create: %zu bytes requested, %zu free", bytes, freeb);
    return QS_ENOMEM;
  }
  qs_sim* s = new (std::nothrow) qs_sim;
  if (!s) return QS_ENOMEM;
  qs_status st = init_handle(s, N, enc, cuda_stream);
  if (st != QS_OK) { if (s->a2dev) cudaFree(s->a2dev); delete s; return st; }
  cudaError_t e = cudaMalloc(&s->state, bytes);
  if (e != cudaSuccess) {
    if (s->a2dev) cudaFree(s->a2dev);
    delete s;
    qs_set_error("sim_create: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    return QS_ENOMEM;
  }
  s->bytes = bytes;
  s->owns = true;
  s->lazy_reset = true;
  st = do_reset(s);
  if (st != QS_OK) { cudaFree(s->state); if (s->a2dev) cudaFree(s->a2dev); delete s; return st; }
  *out = s;
  return QS_OK;
}

extern "C" qs_status sim_create_in(int N, qs_encoding enc, void* dev_ptr, size_t bytes, void* cuda_stream,
                                   qs_sim** out) {
  CHECK_ARG(out != nullptr, "sim_create_in: null out");
  *out = nullptr;
  CHECK_ARG(N > 1 && N < 64, "sim_create_in: N = %d must satisfy 1 < N < 64", N);
  CHECK_ARG(enc == QS_C128 || enc == QS_C64 || enc == QS_ADAPT2, "sim_create_in: bad encoding %d", (int)enc);
  CHECK_ARG(N <= 44, "sim_create_in: N = %d too large", N);
  CHECK_ARG(dev_ptr != nullptr, "sim_create_in: null buffer");
  CHECK_ARG(((uintptr_t)dev_ptr & 255) == 0, "sim_create_in: buffer must be 256-byte aligned");
  const size_t need = qs_amp_bytes(enc) << N;
  CHECK_ARG(bytes >= need, "sim_create_in: buffer of %zu bytes, need %zu", bytes, need);
  qs_sim* s = new (std::nothrow) qs_sim;
  if (!s) return QS_ENOMEM;
  qs_status st = init_handle(s, N, enc, cuda_stream);
  if (st != QS_OK) { if (s->a2dev) cudaFree(s->a2dev); delete s; return st; }
  s->state = dev_ptr;
  s->bytes = need;
  s->owns = false;
  st = do_reset(s);
  if (st != QS_OK) { if (s->a2dev) cudaFree(s->a2dev); delete s; return st; }
  *out = s;
  return QS_OK;
}

extern "C" qs_status sim_destroy(qs_sim* s) {
  if (!s) return QS_OK;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (s->scratch) cudaFree(s->scratch);
  if (s->hbuf) cudaFreeHost(s->hbuf);
  if (s->owns && s->state) cudaFree(s->state);
  if (s->a2dev) cudaFree(s->a2dev);
  for (int i = 0; i < s->evpool_n; ++i) cudaEventDestroy(s->evpool[i]);
  free(s->evpool);
  delete s;
  if (e != cudaSuccess) {
    qs_set_error("sim_destroy: %s", cudaGetErrorString(e));
    return QS_ECUDA;
  }
  return QS_OK;
}

extern "C" qs_status sim_info(const qs_sim* s, int* N, int* enc, void** dev_ptr, size_t* bytes) {
  QS_TRY(check_sim(s));
  // the caller may read the amplitudes through the pointer
  if (dev_ptr) QS_TRY(materialize_state(const_cast<qs_sim*>(s)));
  if (N) *N = s->N;
  if (enc) *enc = (int)s->enc;
  if (dev_ptr) *dev_ptr = s->state;
  if (bytes) *bytes = s->bytes;
  return QS_OK;
}

extern "C" qs_status sim_reset(qs_sim* s) {
  QS_TRY(check_sim(s));
  return do_reset(s);
}

extern "C" qs_status sim_set_lazy_reset(qs_sim* s, int on) {
  QS_TRY(check_sim(s));
  if (!on) QS_TRY(materialize_state(s));
  s->lazy_reset = on != 0;
  return QS_OK;
}

extern "C" qs_status sim_set_product_start(qs_sim* s, int on) {
  QS_TRY(check_sim(s));
  s->product_start = on != 0;
  return QS_OK;
}

static std::atomic<uint32_t> g_pipe_spins{1u << 20};
uint32_t pipeline_wait_spins(void) { return g_pipe_spins.load(); }

extern "C" qs_status qs_set_pipeline_wait_limit(int64_t us) {
  CHECK_ARG(us >= -1, "qs_set_pipeline_wait_limit: us = %lld", (long long)us);
  g_pipe_spins.store(us < 0 ? (1u << 20) : (uint32_t)(us > (1ll << 30) ? (1ll << 30) : us));
  return QS_OK;
}

extern "C" qs_status sim_set_fp64_emulation(qs_sim* s, int on) {
  QS_TRY(check_sim(s));
  CHECK_ARG(on >= 0 && on <= 2, "sim_set_fp64_emulation: %d not in 0..2", on);
  s->c128_df = on;
  return QS_OK;
}

extern "C" qs_status sim_sync(qs_sim* s) {
  QS_TRY(check_sim(s));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}

// ---- gates ------------------------------------------------------------------------
static qs_status check_u2(const double* U) {
  CHECK_ARG(U != nullptr, "null matrix");
  for (int i = 0; i < 8; ++i) CHECK_ARG(isfinite(U[i]), "matrix entry %d is not finite", i);
  double d = unitarity_defect(U, 2);
  if (!(d <= 1e-10)) {
    qs_set_error("matrix is not unitary (defect %.3g > 1e-10)", d);
    return QS_ENOTUNITARY;
  }
  return QS_OK;
}

static qs_status apply_u2_checked(qs_sim* s, const int* controls, int nc, int target, const double* U) {
  if (s->enc == QS_ADAPT2) return a2_apply_u2(s, controls, nc, target, U);
  QS_TRY(materialize_state(s));
  return launch_u2(s, controls, nc, target, U);
}

extern "C" qs_status apply_gate(qs_sim* s, int target, const double U[8]) {
  QS_TRY(check_sim(s));
  QS_TRY(check_qubits(s, &target, 1, "apply_gate"));
  QS_TRY(check_u2(U));
  return apply_u2_checked(s, nullptr, 0, target, U);
}

extern "C" qs_status apply_controlled(qs_sim* s, const int* controls, int nc, int target, const double U[8]) {
  QS_TRY(check_sim(s));
  CHECK_ARG(nc >= 0 && nc <= 2, "apply_controlled: nc = %d not in {0,1,2}", nc);
  int q[3];
  for (int i = 0; i < nc; ++i) {
    CHECK_ARG(controls != nullptr, "apply_controlled: null controls");
    q[i] = controls[i];
  }
  q[nc] = target;
  QS_TRY(check_qubits(s, q, nc + 1, "apply_controlled"));
  QS_TRY(check_u2(U));
  return apply_u2_checked(s, controls, nc, target, U);
}

extern "C" qs_status apply_fused(qs_sim* s, const int* qubits, int k, const double* U) {
  QS_TRY(check_sim(s));
  CHECK_ARG(k >= 1 && k <= 5, "apply_fused: k = %d not in 1..5", k);
  QS_TRY(check_qubits(s, qubits, k, "apply_fused"));
  CHECK_ARG(U != nullptr, "apply_fused: null matrix");
  const int d = 1 << k;
  for (int i = 0; i < 2 * d * d; ++i) CHECK_ARG(isfinite(U[i]), "apply_fused: entry %d not finite", i);
  double def = unitarity_defect(U, d);
  if (!(def <= 1e-10)) {
    qs_set_error("apply_fused: matrix is not unitary (defect %.3g)", def);
    return QS_ENOTUNITARY;
  }
  if (s->enc == QS_ADAPT2) { qs_set_error("apply_fused: not available for QS_ADAPT2"); return QS_EUNSUPPORTED; }
  QS_TRY(materialize_state(s));
  return launch_fused_dense(s, qubits, k, U);
}

extern "C" qs_status sim_set_fused_engine(qs_sim* s, int engine) {
  QS_TRY(check_sim(s));
  CHECK_ARG(engine == QS_FUSED_AUTO || engine == QS_FUSED_CUDA_CORES || engine == QS_FUSED_MMA_SYNC,
            "sim_set_fused_engine: unknown engine %d", engine);
  s->fused_engine = engine;
  return QS_OK;
}

extern "C" qs_status modmul_table(uint64_t a, uint64_t G, int width, uint32_t* table) {
  CHECK_ARG(table != nullptr, "modmul_table: null table");
  CHECK_ARG(width >= 1 && width <= 24, "modmul_table: width %d not in 1..24", width);
  CHECK_ARG(G >= 2 && G <= (1ull << width), "modmul_table: G out of range");
  uint64_t x = a % G, y = G;
  while (y) { uint64_t t = x % y; x = y; y = t; }
  CHECK_ARG(x == 1, "modmul_table: gcd(a, G) != 1");
  for (uint64_t f = 0; f < (1ull << width); ++f) table[f] = (uint32_t)(f < G ? ((a % G) * f) % G : f);
  return QS_OK;
}

extern "C" qs_status apply_permutation(qs_sim* s, const int* controls, int nc, int reg_lo, int reg_w,
                                       const uint32_t* table) {
  QS_TRY(check_sim(s));
  CHECK_ARG(reg_w >= 1 && reg_w <= 12, "apply_permutation: reg_w = %d not in 1..12", reg_w);
  CHECK_ARG(reg_lo >= 0 && reg_lo + reg_w <= s->N, "apply_permutation: register out of range");
  CHECK_ARG(nc >= 0 && nc <= 8, "apply_permutation: nc = %d not in 0..8", nc);
  CHECK_ARG(table != nullptr, "apply_permutation: null table");
  QS_TRY(check_qubits(s, controls, nc, "apply_permutation"));
  for (int i = 0; i < nc; ++i)
    CHECK_ARG(controls[i] < reg_lo || controls[i] >= reg_lo + reg_w, "apply_permutation: control %d inside register",
              controls[i]);
  const size_t W = (size_t)1 << reg_w;
  unsigned char* seen = (unsigned char*)calloc(W, 1);
  if (!seen) return QS_ENOMEM;
  for (size_t i = 0; i < W; ++i) {
    if (table[i] >= W || seen[table[i]]) {
      free(seen);
      qs_set_error("apply_permutation: table is not a bijection on [0, %zu)", W);
      return QS_ENOTBIJECTIVE;
    }
    seen[table[i]] = 1;
  }
  free(seen);
  QS_TRY(materialize_state(s));
  return launch_permutation(s, controls, nc, reg_lo, reg_w, table);
}

extern "C" qs_status shorbox_init(qs_sim* s, int nx, uint64_t G, uint64_t y) {
  QS_TRY(check_sim(s));
  CHECK_ARG(nx >= 1 && nx < s->N, "shorbox_init: nx = %d not in 1..N-1", nx);
  CHECK_ARG(G >= 2 && G <= (1ull << (s->N - nx)) && G < (1ull << 32), "shorbox_init: G out of range");
  CHECK_ARG(y >= 1 && y < G, "shorbox_init: y out of range");
  s->zero_pending = false;   // every amplitude is written
  return (s->enc == QS_ADAPT2) ? a2_shorbox(s, nx, G, y) : launch_shorbox(s, nx, G, y);
}

// ---- circuits -----------------------------------------------------------------------
static qs_status check_gate(const qs_sim* s, const qs_gate& g) {
  CHECK_ARG(g.nc >= 0 && g.nc <= 2, "gate: nc = %d", g.nc);
  int q[3];
  for (int i = 0; i < g.nc; ++i) q[i] = g.controls[i];
  q[g.nc] = g.target;
  QS_TRY(check_qubits(s, q, g.nc + 1, "circuit_run"));
  QS_TRY(check_u2(g.u));
  return QS_OK;
}

// Runs the gate list; when ev is non-null, records an event pair around each
// sweep (ev[2*i], ev[2*i+1]) for the first max_ev sweeps.
static qs_status run_gates(qs_sim* s, const qs_gate* gates, int n, int mode, int* n_passes, cudaEvent_t* ev,
                           int max_ev) {
  QS_TRY(check_sim(s));
  CHECK_ARG(n >= 0 && (n == 0 || gates != nullptr), "circuit_run: bad gate list");
  CHECK_ARG(mode >= 0 && mode <= 3, "circuit_run: mode %d", mode);
  for (int i = 0; i < n; ++i) QS_TRY(check_gate(s, gates[i]));
  int passes = 0;
  PassTimer timer = {ev, max_ev, 0};
  if (mode == 0 || s->enc == QS_ADAPT2 || s->N < tile_bits(s->enc)) {
    for (int i = 0; i < n; ++i) {
      const qs_gate& g = gates[i];
      if (classify_u2(g.u).kind == GK_IDENT) continue;
      const bool timed = ev && timer.n < max_ev;
      if (timed) QS_CUDA(cudaEventRecord(ev[2 * timer.n], s->stream));
      QS_TRY(apply_u2_checked(s, g.controls, g.nc, g.target, g.u));
      if (timed) QS_CUDA(cudaEventRecord(ev[2 * timer.n + 1], s->stream));
      timer.n++;
      ++passes;
    }
  } else {
    const int jit = mode == 2 ? 1 : (mode == 3 ? 2 : 0);
    QS_TRY(run_tile_passes(s, gates, n, &passes, ev ? &timer : nullptr, jit));
  }
  if (n_passes) *n_passes = passes;
  return QS_OK;
}

extern "C" qs_status circuit_compile(int N, const qs_gate* gates, int n, int mode, int* n_passes) {
  CHECK_ARG(mode == 2 || mode == 3, "circuit_compile: mode %d (2 or 3)", mode);
  CHECK_ARG(N >= tile_bits(QS_C64) && N < 64, "circuit_compile: N = %d must be in %d..63", N, tile_bits(QS_C64));
  CHECK_ARG(n >= 0 && (n == 0 || gates != nullptr), "circuit_compile: bad gate list");
  qs_sim probe;
  probe.N = N;
  probe.enc = QS_C64;
  for (int i = 0; i < n; ++i) QS_TRY(check_gate(&probe, gates[i]));
  if (!tile_jit_available()) {
    qs_set_error("circuit_compile: NVRTC could not be loaded");
    return QS_EUNSUPPORTED;
  }
  return compile_tile_passes(N, gates, n, n_passes, mode == 3);
}

extern "C" qs_status circuit_product_start(int N, const qs_gate* gates, int n, int* n_prefix, double* factors) {
  CHECK_ARG(N >= 1 && N < 64, "circuit_product_start: N = %d must be in 1..63", N);
  CHECK_ARG(n >= 0 && (n == 0 || gates != nullptr), "circuit_product_start: bad gate list");
  CHECK_ARG(n_prefix != nullptr, "circuit_product_start: null n_prefix");
  qs_sim probe;
  probe.N = N;
  probe.enc = QS_C64;
  for (int i = 0; i < n; ++i) QS_TRY(check_gate(&probe, gates[i]));
  *n_prefix = product_start_factors(N, gates, n, factors);
  return QS_OK;
}

extern "C" qs_status circuit_plan(int N, int enc, const qs_gate* gates, int n, int* order, int* pass_start,
                                  int* n_passes) {
  CHECK_ARG(enc == QS_C128 || enc == QS_C64, "circuit_plan: encoding %d has no tile passes", enc);
  CHECK_ARG(N >= tile_bits((qs_encoding)enc) && N < 64, "circuit_plan: N = %d below the tile size", N);
  CHECK_ARG(n >= 0 && (n == 0 || gates != nullptr), "circuit_plan: bad gate list");
  CHECK_ARG(order != nullptr && pass_start != nullptr && n_passes != nullptr, "circuit_plan: null output");
  qs_sim probe;
  probe.N = N;
  probe.enc = (qs_encoding)enc;
  for (int i = 0; i < n; ++i) QS_TRY(check_gate(&probe, gates[i]));
  return plan_tile_pass_order(N, (qs_encoding)enc, gates, n, order, pass_start, n_passes);
}

extern "C" qs_status tile_compiler_info(int* available, long* compiles) {
  if (available) *available = tile_jit_available() ? 1 : 0;
  if (compiles) *compiles = tile_jit_compiles();
  return QS_OK;
}

extern "C" qs_status circuit_run(qs_sim* s, const qs_gate* gates, int n, int mode, int* n_passes) {
  return run_gates(s, gates, n, mode, n_passes, nullptr, 0);
}

extern "C" qs_status circuit_run_timed(qs_sim* s, const qs_gate* gates, int n, int mode, int* n_passes,
                                       float* pass_ms, int max_passes) {
  QS_TRY(check_sim(s));
  CHECK_ARG(max_passes >= 0 && max_passes <= 65536, "circuit_run_timed: max_passes");
  // the events stay with the handle between calls (creating them is host
  // work that would otherwise sit between the kernels of every call)
  cudaEvent_t* ev = nullptr;
  int nev = max_passes;
  if (pass_ms && nev > 0) {
    if (s->evpool_n < 2 * nev) {
      cudaEvent_t* p = (cudaEvent_t*)realloc(s->evpool, sizeof(cudaEvent_t) * (size_t)2 * nev);
      if (!p) return QS_ENOMEM;
      s->evpool = p;
      for (; s->evpool_n < 2 * nev; ++s->evpool_n)
        if (cudaEventCreate(&s->evpool[s->evpool_n]) != cudaSuccess) {
          qs_set_error("circuit_run_timed: cudaEventCreate failed");
          return QS_ECUDA;
        }
    }
    ev = s->evpool;
  }
  int np = 0;
  qs_status st = run_gates(s, gates, n, mode, &np, ev, nev);
  if (st == QS_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) {
    qs_set_error("circuit_run_timed: stream synchronize failed");
    st = QS_ECUDA;
  }
  if (ev) {
    for (int i = 0; st == QS_OK && i < np && i < nev; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) {
        qs_set_error("circuit_run_timed: event timing failed");
        st = QS_ECUDA;
      }
      pass_ms[i] = ms;
    }
  }
  if (n_passes) *n_passes = np;
  return st;
}

// ---- reductions ------------------------------------------------------------------------
extern "C" qs_status sim_norm(qs_sim* s, double* out) {
  QS_TRY(check_sim(s));
  CHECK_ARG(out != nullptr, "sim_norm: null out");
  QS_TRY(materialize_state(s));
  return (s->enc == QS_ADAPT2) ? a2_norm(s, out) : launch_norm(s, out);
}

extern "C" qs_status expect_xyz(qs_sim* s, double* qx, double* qy, double* qz) {
  QS_TRY(check_sim(s));
  CHECK_ARG(qx && qy && qz, "expect_xyz: null output");
  QS_TRY(materialize_state(s));
  return launch_expect(s, qx, qy, qz);
}

extern "C" qs_status expect_xyz_norm(qs_sim* s, double* qx, double* qy, double* qz, double* norm) {
  QS_TRY(check_sim(s));
  CHECK_ARG(qx && qy && qz && norm, "expect_xyz_norm: null output");
  QS_TRY(materialize_state(s));
  return launch_expect_norm(s, qx, qy, qz, norm);
}

extern "C" qs_status measure_probs(qs_sim* s, const int* qubits, int nq, double* out) {
  QS_TRY(check_sim(s));
  CHECK_ARG(nq >= 1 && nq <= 24 && nq <= s->N, "measure_probs: nq = %d not in 1..min(24, N)", nq);
  CHECK_ARG(out != nullptr, "measure_probs: null out");
  QS_TRY(check_qubits(s, qubits, nq, "measure_probs"));
  QS_TRY(materialize_state(s));
  return launch_marginal(s, qubits, nq, out);
}

// ---- raw access --------------------------------------------------------------------------
extern "C" qs_status sim_copy_out(qs_sim* s, void* host, size_t bytes, double* r0r1) {
  QS_TRY(check_sim(s));
  CHECK_ARG(host != nullptr && bytes == s->bytes, "sim_copy_out: need %zu bytes", s->bytes);
  QS_TRY(materialize_state(s));
  QS_CUDA(cudaMemcpyAsync(host, s->state, bytes, cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  if (r0r1) {
    r0r1[0] = r0r1[1] = 0.0;
    if (s->enc == QS_ADAPT2) QS_TRY(a2_get_range(s, &r0r1[0], &r0r1[1]));
  }
  return QS_OK;
}

extern "C" qs_status sim_copy_in(qs_sim* s, const void* host, size_t bytes, const double* r0r1) {
  QS_TRY(check_sim(s));
  CHECK_ARG(host != nullptr && bytes == s->bytes, "sim_copy_in: need %zu bytes", s->bytes);
  if (s->enc == QS_ADAPT2) {
    CHECK_ARG(r0r1 != nullptr, "sim_copy_in: ADAPT2 needs (r0, r1)");
    CHECK_ARG(r0r1[0] >= 0 && r0r1[1] >= r0r1[0] && r0r1[1] < 1.0, "sim_copy_in: need 0 <= r0 <= r1 < 1");
    QS_TRY(a2_set_range(s, r0r1[0], r0r1[1]));
  }
  s->zero_pending = false;   // every amplitude is written
  QS_CUDA(cudaMemcpyAsync(s->state, host, bytes, cudaMemcpyHostToDevice, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}
