// Batched small states: many independent N-qubit states (N <= 14 for
// complex64, N <= 13 for complex128) advance through their own gate lists in
// one launch.  Each state is held in shared memory for the whole gate list,
// so one launch reads and writes every state once, whatever the number of
// gates (the pair update of Eq. (NUM2) for every gate, applied in shared
// memory).  Two layouts: one CTA per state (larger N) or one warp per state
// (N <= 9, several states per CTA); the autotuner times both and a few CTA
// sizes and keeps the fastest.  A run can be captured once in a CUDA graph
// and replayed.
#include "internal.cuh"
#include "cplx.cuh"
#include "batch_common.cuh"
#include <stdlib.h>
#include <string.h>
#include <new>

namespace {

// One CTA per state.
template <typename R>
__global__ void k_batch_cta(Cx<R>* __restrict__ states, int N, const BGate<R>* __restrict__ gates,
                            const int* __restrict__ offs, int nstates) {
  extern __shared__ unsigned char smraw[];
  Cx<R>* st = (Cx<R>*)smraw;
  const int s = blockIdx.x;
  if (s >= nstates) return;
  const int n = 1 << N;
  Cx<R>* gs = states + (size_t)s * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) st[i] = gs[i];
  __syncthreads();
  for (int k = offs[s]; k < offs[s + 1]; ++k) {
    apply_gate_range<R>(st, N, gates[k], threadIdx.x, blockDim.x);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) gs[i] = st[i];
}

// One warp per state (small N).
template <typename R>
__global__ void k_batch_warp(Cx<R>* __restrict__ states, int N, const BGate<R>* __restrict__ gates,
                             const int* __restrict__ offs, int nstates) {
  extern __shared__ unsigned char smraw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * (blockDim.x >> 5) + w;
  const int n = 1 << N;
  Cx<R>* st = (Cx<R>*)smraw + (size_t)w * n;
  if (s >= nstates) return;   // the whole warp leaves together
  Cx<R>* gs = states + (size_t)s * n;
  for (int i = lane; i < n; i += 32) st[i] = gs[i];
  __syncwarp();
  for (int k = offs[s]; k < offs[s + 1]; ++k) {
    apply_gate_range<R>(st, N, gates[k], lane, 32);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) gs[i] = st[i];
}

template <typename R>
__global__ void k_batch_reset(Cx<R>* __restrict__ states, uint64_t n_total, int N) {
  const uint64_t mask = (1ull << N) - 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_total; i += (uint64_t)gridDim.x * blockDim.x)
    states[i] = cx<R>((i & mask) == 0 ? (R)1 : (R)0, (R)0);
}

// sum |a|^2 per state, FP64, one CTA per state, fixed order
template <typename R>
__global__ void k_batch_norms(const Cx<R>* __restrict__ states, int N, double* out) {
  __shared__ double sh[32];
  const int s = blockIdx.x;
  const int n = 1 << N;
  const Cx<R>* gs = states + (size_t)s * n;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += (double)gs[i].x * gs[i].x + (double)gs[i].y * gs[i].y;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    out[s] = r;
  }
}

}  // namespace

struct qs_batch {  // opaque to callers (include/qsim.h)
  int N, nstates;
  qs_encoding enc;
  cudaStream_t stream;
  void* states;          // nstates * 2^N amplitudes, state s at offset s * 2^N
  size_t bytes;
  void* gates;           // device BGate<R> array
  int* offs;             // device, nstates + 1
  int ngates;
  int layout;            // 0: CTA per state, 1: warp per state
  int threads;           // CTA size
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  double* dnorm;
};

static size_t amp_bytes(qs_encoding e) { return e == QS_C128 ? 16 : 8; }

extern "C" qs_status batch_create(int N, qs_encoding enc, int nstates, void* cuda_stream, qs_batch** out) {
  if (!out) { qs_set_error("batch_create: null out"); return QS_EINVAL; }
  *out = nullptr;
  if (enc != QS_C64 && enc != QS_C128) { qs_set_error("batch_create: encoding must be QS_C64 or QS_C128"); return QS_EUNSUPPORTED; }
  const int nmax = (enc == QS_C64) ? 14 : 13;
  if (N < 2 || N > nmax) { qs_set_error("batch_create: N = %d not in 2..%d", N, nmax); return QS_EINVAL; }
  if (nstates < 1 || nstates > (1 << 24)) { qs_set_error("batch_create: nstates = %d", nstates); return QS_EINVAL; }
  qs_batch* b = new (std::nothrow) qs_batch;
  if (!b) return QS_ENOMEM;
  memset(b, 0, sizeof *b);
  b->N = N; b->nstates = nstates; b->enc = enc; b->stream = (cudaStream_t)cuda_stream;
  b->bytes = ((size_t)nstates << N) * amp_bytes(enc);
  b->layout = (N <= 9) ? 1 : 0;
  b->threads = 256;
  cudaError_t e = cudaMalloc(&b->states, b->bytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->offs, sizeof(int) * (size_t)(nstates + 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->dnorm, sizeof(double) * (size_t)nstates);
  if (e != cudaSuccess) {
    if (b->states) cudaFree(b->states);
    if (b->offs) cudaFree(b->offs);
    delete b;
    qs_set_error("batch_create: %s", cudaGetErrorString(e));
    return QS_ENOMEM;
  }
  QS_CUDA(cudaMemsetAsync(b->offs, 0, sizeof(int) * (size_t)(nstates + 1), b->stream));
  *out = b;
  return batch_reset(b);
}

extern "C" qs_status batch_destroy(qs_batch* b) {
  if (!b) return QS_OK;
  cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->states);
  cudaFree(b->offs);
  if (b->gates) cudaFree(b->gates);
  cudaFree(b->dnorm);
  delete b;
  return QS_OK;
}

extern "C" qs_status batch_reset(qs_batch* b) {
  if (!b) { qs_set_error("batch_reset: null"); return QS_EINVAL; }
  const uint64_t n = (uint64_t)b->nstates << b->N;
  const unsigned grid = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (b->enc == QS_C64) k_batch_reset<float><<<grid, 256, 0, b->stream>>>((Cx<float>*)b->states, n, b->N);
  else k_batch_reset<double><<<grid, 256, 0, b->stream>>>((Cx<double>*)b->states, n, b->N);
  QS_LAUNCH_CHECK();
  return QS_OK;
}

extern "C" qs_status batch_set_circuits(qs_batch* b, const qs_gate* gates, const int* offsets) {
  if (!b || !offsets || (offsets[b->nstates] > 0 && !gates)) { qs_set_error("batch_set_circuits: null argument"); return QS_EINVAL; }
  if (offsets[0] != 0) { qs_set_error("batch_set_circuits: offsets[0] must be 0"); return QS_EINVAL; }
  for (int s = 0; s < b->nstates; ++s)
    if (offsets[s + 1] < offsets[s]) { qs_set_error("batch_set_circuits: offsets must not decrease"); return QS_EINVAL; }
  const int ng = offsets[b->nstates];
  for (int k = 0; k < ng; ++k) {
    const qs_gate& g = gates[k];
    if (g.nc < 0 || g.nc > 2) { qs_set_error("batch_set_circuits: gate %d: nc = %d", k, g.nc); return QS_EINVAL; }
    int q[3] = {g.controls[0], g.controls[1], g.target};
    q[g.nc] = g.target;
    for (int i = 0; i <= g.nc; ++i) {
      if (q[i] < 0 || q[i] >= b->N) { qs_set_error("batch_set_circuits: gate %d: qubit %d out of range", k, q[i]); return QS_EINVAL; }
      for (int j = 0; j < i; ++j)
        if (q[i] == q[j]) { qs_set_error("batch_set_circuits: gate %d: qubit %d repeated", k, q[i]); return QS_EINVAL; }
    }
    double d = unitarity_defect(g.u, 2);
    if (!(d <= 1e-10)) { qs_set_error("batch_set_circuits: gate %d not unitary", k); return QS_ENOTUNITARY; }
  }
  const size_t gsz = (b->enc == QS_C64) ? sizeof(BGate<float>) : sizeof(BGate<double>);
  void* host = malloc(gsz * (size_t)(ng > 0 ? ng : 1));
  if (!host) return QS_ENOMEM;
  for (int k = 0; k < ng; ++k) {
    const qs_gate& g = gates[k];
    if (b->enc == QS_C64) {
      BGate<float>& o = ((BGate<float>*)host)[k];
      o.nc = g.nc; o.c0 = g.controls[0]; o.c1 = g.controls[1]; o.t = g.target;
      for (int i = 0; i < 8; ++i) o.u[i] = (float)g.u[i];
    } else {
      BGate<double>& o = ((BGate<double>*)host)[k];
      o.nc = g.nc; o.c0 = g.controls[0]; o.c1 = g.controls[1]; o.t = g.target;
      for (int i = 0; i < 8; ++i) o.u[i] = g.u[i];
    }
  }
  if (b->gates) { cudaFree(b->gates); b->gates = nullptr; }
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  cudaError_t e = cudaMalloc(&b->gates, gsz * (size_t)(ng > 0 ? ng : 1));
  if (e != cudaSuccess) { free(host); qs_set_error("batch_set_circuits: %s", cudaGetErrorString(e)); return QS_ENOMEM; }
  e = cudaMemcpyAsync(b->gates, host, gsz * (size_t)ng, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->offs, offsets, sizeof(int) * (size_t)(b->nstates + 1), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  free(host);
  if (e != cudaSuccess) { qs_set_error("batch_set_circuits: %s", cudaGetErrorString(e)); return QS_ECUDA; }
  b->ngates = ng;
  return QS_OK;
}

static qs_status launch_batch(qs_batch* b, int layout, int threads) {
  const size_t ab = amp_bytes(b->enc);
  if (layout == 0) {
    const size_t smem = ab << b->N;
    if (b->enc == QS_C64) {
      QS_CUDA(cudaFuncSetAttribute(k_batch_cta<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_batch_cta<float><<<b->nstates, threads, smem, b->stream>>>((Cx<float>*)b->states, b->N,
                                                                   (const BGate<float>*)b->gates, b->offs, b->nstates);
    } else {
      QS_CUDA(cudaFuncSetAttribute(k_batch_cta<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_batch_cta<double><<<b->nstates, threads, smem, b->stream>>>((Cx<double>*)b->states, b->N,
                                                                    (const BGate<double>*)b->gates, b->offs, b->nstates);
    }
  } else {
    const int wpb = threads / 32;
    const size_t smem = (ab << b->N) * (size_t)wpb;
    const unsigned grid = (unsigned)((b->nstates + wpb - 1) / wpb);
    if (b->enc == QS_C64) {
      QS_CUDA(cudaFuncSetAttribute(k_batch_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_batch_warp<float><<<grid, threads, smem, b->stream>>>((Cx<float>*)b->states, b->N,
                                                              (const BGate<float>*)b->gates, b->offs, b->nstates);
    } else {
      QS_CUDA(cudaFuncSetAttribute(k_batch_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_batch_warp<double><<<grid, threads, smem, b->stream>>>((Cx<double>*)b->states, b->N,
                                                               (const BGate<double>*)b->gates, b->offs, b->nstates);
    }
  }
  QS_LAUNCH_CHECK();
  return QS_OK;
}

static bool layout_ok(const qs_batch* b, int layout, int threads) {
  const size_t ab = amp_bytes(b->enc);
  if (layout == 1) return b->N <= 9 && (ab << b->N) * (size_t)(threads / 32) <= 200 * 1024;
  return (ab << b->N) <= 200 * 1024;
}

extern "C" qs_status batch_run(qs_batch* b) {
  if (!b) { qs_set_error("batch_run: null"); return QS_EINVAL; }
  if (!b->gates) return QS_OK;
  if (b->gexec) {
    QS_CUDA(cudaGraphLaunch(b->gexec, b->stream));
    return QS_OK;
  }
  return launch_batch(b, b->layout, b->threads);
}

extern "C" qs_status batch_capture(qs_batch* b) {
  if (!b) { qs_set_error("batch_capture: null"); return QS_EINVAL; }
  if (!b->gates) { qs_set_error("batch_capture: no circuits set"); return QS_EINVAL; }
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  // capture on a private stream (the legacy default stream cannot be
  // captured); the graph is later launched on the handle's stream
  cudaStream_t cs = nullptr;
  QS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t user = b->stream;
  b->stream = cs;
  cudaError_t e0 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  qs_status st = (e0 == cudaSuccess) ? launch_batch(b, b->layout, b->threads) : QS_ECUDA;
  cudaGraph_t g = nullptr;
  cudaError_t e = (e0 == cudaSuccess) ? cudaStreamEndCapture(cs, &g) : e0;
  b->stream = user;
  cudaStreamDestroy(cs);
  if (st != QS_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st == QS_OK) qs_set_error("batch_capture: %s", cudaGetErrorString(e));
    return st != QS_OK ? st : QS_ECUDA;
  }
  b->graph = g;
  QS_CUDA(cudaGraphInstantiate(&b->gexec, g, 0));
  return QS_OK;
}

extern "C" qs_status batch_autotune(qs_batch* b, int* layout_out, int* threads_out, float* best_ms_out) {
  if (!b || !b->gates) { qs_set_error("batch_autotune: no circuits set"); return QS_EINVAL; }
  // the states are advanced by the timed runs: snapshot and restore them
  void* save = nullptr;
  QS_CUDA(cudaMalloc(&save, b->bytes));
  QS_CUDA(cudaMemcpyAsync(save, b->states, b->bytes, cudaMemcpyDeviceToDevice, b->stream));
  cudaEvent_t e0, e1;
  QS_CUDA(cudaEventCreate(&e0));
  QS_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bl = b->layout, bt = b->threads;
  const int cand_threads[] = {64, 128, 256, 512, 1024};
  for (int layout = 0; layout < 2; ++layout) {
    for (int ti = 0; ti < 5; ++ti) {
      const int th = cand_threads[ti];
      if (!layout_ok(b, layout, th)) continue;
      if (layout == 0 && th > (1 << (b->N - 1)) && th > 64) continue;
      QS_TRY(launch_batch(b, layout, th));  // warm-up
      QS_CUDA(cudaEventRecord(e0, b->stream));
      for (int r = 0; r < 3; ++r) QS_TRY(launch_batch(b, layout, th));
      QS_CUDA(cudaEventRecord(e1, b->stream));
      QS_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      QS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms /= 3.f;
      if (ms < best) { best = ms; bl = layout; bt = th; }
    }
  }
  QS_CUDA(cudaMemcpyAsync(b->states, save, b->bytes, cudaMemcpyDeviceToDevice, b->stream));
  QS_CUDA(cudaStreamSynchronize(b->stream));
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->layout = bl;
  b->threads = bt;
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  if (layout_out) *layout_out = bl;
  if (threads_out) *threads_out = bt;
  if (best_ms_out) *best_ms_out = best;
  return QS_OK;
}

extern "C" qs_status batch_norms(qs_batch* b, double* out) {
  if (!b || !out) { qs_set_error("batch_norms: null argument"); return QS_EINVAL; }
  if (b->enc == QS_C64) k_batch_norms<float><<<b->nstates, 256, 0, b->stream>>>((const Cx<float>*)b->states, b->N, b->dnorm);
  else k_batch_norms<double><<<b->nstates, 256, 0, b->stream>>>((const Cx<double>*)b->states, b->N, b->dnorm);
  QS_LAUNCH_CHECK();
  QS_CUDA(cudaMemcpyAsync(out, b->dnorm, sizeof(double) * (size_t)b->nstates, cudaMemcpyDeviceToHost, b->stream));
  QS_CUDA(cudaStreamSynchronize(b->stream));
  return QS_OK;
}

extern "C" qs_status batch_copy_out(qs_batch* b, void* host, size_t bytes) {
  if (!b || !host || bytes != b->bytes) { qs_set_error("batch_copy_out: need %zu bytes", b ? b->bytes : 0); return QS_EINVAL; }
  QS_CUDA(cudaMemcpyAsync(host, b->states, bytes, cudaMemcpyDeviceToHost, b->stream));
  QS_CUDA(cudaStreamSynchronize(b->stream));
  return QS_OK;
}

extern "C" qs_status batch_copy_in(qs_batch* b, const void* host, size_t bytes) {
  if (!b || !host || bytes != b->bytes) { qs_set_error("batch_copy_in: need %zu bytes", b ? b->bytes : 0); return QS_EINVAL; }
  QS_CUDA(cudaMemcpyAsync(b->states, host, bytes, cudaMemcpyHostToDevice, b->stream));
  QS_CUDA(cudaStreamSynchronize(b->stream));
  return QS_OK;
}

extern "C" qs_status batch_info(const qs_batch* b, int* layout, int* threads, void** dev_states) {
  if (!b) { qs_set_error("batch_info: null"); return QS_EINVAL; }
  if (layout) *layout = b->layout;
  if (threads) *threads = b->threads;
  if (dev_states) *dev_states = b->states;
  return QS_OK;
}
