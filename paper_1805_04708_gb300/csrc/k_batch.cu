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
#include <algorithm>
#include <complex>
#include <new>
#include <vector>

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

// Fused gates: a dense 2^m x 2^m block (m <= 4) on the qubits q[0..m-1]
// (ascending); bit j of a block's local index is the value of qubit q[j].
struct FGate {
  int m;
  int q[4];
  int coef;   // offset of the row-major 4^m coefficients
};

// S = 2^sb states per CTA, blockDim.x / S threads per state; every state
// held in shared memory for its whole fused gate list; the block's
// coefficients staged in shared memory per gate.
template <typename R>
__global__ void k_batch_fused(Cx<R>* __restrict__ states, int N, int sb, const FGate* __restrict__ fg,
                              const int* __restrict__ foffs, const Cx<R>* __restrict__ coef, int nstates) {
  extern __shared__ unsigned char smraw[];
  const int S = 1 << sb;
  const int tps = blockDim.x >> sb;            // threads per state
  const int ls = threadIdx.x / tps, lt = threadIdx.x % tps;
  const int s = blockIdx.x * S + ls;
  const int n = 1 << N;
  Cx<R>* cbuf = (Cx<R>*)smraw + (size_t)ls * 256;           // 4^4 coefficients per state
  Cx<R>* st = (Cx<R>*)smraw + (size_t)S * 256 + (size_t)ls * n;
  const bool live = s < nstates;
  Cx<R>* gs = states + (size_t)(live ? s : 0) * n;
  if (live)
    for (int i = lt; i < n; i += tps) st[i] = gs[i];
  // the CTA runs to the longest list among its states
  __shared__ int maxlen;
  if (threadIdx.x == 0) maxlen = 0;
  __syncthreads();
  const int f0 = live ? foffs[s] : 0, f1 = live ? foffs[s + 1] : 0;
  if (lt == 0) atomicMax(&maxlen, f1 - f0);
  __syncthreads();
  const int L = maxlen;
  for (int k = 0; k < L; ++k) {
    const bool mine = live && f0 + k < f1;
    FGate g;
    if (mine) g = fg[f0 + k];
    else g.m = 0;
    if (mine) {
      const int nc = 1 << (2 * g.m);
      for (int i = lt; i < nc; i += tps) cbuf[i] = coef[g.coef + i];
    }
    __syncthreads();
    if (mine) {
      const int m = g.m, d = 1 << m;
      const int ngroups = n >> m;
      for (int grp = lt; grp < ngroups; grp += tps) {
        // insert zero bits at the block's qubits (ascending)
        uint32_t base = (uint32_t)grp;
        for (int j = 0; j < m; ++j) {
          const uint32_t lo = base & ((1u << g.q[j]) - 1);
          base = ((base >> g.q[j]) << (g.q[j] + 1)) | lo;
        }
        Cx<R> vin[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (j >= d) break;
          uint32_t idx = base;
          for (int b = 0; b < m; ++b)
            if ((j >> b) & 1) idx |= 1u << g.q[b];
          vin[j] = st[idx];
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if (r >= d) break;
          R re = 0, im = 0;
          for (int j = 0; j < d; ++j) {
            const Cx<R> u = cbuf[r * d + j];
            re = fma(u.x, vin[j].x, fma(-u.y, vin[j].y, re));
            im = fma(u.x, vin[j].y, fma(u.y, vin[j].x, im));
          }
          uint32_t idx = base;
          for (int b = 0; b < m; ++b)
            if ((r >> b) & 1) idx |= 1u << g.q[b];
          st[idx] = cx<R>(re, im);
        }
      }
    }
    __syncthreads();
  }
  if (live)
    for (int i = lt; i < n; i += tps) gs[i] = st[i];
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
  int layout;            // 0: CTA per state, 1: warp per state (fuse_k == 0)
  int threads;           // CTA size
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  double* dnorm;
  // fused form: blocks of up to fuse_k qubits (fuse_k = 0: one kernel step
  // per gate), 2^(tile_bits - N) states per CTA
  int fuse_k, tile_bits;
  int fused_for;         // fuse_k the device lists below were built for (-1: none)
  FGate* fgates;         // device
  int* foffs;            // device, nstates + 1
  void* fcoef;           // device Cx<R>
  std::vector<qs_gate>* hgates;   // host copies of the gate lists
  std::vector<int>* hoffs;
};

// ---- fusion (host, FP64) ---------------------------------------------------------------
using cd = std::complex<double>;
// matrix of a controlled 2x2 on the block qubits Q (ascending, m of them)
static void gate_on_block(const qs_gate& g, const int* Q, int m, std::vector<cd>& F) {
  const int d = 1 << m;
  auto pos = [&](int q) { for (int i = 0; i < m; ++i) if (Q[i] == q) return i; return -1; };
  const int tb = pos(g.target);
  int cm = 0;
  for (int c = 0; c < g.nc; ++c) cm |= 1 << pos(g.controls[c]);
  F.assign((size_t)d * d, cd(0, 0));
  for (int c = 0; c < d; ++c) {
    if ((c & cm) != cm) { F[(size_t)c * d + c] = 1.0; continue; }
    const int cb = (c >> tb) & 1;
    for (int rb = 0; rb < 2; ++rb) {
      const int r = (c & ~(1 << tb)) | (rb << tb);
      F[(size_t)r * d + c] = cd(g.u[2 * (2 * rb + cb)], g.u[2 * (2 * rb + cb) + 1]);
    }
  }
}
// M on Q (m qubits) embedded on Q2 (m2 qubits, Q subset of Q2)
static void embed(const std::vector<cd>& M, const int* Q, int m, const int* Q2, int m2, std::vector<cd>& out) {
  const int d2 = 1 << m2;
  int map[4];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m2; ++j)
      if (Q2[j] == Q[i]) map[i] = j;
  int qmask = 0;
  for (int i = 0; i < m; ++i) qmask |= 1 << map[i];
  out.assign((size_t)d2 * d2, cd(0, 0));
  const int d = 1 << m;
  for (int r2 = 0; r2 < d2; ++r2)
    for (int c2 = 0; c2 < d2; ++c2) {
      if ((r2 & ~qmask) != (c2 & ~qmask)) continue;
      int r = 0, c = 0;
      for (int i = 0; i < m; ++i) { r |= ((r2 >> map[i]) & 1) << i; c |= ((c2 >> map[i]) & 1) << i; }
      out[(size_t)r2 * d2 + c2] = M[(size_t)r * d + c];
    }
}
// greedy fusion of one state's gates into blocks of at most k qubits (a
// single gate wider than k is its own block); coefficients appended to coef
static void fuse_list(const qs_gate* g, int n, int k, std::vector<FGate>& out, std::vector<cd>& coef) {
  int Q[4], m = 0;
  std::vector<cd> M, F, E;
  auto flush = [&]() {
    if (m == 0) return;
    FGate f;
    f.m = m;
    for (int i = 0; i < 4; ++i) f.q[i] = i < m ? Q[i] : 0;
    f.coef = (int)coef.size();
    coef.insert(coef.end(), M.begin(), M.end());
    out.push_back(f);
    m = 0;
  };
  for (int i = 0; i < n; ++i) {
    int G[3], ng = 0;
    for (int c = 0; c < g[i].nc; ++c) G[ng++] = g[i].controls[c];
    G[ng++] = g[i].target;
    int U[8], nu = 0;   // Q union G, ascending
    for (int j = 0; j < m; ++j) U[nu++] = Q[j];
    for (int j = 0; j < ng; ++j) {
      bool have = false;
      for (int t = 0; t < nu; ++t) have |= (U[t] == G[j]);
      if (!have) U[nu++] = G[j];
    }
    std::sort(U, U + nu);
    if (m > 0 && nu > k) {
      flush();
      nu = 0;
      for (int j = 0; j < ng; ++j) U[nu++] = G[j];
      std::sort(U, U + nu);
    }
    if (m == 0) {   // start a block on the gate's own qubits
      for (int j = 0; j < nu; ++j) Q[j] = U[j];
      m = nu;
      const int d = 1 << m;
      M.assign((size_t)d * d, cd(0, 0));
      for (int j = 0; j < d; ++j) M[(size_t)j * d + j] = 1.0;
    } else if (nu > m) {
      embed(M, Q, m, U, nu, E);
      M.swap(E);
      for (int j = 0; j < nu; ++j) Q[j] = U[j];
      m = nu;
    }
    gate_on_block(g[i], Q, m, F);
    const int d = 1 << m;
    E.assign((size_t)d * d, cd(0, 0));
    for (int r = 0; r < d; ++r)
      for (int t = 0; t < d; ++t) {
        const cd f = F[(size_t)r * d + t];
        if (f == cd(0, 0)) continue;
        for (int c = 0; c < d; ++c) E[(size_t)r * d + c] += f * M[(size_t)t * d + c];
      }
    M.swap(E);
  }
  flush();
}

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
  b->fuse_k = 0;
  b->tile_bits = N;
  b->fused_for = -1;
  b->hgates = new (std::nothrow) std::vector<qs_gate>();
  b->hoffs = new (std::nothrow) std::vector<int>();
  if (!b->hgates || !b->hoffs) { delete b->hgates; delete b->hoffs; delete b; return QS_ENOMEM; }
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
  if (b->fgates) cudaFree(b->fgates);
  if (b->foffs) cudaFree(b->foffs);
  if (b->fcoef) cudaFree(b->fcoef);
  delete b->hgates;
  delete b->hoffs;
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
  b->hgates->assign(gates, gates + ng);
  b->hoffs->assign(offsets, offsets + b->nstates + 1);
  b->fused_for = -1;
  return QS_OK;
}

// fused device lists for fusion width k (host fusion in FP64, coefficients
// rounded once to the state's precision)
static qs_status build_fused(qs_batch* b, int k) {
  if (b->fused_for == k) return QS_OK;
  std::vector<FGate> fg;
  std::vector<cd> coef;
  std::vector<int> fo(b->nstates + 1, 0);
  const std::vector<qs_gate>& G = *b->hgates;
  const std::vector<int>& O = *b->hoffs;
  for (int st = 0; st < b->nstates; ++st) {
    fuse_list(G.data() + O[st], O[st + 1] - O[st], k, fg, coef);
    fo[st + 1] = (int)fg.size();
  }
  if (fg.empty()) { fg.push_back(FGate{}); }
  if (coef.empty()) coef.push_back(cd(0, 0));
  if (b->fgates) { cudaFree(b->fgates); b->fgates = nullptr; }
  if (b->foffs) { cudaFree(b->foffs); b->foffs = nullptr; }
  if (b->fcoef) { cudaFree(b->fcoef); b->fcoef = nullptr; }
  const size_t ab = amp_bytes(b->enc);
  QS_CUDA(cudaMalloc(&b->fgates, sizeof(FGate) * fg.size()));
  QS_CUDA(cudaMalloc(&b->foffs, sizeof(int) * fo.size()));
  QS_CUDA(cudaMalloc(&b->fcoef, ab * coef.size()));
  std::vector<unsigned char> cbuf(ab * coef.size());
  for (size_t i = 0; i < coef.size(); ++i) {
    if (b->enc == QS_C64) {
      const float v[2] = {(float)coef[i].real(), (float)coef[i].imag()};
      memcpy(&cbuf[i * 8], v, 8);
    } else {
      const double v[2] = {coef[i].real(), coef[i].imag()};
      memcpy(&cbuf[i * 16], v, 16);
    }
  }
  QS_CUDA(cudaMemcpyAsync(b->fgates, fg.data(), sizeof(FGate) * fg.size(), cudaMemcpyHostToDevice, b->stream));
  QS_CUDA(cudaMemcpyAsync(b->foffs, fo.data(), sizeof(int) * fo.size(), cudaMemcpyHostToDevice, b->stream));
  QS_CUDA(cudaMemcpyAsync(b->fcoef, cbuf.data(), cbuf.size(), cudaMemcpyHostToDevice, b->stream));
  QS_CUDA(cudaStreamSynchronize(b->stream));
  b->fused_for = k;
  return QS_OK;
}

static size_t fused_smem(const qs_batch* b, int sb) {
  return ((size_t)1 << sb) * (256 + ((size_t)1 << b->N)) * amp_bytes(b->enc);
}
static bool fused_ok(const qs_batch* b, int k, int tile_bits, int threads) {
  const int sb = tile_bits - b->N;
  return k >= 1 && k <= 4 && sb >= 0 && sb <= 5 && (threads >> sb) >= 32 && threads <= 1024 &&
         fused_smem(b, sb) <= 200 * 1024;
}
static qs_status launch_fused(qs_batch* b, int k, int tile_bits, int threads) {
  QS_TRY(build_fused(b, k));
  const int sb = tile_bits - b->N;
  const size_t smem = fused_smem(b, sb);
  const unsigned grid = (unsigned)((b->nstates + (1 << sb) - 1) >> sb);
  if (b->enc == QS_C64) {
    QS_CUDA(cudaFuncSetAttribute(k_batch_fused<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_batch_fused<float><<<grid, threads, smem, b->stream>>>((Cx<float>*)b->states, b->N, sb, b->fgates, b->foffs,
                                                            (const Cx<float>*)b->fcoef, b->nstates);
  } else {
    QS_CUDA(cudaFuncSetAttribute(k_batch_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_batch_fused<double><<<grid, threads, smem, b->stream>>>((Cx<double>*)b->states, b->N, sb, b->fgates, b->foffs,
                                                             (const Cx<double>*)b->fcoef, b->nstates);
  }
  QS_LAUNCH_CHECK();
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
  if (b->fuse_k > 0) return launch_fused(b, b->fuse_k, b->tile_bits, b->threads);
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
  if (b->fuse_k > 0) {   // the fused lists are built (and uploaded) before the capture
    b->stream = user;
    qs_status sf = build_fused(b, b->fuse_k);
    b->stream = cs;
    if (sf != QS_OK) { b->stream = user; cudaStreamDestroy(cs); return sf; }
  }
  cudaError_t e0 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  qs_status st = (e0 != cudaSuccess) ? QS_ECUDA
                 : (b->fuse_k > 0 ? launch_fused(b, b->fuse_k, b->tile_bits, b->threads)
                                  : launch_batch(b, b->layout, b->threads));
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
  int bl = b->layout, bt = b->threads, bk = 0, bb = b->N;
  const int cand_threads[] = {64, 128, 256, 512, 1024};
  auto time3 = [&](auto launch, float* ms) -> qs_status {
    QS_TRY(launch());   // warm-up (and the fused lists' build)
    QS_CUDA(cudaEventRecord(e0, b->stream));
    for (int r = 0; r < 3; ++r) QS_TRY(launch());
    QS_CUDA(cudaEventRecord(e1, b->stream));
    QS_CUDA(cudaEventSynchronize(e1));
    QS_CUDA(cudaEventElapsedTime(ms, e0, e1));
    *ms /= 3.f;
    return QS_OK;
  };
  // one kernel step per gate: the two layouts and the CTA sizes
  for (int layout = 0; layout < 2; ++layout) {
    for (int ti = 0; ti < 5; ++ti) {
      const int th = cand_threads[ti];
      if (!layout_ok(b, layout, th)) continue;
      if (layout == 0 && th > (1 << (b->N - 1)) && th > 64) continue;
      float ms = 0.f;
      QS_TRY(time3([&]() { return launch_batch(b, layout, th); }, &ms));
      if (ms < best) { best = ms; bl = layout; bt = th; bk = 0; bb = b->N; }
    }
  }
  // fused blocks of k <= 4 qubits, 2^(tile_bits - N) states per CTA
  for (int k = 1; k <= 4; ++k)
    for (int sb = 0; sb <= 5; ++sb)
      for (int ti = 1; ti < 4; ++ti) {
        const int th = cand_threads[ti];
        if (!fused_ok(b, k, b->N + sb, th)) continue;
        if ((th >> sb) > (1 << (b->N - 1)) && (th >> sb) > 32) continue;
        float ms = 0.f;
        QS_TRY(time3([&]() { return launch_fused(b, k, b->N + sb, th); }, &ms));
        if (ms < best) { best = ms; bt = th; bk = k; bb = b->N + sb; }
      }
  QS_CUDA(cudaMemcpyAsync(b->states, save, b->bytes, cudaMemcpyDeviceToDevice, b->stream));
  QS_CUDA(cudaStreamSynchronize(b->stream));
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->layout = bl;
  b->threads = bt;
  b->fuse_k = bk;
  b->tile_bits = bb;
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  if (layout_out) *layout_out = bk > 0 ? 2 : bl;
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

extern "C" qs_status batch_set_tuning(qs_batch* b, int fuse_k, int tile_bits, int threads) {
  if (!b) { qs_set_error("batch_set_tuning: null"); return QS_EINVAL; }
  if (fuse_k == 0) {
    const int layout = tile_bits > b->N ? 1 : 0;
    if (!layout_ok(b, layout, threads) || (threads & 31) || threads < 32 || threads > 1024) {
      qs_set_error("batch_set_tuning: %d threads, tile bits %d do not fit the per-gate kernels", threads, tile_bits);
      return QS_EINVAL;
    }
    b->layout = layout;
  } else if (!fused_ok(b, fuse_k, tile_bits, threads)) {
    qs_set_error("batch_set_tuning: fuse_k %d, tile bits %d, %d threads: not a valid configuration", fuse_k,
                 tile_bits, threads);
    return QS_EINVAL;
  }
  b->fuse_k = fuse_k;
  b->tile_bits = fuse_k ? tile_bits : b->N;
  b->threads = threads;
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  return QS_OK;
}

extern "C" qs_status batch_get_tuning(const qs_batch* b, int* fuse_k, int* tile_bits, int* threads) {
  if (!b) { qs_set_error("batch_get_tuning: null"); return QS_EINVAL; }
  if (fuse_k) *fuse_k = b->fuse_k;
  if (tile_bits) *tile_bits = b->fuse_k ? b->tile_bits : (b->layout == 1 ? b->N + 3 : b->N);
  if (threads) *threads = b->threads;
  return QS_OK;
}
