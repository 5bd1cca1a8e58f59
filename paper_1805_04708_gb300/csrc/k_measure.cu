// The stochastic instructions of Appendix A on the device: M (projective
// measurement of one qubit), CLEAR / SET (projection onto |0> / |1> with
// renormalisation), GENERATE EVENTS (basis states sampled from |a_i|^2), and
// the DEPOLARIZING CHANNEL (Pauli errors inserted after every gate).
//
// Every random number is an input (a uniform draw in [0, 1)), or comes from
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) evaluated at (seed, counter),
// so that a run is reproducible and the draws of the device and the host
// agree bit for bit.
//
// GENERATE EVENTS is inverse-CDF sampling in index order: event k is the
// smallest index i with C_i > u_k C_last, C_i = sum_{j <= i} |a_j|^2.  Three
// sweeps of small arrays after one read of the state:
//   k_ev_chunks  : FP64 sum of |a|^2 over each chunk of 1024 amplitudes
//                  (one warp per chunk; each lane's squares exact and summed
//                  in float-float for complex64 and the adaptive encoding);
//   k_scan_*     : exclusive prefix of the chunk sums in a fixed tree order;
//   k_ev_sample  : one warp per event: binary search of the chunk prefix for
//                  the first chunk whose end exceeds the target, then the
//                  lane sums of the chunk's 32 segments of 32 amplitudes, a
//                  warp scan to find the segment, and a warp scan inside it.
// Results are deterministic (no atomics on sums).  Where rounding moves a
// target across a boundary the event is the neighbouring index, and an event
// never lands on an amplitude that is exactly zero.
#include "internal.cuh"
#include "cplx.cuh"
#include "a2codec.cuh"
#include <math.h>
#include <string.h>
#include <vector>

namespace {

constexpr int TPB = 256;
constexpr int CH_LOG = 10;           // amplitudes per chunk: 1024 = 32 segments of 32
constexpr int SCAN_PER_THREAD = 8;   // chunk sums per thread in the prefix kernels
constexpr int SCAN_BLOCK = TPB * SCAN_PER_THREAD;

// ---- SplitMix64 at (seed, counter) ------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double uniform_at(uint64_t seed, uint64_t counter) {
  return (double)(splitmix64_at(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

// ---- |a|^2 in FP64 for each encoding --------------------------------------------------
template <typename A> struct Prob;
template <> struct Prob<double2> {
  static __device__ __forceinline__ double at(const double2* s, uint64_t i, const float*) {
    const double2 a = s[i];
    return a.x * a.x + a.y * a.y;
  }
};
template <> struct Prob<float2> {
  static __device__ __forceinline__ double at(const float2* s, uint64_t i, const float*) {
    const float2 a = s[i];
    return (double)a.x * a.x + (double)a.y * a.y;   // exact products
  }
};
template <> struct Prob<uint16_t> {
  static __device__ __forceinline__ double at(const uint16_t* s, uint64_t i, const float* r) {
    const double m = (double)r[(s[i] & 0xFFu) ^ 0x80u];
    return m * m;
  }
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// inclusive scan over the warp (Kogge-Stone, fixed order)
__device__ __forceinline__ double warp_incl_scan(double x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// a lane's sum of squares in float-float: each square formed exactly (p + e
// by FMA) and added with a TwoSum, so the FP64 units do nothing per amplitude
struct SqAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_sq(float a) {
    const float p = __fmul_rn(a, a);
    const float e = __fmaf_rn(a, a, -p);
    const float t = __fadd_rn(hi, p);
    const float bp = __fsub_rn(t, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
    lo = __fadd_rn(lo, e);
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <typename A>
__device__ __forceinline__ double lane_chunk_sum(const A* s, uint64_t i0, uint64_t len, int lane, const float* r) {
  double acc = 0.0;
  for (uint64_t j = lane; j < len; j += 32) acc += Prob<A>::at(s, i0 + j, r);
  return acc;
}
template <>
__device__ __forceinline__ double lane_chunk_sum<float2>(const float2* s, uint64_t i0, uint64_t len, int lane,
                                                         const float*) {
  SqAcc f;
  for (uint64_t j = lane; j < len; j += 32) {
    const float2 a = s[i0 + j];
    f.add_sq(a.x);
    f.add_sq(a.y);
  }
  return f.value();
}
template <>
__device__ __forceinline__ double lane_chunk_sum<uint16_t>(const uint16_t* s, uint64_t i0, uint64_t len, int lane,
                                                           const float* r) {
  SqAcc f;
  for (uint64_t j = lane; j < len; j += 32) f.add_sq(r[(s[i0 + j] & 0xFFu) ^ 0x80u]);
  return f.value();
}

// chunk sums: one warp per chunk of 2^clog amplitudes; lane l sums the
// amplitudes l, l + 32, ... of the chunk (coalesced), then a warp tree
template <typename A>
__global__ void __launch_bounds__(TPB) k_ev_chunks(const A* __restrict__ s, uint64_t nchunks, int clog,
                                                   double* __restrict__ sums, const A2Dev* a2) {
  __shared__ Luts L;
  if (a2) build_luts(L, a2->r0, a2->r1);
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * TPB + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * TPB) >> 5;
  const uint64_t len = 1ull << clog;
  for (uint64_t c = w0; c < nchunks; c += nw) {
    double acc = lane_chunk_sum<A>(s, c << clog, len, lane, L.r);
    acc = warp_sum(acc);
    if (lane == 0) sums[c] = acc;
  }
}

// CLEAR / SET and the projection of M: on every pair of Eq. (NUM2) along
// qubit q, the element with bit q = `bit` is scaled by c and the other is set
// to zero without being read (one read of half the state, one write of all).
template <typename A, typename F>
__global__ void __launch_bounds__(TPB) k_project(A* __restrict__ s, uint64_t npairs, int q, int bit, F c) {
  const uint64_t low = (1ull << q) - 1, qb = 1ull << q;
  const uint64_t stride = (uint64_t)gridDim.x * TPB;
  for (uint64_t j = (uint64_t)blockIdx.x * TPB + threadIdx.x; j < npairs; j += stride) {
    const uint64_t i0 = ((j & ~low) << 1) | (j & low);
    const uint64_t keep = bit ? (i0 | qb) : i0;
    A a = s[keep];
    a.x *= c;
    a.y *= c;
    s[keep] = a;
    s[keep ^ qb] = A{};
  }
}

// block-level exclusive scan of one value per thread (Kogge-Stone in shared
// memory, fixed order); returns the exclusive prefix, *total the block sum
__device__ double block_excl_scan(double x, double* total) {
  __shared__ double sh[TPB];
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int o = 1; o < TPB; o <<= 1) {
    const double y = (threadIdx.x >= (unsigned)o) ? sh[threadIdx.x - o] : 0.0;
    __syncthreads();
    sh[threadIdx.x] += y;
    __syncthreads();
  }
  const double excl = threadIdx.x ? sh[threadIdx.x - 1] : 0.0;
  *total = sh[TPB - 1];
  __syncthreads();
  return excl;
}

// per-thread sum of its SCAN_PER_THREAD entries (sequential)
__device__ __forceinline__ double thread_run(const double* v, uint64_t n, uint64_t i0) {
  double a = 0.0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k)
    if (i0 + k < n) a += v[i0 + k];
  return a;
}

// phase 1: block totals of the per-thread runs
__global__ void __launch_bounds__(TPB) k_scan_blocks(const double* __restrict__ v, uint64_t n,
                                                     double* __restrict__ bsum) {
  const uint64_t i0 = ((uint64_t)blockIdx.x * TPB + threadIdx.x) * SCAN_PER_THREAD;
  double tot;
  (void)block_excl_scan(thread_run(v, n, i0), &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}
// phase 2: one block, exclusive prefix of the block totals (sequential runs of
// per-thread segments, then a block scan); boff[nb] = the grand total
__global__ void __launch_bounds__(TPB) k_scan_top(const double* __restrict__ bsum, uint64_t nb,
                                                  double* __restrict__ boff) {
  const uint64_t per = (nb + TPB - 1) / TPB;
  const uint64_t i0 = threadIdx.x * per;
  double run = 0.0;
  for (uint64_t k = 0; k < per; ++k)
    if (i0 + k < nb) run += bsum[i0 + k];
  double tot;
  double base = block_excl_scan(run, &tot);
  for (uint64_t k = 0; k < per; ++k)
    if (i0 + k < nb) {
      boff[i0 + k] = base;
      base += bsum[i0 + k];
    }
  if (threadIdx.x == 0) boff[nb] = tot;
}
// phase 3: prefix[i] = boff[block] + in-block exclusive prefix (same runs as
// phase 1); prefix[n] = the grand total
__global__ void __launch_bounds__(TPB) k_scan_down(const double* __restrict__ v, uint64_t n,
                                                   const double* __restrict__ boff, uint64_t nb,
                                                   double* __restrict__ prefix) {
  const uint64_t i0 = ((uint64_t)blockIdx.x * TPB + threadIdx.x) * SCAN_PER_THREAD;
  double tot;
  double base = boff[blockIdx.x] + block_excl_scan(thread_run(v, n, i0), &tot);
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k)
    if (i0 + k < n) {
      prefix[i0 + k] = base;
      base += v[i0 + k];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) prefix[n] = boff[nb];
}
// the last chunk with a nonzero sum (for targets at or beyond the total)
__global__ void k_last_nonzero(const double* __restrict__ sums, uint64_t n, unsigned long long* out) {
  unsigned long long best = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB)
    if (sums[i] > 0.0) best = i;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
    best = y > best ? y : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

// first index in [lo, hi) whose value exceeds t (binary search; hi if none)
__device__ __forceinline__ uint64_t first_above(const double* incl, uint64_t lo, uint64_t hi, double t) {
  while (lo < hi) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    if (incl[mid] > t) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// one warp per event
template <typename A>
__global__ void __launch_bounds__(TPB) k_ev_sample(const A* __restrict__ s, int clog, uint64_t nchunks,
                                                   const double* __restrict__ sums,
                                                   const double* __restrict__ prefix,
                                                   const unsigned long long* __restrict__ last_nz,
                                                   const double* __restrict__ u, uint64_t seed, uint64_t first,
                                                   uint64_t nev, unsigned long long* __restrict__ out,
                                                   const A2Dev* a2) {
  __shared__ Luts L;
  if (a2) build_luts(L, a2->r0, a2->r1);
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * TPB + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * TPB) >> 5;
  const double T = prefix[nchunks];
  const uint64_t len = 1ull << clog;
  const int seg_log = clog > 5 ? clog - 5 : 0;     // amplitudes per lane segment
  const uint64_t seg = 1ull << seg_log;
  for (uint64_t e = w0; e < nev; e += nw) {
    const double ue = u ? u[e] : uniform_at(seed, first + e);
    const double t = ue * T;
    // chunk: the first whose end prefix[c + 1] exceeds t, else the last nonzero
    uint64_t c = first_above(prefix + 1, 0, nchunks, t);
    if (c >= nchunks) c = *last_nz;
    const uint64_t base_i = c << clog;
    // lane segments of the chunk (lane l: amplitudes l*seg .. l*seg + seg - 1)
    double ls = 0.0;
    if ((uint64_t)lane * seg < len)
      for (uint64_t j = 0; j < seg; ++j) ls += Prob<A>::at(s, base_i + (uint64_t)lane * seg + j, L.r);
    const double lscan = warp_incl_scan(ls, lane);
    double lexcl = __shfl_up_sync(0xffffffffu, lscan, 1);
    if (lane == 0) lexcl = 0.0;
    const double lincl = prefix[c] + lscan;
    unsigned m = __ballot_sync(0xffffffffu, lincl > t && ls > 0.0);
    int sl;
    if (m) {
      sl = __ffs(m) - 1;
    } else {
      const unsigned nzm = __ballot_sync(0xffffffffu, ls > 0.0);
      sl = nzm ? 31 - __clz(nzm) : 0;
    }
    // inside the segment: one amplitude per lane (seg <= 32)
    const double sbase = prefix[c] + __shfl_sync(0xffffffffu, lexcl, sl);
    const uint64_t i0 = base_i + (uint64_t)sl * seg;
    const double p = ((uint64_t)lane < seg) ? Prob<A>::at(s, i0 + lane, L.r) : 0.0;
    const double pin = sbase + warp_incl_scan(p, lane);
    m = __ballot_sync(0xffffffffu, pin > t && p > 0.0);
    int k;
    if (m) {
      k = __ffs(m) - 1;
    } else {
      const unsigned nzm = __ballot_sync(0xffffffffu, p > 0.0);
      k = nzm ? 31 - __clz(nzm) : 0;
    }
    if (lane == 0) out[e] = i0 + (uint64_t)k;
  }
}

}  // namespace

// =========================================================================================
// host side
// =========================================================================================
static unsigned grid_for(const qs_sim* s, uint64_t warps) {
  const uint64_t blocks = (warps * 32 + TPB - 1) / TPB;
  const uint64_t cap = (uint64_t)s->num_sms * 8;
  return (unsigned)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

template <typename A>
static qs_status events_impl(qs_sim* s, const double* u_host, uint64_t seed, uint64_t nev, uint64_t* out) {
  const int clog = s->N < CH_LOG ? s->N : CH_LOG;
  const uint64_t nchunks = 1ull << (s->N - clog);
  const uint64_t nb = (nchunks + SCAN_BLOCK - 1) / SCAN_BLOCK;
  // scratch: sums[nchunks], prefix[nchunks + 1], bsum[nb], boff[nb + 1],
  // last-nonzero (8 B), u[nev], out[nev]
  const size_t dbl = nchunks + (nchunks + 1) + nb + (nb + 1) + 1;
  const size_t bytes = (dbl + (u_host ? nev : 0) + nev) * 8;
  QS_TRY(ensure_scratch(s, bytes));
  double* sums = (double*)s->scratch;
  double* prefix = sums + nchunks;
  double* bsum = prefix + nchunks + 1;
  double* boff = bsum + nb;
  unsigned long long* lastnz = (unsigned long long*)(boff + nb + 1);
  double* ud = (double*)(lastnz + 1);
  unsigned long long* od = (unsigned long long*)(ud + (u_host ? nev : 0));
  const A2Dev* a2 = (const A2Dev*)s->a2dev;
  k_ev_chunks<A><<<grid_for(s, nchunks), TPB, 0, s->stream>>>((const A*)s->state, nchunks, clog, sums, a2);
  QS_LAUNCH_CHECK();
  k_scan_blocks<<<(unsigned)nb, TPB, 0, s->stream>>>(sums, nchunks, bsum);
  QS_LAUNCH_CHECK();
  k_scan_top<<<1, TPB, 0, s->stream>>>(bsum, nb, boff);
  QS_LAUNCH_CHECK();
  k_scan_down<<<(unsigned)nb, TPB, 0, s->stream>>>(sums, nchunks, boff, nb, prefix);
  QS_LAUNCH_CHECK();
  QS_CUDA(cudaMemsetAsync(lastnz, 0, sizeof(unsigned long long), s->stream));
  k_last_nonzero<<<grid_for(s, (nchunks + 31) / 32), TPB, 0, s->stream>>>(sums, nchunks, lastnz);
  QS_LAUNCH_CHECK();
  if (u_host) QS_CUDA(cudaMemcpyAsync(ud, u_host, nev * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  k_ev_sample<A><<<grid_for(s, nev), TPB, 0, s->stream>>>((const A*)s->state, clog, nchunks, sums, prefix, lastnz,
                                                         u_host ? ud : nullptr, seed, 0, nev, od, a2);
  QS_LAUNCH_CHECK();
  QS_CUDA(cudaMemcpyAsync(out, od, nev * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}

static qs_status events_dispatch(qs_sim* s, const double* u, uint64_t seed, uint64_t n, uint64_t* out) {
  if (s->enc == QS_C128) return events_impl<double2>(s, u, seed, n, out);
  if (s->enc == QS_C64) return events_impl<float2>(s, u, seed, n, out);
  return events_impl<uint16_t>(s, u, seed, n, out);
}

#define CHECK_ARG(cond, ...)            \
  do {                                  \
    if (!(cond)) {                      \
      qs_set_error(__VA_ARGS__);        \
      return QS_EINVAL;                 \
    }                                   \
  } while (0)

extern "C" qs_status qs_uniforms(uint64_t seed, uint64_t first, int64_t n, double* out) {
  CHECK_ARG(n >= 0 && (n == 0 || out), "qs_uniforms: bad output");
  for (int64_t k = 0; k < n; ++k) out[k] = uniform_at(seed, first + (uint64_t)k);
  return QS_OK;
}

extern "C" qs_status generate_events(qs_sim* s, const double* u, int64_t n, uint64_t* events) {
  CHECK_ARG(s != nullptr, "null handle");
  CHECK_ARG(n >= 1 && n <= (1ll << 31), "generate_events: n = %lld not in 1..2^31", (long long)n);
  CHECK_ARG(u != nullptr && events != nullptr, "generate_events: null array");
  for (int64_t k = 0; k < n; ++k)
    CHECK_ARG(u[k] >= 0.0 && u[k] < 1.0, "generate_events: draw %lld = %g not in [0, 1)", (long long)k, u[k]);
  QS_TRY(materialize_state(s));
  return events_dispatch(s, u, 0, (uint64_t)n, events);
}

extern "C" qs_status generate_events_seeded(qs_sim* s, uint64_t seed, int64_t n, uint64_t* events) {
  CHECK_ARG(s != nullptr, "null handle");
  CHECK_ARG(n >= 1 && n <= (1ll << 31), "generate_events_seeded: n = %lld not in 1..2^31", (long long)n);
  CHECK_ARG(events != nullptr, "generate_events_seeded: null array");
  QS_TRY(materialize_state(s));
  return events_dispatch(s, nullptr, seed, (uint64_t)n, events);
}

// projection onto `bit` of qubit q, scaled by c (a diagonal update with the
// entries (c, 0) or (0, c) on the pair of Eq. (NUM2))
static qs_status project_scaled(qs_sim* s, int q, int bit, double c) {
  if (s->enc == QS_ADAPT2) {
    double u[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (bit == 0) u[0] = c; else u[6] = c;
    return a2_apply_arith(s, nullptr, 0, q, u);
  }
  QS_TRY(materialize_state(s));
  const uint64_t npairs = 1ull << (s->N - 1);
  const unsigned grid = grid_for(s, (npairs + 31) / 32);
  if (s->enc == QS_C128)
    k_project<double2, double><<<grid, TPB, 0, s->stream>>>((double2*)s->state, npairs, q, bit, c);
  else
    k_project<float2, float><<<grid, TPB, 0, s->stream>>>((float2*)s->state, npairs, q, bit, (float)c);
  QS_LAUNCH_CHECK();
  return QS_OK;
}

static qs_status qubit_probs(qs_sim* s, int q, double* p0, double* p1) {
  QS_TRY(materialize_state(s));
  return launch_qubit_probs(s, q, p0, p1);
}

extern "C" qs_status project_qubit(qs_sim* s, int q, int bit, double* prob) {
  CHECK_ARG(s != nullptr, "null handle");
  CHECK_ARG(q >= 0 && q < s->N, "project_qubit: qubit %d out of range", q);
  CHECK_ARG(bit == 0 || bit == 1, "project_qubit: bit must be 0 or 1");
  double p0, p1;
  QS_TRY(qubit_probs(s, q, &p0, &p1));
  const double p = bit ? p1 : p0;
  if (prob) *prob = p;
  if (p == 0.0) {
    qs_set_error("project_qubit: the projection of qubit %d onto %d gives a zero state", q, bit);
    return QS_EZEROPROJ;
  }
  return project_scaled(s, q, bit, 1.0 / sqrt(p));
}

extern "C" qs_status measure_qubit(qs_sim* s, int q, double u, int* outcome, double* probs) {
  CHECK_ARG(s != nullptr, "null handle");
  CHECK_ARG(q >= 0 && q < s->N, "measure_qubit: qubit %d out of range", q);
  CHECK_ARG(u >= 0.0 && u < 1.0, "measure_qubit: draw %g not in [0, 1)", u);
  double p0, p1;
  QS_TRY(qubit_probs(s, q, &p0, &p1));
  const int o = (u * (p0 + p1) < p0) ? 0 : 1;
  if (outcome) *outcome = o;
  if (probs) { probs[0] = p0; probs[1] = p1; }
  const double p = o ? p1 : p0;
  if (p == 0.0) {   // only for a zero state, which M cannot project
    qs_set_error("measure_qubit: the state has zero norm");
    return QS_EZEROPROJ;
  }
  return project_scaled(s, q, o, 1.0 / sqrt(p));
}

extern "C" qs_status depolarize_circuit(int N, const qs_gate* gates, int n, double px, double py, double pz,
                                        uint64_t seed, int64_t first_gate, qs_gate* out, int cap, int* n_out) {
  CHECK_ARG(N > 1 && N < 64, "depolarize_circuit: N = %d out of range", N);
  CHECK_ARG(n >= 0 && (n == 0 || gates), "depolarize_circuit: bad gate list");
  CHECK_ARG(px >= 0 && py >= 0 && pz >= 0 && px + py + pz <= 1.0,
            "depolarize_circuit: need 0 <= p_x, p_y, p_z and p_x + p_y + p_z <= 1");
  CHECK_ARG(first_gate >= 0 && n_out != nullptr, "depolarize_circuit: bad arguments");
  static const double X[8] = {0, 0, 1, 0, 1, 0, 0, 0};
  static const double Y[8] = {0, 0, 0, -1, 0, 1, 0, 0};
  static const double Z[8] = {1, 0, 0, 0, 0, 0, -1, 0};
  int k = 0;
  auto put = [&](const qs_gate& g) {
    if (out && k < cap) out[k] = g;
    ++k;
  };
  for (int g = 0; g < n; ++g) {
    put(gates[g]);
    for (int q = 0; q < N; ++q) {
      const double r = uniform_at(seed, (uint64_t)(first_gate + g) * (uint64_t)N + (uint64_t)q);
      const double* P = r < px ? X : (r < px + py ? Y : (r < px + py + pz ? Z : nullptr));
      if (!P) continue;
      qs_gate e;
      e.nc = 0;
      e.controls[0] = e.controls[1] = 0;
      e.target = q;
      memcpy(e.u, P, sizeof e.u);
      put(e);
    }
  }
  *n_out = k;
  if (!out || k > cap) {
    qs_set_error("depolarize_circuit: %d records need room (cap %d)", k, cap);
    return out ? QS_EINVAL : QS_OK;
  }
  return QS_OK;
}
