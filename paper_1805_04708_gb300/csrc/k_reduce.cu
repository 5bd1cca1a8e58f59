// Reductions over the dense encodings (complex128 / complex64):
//   norm          sum |a_i|^2                                   (Eq. (STAT1))
//   expect_xyz    w_n = sum_{bit n = 0} conj(a_i) a_{i+2^n},  P_n(1)  (BEGIN MEASUREMENT)
//   marginal      P(k) over a register                           (Sec. 2)
//
// All sums are FP64 with a fixed grid and a fixed tree order, so results are
// bit-stable from run to run on a given GPU.  complex64 products are formed
// exactly (a*b = p + e with e = fma(a, b, -p)) and summed in float-float pairs
// before being folded into FP64, which keeps the work on the FP32 pipes.
#include "internal.cuh"
#include "cplx.cuh"
#include "a2codec.cuh"
#include <string.h>

namespace {

constexpr int TPB = 256;

// ---- float-float accumulation ----------------------------------------------------
struct FF { float hi, lo; };
__device__ __forceinline__ void ff_add(FF& s, float p) {
  float t = s.hi + p;
  float bp = t - s.hi;
  float e = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += e;
}
// s += a*b exactly up to the final roundings of the pair.
__device__ __forceinline__ void ff_add_prod(FF& s, float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  ff_add(s, p);
  s.lo += e;
}
__device__ __forceinline__ double ff_val(const FF& s) { return (double)s.hi + (double)s.lo; }

// ---- block reduction in a fixed order -----------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// Sum over the block; result valid in thread 0.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;
}

// ---- norm -----------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_norm_c128(const double2* __restrict__ s, uint64_t n, double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (uint64_t i = (uint64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB) {
    double2 a = s[i];
    acc = fma(a.x, a.x, acc);
    acc = fma(a.y, a.y, acc);
  }
  double r = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void __launch_bounds__(TPB) k_norm_c64(const float4* __restrict__ s, uint64_t n, double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * TPB;
  uint64_t i = (uint64_t)blockIdx.x * TPB + threadIdx.x;
  // four independent loads in flight per thread; products exact (p + e),
  // summed in float-float, folded into FP64 every iteration
  for (; i + 3 * stride < n; i += 4 * stride) {
    float4 a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = s[i + u * stride];
    FF f = {0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ff_add_prod(f, a[u].x, a[u].x);
      ff_add_prod(f, a[u].y, a[u].y);
      ff_add_prod(f, a[u].z, a[u].z);
      ff_add_prod(f, a[u].w, a[u].w);
    }
    acc += ff_val(f);
  }
  FF f = {0.f, 0.f};
  for (; i < n; i += stride) {
    float4 a = s[i];
    ff_add_prod(f, a.x, a.x);
    ff_add_prod(f, a.y, a.y);
    ff_add_prod(f, a.z, a.z);
    ff_add_prod(f, a.w, a.w);
  }
  acc += ff_val(f);
  double r = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// Neumaier sum of n values per column (stride `cols`), one column per thread
// block x; fixed order.  out[c] = sum_r part[r * cols + c].
__global__ void k_sum_columns(const double* __restrict__ part, int rows, int cols, double* out) {
  __shared__ double shs[TPB], shc[TPB];
  const int c = blockIdx.x;
  double s = 0.0, comp = 0.0;
  for (int r = threadIdx.x; r < rows; r += TPB) {
    double x = part[(size_t)r * cols + c];
    double t = s + x;
    comp += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  shs[threadIdx.x] = s;
  shc[threadIdx.x] = comp;
  __syncthreads();
  for (int h = TPB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      double a = shs[threadIdx.x], b = shs[threadIdx.x + h];
      double t = a + b;
      double e = (fabs(a) >= fabs(b)) ? ((a - t) + b) : ((b - t) + a);
      shs[threadIdx.x] = t;
      shc[threadIdx.x] += shc[threadIdx.x + h] + e;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = shs[0] + shc[0];
}

__device__ __forceinline__ uint64_t deposit(uint64_t x, uint64_t mask) {
  uint64_t r = 0;
  for (uint64_t m = mask; m; m &= m - 1) {
    if (x & 1) r |= m & (~m + 1);
    x >>= 1;
  }
  return r;
}
__device__ __forceinline__ double sq(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double sq(float2 a) { return (double)a.x * a.x + (double)a.y * a.y; }

// ---- expect_xyz for small states (N <= 12): one CTA, FP64 throughout -------------------
template <typename A>
__device__ __forceinline__ double2 to_d2(const A& a, const Luts& L) { return make_double2((double)a.x, (double)a.y); }
template <>
__device__ __forceinline__ double2 to_d2<uint16_t>(const uint16_t& w, const Luts& L) {
  Cx<float> z = a2_dec(L, w);
  return make_double2((double)z.x, (double)z.y);
}
template <typename A>
__global__ void __launch_bounds__(TPB) k_expect_small(const A* __restrict__ s, int N, double* out, const A2Dev* a2) {
  __shared__ double2 t[4096];
  __shared__ double sh[32];
  __shared__ Luts L;
  if (a2) build_luts(L, a2->r0, a2->r1);
  const int n = 1 << N;
  for (int i = threadIdx.x; i < n; i += TPB) t[i] = to_d2<A>(s[i], L);
  __syncthreads();
  double tot = 0.0;
  for (int i = threadIdx.x; i < n; i += TPB) tot += t[i].x * t[i].x + t[i].y * t[i].y;
  tot = block_sum(tot, sh);
  if (threadIdx.x == 0) out[0] = tot;
  for (int q = 0; q < N; ++q) {
    double re = 0.0, im = 0.0, p1 = 0.0;
    for (int j = threadIdx.x; j < n / 2; j += TPB) {
      const int l0 = (int)ins0((uint64_t)j, q), l1 = l0 | (1 << q);
      const double2 a = t[l0], b = t[l1];
      re += a.x * b.x + a.y * b.y;
      im += a.x * b.y - a.y * b.x;
      p1 += b.x * b.x + b.y * b.y;
    }
    re = block_sum(re, sh);
    __syncthreads();
    im = block_sum(im, sh);
    __syncthreads();
    p1 = block_sum(p1, sh);
    __syncthreads();
    if (threadIdx.x == 0) { out[1 + 3 * q] = re; out[2 + 3 * q] = im; out[3 + 3 * q] = p1; }
  }
}

// ---- expect_xyz: register-tile passes -----------------------------------------------------
// A pass reads the state once in tiles of 2^(RB+8) amplitudes: inside a CTA of
// 256 threads, local bit 0 and RB-1 chosen qubits are register slots (each
// thread holds 2^RB amplitudes), index bits 1..5 are the 32 lanes, and 3 more
// qubits are the 8 warps.  For a register-slot qubit n the pairs
// (a(*0_n*), a(*1_n*)) sit in one thread's registers; for a lane qubit the
// partner comes by a warp shuffle.  Pass 0 computes w_n for qubit 0, the lane
// qubits 1..5 and its slot qubits, plus sum |a|^2 per register slot and lane
// bit and per tile and warp (from which P_n(1) of every qubit follows); later
// passes compute w_n for RB-1 new slot qubits each.
//
// Per-thread sums are formed per tile in the arithmetic type (FP32 for
// complex64, FP64 for complex128) and folded into per-thread accumulators in
// shared memory (float-float / FP64), then reduced over the CTA and the grid
// in a fixed order.
constexpr int ETPB = 256;

struct RedParams {
  int N, RB;
  int first;                 // pass 0
  int nslots_new;            // slots 1..nslots_new carry new qubits (pass 0: also slot 0)
  uint8_t slot_g[8];         // global qubit of slot s (slot_g[0] = 0)
  uint8_t warp_g[3];         // global qubit of warp bit k
  uint64_t out_mask;         // global bits outside the tile
};

template <typename R> struct SAcc;
template <> struct SAcc<float> {
  // float-float accumulators, [acc][thread] in shared memory
  float* hi; float* lo;
  __device__ void init(unsigned char* base, int nacc) {
    hi = (float*)base; lo = hi + nacc * ETPB;
    for (int i = 0; i < nacc; ++i) { hi[i * ETPB + threadIdx.x] = 0.f; lo[i * ETPB + threadIdx.x] = 0.f; }
  }
  __device__ __forceinline__ void add(int i, float x) {
    FF f = {hi[i * ETPB + threadIdx.x], lo[i * ETPB + threadIdx.x]};
    ff_add(f, x);
    hi[i * ETPB + threadIdx.x] = f.hi; lo[i * ETPB + threadIdx.x] = f.lo;
  }
  __device__ double get(int i) const { return (double)hi[i * ETPB + threadIdx.x] + (double)lo[i * ETPB + threadIdx.x]; }
  __host__ __device__ static size_t bytes(int nacc) { return (size_t)nacc * ETPB * 8; }
};
template <> struct SAcc<double> {
  double* a;
  __device__ void init(unsigned char* base, int nacc) {
    a = (double*)base;
    for (int i = 0; i < nacc; ++i) a[i * ETPB + threadIdx.x] = 0.0;
  }
  __device__ __forceinline__ void add(int i, double x) { a[i * ETPB + threadIdx.x] += x; }
  __device__ double get(int i) const { return a[i * ETPB + threadIdx.x]; }
  __host__ __device__ static size_t bytes(int nacc) { return (size_t)nacc * ETPB * 8; }
};

template <typename R> __device__ __forceinline__ R shfx(R x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }

// sum over pairs (j, j | 2^S) of conj(v[j]) v[j | 2^S]
template <typename R, int RB, int S>
__device__ __forceinline__ void slot_w(const Cx<R>* v, R& re, R& im) {
  re = 0; im = 0;
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if ((j >> S) & 1) continue;
    const Cx<R> a = v[j], b = v[j | (1 << S)];
    re = fma(a.x, b.x, re); re = fma(a.y, b.y, re);
    im = fma(a.x, b.y, im); im = fma(-a.y, b.x, im);
  }
}
template <typename R, int RB>
__device__ __forceinline__ void slot_w_rt(const Cx<R>* v, int s, R& re, R& im) {
  switch (s) {
    case 0: slot_w<R, RB, 0>(v, re, im); break;
    case 1: slot_w<R, RB, 1>(v, re, im); break;
    case 2: slot_w<R, RB, 2>(v, re, im); break;
    case 3: slot_w<R, RB, 3>(v, re, im); break;
    default: slot_w<R, RB, (RB > 4 ? 4 : 3)>(v, re, im); break;
  }
}

// ENC: 0 complex64, 1 complex128, 2 adaptive 2-byte words (decoded to FP32)
template <typename R, int RB, int ENC>
__global__ void __launch_bounds__(ETPB, 2) k_expect2(const void* __restrict__ s, const __grid_constant__ RedParams P,
                                                      double* __restrict__ tile_tot, double* __restrict__ part,
                                                      const A2Dev* __restrict__ a2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ Luts L;
  if (ENC == 2) build_luts(L, a2->r0, a2->r1);
  constexpr int NR = 1 << RB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // accumulators: pass 0: [w re/im: slot 0, lanes 0..4, slots 1..ns] [P1: slots 0..RB-1, lanes 0..4]
  //               later : [w re/im: slots 1..ns]
  const int nw = P.first ? (1 + 5 + P.nslots_new) : P.nslots_new;
  const int nacc = 2 * nw + (P.first ? (RB + 5) : 0);
  uint64_t* roff = (uint64_t*)smraw;                    // NR/2 register-pair offsets
  SAcc<R> acc;
  acc.init(smraw + 256, nacc);
  if (threadIdx.x < NR / 2) {
    uint64_t g = 0;
    for (int sl = 1; sl < RB; ++sl)
      if (((2 * threadIdx.x) >> sl) & 1) g |= 1ull << P.slot_g[sl];
    roff[threadIdx.x] = g;
  }
  uint64_t woff = ((uint64_t)lane << 1);
  for (int k = 0; k < 3; ++k)
    if ((warp >> k) & 1) woff |= 1ull << P.warp_g[k];
  __syncthreads();
  const uint64_t ntiles = 1ull << (P.N - RB - 8);
  Cx<R> v[NR];
  for (uint64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
    const uint64_t base = deposit(tau, P.out_mask) | woff;
    if constexpr (ENC == 2) {
      const unsigned int* s2 = (const unsigned int*)s;
#pragma unroll
      for (int jj = 0; jj < NR / 2; ++jj) {
        const unsigned int w = s2[(base + roff[jj]) >> 1];
        v[2 * jj] = a2_dec(L, w & 0xFFFFu);
        v[2 * jj + 1] = a2_dec(L, w >> 16);
      }
    } else if constexpr (sizeof(R) == 4) {
      const float4* s4 = (const float4*)s;
#pragma unroll
      for (int jj = 0; jj < NR / 2; ++jj) {
        float4 x = s4[(base + roff[jj]) >> 1];
        v[2 * jj] = cx<float>(x.x, x.y);
        v[2 * jj + 1] = cx<float>(x.z, x.w);
      }
    } else {
      const double2* s2 = (const double2*)s;
#pragma unroll
      for (int jj = 0; jj < NR / 2; ++jj) {
        double2 x = s2[base + roff[jj]], y = s2[base + roff[jj] + 1];
        v[2 * jj] = cx<double>(x.x, x.y);
        v[2 * jj + 1] = cx<double>(y.x, y.y);
      }
    }
    int ai = 0;
    if (P.first) {
      R re, im;
      slot_w<R, RB, 0>(v, re, im);
      acc.add(ai++, re); acc.add(ai++, im);
      for (int k = 0; k < 5; ++k) {
        const int m = 1 << k;
        const bool lo = !((lane >> k) & 1);
        R r2 = 0, i2 = 0;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          const R px = shfx<R>(v[j].x, m), py = shfx<R>(v[j].y, m);
          r2 = fma(v[j].x, px, r2); r2 = fma(v[j].y, py, r2);
          i2 = fma(v[j].x, py, i2); i2 = fma(-v[j].y, px, i2);
        }
        acc.add(ai++, lo ? r2 : (R)0); acc.add(ai++, lo ? i2 : (R)0);
      }
    }
    for (int sl = 1; sl <= P.nslots_new; ++sl) {
      R re, im;
      slot_w_rt<R, RB>(v, sl, re, im);
      acc.add(ai++, re); acc.add(ai++, im);
    }
    if (P.first) {
      R p[NR];
      R T = 0;
#pragma unroll
      for (int j = 0; j < NR; ++j) { p[j] = fma(v[j].x, v[j].x, v[j].y * v[j].y); T += p[j]; }
#pragma unroll
      for (int sl = 0; sl < RB; ++sl) {
        R q = 0;
#pragma unroll
        for (int j = 0; j < NR; ++j)
          if ((j >> sl) & 1) q += p[j];
        acc.add(ai++, q);
      }
      for (int k = 0; k < 5; ++k) acc.add(ai++, ((lane >> k) & 1) ? T : (R)0);
      double t = warp_sum((double)T);
      if (lane == 0) tile_tot[tau * 8 + warp] = t;
    }
  }
  // CTA reduction of every accumulator in a fixed order
  __syncthreads();
  double* red = (double*)(smraw + 256 + SAcc<R>::bytes(nacc));   // [8 warps]
  for (int i = 0; i < nacc; ++i) {
    double x = warp_sum(acc.get(i));
    if (lane == 0) red[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < ETPB / 32; ++w) t += red[w];
      part[(size_t)blockIdx.x * nacc + i] = t;
    }
    __syncthreads();
  }
}

// P1 of the warp and outer qubits from the per-(tile, warp) totals: one
// column per qubit (col 0 = total), rows = CTAs of a grid-stride sum.
__global__ void k_tile_bits(const double* __restrict__ tile_tot, uint64_t ntiles, RedParams P, int nq_out,
                            const uint8_t* __restrict__ qlist, double* __restrict__ part) {
  // thread handles (tile, warp) entries in a grid-stride loop; per-thread sums
  // for the total and for each listed qubit (<= 40)
  double acc[41];
  for (int i = 0; i <= nq_out; ++i) acc[i] = 0.0;
  const uint64_t n = ntiles * 8;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t tau = e >> 3;
    const int w = (int)(e & 7);
    uint64_t g = deposit(tau, P.out_mask);
    for (int k = 0; k < 3; ++k)
      if ((w >> k) & 1) g |= 1ull << P.warp_g[k];
    const double x = tile_tot[e];
    acc[0] += x;
    for (int i = 0; i < nq_out; ++i)
      if ((g >> qlist[i]) & 1) acc[i + 1] += x;
  }
  __shared__ double sh[32];
  for (int i = 0; i <= nq_out; ++i) {
    double r = block_sum(acc[i], sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * (nq_out + 1) + i] = r;
    __syncthreads();
  }
}

// ---- marginal -------------------------------------------------------------------------------
// Thread t handles register value t (bits in ascending qubit order) and one
// segment of the complement; part[seg * R + kout] = sum over the segment.
struct MargGeo {
  int N, nq;
  int sq[24];       // register qubits, ascending
  int outbit[24];   // output bit of sq[m]
  uint64_t cmask;   // complement mask
  uint64_t seglen;  // complement values per segment (power of two)
  int nseg_log;
};

template <typename A>
__device__ __forceinline__ double sqa(const A& a, const float* r) { return sq(a); }
template <>
__device__ __forceinline__ double sqa<uint16_t>(const uint16_t& w, const float* r) {
  const double m = (double)r[(w & 0xFFu) ^ 0x80u];
  return m * m;
}
template <typename A>
__global__ void __launch_bounds__(TPB) k_marginal(const A* __restrict__ s, MargGeo g, double* part, const A2Dev* a2) {
  __shared__ Luts L;
  if (a2) build_luts(L, a2->r0, a2->r1);
  const uint64_t R = 1ull << g.nq;
  const uint64_t tid = (uint64_t)blockIdx.x * TPB + threadIdx.x;
  if (tid >= (R << g.nseg_log)) return;
  const uint64_t t = tid & (R - 1);
  const uint64_t seg = tid >> g.nq;
  uint64_t ireg = 0, kout = 0;
  for (int m = 0; m < g.nq; ++m) {
    uint64_t bit = (t >> m) & 1ull;
    ireg |= bit << g.sq[m];
    kout |= bit << g.outbit[m];
  }
  // first complement value of this segment: deposit(seg * seglen, cmask)
  uint64_t x = deposit(seg * g.seglen, g.cmask);
  double acc = 0.0;
  for (uint64_t j = 0; j < g.seglen; ++j) {
    acc += sqa<A>(s[ireg | x], L.r);
    x = (x - g.cmask) & g.cmask;  // next subset of cmask in increasing order
  }
  part[seg * R + kout] = acc;
}

}  // namespace

// =====================================================================================
qs_status ensure_scratch(qs_sim* s, size_t bytes) {
  if (s->scratch_bytes >= bytes) return QS_OK;
  if (s->scratch) QS_CUDA(cudaFreeAsync(s->scratch, s->stream));
  s->scratch = nullptr;
  s->scratch_bytes = 0;
  QS_CUDA(cudaMallocAsync(&s->scratch, bytes, s->stream));
  s->scratch_bytes = bytes;
  return QS_OK;
}
qs_status ensure_hbuf(qs_sim* s, size_t bytes) {
  if (s->hbuf_bytes >= bytes) return QS_OK;
  if (s->hbuf) {
    QS_CUDA(cudaStreamSynchronize(s->stream));
    QS_CUDA(cudaFreeHost(s->hbuf));
  }
  s->hbuf = nullptr;
  s->hbuf_bytes = 0;
  QS_CUDA(cudaMallocHost(&s->hbuf, bytes));
  s->hbuf_bytes = bytes;
  return QS_OK;
}

static int reduce_grid(qs_sim* s) { return s->num_sms * 8; }

qs_status launch_norm(qs_sim* s, double* out) {
  const int G = reduce_grid(s);
  QS_TRY(ensure_scratch(s, (size_t)(G + 1) * sizeof(double)));
  double* part = (double*)s->scratch;
  if (s->enc == QS_C128) {
    k_norm_c128<<<G, TPB, 0, s->stream>>>((const double2*)s->state, 1ull << s->N, part);
  } else if (s->enc == QS_C64) {
    k_norm_c64<<<G, TPB, 0, s->stream>>>((const float4*)s->state, 1ull << (s->N - 1), part);
  } else {
    return QS_EUNSUPPORTED;
  }
  QS_LAUNCH_CHECK();
  k_sum_columns<<<1, TPB, 0, s->stream>>>(part, G, 1, part + G);
  QS_LAUNCH_CHECK();
  QS_TRY(ensure_hbuf(s, sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(s->hbuf, part + G, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  *out = *(double*)s->hbuf;
  return QS_OK;
}

template <typename R, int RB, int ENC>
static qs_status expect_impl(qs_sim* s, double* qx, double* qy, double* qz) {
  const int N = s->N;
  const int b = RB + 8;
  if (N < b) return QS_EUNSUPPORTED;  // small states use the generic path
  const int G = s->num_sms * 2;
  const uint64_t ntiles = 1ull << (N - b);
  const int grid = (int)(ntiles < (uint64_t)G ? ntiles : (uint64_t)G);
  // pass list: pass 0 = qubits 0..5 (slot 0 + lanes) + slots 1..RB-1 = qubits 6..RB+4,
  // warps = the next 3 qubits; later passes take RB-1 new qubits as slots.
  struct Pass { RedParams P; int qs[8]; };
  Pass passes[32];
  int np = 0;
  int next = 6;
  while (next < N || np == 0) {
    Pass& ps = passes[np];
    memset(&ps, 0, sizeof ps);
    RedParams& P = ps.P;
    P.N = N; P.RB = RB; P.first = (np == 0);
    uint64_t tmask = 63ull;
    P.slot_g[0] = 0;
    int ns = 0;
    for (int sl = 1; sl < RB && next < N; ++sl) { P.slot_g[sl] = (uint8_t)next; tmask |= 1ull << next; ps.qs[ns++] = next++; }
    P.nslots_new = ns;
    // fill the remaining slots and the warp bits with unused qubits (not new)
    int fill = 6;
    auto take = [&]() { while ((tmask >> fill) & 1) ++fill; tmask |= 1ull << fill; return fill; };
    for (int sl = ns + 1; sl < RB; ++sl) P.slot_g[sl] = (uint8_t)take();
    for (int k = 0; k < 3; ++k) P.warp_g[k] = (uint8_t)take();
    const uint64_t all = (N >= 64) ? ~0ull : ((1ull << N) - 1);
    P.out_mask = all & ~tmask;
    ++np;
  }
  // scratch: per pass partials, tile totals, column results
  const int nacc0 = 2 * (1 + 5 + passes[0].P.nslots_new) + RB + 5;
  const int nq_out = N - 6 - (RB - 1) >= 0 ? (3 + (N - b)) : 0;
  size_t off = 0;
  size_t part_off[32], res_off[32];
  int nacc_of[32];
  for (int i = 0; i < np; ++i) {
    nacc_of[i] = (i == 0) ? nacc0 : 2 * passes[i].P.nslots_new;
    part_off[i] = off; off += (size_t)grid * nacc_of[i];
    res_off[i] = off; off += nacc_of[i];
  }
  const size_t tt_off = off; off += ntiles * 8;
  const int gtb = 64;
  const size_t tbp_off = off; off += (size_t)gtb * (nq_out + 1);
  const size_t tbr_off = off; off += nq_out + 1;
  const size_t ql_off = off; off += 8;   // 64 bytes of qubit list
  QS_TRY(ensure_scratch(s, off * sizeof(double)));
  double* sc = (double*)s->scratch;
  // warp + outer qubits of pass 0, in the order used by k_tile_bits
  uint8_t ql[64];
  int nql = 0;
  {
    const RedParams& P0 = passes[0].P;
    for (int k = 0; k < 3; ++k) ql[nql++] = P0.warp_g[k];
    for (int q = 0; q < N; ++q)
      if ((P0.out_mask >> q) & 1) ql[nql++] = (uint8_t)q;
  }
  QS_CUDA(cudaMemcpyAsync(sc + ql_off, ql, 64, cudaMemcpyHostToDevice, s->stream));
  for (int i = 0; i < np; ++i) {
    const size_t smem = 256 + SAcc<R>::bytes(nacc_of[i]) + 8 * sizeof(double);
    QS_CUDA(cudaFuncSetAttribute(k_expect2<R, RB, ENC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_expect2<R, RB, ENC><<<grid, ETPB, smem, s->stream>>>(s->state, passes[i].P, sc + tt_off, sc + part_off[i],
                                                           (const A2Dev*)s->a2dev);
    QS_LAUNCH_CHECK();
    k_sum_columns<<<nacc_of[i], TPB, 0, s->stream>>>(sc + part_off[i], grid, nacc_of[i], sc + res_off[i]);
    QS_LAUNCH_CHECK();
  }
  k_tile_bits<<<gtb, TPB, 0, s->stream>>>(sc + tt_off, ntiles, passes[0].P, nql, (const uint8_t*)(sc + ql_off),
                                          sc + tbp_off);
  QS_LAUNCH_CHECK();
  k_sum_columns<<<nql + 1, TPB, 0, s->stream>>>(sc + tbp_off, gtb, nql + 1, sc + tbr_off);
  QS_LAUNCH_CHECK();
  QS_TRY(ensure_hbuf(s, off * sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(s->hbuf, sc, off * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  const double* h = (const double*)s->hbuf;
  const double* t = h + tbr_off;
  const double nrm = t[0];
  for (int i = 0; i < nql; ++i) qz[ql[i]] = t[i + 1];
  const double* r0 = h + res_off[0];
  const RedParams& P0 = passes[0].P;
  // pass 0 layout: w(slot 0), w(lanes 0..4), w(slots 1..ns), P1(slots 0..RB-1), P1(lanes 0..4)
  int ai = 0;
  auto setw = [&](int q, const double* r) { qx[q] = 0.5 * nrm - r[0]; qy[q] = 0.5 * nrm - r[1]; };
  setw(0, r0 + ai); ai += 2;
  for (int k = 0; k < 5; ++k) { setw(k + 1, r0 + ai); ai += 2; }
  for (int sl = 1; sl <= P0.nslots_new; ++sl) { setw(P0.slot_g[sl], r0 + ai); ai += 2; }
  for (int sl = 0; sl < RB; ++sl) { qz[P0.slot_g[sl]] = r0[ai]; ++ai; }
  for (int k = 0; k < 5; ++k) { qz[k + 1] = r0[ai]; ++ai; }
  for (int i = 1; i < np; ++i) {
    const double* r = h + res_off[i];
    for (int sl = 1; sl <= passes[i].P.nslots_new; ++sl) setw(passes[i].P.slot_g[sl], r + 2 * (sl - 1));
  }
  return QS_OK;
}

static qs_status expect_small(qs_sim* s, double* qx, double* qy, double* qz) {
  if (s->N > 12) return QS_EUNSUPPORTED;
  QS_TRY(ensure_scratch(s, sizeof(double) * (1 + 3 * s->N)));
  double* d = (double*)s->scratch;
  if (s->enc == QS_C128) k_expect_small<double2><<<1, TPB, 0, s->stream>>>((const double2*)s->state, s->N, d, nullptr);
  else if (s->enc == QS_C64) k_expect_small<float2><<<1, TPB, 0, s->stream>>>((const float2*)s->state, s->N, d, nullptr);
  else k_expect_small<uint16_t><<<1, TPB, 0, s->stream>>>((const uint16_t*)s->state, s->N, d, (const A2Dev*)s->a2dev);
  QS_LAUNCH_CHECK();
  QS_TRY(ensure_hbuf(s, sizeof(double) * (1 + 3 * s->N)));
  QS_CUDA(cudaMemcpyAsync(s->hbuf, d, sizeof(double) * (1 + 3 * s->N), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  const double* h = (const double*)s->hbuf;
  for (int q = 0; q < s->N; ++q) {
    qx[q] = 0.5 * h[0] - h[1 + 3 * q];
    qy[q] = 0.5 * h[0] - h[2 + 3 * q];
    qz[q] = h[3 + 3 * q];
  }
  return QS_OK;
}

qs_status launch_expect(qs_sim* s, double* qx, double* qy, double* qz) {
  if (s->enc == QS_C128 && s->N >= 12) return expect_impl<double, 4, 1>(s, qx, qy, qz);
  if (s->enc == QS_C64 && s->N >= 13) return expect_impl<float, 5, 0>(s, qx, qy, qz);
  if (s->enc == QS_ADAPT2 && s->N >= 13) return expect_impl<float, 5, 2>(s, qx, qy, qz);
  return expect_small(s, qx, qy, qz);
}

template <typename A>
static qs_status marginal_impl(qs_sim* s, const int* qubits, int nq, double* out) {
  MargGeo g;
  g.N = s->N; g.nq = nq;
  int idx[24];
  for (int m = 0; m < nq; ++m) idx[m] = m;
  for (int i = 0; i < nq; ++i)
    for (int j = i + 1; j < nq; ++j)
      if (qubits[idx[j]] < qubits[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
  uint64_t qmask = 0;
  for (int m = 0; m < nq; ++m) { g.sq[m] = qubits[idx[m]]; g.outbit[m] = idx[m]; qmask |= 1ull << qubits[m]; }
  const uint64_t all = (s->N >= 64) ? ~0ull : ((1ull << s->N) - 1);
  g.cmask = all & ~qmask;
  const int cbits = s->N - nq;
  // enough threads: R * nseg >= 2^20 when possible
  int nseg_log = 0;
  while (nq + nseg_log < 20 && nseg_log < cbits) ++nseg_log;
  g.nseg_log = nseg_log;
  g.seglen = 1ull << (cbits - nseg_log);
  const uint64_t R = 1ull << nq;
  const uint64_t nthreads = R << nseg_log;
  QS_TRY(ensure_scratch(s, (size_t)(nthreads + R) * sizeof(double)));
  double* part = (double*)s->scratch;
  k_marginal<A><<<(unsigned)((nthreads + TPB - 1) / TPB), TPB, 0, s->stream>>>((const A*)s->state, g, part,
                                                                             (const A2Dev*)s->a2dev);
  QS_LAUNCH_CHECK();
  double* res = part + nthreads;
  // column sums over the 2^nseg_log segment rows, fixed order
  for (uint64_t c0 = 0; c0 < R; c0 += 65535) {
    uint64_t nc = (R - c0) < 65535 ? (R - c0) : 65535;
    // sum rows r of column c: part[r * R + c]; emulate with a shifted base
    k_sum_columns<<<(unsigned)nc, TPB, 0, s->stream>>>(part + c0, 1 << nseg_log, (int)R, res + c0);
    QS_LAUNCH_CHECK();
  }
  QS_TRY(ensure_hbuf(s, R * sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(s->hbuf, res, R * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  memcpy(out, s->hbuf, R * sizeof(double));
  return QS_OK;
}

qs_status launch_marginal(qs_sim* s, const int* qubits, int nq, double* out) {
  if (s->enc == QS_C128) return marginal_impl<double2>(s, qubits, nq, out);
  if (s->enc == QS_C64) return marginal_impl<float2>(s, qubits, nq, out);
  return marginal_impl<uint16_t>(s, qubits, nq, out);
}

qs_status sum_partials(qs_sim* s, const double* part, int n, double* out) {
  k_sum_columns<<<1, TPB, 0, s->stream>>>(part, n, 1, out);
  QS_LAUNCH_CHECK();
  return QS_OK;
}

// =====================================================================================
// measure_probs_static: the register marginal without any allocation.
//
// Some callers cannot allocate device memory: a host framework whose memory
// pool already owns the device's memory, or a latency-critical loop that must
// not enter the driver's allocator.  This entry point works on a device buffer
// the caller already holds and keeps its scratch in a fixed array in the
// library's device memory (QS_STATIC_SCRATCH_DOUBLES doubles, 2.5 MiB, held by
// every GPU that loads the library until the process exits).
// =====================================================================================
#include <mutex>

#define QS_STATIC_MAX_NQ 16
#define QS_STATIC_PARTIALS (1 << 18)
#define QS_STATIC_SCRATCH_DOUBLES (QS_STATIC_PARTIALS + (1 << QS_STATIC_MAX_NQ))
#define QS_STATIC_MAX_DEVICES 64

static __device__ __align__(256) double g_static_scratch[QS_STATIC_SCRATCH_DOUBLES];

static std::mutex g_static_mu;
static double* g_static_addr[QS_STATIC_MAX_DEVICES];

// Device address of g_static_scratch on the current device.  The name of the
// array in host code is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
static qs_status static_scratch_addr(double** out) {
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= QS_STATIC_MAX_DEVICES) {
    qs_set_error("measure_probs_static: device %d beyond the %d supported", dev, QS_STATIC_MAX_DEVICES);
    return QS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      qs_set_error("measure_probs_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return QS_ECUDA;
    }
    g_static_addr[dev] = (double*)p;
  }
  *out = g_static_addr[dev];
  return QS_OK;
}

template <typename A>
static qs_status marginal_static_impl(const void* state, int N, const int* qubits, int nq, double* out,
                                      cudaStream_t stream, double* scratch) {
  MargGeo g;
  g.N = N; g.nq = nq;
  int idx[24];
  for (int m = 0; m < nq; ++m) idx[m] = m;
  for (int i = 0; i < nq; ++i)
    for (int j = i + 1; j < nq; ++j)
      if (qubits[idx[j]] < qubits[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
  uint64_t qmask = 0;
  for (int m = 0; m < nq; ++m) { g.sq[m] = qubits[idx[m]]; g.outbit[m] = idx[m]; qmask |= 1ull << qubits[m]; }
  const uint64_t all = (N >= 64) ? ~0ull : ((1ull << N) - 1);
  g.cmask = all & ~qmask;
  const int cbits = N - nq;
  // at most QS_STATIC_PARTIALS partial sums: R * 2^nseg_log <= 2^18
  int nseg_log = 0;
  while (nq + nseg_log < 18 && nseg_log < cbits) ++nseg_log;
  g.nseg_log = nseg_log;
  g.seglen = 1ull << (cbits - nseg_log);
  const uint64_t R = 1ull << nq;
  const uint64_t nthreads = R << nseg_log;
  double* part = scratch;                       // every entry written by k_marginal
  double* res = scratch + QS_STATIC_PARTIALS;   // every entry written by k_sum_columns
  k_marginal<A><<<(unsigned)((nthreads + TPB - 1) / TPB), TPB, 0, stream>>>((const A*)state, g, part, nullptr);
  QS_LAUNCH_CHECK();
  k_sum_columns<<<(unsigned)R, TPB, 0, stream>>>(part, 1 << nseg_log, (int)R, res);
  QS_LAUNCH_CHECK();
  QS_CUDA(cudaMemcpyAsync(out, res, R * sizeof(double), cudaMemcpyDeviceToHost, stream));
  QS_CUDA(cudaStreamSynchronize(stream));
  return QS_OK;
}

extern "C" qs_status measure_probs_static(const void* state, int N, qs_encoding enc, const int* qubits, int nq,
                                          double* out, void* cuda_stream) {
  if (!state || !qubits || !out) { qs_set_error("measure_probs_static: null argument"); return QS_EINVAL; }
  if (N < 2 || N > 44) { qs_set_error("measure_probs_static: N = %d not in 2..44", N); return QS_EINVAL; }
  if (enc != QS_C128 && enc != QS_C64) {
    qs_set_error("measure_probs_static: only QS_C128 and QS_C64 states");
    return QS_EUNSUPPORTED;
  }
  if (nq < 1 || nq > N || nq > QS_STATIC_MAX_NQ) {
    qs_set_error("measure_probs_static: nq = %d not in 1..min(N, %d): the static scratch holds %d doubles", nq,
                 QS_STATIC_MAX_NQ, QS_STATIC_SCRATCH_DOUBLES);
    return QS_EINVAL;
  }
  for (int i = 0; i < nq; ++i) {
    if (qubits[i] < 0 || qubits[i] >= N) { qs_set_error("measure_probs_static: qubit %d out of range", qubits[i]); return QS_EINVAL; }
    for (int j = 0; j < i; ++j)
      if (qubits[i] == qubits[j]) { qs_set_error("measure_probs_static: qubit %d repeated", qubits[i]); return QS_EINVAL; }
  }
  double* scratch = nullptr;
  QS_TRY(static_scratch_addr(&scratch));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (enc == QS_C128) return marginal_static_impl<double2>(state, N, qubits, nq, out, st, scratch);
  return marginal_static_impl<float2>(state, N, qubits, nq, out, st, scratch);
}
