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
#include "tma.cuh"
#include <string.h>
#include <type_traits>

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

// ---- expect_xyz for complex128: register-tile passes ---------------------------------------
// (complex64 and the adaptive words use the shared-memory views further down.)
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
// Per-thread sums are formed per tile in FP64 and folded into per-thread
// accumulators in shared memory, then reduced over the CTA and the grid in a
// fixed order.
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

template <typename R, int RB>
__global__ void __launch_bounds__(ETPB, 2) k_expect2(const void* __restrict__ s, const __grid_constant__ RedParams P,
                                                      double* __restrict__ tile_tot, double* __restrict__ part) {
  static_assert(sizeof(R) == 8, "complex128 only");
  extern __shared__ __align__(16) unsigned char smraw[];
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
    const double2* s2 = (const double2*)s;
#pragma unroll
    for (int jj = 0; jj < NR / 2; ++jj) {
      double2 x = s2[base + roff[jj]], y = s2[base + roff[jj] + 1];
      v[2 * jj] = cx<double>(x.x, x.y);
      v[2 * jj + 1] = cx<double>(y.x, y.y);
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

// ---- expect_xyz for complex64 and adaptive words: shared-memory views ------------------
// A tile is 2^13 amplitudes: local bits 0..3 are index bits 0..3 (128-byte
// runs of complex64), local bits 4..3+f the qubits 4..3+f and local bits
// 4+f..12 a run of 9-f consecutive qubits b..b+8-f.  Pass 0 takes qubits
// 0..12 (f = 0, b = 4); the later passes split qubits 13..N-1 into runs of
// near-equal length (at most 9), each padded with the low qubits 4.. (already
// served).  Each of 256 threads holds 32 amplitudes of the tile in
// registers, in one of three views (register bits; the thread index covers
// the other 8 local bits):
//   view A: local {0, 6, 7, 8, 9}    lanes = local 1..5, warps = local 10..12
//   view B: local {4, 5, 10, 11, 12}
//   view C: local {1, 2, 3, 7, 8}    (the last pass only)
// A qubit that is a register bit of a view gets w_n from pairs held by one
// thread, so pass 0 serves qubits 0 and 4..12, the last pass qubits 1..3,
// and every later pass up to 9 new qubits (3 passes at N = 30: 0..12,
// 13..21, 4 + 22..29).  Splitting the runs evenly keeps a tile within 2^8 of
// the 2 MB pages of the state where it can: tiles spread over 2^9 pages
// measured 1.1-1.5x slower.  The tile sits in shared memory in the 128-byte swizzle
// of the tensor loads (complex64 units: local bits 4..6 flip bits 1..3),
// under which all three views read without bank conflicts.
//
// Per tile each thread forms FP32 leaf sums (at most 16 pairs or 16 |a|^2)
// and folds them into float-float accumulators in registers; the CTA sums
// those in FP64 in a fixed order at the end, the grid by k_sum_columns.
namespace xv {
constexpr int TB = 13;      // tile bits
constexpr int NV = 16;      // values per view: w re/im of 5 slots, then P1 of 5 slots
constexpr int NVIEW = 3;
constexpr int NCOL = NV * NVIEW;
constexpr uint8_t REG_A[5] = {0, 6, 7, 8, 9};
constexpr uint8_t REG_B[5] = {4, 5, 10, 11, 12};
constexpr uint8_t REG_C[5] = {1, 2, 3, 7, 8};
__host__ __device__ constexpr uint32_t phys(uint32_t l) { return l ^ (((l >> 4) & 7u) << 1); }
__host__ __device__ constexpr uint32_t reg_a(int j) { return (uint32_t)(j & 1) | ((uint32_t)(j >> 1) << 6); }
__host__ __device__ constexpr uint32_t reg_b(int j) { return ((uint32_t)(j & 3) << 4) | ((uint32_t)(j >> 2) << 10); }
__host__ __device__ constexpr uint32_t reg_c(int j) { return ((uint32_t)(j & 7) << 1) | ((uint32_t)(j >> 3) << 7); }
__device__ __forceinline__ uint32_t thr_a(int t) { return ((uint32_t)(t & 31) << 1) | ((uint32_t)(t >> 5) << 10); }
__device__ __forceinline__ uint32_t thr_b(int t) { return (uint32_t)(t & 15) | ((uint32_t)(t >> 4) << 6); }
__device__ __forceinline__ uint32_t thr_c(int t) {
  return (uint32_t)(t & 1) | ((uint32_t)((t >> 1) & 7) << 4) | ((uint32_t)(t >> 4) << 9);
}
}  // namespace xv

struct XParams {
  int N;
  int f, b;               // local bits 4..3+f: qubits 4..3+f; 4+f..12: qubits b..b+8-f
  int lo_bits;            // tile-index bits below the run (qubits 4+f..b-1)
  uint64_t out_mask;      // global bits outside the tile
  uint64_t roff_a[16];    // register loads: global offset of view-A register pair (2jj, 2jj+1)
  uint8_t gpos[16];       // global qubit of local bit k
};

// Per-thread float-float accumulators of one pass: view A and B hold w re/im
// of their 5 register slots (and in the first pass P1 of each slot), view C
// (VC: the last pass, whose ALU load is lighter) w and P1 of its slots 0..2,
// qubits 1..3, which every tile holds.
// NORM: one more accumulator, sum |a|^2 from exact products (column 15).
template <bool FIRST, bool VC, bool NORM = false>
struct XAcc {
  static constexpr int NA = FIRST ? 15 : 10, NC = VC ? 9 : 0, N = 2 * NA + NC + (NORM ? 1 : 0);
  FF f[N];
  // output column of accumulator i (16 columns per view: w re/im of slot s at
  // 2s, 2s+1, P1 of slot s at 10+s; the norm at 15)
  __host__ __device__ static constexpr int col(int i) {
    return i < NA ? i
           : i < 2 * NA ? xv::NV + (i - NA)
           : i < 2 * NA + NC ? 2 * xv::NV + (i - 2 * NA < 6 ? i - 2 * NA : 4 + (i - 2 * NA))
                             : xv::NV - 1;
  }
};
constexpr int XNORM_COL = xv::NV - 1;

// Fold one view's per-thread leaf sums (FP32, at most 16 pairs each) into
// acc[0 .. 2NS-1] (w re/im of slots 0..NS-1) and, with P1, acc[2NS ..
// 3NS-1] (P1 of the slots); T = sum of all |a|^2 of the thread.
template <int NS, bool P1>
__device__ __forceinline__ void view_fold(const Cx<float>* v, FF* acc, float& T) {
  float re, im;
  slot_w<float, 5, 0>(v, re, im); ff_add(acc[0], re); ff_add(acc[1], im);
  slot_w<float, 5, 1>(v, re, im); ff_add(acc[2], re); ff_add(acc[3], im);
  slot_w<float, 5, 2>(v, re, im); ff_add(acc[4], re); ff_add(acc[5], im);
  if constexpr (NS > 3) { slot_w<float, 5, 3>(v, re, im); ff_add(acc[6], re); ff_add(acc[7], im); }
  if constexpr (NS > 4) { slot_w<float, 5, 4>(v, re, im); ff_add(acc[8], re); ff_add(acc[9], im); }
  T = 0.f;
  if constexpr (P1) {
    // halving tree: at level s the sums over register bits < s are paired;
    // P1 of slot s is the sum of the odd members of level s
    float p[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) p[j] = fmaf(v[j].x, v[j].x, v[j].y * v[j].y);
#pragma unroll
    for (int sl = 0, n = 32; sl < 5; ++sl, n >>= 1) {
      if (sl < NS) {
        float q = p[1];
#pragma unroll
        for (int i = 3; i < n; i += 2) q += p[i];
        ff_add(acc[2 * NS + sl], q);
      }
#pragma unroll
      for (int i = 0; i < n / 2; ++i) p[i] = p[2 * i] + p[2 * i + 1];
    }
    T = p[0];
  }
}

// View A is in v; folds it, then views C (VC) and B read from the shared
// tile xt.  FIRST also writes the per-(tile, warp) total of |a|^2.
template <bool FIRST, bool VC, bool NORM>
__device__ __forceinline__ void tile_views(const float2* xt, Cx<float> (&v)[32], XAcc<FIRST, VC, NORM>& acc,
                                           uint64_t tau, double* __restrict__ tile_tot) {
  const int t = threadIdx.x;
  constexpr int NA = XAcc<FIRST, VC, NORM>::NA;
  if constexpr (NORM) {   // sum |a|^2 of view A's registers, products exact
    FF& f = acc.f[XAcc<FIRST, VC, NORM>::N - 1];
#pragma unroll
    for (int j = 0; j < 32; ++j) { ff_add_prod(f, v[j].x, v[j].x); ff_add_prod(f, v[j].y, v[j].y); }
  }
  float T;
  view_fold<5, FIRST>(v, acc.f, T);
  if (FIRST) {
    const double tt = warp_sum((double)T);
    if ((t & 31) == 0) tile_tot[tau * 8 + (t >> 5)] = tt;
  }
  if constexpr (VC) {
    const uint32_t pc = xv::phys(xv::thr_c(t));
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float2 q = xt[pc ^ xv::phys(xv::reg_c(j))];
      v[j] = cx<float>(q.x, q.y);
    }
    view_fold<3, true>(v, acc.f + 2 * NA, T);
  }
  const uint32_t pb = xv::phys(xv::thr_b(t));
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float2 q = xt[pb ^ xv::phys(xv::reg_b(j))];
    v[j] = cx<float>(q.x, q.y);
  }
  view_fold<5, FIRST>(v, acc.f + NA, T);
}

// CTA sum of the accumulators in FP64 in a fixed order (warp tree, then the 8
// warps in order) into part[block][column]; red: XAcc::N * 8 doubles of
// shared memory.  Columns no accumulator maps to are written as 0.
template <bool FIRST, bool VC, bool NORM>
__device__ __forceinline__ void views_to_part(const XAcc<FIRST, VC, NORM>& acc, double* red,
                                              double* __restrict__ part) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int M = XAcc<FIRST, VC, NORM>::N;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const double d = warp_sum((double)acc.f[i].hi + (double)acc.f[i].lo);
    if (lane == 0) red[i * 8 + warp] = d;
  }
  __syncthreads();
  if (t < xv::NCOL) part[(size_t)blockIdx.x * xv::NCOL + t] = 0.0;
  __syncthreads();
  if (t < M) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += red[t * 8 + w];
    part[(size_t)blockIdx.x * xv::NCOL + XAcc<FIRST, VC, NORM>::col(t)] = sum;
  }
}

// complex64: one persistent CTA per SM; thread 0 streams the CTA's tiles
// through a ring of XSTAGES shared-memory buffers with 5-D tensor loads
// (dims: qubits 0..3, the two tile segments, then the qubits below and above
// the run: the tile index, low bits first), the whole CTA
// consumes them in order.  A wait that runs out makes every thread leave the
// loop; thread 0 then waits (bounded) for the loads still in flight and sets
// *err.
constexpr int XSTAGES = 3;
constexpr uint32_t XTILE_BYTES = 8u << xv::TB;
constexpr size_t XTMA_SMEM = (size_t)XSTAGES * XTILE_BYTES + 1024 + 64;

template <bool FIRST, bool VC, bool NORM>
__global__ void __launch_bounds__(ETPB, 1) k_expect_tma(const __grid_constant__ CUtensorMap map,
                                                         const __grid_constant__ XParams P,
                                                         double* __restrict__ tile_tot, double* __restrict__ part,
                                                         int* __restrict__ err, uint32_t spins) {
  using namespace qs_tma;
  extern __shared__ unsigned char xraw[];
  const uint32_t raw_s = smem_u32(xraw);
  unsigned char* buf = xraw + (((raw_s + 1023u) & ~1023u) - raw_s);   // the swizzle repeats every 1024 bytes
  uint64_t* full = (uint64_t*)(buf + XSTAGES * XTILE_BYTES);
  volatile int* abort_flag = (volatile int*)(full + XSTAGES);
  const int t = threadIdx.x;
  if (t == 0) {
    for (int st = 0; st < XSTAGES; ++st) mbar_init(smem_u32(&full[st]), 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const uint64_t ntiles = 1ull << (P.N - xv::TB);
  const uint64_t nmine = (uint64_t)blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int lo_bits = P.lo_bits;
  uint64_t issued = 0;           // thread 0 only
  auto issue = [&]() {
    const uint64_t tau = blockIdx.x + issued * gridDim.x;
    const int st = (int)(issued % XSTAGES);
    const uint32_t bar = smem_u32(&full[st]);
    mbar_expect_tx(bar, XTILE_BYTES);
    tma_load_5d(smem_u32(buf + st * XTILE_BYTES), &map, 0, 0, 0, (int)(tau & ((1ull << lo_bits) - 1)),
                (int)(tau >> lo_bits), bar);
    ++issued;
  };
  if (t == 0)
    while (issued < nmine && issued < (uint64_t)XSTAGES) issue();
  const uint32_t pa = xv::phys(xv::thr_a(t));
  XAcc<FIRST, VC, NORM> acc;
#pragma unroll
  for (int i = 0; i < XAcc<FIRST, VC, NORM>::N; ++i) acc.f[i] = {0.f, 0.f};
  Cx<float> v[32];
  uint64_t k = 0;
  bool ok = true;
  for (; k < nmine; ++k) {
    const int st = (int)(k % XSTAGES);
    const float2* xt = (const float2*)(buf + st * XTILE_BYTES);
    const bool got = mbar_wait_or_abort(smem_u32(&full[st]), (uint32_t)((k / XSTAGES) & 1), abort_flag, spins);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const float4 q = *(const float4*)&xt[pa ^ xv::phys(xv::reg_a(2 * jj))];
      v[2 * jj] = cx<float>(q.x, q.y);
      v[2 * jj + 1] = cx<float>(q.z, q.w);
    }
    tile_views<FIRST, VC, NORM>(xt, v, acc, blockIdx.x + k * gridDim.x, tile_tot);
    if (!bar_and(1, ETPB, got)) { ok = false; break; }   // also: the stage is free again
    if (t == 0 && issued < nmine) issue();
  }
  if (!ok) {
    if (t == 0) {
      for (uint64_t kk = k; kk < issued; ++kk) mbar_wait(smem_u32(&full[kk % XSTAGES]), (uint32_t)((kk / XSTAGES) & 1));
      atomicExch(err, 1);
    }
    return;
  }
  views_to_part<FIRST, VC, NORM>(acc, (double*)buf, part);
}

// adaptive 2-byte words: each thread loads its view-A words from global memory
// and decodes them, the tile goes through shared memory for views C and B.
template <bool FIRST, bool VC>
__global__ void __launch_bounds__(ETPB, FIRST || VC ? 1 : 2) k_expect_ld(const unsigned int* __restrict__ s2,
                                                        const __grid_constant__ XParams P,
                                                        double* __restrict__ tile_tot, double* __restrict__ part,
                                                        const A2Dev* __restrict__ a2) {
  extern __shared__ __align__(16) float2 xt[];   // the tile, 2^13 complex64, swizzled
  __shared__ Luts L;
  build_luts(L, a2->r0, a2->r1);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t pa = xv::phys(xv::thr_a(t));
  uint64_t woff = 0;
  for (int k = 0; k < 5; ++k)
    if ((lane >> k) & 1) woff |= 1ull << P.gpos[1 + k];
  for (int k = 0; k < 3; ++k)
    if ((warp >> k) & 1) woff |= 1ull << P.gpos[10 + k];
  XAcc<FIRST, VC, false> acc;
#pragma unroll
  for (int i = 0; i < XAcc<FIRST, VC, false>::N; ++i) acc.f[i] = {0.f, 0.f};
  const uint64_t ntiles = 1ull << (P.N - xv::TB);
  Cx<float> v[32];
  for (uint64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
    const uint64_t base = deposit(tau, P.out_mask) | woff;
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const unsigned int w = s2[(base + P.roff_a[jj]) >> 1];
      v[2 * jj] = a2_dec(L, w & 0xFFFFu);
      v[2 * jj + 1] = a2_dec(L, w >> 16);
    }
    __syncthreads();   // every view read of the previous tile is done
#pragma unroll
    for (int jj = 0; jj < 16; ++jj)
      *(float4*)&xt[pa ^ xv::phys(xv::reg_a(2 * jj))] =
          make_float4(v[2 * jj].x, v[2 * jj].y, v[2 * jj + 1].x, v[2 * jj + 1].y);
    __syncthreads();
    tile_views<FIRST, VC, false>(xt, v, acc, tau, tile_tot);
  }
  __syncthreads();
  views_to_part<FIRST, VC, false>(acc, (double*)xt, part);
}

// ---- marginal -------------------------------------------------------------------------------
// Thread t handles register value t (bits in ascending qubit order) and one
// segment of the complement; part[seg * R + kout] = sum over the segment.
struct MargGeo {
  int N, nq;
  int sq[24];       // register qubits, ascending
  int outbit[24];   // output bit of sq[m]
  uint64_t cmask;   // complement mask
  uint64_t seglen;  // complement values per thread (power of two)
  int nseg_log;     // 2^nseg_log threads per register value
};

// |a|^2 of a complex128 amplitude (FP64 units)
__device__ __forceinline__ double sqa(const double2& a, const float*) { return sq(a); }
// |a|^2 into a float-float sum: complex64 products exact, adaptive-encoding
// magnitudes from the decode table
__device__ __forceinline__ void ff_add_sq(FF& f, const float2& a, const float*) {
  ff_add_prod(f, a.x, a.x);
  ff_add_prod(f, a.y, a.y);
}
__device__ __forceinline__ void ff_add_sq(FF& f, const uint16_t& w, const float* r) {
  const float m = r[(w & 0xFFu) ^ 0x80u];
  ff_add_prod(f, m, m);
}

// Thread (v, u) sums P over register value v's complement values u, u + T,
// u + 2T, ... (T = 2^nseg_log threads per value): consecutive threads read
// consecutive complement values, so a warp's loads are contiguous wherever
// the low index bits lie outside the register.  The next complement value is
// an addition in the deposited domain.  part[u * R + k] = the thread's sum.
template <typename A>
__global__ void __launch_bounds__(TPB) k_marginal(const A* __restrict__ s, MargGeo g, double* part, const A2Dev* a2) {
  __shared__ Luts L;
  if (a2) build_luts(L, a2->r0, a2->r1);
  const uint64_t R = 1ull << g.nq;
  const uint64_t tid = (uint64_t)blockIdx.x * TPB + threadIdx.x;
  if (tid >= (R << g.nseg_log)) return;
  const uint64_t t = tid >> g.nseg_log;
  const uint64_t u = tid & ((1ull << g.nseg_log) - 1);
  uint64_t ireg = 0, kout = 0;
  for (int m = 0; m < g.nq; ++m) {
    uint64_t bit = (t >> m) & 1ull;
    ireg |= bit << g.sq[m];
    kout |= bit << g.outbit[m];
  }
  uint64_t x = deposit(u, g.cmask);
  const uint64_t step = deposit(1ull << g.nseg_log, g.cmask);
  double acc = 0.0;
  if constexpr (std::is_same<A, double2>::value) {
    for (uint64_t j = 0; j < g.seglen; ++j) {
      acc += sqa(s[ireg | x], L.r);
      x = ((x | ~g.cmask) + step) & g.cmask;
    }
  } else {
    // float-float sums of up to 8 values folded into FP64
    for (uint64_t j = 0; j < g.seglen; j += 8) {
      FF f = {0.f, 0.f};
      const uint64_t n = g.seglen - j < 8 ? g.seglen - j : 8;
      for (uint64_t e = 0; e < n; ++e) {
        ff_add_sq(f, s[ireg | x], L.r);
        x = ((x | ~g.cmask) + step) & g.cmask;
      }
      acc += ff_val(f);
    }
  }
  part[u * R + kout] = acc;
}

template <typename A> __device__ __forceinline__ A zero_amp() { return A{}; }
template <> __device__ __forceinline__ uint16_t zero_amp<uint16_t>() { return (uint16_t)0x80u; }

// ---- P(bit q = 0), P(bit q = 1) of one qubit ----------------------------------------
// Pair j (of 2^(N-1)) is i0 = j with a 0 inserted at bit q and i1 = i0 | 2^q,
// the pair of Eq. (NUM2); consecutive threads take consecutive j, so both
// loads of a warp cover contiguous runs for every q and no lane diverges.
// Each block leaves its two sums in part[2 * block + {0, 1}].
__device__ __forceinline__ uint64_t pair_lo(uint64_t j, int q) {
  const uint64_t low = (1ull << q) - 1;
  return ((j & ~low) << 1) | (j & low);
}
template <typename A>
__global__ void __launch_bounds__(TPB) k_qubit_probs(const A* __restrict__ s, uint64_t npairs, int q, double* part,
                                                     const A2Dev* a2) {
  __shared__ double sh[32];
  __shared__ Luts L;
  if (a2) build_luts(L, a2->r0, a2->r1);
  const uint64_t stride = (uint64_t)gridDim.x * TPB;
  const uint64_t bit = 1ull << q;
  double acc0 = 0.0, acc1 = 0.0;
  uint64_t j = (uint64_t)blockIdx.x * TPB + threadIdx.x;
  if constexpr (std::is_same<A, double2>::value) {
    for (; j < npairs; j += stride) {
      const uint64_t i0 = pair_lo(j, q);
      const double2 a = s[i0], b = s[i0 | bit];
      acc0 = fma(a.x, a.x, acc0);
      acc0 = fma(a.y, a.y, acc0);
      acc1 = fma(b.x, b.x, acc1);
      acc1 = fma(b.y, b.y, acc1);
    }
  } else {
    // complex64: products exact (p + e), four pairs per thread in flight,
    // float-float sums folded into FP64 every round; the adaptive encoding
    // squares its decoded magnitudes the same way
    constexpr int U = 4;
    for (; j < npairs; j += U * stride) {
      A a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t ju = j + u * stride;
        if (ju < npairs) {
          const uint64_t i0 = pair_lo(ju, q);
          a[u] = s[i0];
          b[u] = s[i0 | bit];
        } else {   // amplitude zero: (0, 0), or magnitude code -128
          a[u] = zero_amp<A>();
          b[u] = zero_amp<A>();
        }
      }
      FF f0 = {0.f, 0.f}, f1 = {0.f, 0.f};
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if constexpr (std::is_same<A, float2>::value) {
          ff_add_prod(f0, a[u].x, a[u].x);
          ff_add_prod(f0, a[u].y, a[u].y);
          ff_add_prod(f1, b[u].x, b[u].x);
          ff_add_prod(f1, b[u].y, b[u].y);
        } else {
          const float ma = L.r[(a[u] & 0xFFu) ^ 0x80u], mb = L.r[(b[u] & 0xFFu) ^ 0x80u];
          ff_add_prod(f0, ma, ma);
          ff_add_prod(f1, mb, mb);
        }
      }
      acc0 += ff_val(f0);
      acc1 += ff_val(f1);
    }
  }
  const double r0 = block_sum(acc0, sh);
  const double r1 = block_sum(acc1, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r0;
    part[2 * blockIdx.x + 1] = r1;
  }
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

template <typename R, int RB>
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
    QS_CUDA(cudaFuncSetAttribute(k_expect2<R, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_expect2<R, RB><<<grid, ETPB, smem, s->stream>>>(s->state, passes[i].P, sc + tt_off, sc + part_off[i]);
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

// Tensor map of one complex64 pass (see k_expect_tma): 5 dims of floats, the
// box one 64 KB tile in the 128-byte swizzle.  Dims 1 and 2 are the tile's
// two segments (f = 0: the run split 5 + 4), dims 3 and 4 the qubits below
// and above the run.
static qs_status expect_tensor_map(const qs_sim* s, const XParams& P, CUtensorMap* map) {
  qs_tma::EncodeTiledFn enc = qs_tma::encode_fn();
  if (!enc) {
    qs_set_error("expect_xyz: cuTensorMapEncodeTiled is not available from the driver");
    return QS_ECUDA;
  }
  const int N = s->N, f = P.f, b = P.b;
  const cuuint64_t el = 8;   // bytes per amplitude
  const int top = b + 9 - f;  // first qubit above the run
  const cuuint64_t hi_stride = el << top;
  const cuuint64_t lo_stride = el << (4 + f);
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5];
  dims[0] = 32; box[0] = 32;
  if (f == 0) {
    dims[1] = 32; box[1] = 32; strides[0] = el << b;
    dims[2] = 16; box[2] = 16; strides[1] = el << (b + 5);
  } else {
    dims[1] = 1ull << f; box[1] = 1u << f; strides[0] = el * 16;
    dims[2] = 1ull << (9 - f); box[2] = 1u << (9 - f); strides[1] = el << b;
  }
  dims[3] = 1ull << P.lo_bits; box[3] = 1; strides[2] = P.lo_bits > 0 ? lo_stride : hi_stride;
  dims[4] = 1ull << (N - top); box[4] = 1; strides[3] = hi_stride;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, s->state, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    qs_set_error("expect_xyz: cuTensorMapEncodeTiled failed (%d)", (int)cr);
    return QS_ECUDA;
  }
  return QS_OK;
}

// norm_out (complex64 with a pass that has neither P1 nor view C, N >= 23):
// that pass also sums |a|^2 from exact products; else null or not filled.
template <int ENC>
static qs_status expect_views_impl(qs_sim* s, double* qx, double* qy, double* qz, double* norm_out,
                                   bool* norm_done) {
  const int N = s->N;
  if (N < xv::TB) return QS_EUNSUPPORTED;
  const uint64_t ntiles = 1ull << (N - xv::TB);
  const int G = ENC == 0 ? s->num_sms : s->num_sms * 2;
  const int grid = (int)(ntiles < (uint64_t)G ? ntiles : (uint64_t)G);
  const uint64_t all = (N >= 64) ? ~0ull : ((1ull << N) - 1);
  // pass 0: qubits 0..12; then qubits 13..N-1 in runs of near-equal length
  // (the longer ones first), each run new in its pass
  XParams ps[8];
  int first_new[8];
  int np = 0;
  auto add_pass = [&](int f, int b) {
    XParams& P = ps[np];
    memset(&P, 0, sizeof P);
    P.N = N; P.f = f; P.b = b; P.lo_bits = b - 4 - f;
    first_new[np] = np == 0 ? 0 : b;
    uint64_t tmask = 0;
    for (int k = 0; k < xv::TB; ++k) {
      P.gpos[k] = (uint8_t)(k < 4 + f ? k : b + (k - 4 - f));
      tmask |= 1ull << P.gpos[k];
    }
    P.out_mask = all & ~tmask;
    for (int jj = 0; jj < 16; ++jj) {
      const uint32_t l = xv::reg_a(2 * jj);
      uint64_t g = 0;
      for (int k = 0; k < xv::TB; ++k)
        if ((l >> k) & 1) g |= 1ull << P.gpos[k];
      P.roff_a[jj] = g;
    }
    ++np;
  };
  add_pass(0, 4);
  const int rem = N - xv::TB, nl = (rem + 8) / 9;
  for (int p = 0, b = xv::TB; p < nl; ++p) {
    const int len = rem / nl + (p < rem % nl ? 1 : 0);
    add_pass(9 - len, b);
    b += len;
  }
  // scratch: per pass partials and column sums, tile totals, outer-qubit P1,
  // the error word
  const int nq_out = N - xv::TB;
  size_t off = 0;
  size_t part_off[8], res_off[8];
  for (int i = 0; i < np; ++i) {
    part_off[i] = off; off += (size_t)grid * xv::NCOL;
    res_off[i] = off; off += xv::NCOL;
  }
  const size_t tt_off = off; off += ntiles * 8;
  const int gtb = 64;
  const size_t tbp_off = off; off += (size_t)gtb * (nq_out + 1);
  const size_t tbr_off = off; off += nq_out + 1;
  const size_t ql_off = off; off += 8;    // 64 bytes of qubit list
  const size_t err_off = off; off += 1;
  QS_TRY(ensure_scratch(s, off * sizeof(double)));
  double* sc = (double*)s->scratch;
  // k_tile_bits: P1 of the qubits outside the pass-0 tile
  RedParams rp;
  memset(&rp, 0, sizeof rp);
  rp.N = N;
  rp.out_mask = ps[0].out_mask;
  for (int k = 0; k < 3; ++k) rp.warp_g[k] = ps[0].gpos[10 + k];
  uint8_t ql[64];
  int nql = 0;
  for (int q = 0; q < N; ++q)
    if ((rp.out_mask >> q) & 1) ql[nql++] = (uint8_t)q;
  QS_CUDA(cudaMemcpyAsync(sc + ql_off, ql, 64, cudaMemcpyHostToDevice, s->stream));
  int* err = (int*)(sc + err_off);
  QS_CUDA(cudaMemsetAsync(err, 0, sizeof(double), s->stream));
  // the pass that also sums |a|^2: the first one with neither P1 nor view C
  const int norm_pass = (ENC == 0 && norm_out && np >= 3) ? 1 : -1;
  if (norm_done) *norm_done = norm_pass >= 0;
  for (int i = 0; i < np; ++i) {
    if (ENC == 0) {
      CUtensorMap map;
      QS_TRY(expect_tensor_map(s, ps[i], &map));
      auto go = [&](auto kern) -> qs_status {
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XTMA_SMEM));
        kern<<<grid, ETPB, XTMA_SMEM, s->stream>>>(map, ps[i], sc + tt_off, sc + part_off[i], err,
                                                   pipeline_wait_spins());
        return QS_OK;
      };
      const bool vc = i == np - 1;
      if (i == norm_pass) QS_TRY(go(k_expect_tma<false, false, true>));
      else QS_TRY(i == 0 ? (vc ? go(k_expect_tma<true, true, false>) : go(k_expect_tma<true, false, false>))
                         : (vc ? go(k_expect_tma<false, true, false>) : go(k_expect_tma<false, false, false>)));
    } else {
      const size_t smem = sizeof(float2) << xv::TB;
      auto go = [&](auto kern) -> qs_status {
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, ETPB, smem, s->stream>>>((const unsigned int*)s->state, ps[i], sc + tt_off, sc + part_off[i],
                                              (const A2Dev*)s->a2dev);
        return QS_OK;
      };
      const bool vc = i == np - 1;
      QS_TRY(i == 0 ? (vc ? go(k_expect_ld<true, true>) : go(k_expect_ld<true, false>))
                    : (vc ? go(k_expect_ld<false, true>) : go(k_expect_ld<false, false>)));
    }
    QS_LAUNCH_CHECK();
    k_sum_columns<<<xv::NCOL, TPB, 0, s->stream>>>(sc + part_off[i], grid, xv::NCOL, sc + res_off[i]);
    QS_LAUNCH_CHECK();
  }
  // the total and P1 of the qubits outside the pass-0 tile
  k_tile_bits<<<gtb, TPB, 0, s->stream>>>(sc + tt_off, ntiles, rp, nql, (const uint8_t*)(sc + ql_off), sc + tbp_off);
  QS_LAUNCH_CHECK();
  k_sum_columns<<<nql + 1, TPB, 0, s->stream>>>(sc + tbp_off, gtb, nql + 1, sc + tbr_off);
  QS_LAUNCH_CHECK();
  QS_TRY(ensure_hbuf(s, off * sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(s->hbuf, sc, off * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  const double* h = (const double*)s->hbuf;
  if (*(const int*)(h + err_off)) {
    qs_set_error("expect_xyz: a tensor-load wait ran out of time");
    return QS_ETIMEOUT;
  }
  const double nrm = h[tbr_off];
  for (int i = 0; i < nql; ++i) qz[ql[i]] = h[tbr_off + i + 1];
  // each qubit once: views A and B of pass 0 and the new qubits of views A
  // and B of the later passes; view C (qubits 1..3) of the last pass
  const uint8_t* regs[3] = {xv::REG_A, xv::REG_B, xv::REG_C};
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < xv::NVIEW; ++k) {
      if (k == 2 && i != np - 1) continue;
      for (int sl = 0; sl < (k == 2 ? 3 : 5); ++sl) {
        const int q = ps[i].gpos[regs[k][sl]];
        if (k < 2 && q < first_new[i]) continue;
        const double* c = h + res_off[i] + k * xv::NV;
        qx[q] = 0.5 * nrm - c[2 * sl];
        qy[q] = 0.5 * nrm - c[2 * sl + 1];
        if (i == 0 || k == 2) qz[q] = c[10 + sl];
      }
    }
  if (norm_pass >= 0) *norm_out = h[res_off[norm_pass] + XNORM_COL];
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
  if (s->enc == QS_C128 && s->N >= 12) return expect_impl<double, 4>(s, qx, qy, qz);
  if (s->enc == QS_C64 && s->N >= 13) return expect_views_impl<0>(s, qx, qy, qz, nullptr, nullptr);
  if (s->enc == QS_ADAPT2 && s->N >= 13) return expect_views_impl<2>(s, qx, qy, qz, nullptr, nullptr);
  return expect_small(s, qx, qy, qz);
}

qs_status launch_expect_norm(qs_sim* s, double* qx, double* qy, double* qz, double* norm) {
  bool done = false;
  if (s->enc == QS_C64 && s->N >= 13) QS_TRY(expect_views_impl<0>(s, qx, qy, qz, norm, &done));
  else QS_TRY(launch_expect(s, qx, qy, qz));
  if (done) return QS_OK;
  return (s->enc == QS_ADAPT2) ? a2_norm(s, norm) : launch_norm(s, norm);
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

qs_status launch_qubit_probs(qs_sim* s, int q, double* p0, double* p1) {
  const uint64_t npairs = 1ull << (s->N - 1);
  const uint64_t want = (npairs + TPB - 1) / TPB;
  const int G = (int)(want < (uint64_t)reduce_grid(s) ? want : (uint64_t)reduce_grid(s));
  QS_TRY(ensure_scratch(s, (size_t)(2 * G + 2) * sizeof(double)));
  double* part = (double*)s->scratch;
  if (s->enc == QS_C128)
    k_qubit_probs<double2><<<G, TPB, 0, s->stream>>>((const double2*)s->state, npairs, q, part, nullptr);
  else if (s->enc == QS_C64)
    k_qubit_probs<float2><<<G, TPB, 0, s->stream>>>((const float2*)s->state, npairs, q, part, nullptr);
  else
    k_qubit_probs<uint16_t><<<G, TPB, 0, s->stream>>>((const uint16_t*)s->state, npairs, q, part,
                                                      (const A2Dev*)s->a2dev);
  QS_LAUNCH_CHECK();
  k_sum_columns<<<2, TPB, 0, s->stream>>>(part, G, 2, part + 2 * G);
  QS_LAUNCH_CHECK();
  QS_TRY(ensure_hbuf(s, 2 * sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(s->hbuf, part + 2 * G, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  *p0 = ((const double*)s->hbuf)[0];
  *p1 = ((const double*)s->hbuf)[1];
  return QS_OK;
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
