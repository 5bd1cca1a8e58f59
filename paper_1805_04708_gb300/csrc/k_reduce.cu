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
__device__ __forceinline__ void ff_sub_prod(FF& s, float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  ff_add(s, -p);
  s.lo -= e;
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
  FF f = {0.f, 0.f};
  int cnt = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB) {
    float4 a = s[i];
    ff_add_prod(f, a.x, a.x);
    ff_add_prod(f, a.y, a.y);
    ff_add_prod(f, a.z, a.z);
    ff_add_prod(f, a.w, a.w);
    if (++cnt == 8) { acc += ff_val(f); f.hi = f.lo = 0.f; cnt = 0; }
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

// ---- expect_xyz tile passes -------------------------------------------------------------
// A tile is the 2^b amplitudes whose index bits outside `bits` are fixed:
// bits[0..L-1] are the low L index bits (contiguous runs of 2^L amplitudes),
// bits[L..b-1] are higher bits.  For the local bits p >= p_new the pass
// accumulates, per tile, Re/Im of sum conj(a(l)) a(l | 2^p) over l with bit
// p = 0, and P(bit = 1); pass 0 also accumulates the total |a|^2.
struct TileGeo {
  int N, b, L, p_new;
  uint64_t hi_mask;        // global mask of bits[L..b-1]
  uint64_t out_mask;       // global mask of the bits outside the tile
  int hb[16];              // global positions of bits[L..b-1]
};

__device__ __forceinline__ uint64_t deposit(uint64_t x, uint64_t mask) {
  uint64_t r = 0;
  for (uint64_t m = mask; m; m &= m - 1) {
    if (x & 1) r |= m & (~m + 1);
    x >>= 1;
  }
  return r;
}

template <typename A> struct ElemT;
template <> struct ElemT<double2> { using R = double; };
template <> struct ElemT<float2> { using R = float; };

// per-pair accumulation: re += Re(conj(a0) a1), im += Im(conj(a0) a1), p1 += |a1|^2
struct AccD {
  double re, im, p1;
  __device__ void zero() { re = im = p1 = 0.0; }
  __device__ void add(double2 a0, double2 a1) {
    re = fma(a0.x, a1.x, re); re = fma(a0.y, a1.y, re);
    im = fma(a0.x, a1.y, im); im = fma(-a0.y, a1.x, im);
    p1 = fma(a1.x, a1.x, p1); p1 = fma(a1.y, a1.y, p1);
  }
  __device__ double vre() const { return re; }
  __device__ double vim() const { return im; }
  __device__ double vp1() const { return p1; }
};
struct AccF {
  FF re, im, p1;
  __device__ void zero() { re.hi = re.lo = im.hi = im.lo = p1.hi = p1.lo = 0.f; }
  __device__ void add(float2 a0, float2 a1) {
    ff_add_prod(re, a0.x, a1.x); ff_add_prod(re, a0.y, a1.y);
    ff_add_prod(im, a0.x, a1.y); ff_sub_prod(im, a0.y, a1.x);
    ff_add_prod(p1, a1.x, a1.x); ff_add_prod(p1, a1.y, a1.y);
  }
  __device__ double vre() const { return ff_val(re); }
  __device__ double vim() const { return ff_val(im); }
  __device__ double vp1() const { return ff_val(p1); }
};
template <typename A> struct AccT;
template <> struct AccT<double2> { using T = AccD; };
template <> struct AccT<float2> { using T = AccF; };

__device__ __forceinline__ double sq(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double sq(float2 a) { return (double)a.x * a.x + (double)a.y * a.y; }

// partials layout per block: [ (b - p_new) * 3 + 1 ] doubles
template <typename A>
__global__ void __launch_bounds__(TPB) k_expect_tiles(const A* __restrict__ s, TileGeo g, double* part) {
  extern __shared__ unsigned char smraw[];
  A* tile = (A*)smraw;
  const int nb = g.b - g.p_new;
  double* wacc = (double*)(smraw + ((size_t)sizeof(A) << g.b));  // [warps][nb*3+1]
  const int nw = TPB / 32, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stride = nb * 3 + 1;
  for (int i = threadIdx.x; i < nw * stride; i += TPB) wacc[i] = 0.0;
  const uint64_t ntiles = 1ull << (g.N - g.b);
  const int tsize = 1 << g.b;
  const int lmask = (1 << g.L) - 1;
  __syncthreads();
  double tot = 0.0;
  for (uint64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
    const uint64_t base = deposit(tau, g.out_mask);
    for (int l = threadIdx.x; l < tsize; l += TPB) {
      uint64_t h = (uint64_t)(l >> g.L);
      uint64_t gi = base | (uint64_t)(l & lmask);
      for (int k = 0; k < g.b - g.L; ++k) gi |= ((h >> k) & 1ull) << g.hb[k];
      tile[l] = s[gi];
    }
    __syncthreads();
    if (g.p_new == 0)
      for (int l = threadIdx.x; l < tsize; l += TPB) tot += sq(tile[l]);
    for (int p = g.p_new; p < g.b; ++p) {
      typename AccT<A>::T acc;
      acc.zero();
      for (int j = threadIdx.x; j < (tsize >> 1); j += TPB) {
        int l0 = (int)ins0((uint64_t)j, p);
        acc.add(tile[l0], tile[l0 | (1 << p)]);
      }
      double re = warp_sum(acc.vre()), im = warp_sum(acc.vim()), p1 = warp_sum(acc.vp1());
      if (lane == 0) {
        double* d = wacc + w * stride + (p - g.p_new) * 3;
        d[0] += re; d[1] += im; d[2] += p1;
      }
    }
    __syncthreads();
  }
  tot = warp_sum(tot);
  if (lane == 0) wacc[w * stride + nb * 3] += tot;
  __syncthreads();
  for (int i = threadIdx.x; i < stride; i += TPB) {
    double r = 0.0;
    for (int ww = 0; ww < nw; ++ww) r += wacc[ww * stride + i];
    part[(size_t)blockIdx.x * stride + i] = r;
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
__global__ void __launch_bounds__(TPB) k_marginal(const A* __restrict__ s, MargGeo g, double* part) {
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
    acc += sq(s[ireg | x]);
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

static int reduce_grid(qs_sim* s) { return s->num_sms * 4; }

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

template <typename A>
static qs_status expect_impl(qs_sim* s, double* qx, double* qy, double* qz) {
  const int N = s->N;
  const int bmax = (sizeof(A) == 16) ? 12 : 13;
  const int b0 = N < bmax ? N : bmax;
  const int L = N < 5 ? N : 5;
  // pass list: pass 0 covers bits 0..b0-1; then groups of (bmax - L) bits.
  struct P { int b, p_new, first_new; };
  P passes[64];
  int np = 0;
  passes[np++] = {b0, 0, 0};
  for (int q = b0; q < N;) {
    int gsz = bmax - L;
    if (q + gsz > N) gsz = N - q;
    passes[np++] = {L + gsz, L, q};
    q += gsz;
  }
  const int G = reduce_grid(s);
  size_t need = 0;
  for (int i = 0; i < np; ++i) need += (size_t)G * ((passes[i].b - passes[i].p_new) * 3 + 1) + 64;
  QS_TRY(ensure_scratch(s, need * sizeof(double) + 3 * 64 * sizeof(double)));
  double* part = (double*)s->scratch;
  double* res = part;  // per pass results follow the partials
  size_t off = 0;
  size_t res_off[64];
  int stride_of[64];
  for (int i = 0; i < np; ++i) {
    const P& p = passes[i];
    TileGeo g;
    g.N = N; g.b = p.b; g.L = (i == 0) ? p.b : L; g.p_new = p.p_new;
    g.hi_mask = 0;
    uint64_t tmask = 0;
    if (i == 0) {
      tmask = (p.b >= 64) ? ~0ull : ((1ull << p.b) - 1);
    } else {
      tmask = (1ull << L) - 1;
      for (int k = 0; k < p.b - L; ++k) { g.hb[k] = p.first_new + k; g.hi_mask |= 1ull << (p.first_new + k); }
      tmask |= g.hi_mask;
    }
    g.out_mask = ((N >= 64) ? ~0ull : ((1ull << N) - 1)) & ~tmask;
    const uint64_t ntiles = 1ull << (N - p.b);
    int grid = (int)((ntiles < (uint64_t)G) ? ntiles : (uint64_t)G);
    const int stride = (p.b - p.p_new) * 3 + 1;
    size_t smem = ((size_t)sizeof(A) << p.b) + (TPB / 32) * stride * sizeof(double);
    QS_CUDA(cudaFuncSetAttribute(k_expect_tiles<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_expect_tiles<A><<<grid, TPB, smem, s->stream>>>((const A*)s->state, g, part + off);
    QS_LAUNCH_CHECK();
    res_off[i] = off + (size_t)grid * stride;
    stride_of[i] = stride;
    k_sum_columns<<<stride, TPB, 0, s->stream>>>(part + off, grid, stride, part + res_off[i]);
    QS_LAUNCH_CHECK();
    off = res_off[i] + stride;
  }
  QS_TRY(ensure_hbuf(s, off * sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(s->hbuf, part, off * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  const double* h = (const double*)s->hbuf;
  (void)res;
  double nrm = h[res_off[0] + (passes[0].b - passes[0].p_new) * 3];
  for (int i = 0; i < np; ++i) {
    const double* r = h + res_off[i];
    for (int p = passes[i].p_new; p < passes[i].b; ++p) {
      int q = (i == 0) ? p : passes[i].first_new + (p - L);
      const double* d = r + (p - passes[i].p_new) * 3;
      qx[q] = 0.5 * nrm - d[0];
      qy[q] = 0.5 * nrm - d[1];
      qz[q] = d[2];
    }
  }
  (void)stride_of;
  return QS_OK;
}

qs_status launch_expect(qs_sim* s, double* qx, double* qy, double* qz) {
  if (s->enc == QS_C128) return expect_impl<double2>(s, qx, qy, qz);
  if (s->enc == QS_C64) return expect_impl<float2>(s, qx, qy, qz);
  return QS_EUNSUPPORTED;
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
  k_marginal<A><<<(unsigned)((nthreads + TPB - 1) / TPB), TPB, 0, s->stream>>>((const A*)s->state, g, part);
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
  return QS_EUNSUPPORTED;
}
