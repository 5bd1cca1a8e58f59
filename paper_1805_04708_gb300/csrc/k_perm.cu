// Index-permutation kernels (bit-exact amplitude / code moves) and state
// preparation: controlled register permutations (the controlled modular
// multiplications of Shor's algorithm, Sec. 5.4), SHORBOX (Appendix A) and
// |0..0> (Eq. (appa0)).
#include "internal.cuh"
#include <string.h>

namespace {

constexpr int TPB = 256;

struct PermGeo {
  int N, w, reg_lo, Lp;
  int lowpos[8];         // global positions of the Lp low non-register tile bits
  uint64_t out_mask;     // bits outside the tile
  uint64_t cmask;        // all control bits
  uint64_t cmask_out;    // control bits outside the tile
};

__device__ __forceinline__ uint64_t deposit_p(uint64_t x, uint64_t mask) {
  uint64_t r = 0;
  for (uint64_t m = mask; m; m &= m - 1) {
    if (x & 1) r |= m & (~m + 1);
    x >>= 1;
  }
  return r;
}

// One tile = all 2^w register values x 2^Lp low values, for fixed outer bits.
// Read the tile into shared memory, then write every element to its permuted
// register value; the map is a bijection inside the tile, so in place is safe.
template <typename E>
__global__ void __launch_bounds__(TPB) k_perm_tiles(E* __restrict__ s, PermGeo g, const uint32_t* __restrict__ table) {
  extern __shared__ unsigned char smraw[];
  uint32_t* tab = (uint32_t*)smraw;
  E* tile = (E*)(smraw + ((size_t)4 << g.w));
  const int W = 1 << g.w;
  for (int i = threadIdx.x; i < W; i += TPB) tab[i] = table[i];
  const int tsize = 1 << (g.w + g.Lp);
  const uint64_t ntiles = 1ull << (g.N - g.w - g.Lp);
  for (uint64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
    const uint64_t base = deposit_p(tau, g.out_mask);
    if ((base & g.cmask_out) != g.cmask_out) continue;   // uniform over the block
    __syncthreads();
    for (int l = threadIdx.x; l < tsize; l += TPB) {
      uint64_t f = (uint64_t)(l >> g.Lp);
      uint64_t lo = 0;
      for (int k = 0; k < g.Lp; ++k) lo |= (uint64_t)((l >> k) & 1) << g.lowpos[k];
      tile[l] = s[base | lo | (f << g.reg_lo)];
    }
    __syncthreads();
    for (int l = threadIdx.x; l < tsize; l += TPB) {
      uint64_t f = (uint64_t)(l >> g.Lp);
      uint64_t lo = 0;
      for (int k = 0; k < g.Lp; ++k) lo |= (uint64_t)((l >> k) & 1) << g.lowpos[k];
      uint64_t gi = base | lo;
      uint64_t fd = ((gi & g.cmask) == g.cmask) ? (uint64_t)tab[f] : f;
      s[gi | (fd << g.reg_lo)] = tile[l];
    }
  }
}

// SHORBOX: thread x computes f(x) = y^x mod G and writes the column x of the
// 2^nx x 2^F array (amplitude `amp` at f = f(x), zero elsewhere).
template <typename E>
__global__ void k_shorbox(E* __restrict__ s, int nx, int F, uint64_t G, uint64_t y, E amp, E zero) {
  const uint64_t x = (uint64_t)blockIdx.x * TPB + threadIdx.x;
  if (x >= (1ull << nx)) return;
  uint64_t r = 1 % G, b = y % G, e = x;
  while (e) {
    if (e & 1) r = (r * b) % G;
    b = (b * b) % G;
    e >>= 1;
  }
  for (uint64_t f = 0; f < (1ull << F); ++f) s[x + (f << nx)] = (f == r) ? amp : zero;
}

template <typename E>
__global__ void k_fill(E* __restrict__ s, uint64_t n, E v, E v0) {
  for (uint64_t i = (uint64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB)
    s[i] = (i == 0) ? v0 : v;
}

template <typename E>
qs_status perm_impl(qs_sim* s, const int* controls, int nc, int reg_lo, int w, const uint32_t* table) {
  PermGeo g;
  g.N = s->N; g.w = w; g.reg_lo = reg_lo;
  const uint64_t regmask = ((1ull << w) - 1) << reg_lo;
  // choose Lp low non-register bits with 2^(w+Lp) * sizeof(E) <= 96 KB
  int Lp = 0;
  while (Lp < 8 && Lp < s->N - w && ((size_t)sizeof(E) << (w + Lp + 1)) <= 96 * 1024) ++Lp;
  int k = 0;
  uint64_t lomask = 0;
  for (int q = 0; q < s->N && k < Lp; ++q)
    if (!((regmask >> q) & 1)) { g.lowpos[k++] = q; lomask |= 1ull << q; }
  g.Lp = Lp;
  const uint64_t all = (s->N >= 64) ? ~0ull : ((1ull << s->N) - 1);
  g.out_mask = all & ~regmask & ~lomask;
  g.cmask = 0;
  for (int i = 0; i < nc; ++i) g.cmask |= 1ull << controls[i];
  g.cmask_out = g.cmask & g.out_mask;
  uint32_t* dtab = nullptr;
  QS_TRY(ensure_scratch(s, (size_t)4 << w));
  dtab = (uint32_t*)s->scratch;
  QS_CUDA(cudaMemcpyAsync(dtab, table, (size_t)4 << w, cudaMemcpyHostToDevice, s->stream));
  const size_t smem = ((size_t)4 << w) + ((size_t)sizeof(E) << (w + Lp));
  QS_CUDA(cudaFuncSetAttribute(k_perm_tiles<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const uint64_t ntiles = 1ull << (s->N - w - Lp);
  const uint64_t gmax = (uint64_t)s->num_sms * 2;
  k_perm_tiles<E><<<(unsigned)(ntiles < gmax ? ntiles : gmax), TPB, smem, s->stream>>>((E*)s->state, g, dtab);
  QS_LAUNCH_CHECK();
  // the host table must stay valid until the copy is done
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}

}  // namespace

qs_status launch_permutation(qs_sim* s, const int* controls, int nc, int reg_lo, int reg_w,
                             const uint32_t* table) {
  switch (s->enc) {
    case QS_C128: return perm_impl<uint4>(s, controls, nc, reg_lo, reg_w, table);
    case QS_C64: return perm_impl<uint2>(s, controls, nc, reg_lo, reg_w, table);
    default: return perm_impl<uint16_t>(s, controls, nc, reg_lo, reg_w, table);
  }
}

qs_status launch_shorbox(qs_sim* s, int nx, uint64_t G, uint64_t y) {
  const int F = s->N - nx;
  const double amp = pow(2.0, -0.5 * nx);
  const unsigned blocks = (unsigned)(((1ull << nx) + TPB - 1) / TPB);
  if (s->enc == QS_C128) {
    k_shorbox<double2><<<blocks, TPB, 0, s->stream>>>((double2*)s->state, nx, F, G, y,
                                                       make_double2(amp, 0.0), make_double2(0.0, 0.0));
  } else if (s->enc == QS_C64) {
    k_shorbox<float2><<<blocks, TPB, 0, s->stream>>>((float2*)s->state, nx, F, G, y,
                                                      make_float2((float)amp, 0.f), make_float2(0.f, 0.f));
  } else {
    // every nonzero amplitude has |z| = 2^{-nx/2} = r0 = r1: b0 = -127, b1 = 0
    k_shorbox<uint16_t><<<blocks, TPB, 0, s->stream>>>((uint16_t*)s->state, nx, F, G, y,
                                                        (uint16_t)0x0081, (uint16_t)0x0080);
    QS_LAUNCH_CHECK();
    return a2_set_range(s, amp, amp);
  }
  QS_LAUNCH_CHECK();
  return QS_OK;
}

qs_status launch_reset(qs_sim* s) {
  const uint64_t n = 1ull << s->N;
  const unsigned blocks = (unsigned)((n / TPB + 1) < (uint64_t)s->num_sms * 8 ? (n / TPB + 1) : (uint64_t)s->num_sms * 8);
  if (s->enc == QS_C128) {
    k_fill<double2><<<blocks, TPB, 0, s->stream>>>((double2*)s->state, n, make_double2(0, 0), make_double2(1, 0));
  } else if (s->enc == QS_C64) {
    k_fill<float2><<<blocks, TPB, 0, s->stream>>>((float2*)s->state, n, make_float2(0, 0), make_float2(1, 0));
  } else {
    // b0 = -128 (r = 0) everywhere, b0 = 127 (r = 1) at index 0; r0 = r1 = 0
    k_fill<uint16_t><<<blocks, TPB, 0, s->stream>>>((uint16_t*)s->state, n, (uint16_t)0x0080, (uint16_t)0x007F);
    QS_LAUNCH_CHECK();
    return a2_set_range(s, 0.0, 0.0);
  }
  QS_LAUNCH_CHECK();
  return QS_OK;
}
