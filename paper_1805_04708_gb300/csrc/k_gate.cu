// Per-gate sweeps for the dense encodings (complex128 / complex64).
//
// One launch applies one controlled 2x2 update (Eq. (NUM2) with a general U,
// Eq. (AQS0); the groups of four / eight amplitudes of CNOT / TOFFOLI in
// Sec. 2).  Each thread handles U_PER groups; all loads of a thread are issued
// before its stores so that 2*U_PER 16-byte accesses are in flight.
//
// Vector modes for complex64 (8-byte amplitudes): when every qubit involved
// is >= 1, two neighbouring amplitudes (index bit 0 = 0/1) share one 16-byte
// float4 and both are updated with the same pattern ("vec"); a target on
// qubit 0 with controls >= 1 pairs the two halves of one float4 ("inreg").
#include "internal.cuh"
#include "cplx.cuh"

namespace {

constexpr int TPB = 256;
constexpr int U_PER = 4;

struct Geom {
  int nins;          // zero bits inserted into the group index (ascending)
  int pos[4];
  uint64_t setmask;  // bits forced to 1 after insertion
  uint64_t stride;   // pair distance in storage elements
};

__device__ __forceinline__ uint64_t expand(uint64_t g, const Geom& G) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (k < G.nins) g = ins0(g, G.pos[k]);
  return g | G.setmask;
}

// --- element adapters: apply a pair functor to storage elements -------------
// complex128 storage; R = double on the FP64 units, R = DF on FP32 pairs
template <typename Op, typename R = double> struct PairD2 {
  Op op;
  __device__ __forceinline__ void operator()(double2& x, double2& y) const {
    Cx<R> a = from_mem<R>(x), b = from_mem<R>(y); op.pair(a, b); x = to_mem<R>(a); y = to_mem<R>(b);
  }
};
template <typename Op> struct PairF2 {
  Op op;
  __device__ __forceinline__ void operator()(float2& x, float2& y) const {
    Cx<float> a = ld(x), b = ld(y); op.pair(a, b); st(x, a); st(y, b);
  }
};
template <typename Op> struct PairF4 {   // two pairs: (x.lo, y.lo), (x.hi, y.hi)
  Op op;
  __device__ __forceinline__ void operator()(float4& x, float4& y) const {
    Cx<float> a0 = cx<float>(x.x, x.y), b0 = cx<float>(y.x, y.y);
    Cx<float> a1 = cx<float>(x.z, x.w), b1 = cx<float>(y.z, y.w);
    op.pair(a0, b0); op.pair(a1, b1);
    x = make_float4(a0.x, a0.y, a1.x, a1.y);
    y = make_float4(b0.x, b0.y, b1.x, b1.y);
  }
};
template <typename Op> struct InregF4 {  // one pair: (v.lo, v.hi)
  Op op;
  __device__ __forceinline__ void operator()(float4& v) const {
    Cx<float> a = cx<float>(v.x, v.y), b = cx<float>(v.z, v.w);
    op.pair(a, b);
    v = make_float4(a.x, a.y, b.x, b.y);
  }
};
template <typename Op, typename R = double> struct OneD2 {
  Op op;
  __device__ __forceinline__ void operator()(double2& v) const {
    Cx<R> a = from_mem<R>(v); op.one(a); v = to_mem<R>(a);
  }
};
template <typename Op> struct OneF2 {
  Op op;
  __device__ __forceinline__ void operator()(float2& v) const {
    Cx<float> a = ld(v); op.one(a); st(v, a);
  }
};
template <typename Op> struct OneF4 {
  Op op;
  __device__ __forceinline__ void operator()(float4& v) const {
    Cx<float> a = cx<float>(v.x, v.y), b = cx<float>(v.z, v.w);
    op.one(a); op.one(b);
    v = make_float4(a.x, a.y, b.x, b.y);
  }
};

// --- kernels -------------------------------------------------------------------
template <typename V, typename F>
__global__ void __launch_bounds__(TPB) k_pair(V* __restrict__ s, uint64_t ngroups, Geom G, F f) {
  const uint64_t base = (uint64_t)blockIdx.x * (TPB * U_PER) + threadIdx.x;
  V a[U_PER], b[U_PER];
  uint64_t id[U_PER];
#pragma unroll
  for (int u = 0; u < U_PER; ++u) {
    const uint64_t g = base + (uint64_t)u * TPB;
    id[u] = (g < ngroups) ? expand(g, G) : ~0ull;
    if (g < ngroups) { a[u] = s[id[u]]; b[u] = s[id[u] + G.stride]; }
  }
#pragma unroll
  for (int u = 0; u < U_PER; ++u) {
    if (id[u] != ~0ull) {
      f(a[u], b[u]);
      s[id[u]] = a[u];
      s[id[u] + G.stride] = b[u];
    }
  }
}

template <typename V, typename F>
__global__ void __launch_bounds__(TPB) k_one(V* __restrict__ s, uint64_t ngroups, Geom G, F f) {
  const uint64_t base = (uint64_t)blockIdx.x * (TPB * U_PER) + threadIdx.x;
  V a[U_PER];
  uint64_t id[U_PER];
#pragma unroll
  for (int u = 0; u < U_PER; ++u) {
    const uint64_t g = base + (uint64_t)u * TPB;
    id[u] = (g < ngroups) ? expand(g, G) : ~0ull;
    if (g < ngroups) a[u] = s[id[u]];
  }
#pragma unroll
  for (int u = 0; u < U_PER; ++u) {
    if (id[u] != ~0ull) {
      f(a[u]);
      s[id[u]] = a[u];
    }
  }
}

static uint64_t nblocks(uint64_t ngroups) {
  return (ngroups + (uint64_t)TPB * U_PER - 1) / ((uint64_t)TPB * U_PER);
}

// Build the insertion geometry: zero bits at `ins` (any order), ones at `set`.
static Geom make_geom(int* ins, int nins, uint64_t setmask, uint64_t stride) {
  Geom G;
  for (int i = 0; i < nins; ++i)
    for (int j = i + 1; j < nins; ++j)
      if (ins[j] < ins[i]) { int t = ins[i]; ins[i] = ins[j]; ins[j] = t; }
  G.nins = nins;
  for (int i = 0; i < 4; ++i) G.pos[i] = i < nins ? ins[i] : 0;
  G.setmask = setmask;
  G.stride = stride;
  return G;
}

template <typename V, typename F>
qs_status run_pair(qs_sim* s, int space_bits, int* ins, int nins, uint64_t setmask, uint64_t stride, F f) {
  Geom G = make_geom(ins, nins, setmask, stride);
  uint64_t ng = 1ull << (space_bits - nins);
  k_pair<V, F><<<(unsigned)nblocks(ng), TPB, 0, s->stream>>>((V*)s->state, ng, G, f);
  QS_LAUNCH_CHECK();
  return QS_OK;
}
template <typename V, typename F>
qs_status run_one(qs_sim* s, int space_bits, int* ins, int nins, uint64_t setmask, F f) {
  Geom G = make_geom(ins, nins, setmask, 0);
  uint64_t ng = 1ull << (space_bits - nins);
  k_one<V, F><<<(unsigned)nblocks(ng), TPB, 0, s->stream>>>((V*)s->state, ng, G, f);
  QS_LAUNCH_CHECK();
  return QS_OK;
}

template <typename R> Cx<R> hcx(const double* u, int k) { Cx<R> c; c.x = (R)u[2 * k]; c.y = (R)u[2 * k + 1]; return c; }

// Dispatch one controlled 2x2 update for real type R.
template <typename R>
qs_status dispatch(qs_sim* s, const int* controls, int nc, int t, const double* u) {
  GateClass gc = classify_u2(u);
  if (gc.kind == GK_IDENT) return QS_OK;
  const int N = s->N;
  int minc = 64;
  uint64_t cmask = 0;
  for (int i = 0; i < nc; ++i) { minc = controls[i] < minc ? controls[i] : minc; cmask |= 1ull << controls[i]; }

  // One-sided diagonal: only the half with target bit = 1 (or 0) changes.
  if (gc.kind == GK_DIAG && (gc.c0 == 0 || gc.c1 == 0)) {
    const bool upper = (gc.c0 == 0);                 // d0 == 1: multiply bit-1 half by d1
    OpMul<R> op; op.f = hcx<R>(u, upper ? 3 : 0); op.c = upper ? gc.c1 : gc.c0;
    int ins[4]; int n = 0;
    for (int i = 0; i < nc; ++i) ins[n++] = controls[i];
    ins[n++] = t;
    uint64_t set = cmask | (upper ? (1ull << t) : 0ull);
    if constexpr (sizeof(R) == 8) {
      return run_one<double2>(s, N, ins, n, set, OneD2<OpMul<R>, R>{op});
    } else {
      if (minc >= 1 && t >= 1) {
        for (int i = 0; i < n; ++i) ins[i] -= 1;
        return run_one<float4>(s, N - 1, ins, n, set >> 1, OneF4<OpMul<R>>{op});
      }
      return run_one<float2>(s, N, ins, n, set, OneF2<OpMul<R>>{op});
    }
  }

  auto go = [&](auto op) -> qs_status {
    using Op = decltype(op);
    int ins[4]; int n = 0;
    for (int i = 0; i < nc; ++i) ins[n++] = controls[i];
    if constexpr (sizeof(R) == 8) {
      ins[n++] = t;
      return run_pair<double2>(s, N, ins, n, cmask, 1ull << t, PairD2<Op, R>{op});
    } else {
      if (minc >= 1 && t >= 1) {
        ins[n++] = t;
        for (int i = 0; i < n; ++i) ins[i] -= 1;
        return run_pair<float4>(s, N - 1, ins, n, cmask >> 1, 1ull << (t - 1), PairF4<Op>{op});
      }
      if (minc >= 1 && t == 0) {
        for (int i = 0; i < n; ++i) ins[i] -= 1;
        return run_one<float4>(s, N - 1, ins, n, cmask >> 1, InregF4<Op>{op});
      }
      ins[n++] = t;
      return run_pair<float2>(s, N, ins, n, cmask, 1ull << t, PairF2<Op>{op});
    }
  };

  switch (gc.kind) {
    case GK_HAD: { OpHad<R> op; op.s = (R)u[0]; return go(op); }
    case GK_DIAG: { OpDiag<R> op; op.d0 = hcx<R>(u, 0); op.d1 = hcx<R>(u, 3); op.c0 = gc.c0; op.c1 = gc.c1; return go(op); }
    case GK_ANTI: { OpAnti<R> op; op.f01 = hcx<R>(u, 1); op.f10 = hcx<R>(u, 2); op.c0 = gc.c0; op.c1 = gc.c1; return go(op); }
    default: {
      OpDense<R> op; op.u00 = hcx<R>(u, 0); op.u01 = hcx<R>(u, 1); op.u10 = hcx<R>(u, 2); op.u11 = hcx<R>(u, 3);
      return go(op);
    }
  }
}

}  // namespace

qs_status launch_u2(qs_sim* s, const int* controls, int nc, int target, const double u[8]) {
  if (s->enc == QS_C128) {
    // double-float carries 48 significant bits, so gates that only move
    // amplitudes or multiply them by +-1, +-i (X, Y, Z, S, CNOT, TOFFOLI, ...)
    // run in FP64 and stay exact
    const GateClass gc = classify_u2(u);
    const bool moves = (gc.kind == GK_ANTI || gc.kind == GK_DIAG) && gc.c0 < 4 && gc.c1 < 4;
    return (s->c128_df != 0 && !moves) ? dispatch<DF>(s, controls, nc, target, u)
                                  : dispatch<double>(s, controls, nc, target, u);
  }
  if (s->enc == QS_C64) return dispatch<float>(s, controls, nc, target, u);
  return QS_EUNSUPPORTED;
}
