// Shared-memory tile passes: several gates per read and write of the state
// (the gate fusion that the end of Sec. 5.2 proposes for raising arithmetic
// intensity; here every gate keeps its own 2x2 and the fusion is in the data
// movement).
//
// A tile is the 2^b amplitudes whose index bits outside the tile bit set B
// are fixed.  B always holds the low L index bits (contiguous runs of 2^L
// amplitudes, 512 B) plus the targets of the gates in the pass.  A gate may
// join the pass when its target is in B, or when it is diagonal (its target
// bit is then fixed per tile and the gate is a per-tile phase); controls may
// be anywhere (a control outside B is a per-tile condition).  Gate order is
// kept, so the result equals the per-gate sweep up to rounding order.
#include "internal.cuh"
#include "cplx.cuh"
#include <string.h>
#include <stdlib.h>

namespace {

constexpr int TPB = 512;
constexpr int MAX_OPS = 48;

struct TileParams {
  int N, b, L;
  uint64_t out_mask;   // global bits outside the tile
  int hb[16];          // global positions of tile bits L..b-1
  int nops;
  TileOp ops[MAX_OPS];
};

__device__ __forceinline__ uint64_t deposit_t(uint64_t x, uint64_t mask) {
  uint64_t r = 0;
  for (uint64_t m = mask; m; m &= m - 1) {
    if (x & 1) r |= m & (~m + 1);
    x >>= 1;
  }
  return r;
}

template <typename R> __device__ __forceinline__ Cx<R> opc(const TileOp& o, int k) {
  return cx<R>((R)o.u[2 * k], (R)o.u[2 * k + 1]);
}

template <typename R, typename F>
__device__ __forceinline__ void pairs(Cx<R>* t, int b, int p, uint32_t lmask, const F& f) {
  const int npairs = 1 << (b - 1);
  for (int j = threadIdx.x; j < npairs; j += TPB) {
    const uint32_t l0 = (uint32_t)ins0((uint64_t)j, p);
    if ((l0 & lmask) != lmask) continue;
    const uint32_t l1 = l0 | (1u << p);
    Cx<R> a0 = t[l0], a1 = t[l1];
    f.pair(a0, a1);
    t[l0] = a0;
    t[l1] = a1;
  }
}

template <typename R, typename A>
__global__ void __launch_bounds__(TPB) k_tile(A* __restrict__ s, const __grid_constant__ TileParams P) {
  extern __shared__ unsigned char smraw[];
  Cx<R>* t = (Cx<R>*)smraw;
  uint64_t* off = (uint64_t*)(smraw + (sizeof(Cx<R>) << P.b));
  const int nh = 1 << (P.b - P.L);
  for (int h = threadIdx.x; h < nh; h += TPB) {
    uint64_t o = 0;
    for (int k = 0; k < P.b - P.L; ++k) o |= (uint64_t)((h >> k) & 1) << P.hb[k];
    off[h] = o;
  }
  const int tsize = 1 << P.b;
  const int lm = (1 << P.L) - 1;
  const uint64_t ntiles = 1ull << (P.N - P.b);
  __syncthreads();
  for (uint64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
    const uint64_t base = deposit_t(tau, P.out_mask);
    // load (2 amplitudes per 16-byte access for complex64, 1 for complex128)
    if (sizeof(R) == 4) {
      const float4* s4 = (const float4*)s;
      float4* t4 = (float4*)t;
#pragma unroll 4
      for (int v = threadIdx.x; v < tsize / 2; v += TPB) {
        const int l = 2 * v;
        t4[v] = s4[(base + off[l >> P.L] + (l & lm)) >> 1];
      }
    } else {
      const double2* s2 = (const double2*)s;
      double2* t2 = (double2*)t;
#pragma unroll 4
      for (int l = threadIdx.x; l < tsize; l += TPB) t2[l] = s2[base + off[l >> P.L] + (l & lm)];
    }
    __syncthreads();
    for (int i = 0; i < P.nops; ++i) {
      const TileOp& o = P.ops[i];
      if ((base & o.gmask) != o.gmask) continue;  // an outer control is 0 for this tile
      if (o.p < 0) {
        // diagonal gate on a qubit outside the tile: one factor per tile
        const bool one = (base & o.gtbit) != 0;
        const int code = one ? o.c1 : o.c0;
        if (code == 0) continue;
        OpMul<R> m;
        m.f = opc<R>(o, one ? 3 : 0);
        m.c = code;
        for (int l = threadIdx.x; l < tsize; l += TPB)
          if (((uint32_t)l & o.lmask) == o.lmask) m.one(t[l]);
      } else {
        switch (o.kind) {
          case GK_HAD: { OpHad<R> f; f.s = (R)o.u[0]; pairs<R>(t, P.b, o.p, o.lmask, f); break; }
          case GK_DIAG: {
            OpDiag<R> f; f.d0 = opc<R>(o, 0); f.d1 = opc<R>(o, 3); f.c0 = o.c0; f.c1 = o.c1;
            pairs<R>(t, P.b, o.p, o.lmask, f);
            break;
          }
          case GK_ANTI: {
            OpAnti<R> f; f.f01 = opc<R>(o, 1); f.f10 = opc<R>(o, 2); f.c0 = o.c0; f.c1 = o.c1;
            pairs<R>(t, P.b, o.p, o.lmask, f);
            break;
          }
          default: {
            OpDense<R> f; f.u00 = opc<R>(o, 0); f.u01 = opc<R>(o, 1); f.u10 = opc<R>(o, 2); f.u11 = opc<R>(o, 3);
            pairs<R>(t, P.b, o.p, o.lmask, f);
          }
        }
      }
      __syncthreads();
    }
    // store
    if (sizeof(R) == 4) {
      float4* s4 = (float4*)s;
      const float4* t4 = (const float4*)t;
#pragma unroll 4
      for (int v = threadIdx.x; v < tsize / 2; v += TPB) {
        const int l = 2 * v;
        s4[(base + off[l >> P.L] + (l & lm)) >> 1] = t4[v];
      }
    } else {
      double2* s2 = (double2*)s;
      const double2* t2 = (const double2*)t;
#pragma unroll 4
      for (int l = threadIdx.x; l < tsize; l += TPB) s2[base + off[l >> P.L] + (l & lm)] = t2[l];
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------------
// planner
// ---------------------------------------------------------------------------------
static void close_pass(const qs_gate* gates, const int* gidx, int ng, int N, int b, uint64_t S,
                       TilePass* tp, TileOp* ops, int* nops_total) {
  // pad S to b bits with the lowest unused bits
  for (int q = 0; q < N && __builtin_popcountll(S) < b; ++q) S |= 1ull << q;
  tp->b = __builtin_popcountll(S);
  int k = 0;
  int local[64];
  for (int q = 0; q < N; ++q) {
    local[q] = -1;
    if ((S >> q) & 1) { tp->bits[k] = q; local[q] = k; ++k; }
  }
  tp->op_begin = *nops_total;
  tp->nops = 0;
  for (int i = 0; i < ng; ++i) {
    const qs_gate& g = gates[gidx[i]];
    GateClass gc = classify_u2(g.u);
    TileOp o;
    memset(&o, 0, sizeof o);
    o.kind = gc.kind;
    o.c0 = gc.c0;
    o.c1 = gc.c1;
    o.p = local[g.target];
    o.gtbit = (o.p < 0) ? (1ull << g.target) : 0;
    for (int c = 0; c < g.nc; ++c) {
      int q = g.controls[c];
      if (local[q] >= 0) o.lmask |= 1u << local[q];
      else o.gmask |= 1ull << q;
    }
    memcpy(o.u, g.u, sizeof o.u);
    ops[*nops_total + tp->nops] = o;
    tp->nops++;
  }
  *nops_total += tp->nops;
}

int plan_tile_passes(const qs_gate* gates, int n, int N, int b, int L, TilePass* passes, int max_passes,
                     TileOp* ops, int max_ops) {
  (void)max_ops;
  int np = 0, nops = 0;
  const uint64_t lowS = (L >= 64) ? ~0ull : ((1ull << L) - 1);
  uint64_t S = lowS;
  int* gidx = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  int ng = 0;
  for (int i = 0; i < n; ++i) {
    GateClass gc = classify_u2(gates[i].u);
    if (gc.kind == GK_IDENT) continue;
    uint64_t need = (gc.kind == GK_DIAG) ? 0ull : (1ull << gates[i].target);
    uint64_t S2 = S | need;
    if ((__builtin_popcountll(S2) > b || ng >= MAX_OPS) && ng > 0) {
      if (np < max_passes) close_pass(gates, gidx, ng, N, b, S, &passes[np++], ops, &nops);
      ng = 0;
      S = lowS | need;
    } else {
      S = S2;
    }
    gidx[ng++] = i;
  }
  if (ng > 0 && np < max_passes) close_pass(gates, gidx, ng, N, b, S, &passes[np++], ops, &nops);
  free(gidx);
  return np;
}

qs_status launch_tile_pass(qs_sim* s, const TilePass& pass, const TileOp* ops) {
  TileParams P;
  memset(&P, 0, sizeof P);
  P.N = s->N;
  P.b = pass.b;
  // low contiguous bits of the tile
  int L = 0;
  while (L < pass.b && pass.bits[L] == L) ++L;
  P.L = L;
  uint64_t tmask = 0;
  for (int k = 0; k < pass.b; ++k) tmask |= 1ull << pass.bits[k];
  for (int k = L; k < pass.b; ++k) P.hb[k - L] = pass.bits[k];
  const uint64_t all = (s->N >= 64) ? ~0ull : ((1ull << s->N) - 1);
  P.out_mask = all & ~tmask;
  P.nops = pass.nops;
  for (int i = 0; i < pass.nops; ++i) P.ops[i] = ops[i];
  const uint64_t ntiles = 1ull << (s->N - pass.b);
  if (s->enc == QS_C128) {
    const size_t smem = ((size_t)16 << pass.b) + ((size_t)8 << (pass.b - L));
    QS_CUDA(cudaFuncSetAttribute(k_tile<double, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint64_t g = (uint64_t)s->num_sms * 3;
    k_tile<double, double2><<<(unsigned)(ntiles < g ? ntiles : g), TPB, smem, s->stream>>>((double2*)s->state, P);
  } else {
    if (L < 1) { qs_set_error("tile pass: complex64 tiles need bit 0"); return QS_EINVAL; }
    const size_t smem = ((size_t)8 << pass.b) + ((size_t)8 << (pass.b - L));
    QS_CUDA(cudaFuncSetAttribute(k_tile<float, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint64_t g = (uint64_t)s->num_sms * 3;
    k_tile<float, float2><<<(unsigned)(ntiles < g ? ntiles : g), TPB, smem, s->stream>>>((float2*)s->state, P);
  }
  QS_LAUNCH_CHECK();
  return QS_OK;
}
