// Tile passes: several gates per read and write of the state (the gate
// fusion that the end of Sec. 5.2 proposes to raise arithmetic intensity;
// every gate keeps its own 2x2 matrix, the fusion is in the data movement).
//
// A tile is the 2^b amplitudes whose index bits outside the tile bit set are
// fixed; the set holds the low 6 index bits (512-byte runs) plus the targets
// of the pass's gates.  Inside a CTA of 256 threads the b local bits are
// split three ways:
//   local bit 0 and RB-1 more local bits  -> register slots (2^RB amplitudes
//                                             per thread, updated in registers)
//   local bits 1..5                         -> the 32 lanes (updated with one
//                                             warp shuffle per amplitude)
//   the remaining 3 local bits              -> the 8 warps
// A gate on a register bit or a lane bit runs without shared memory; a gate on
// a warp bit first swaps that bit into a register slot by one shared-memory
// transpose.  Diagonal gates run in place whatever their target (the target
// bit is known for every element), and controls may be any bit (a control
// outside the tile is a per-tile condition).  Gate order is kept, so the
// result equals the per-gate sweep up to rounding order.
#include "internal.cuh"
#include "cplx.cuh"
#include <string.h>
#include <stdlib.h>

namespace {

constexpr int TPB = 256;      // 8 warps
constexpr int LANE_BITS = 5;  // local bits 1..5
constexpr int WARP_BITS = 3;
constexpr int MAX_TOPS = 96;
constexpr int LOW_BITS = 4;   // index bits always in the tile (16-amplitude runs)

enum TOpType : uint8_t { T_REG = 0, T_LANE = 1, T_DIAG_REG = 2, T_DIAG_THR = 3, T_DIAG_OUT = 4, T_XPOSE = 5 };

struct TOp {
  uint8_t type, kind, c0, c1;
  uint8_t a;           // T_REG / T_DIAG_REG: register slot; T_LANE: lane bit; T_DIAG_THR: local bit
  uint8_t pad[3];
  uint32_t smask;      // control bits among the register slots (bits of j)
  uint32_t tmask;      // control bits among lane / warp local bits (local-index mask)
  uint64_t gmask;      // control bits outside the tile
  uint64_t gtbit;      // T_DIAG_OUT: the target bit (global)
  float uf[8];
  double ud[8];
};
struct TMap {
  uint8_t reg[8];      // local bit of register slot s (reg[0] = 0)
  uint8_t warp[4];     // local bit of warp bit k
};

struct TileParams2 {
  int N, b;
  uint64_t out_mask;   // global bits outside the tile
  uint8_t gpos[20];    // global position of local bit k
  TMap init, fin;      // register / warp assignment at load and at store
  int nops;
  int last_xpose;      // index of the last transpose op, -1 if none
  TOp ops[MAX_TOPS];   // T_XPOSE ops carry their new map in the next TMap slot
  TMap maps[16];
};

__device__ __forceinline__ uint64_t deposit_t(uint64_t x, uint64_t mask) {
  uint64_t r = 0;
  for (uint64_t m = mask; m; m &= m - 1) {
    if (x & 1) r |= m & (~m + 1);
    x >>= 1;
  }
  return r;
}

template <typename R> __device__ __forceinline__ Cx<R> ucx(const TOp& o, int k);
template <> __device__ __forceinline__ Cx<float> ucx<float>(const TOp& o, int k) { return cx<float>(o.uf[2 * k], o.uf[2 * k + 1]); }
template <> __device__ __forceinline__ Cx<double> ucx<double>(const TOp& o, int k) { return cx<double>(o.ud[2 * k], o.ud[2 * k + 1]); }

// local index of register j under map m, given the thread part tl
template <int RB>
__device__ __forceinline__ uint32_t lidx(const TMap& m, int j, uint32_t tl) {
  uint32_t l = tl;
#pragma unroll
  for (int s = 0; s < RB; ++s)
    if ((j >> s) & 1) l |= 1u << m.reg[s];
  return l;
}
__device__ __forceinline__ uint32_t thread_part(const TMap& m, int lane, int warp) {
  uint32_t l = (uint32_t)lane << 1;
#pragma unroll
  for (int k = 0; k < WARP_BITS; ++k)
    if ((warp >> k) & 1) l |= 1u << m.warp[k];
  return l;
}
// global offset (within the tile) of a local index: local bits 0..3 are
// index bits 0..3, the others map through gpos
__device__ __forceinline__ uint64_t goff(uint32_t l, const uint8_t* gpos, int b) {
  uint64_t g = l & 15u;
  for (int k = 4; k < b; ++k)
    if ((l >> k) & 1) g |= 1ull << gpos[k];
  return g;
}

// --- register-slot pair op, slot S fixed at compile time -----------------------------
template <typename R, int RB, int S, typename F>
__device__ __forceinline__ void reg_pairs(Cx<R>* v, uint32_t smask, const F& f) {
  if (smask == 0) {   // the common case: no control among the register slots
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j)
      if (!((j >> S) & 1)) f.pair(v[j], v[j | (1 << S)]);
  } else {
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
      if ((j >> S) & 1) continue;
      if ((j & (int)smask) != (int)smask) continue;
      f.pair(v[j], v[j | (1 << S)]);
    }
  }
}

// diagonal on register slot S: factor d1 where bit S is 1, d0 where it is 0;
// skip0 / skip1 leave the elements with a unit factor untouched
template <typename R, int RB, int S>
__device__ __forceinline__ void reg_diag(Cx<R>* v, uint32_t smask, Cx<R> d0, Cx<R> d1, bool skip0, bool skip1) {
  if (smask == 0) {
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
      const bool one = (j >> S) & 1;
      if (one ? skip1 : skip0) continue;
      v[j] = cmul_code(v[j], one ? d1 : d0, 4);
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if ((j & (int)smask) != (int)smask) continue;
    const bool one = (j >> S) & 1;
    if (one ? skip1 : skip0) continue;
    v[j] = cmul_code(v[j], one ? d1 : d0, 4);
  }
}
template <typename R, int RB>
__device__ __forceinline__ void reg_diag_rt(Cx<R>* v, int s, uint32_t smask, Cx<R> d0, Cx<R> d1, bool skip0, bool skip1) {
  switch (s) {
    case 0: reg_diag<R, RB, 0>(v, smask, d0, d1, skip0, skip1); break;
    case 1: reg_diag<R, RB, (RB > 1 ? 1 : 0)>(v, smask, d0, d1, skip0, skip1); break;
    case 2: reg_diag<R, RB, (RB > 2 ? 2 : 0)>(v, smask, d0, d1, skip0, skip1); break;
    case 3: reg_diag<R, RB, (RB > 3 ? 3 : 0)>(v, smask, d0, d1, skip0, skip1); break;
    default: reg_diag<R, RB, (RB > 4 ? 4 : 0)>(v, smask, d0, d1, skip0, skip1); break;
  }
}
template <typename R, int RB, typename F>
__device__ __forceinline__ void reg_op(Cx<R>* v, int s, uint32_t smask, const F& f) {
  switch (s) {
    case 0: reg_pairs<R, RB, 0>(v, smask, f); break;
    case 1: if (RB > 1) reg_pairs<R, RB, (RB > 1 ? 1 : 0)>(v, smask, f); break;
    case 2: if (RB > 2) reg_pairs<R, RB, (RB > 2 ? 2 : 0)>(v, smask, f); break;
    case 3: if (RB > 3) reg_pairs<R, RB, (RB > 3 ? 3 : 0)>(v, smask, f); break;
    case 4: if (RB > 4) reg_pairs<R, RB, (RB > 4 ? 4 : 0)>(v, smask, f); break;
    default: if (RB > 5) reg_pairs<R, RB, (RB > 5 ? 5 : 0)>(v, smask, f); break;
  }
}

template <typename R> __device__ __forceinline__ R uscal(const TOp& o) {
  if constexpr (sizeof(R) == 4) return o.uf[0]; else return o.ud[0];
}

template <typename R> __device__ __forceinline__ R shx(R x, int m);
template <> __device__ __forceinline__ float shx<float>(float x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }
template <> __device__ __forceinline__ double shx<double>(double x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }

// lane-bit op: partner values by shuffle, each lane keeps its own output
template <typename R, int RB, bool SWAP>
__device__ __forceinline__ void lane_op(Cx<R>* v, const TOp& o, int lane, bool tok) {
  const int m = 1 << o.a;
  const bool hi = (lane >> o.a) & 1;
  Cx<R> u00 = ucx<R>(o, 0), u01 = ucx<R>(o, 1), u10 = ucx<R>(o, 2), u11 = ucx<R>(o, 3);
  if constexpr (sizeof(R) == 4) {
    if (SWAP && o.kind == GK_ANTI && o.c0 == 0 && o.c1 == 0) {
      // pure swap: every lane takes its partner's value
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const Cx<R> p = cx<R>(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (tok && (j & (int)o.smask) == (int)o.smask) v[j] = p;
      }
      return;
    }
    if (o.kind == GK_REAL) {
      // real coefficients: packed FP32x2 on (re, im)
      const float2 cs = hi ? make_float2(o.uf[6], o.uf[6]) : make_float2(o.uf[0], o.uf[0]);
      const float2 cp = hi ? make_float2(o.uf[4], o.uf[4]) : make_float2(o.uf[2], o.uf[2]);
      const bool all = tok && o.smask == 0;
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const float2 p = make_float2(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (!all && (!tok || (j & (int)o.smask) != (int)o.smask)) continue;
#ifdef QS_HAVE_F32X2
        const float2 r = __ffma2_rn(cs, make_float2(v[j].x, v[j].y), __fmul2_rn(cp, p));
#else
        const float2 r = make_float2(fmaf(cs.x, v[j].x, cp.x * p.x), fmaf(cs.x, v[j].y, cp.x * p.y));
#endif
        v[j] = cx<R>(r.x, r.y);
      }
      return;
    }
    // each lane keeps cs * own + cp * partner, with per-lane coefficients
    const Cx<R> cs = hi ? u11 : u00, cp = hi ? u10 : u01;
    if (o.smask == 0) {
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const Cx<R> p = cx<R>(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (tok) v[j] = cmac2(cs, v[j], cp, p);
      }
    } else {
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const Cx<R> p = cx<R>(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (tok && (j & (int)o.smask) == (int)o.smask) v[j] = cmac2(cs, v[j], cp, p);
      }
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    Cx<R> p = cx<R>(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
    if (!tok || (j & (int)o.smask) != (int)o.smask) continue;
    Cx<R> a0 = hi ? p : v[j], a1 = hi ? v[j] : p;
    switch (o.kind) {
      case GK_HAD: {
        const R s = uscal<R>(o);
        v[j] = hi ? cx<R>((a0.x - a1.x) * s, (a0.y - a1.y) * s) : cx<R>((a0.x + a1.x) * s, (a0.y + a1.y) * s);
        break;
      }
      case GK_ANTI:
        v[j] = hi ? cmul_code(a0, u10, o.c1) : cmul_code(a1, u01, o.c0);
        break;
      case GK_DIAG:
        v[j] = hi ? cmul_code(a1, u11, o.c1) : cmul_code(a0, u00, o.c0);
        break;
      default:
        v[j] = hi ? cmac2(u10, a0, u11, a1) : cmac2(u00, a0, u01, a1);
    }
  }
}

template <typename R, int RB>
__device__ __forceinline__ void load_tile(const void* s, Cx<R>* v, uint64_t base, const uint64_t* roff, uint64_t woff,
                                          int lane) {
  if constexpr (sizeof(R) == 4) {
    const float4* s4 = (const float4*)s;
#pragma unroll
    for (int jj = 0; jj < (1 << (RB - 1)); ++jj) {
      float4 x = s4[(base + woff + roff[jj]) >> 1];
      v[2 * jj] = cx<float>(x.x, x.y);
      v[2 * jj + 1] = cx<float>(x.z, x.w);
    }
  } else {
    const double2* s2 = (const double2*)s;
#pragma unroll
    for (int jj = 0; jj < (1 << (RB - 1)); ++jj) {
      const uint64_t g = base + woff + roff[jj];
      double2 x = s2[g], y = s2[g + 1];
      v[2 * jj] = cx<double>(x.x, x.y);
      v[2 * jj + 1] = cx<double>(y.x, y.y);
    }
  }
}
template <typename R, int RB>
__device__ __forceinline__ void store_tile(void* s, const Cx<R>* v, uint64_t base, const uint64_t* roff, uint64_t woff,
                                           int lane) {
  if constexpr (sizeof(R) == 4) {
    float4* s4 = (float4*)s;
#pragma unroll
    for (int jj = 0; jj < (1 << (RB - 1)); ++jj)
      s4[(base + woff + roff[jj]) >> 1] = make_float4(v[2 * jj].x, v[2 * jj].y, v[2 * jj + 1].x, v[2 * jj + 1].y);
  } else {
    double2* s2 = (double2*)s;
#pragma unroll
    for (int jj = 0; jj < (1 << (RB - 1)); ++jj) {
      const uint64_t g = base + woff + roff[jj];
      s2[g] = make_double2(v[2 * jj].x, v[2 * jj].y);
      s2[g + 1] = make_double2(v[2 * jj + 1].x, v[2 * jj + 1].y);
    }
  }
}

// FEAT: which specialised complex64 paths the pass needs (bit 0: swaps, bit 1:
// Hadamard-shaped); passes without them run a smaller kernel.
constexpr int FEAT_SWAP = 1, FEAT_HAD = 2;   // FEAT_HAD: real-matrix path (packed FP32x2)

// 16-byte global -> shared copies that bypass registers (LDGSTS), so the next
// tile's loads are in flight while the current tile is computed and stored.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Each thread stages exactly the 16-byte chunks it will read back, so the
// stage buffer needs no barrier: the thread's own wait_group orders it.
template <typename R, int RB>
__device__ __forceinline__ void stage_tile(const void* s, Cx<R>* st, uint64_t base, const uint64_t* roff, uint64_t woff,
                                           const TMap& m, uint32_t tl) {
#pragma unroll
  for (int jj = 0; jj < (1 << (RB - 1)); ++jj) {
    const uint32_t l = lidx<RB>(m, 2 * jj, tl);
    const uint64_t g = base + woff + roff[jj];
    if constexpr (sizeof(R) == 4) {
      cp_async16(((float4*)st) + (l >> 1), ((const float4*)s) + (g >> 1));
    } else {
      cp_async16(st + l, ((const double2*)s) + g);
      cp_async16(st + l + 1, ((const double2*)s) + g + 1);
    }
  }
  cp_async_commit();
}
template <typename R, int RB>
__device__ __forceinline__ void unstage_tile(const Cx<R>* st, Cx<R>* v, const TMap& m, uint32_t tl) {
#pragma unroll
  for (int jj = 0; jj < (1 << (RB - 1)); ++jj) {
    const uint32_t l = lidx<RB>(m, 2 * jj, tl);
    if constexpr (sizeof(R) == 4) {
      const float4 x = ((const float4*)st)[l >> 1];
      v[2 * jj] = cx<float>(x.x, x.y);
      v[2 * jj + 1] = cx<float>(x.z, x.w);
    } else {
      v[2 * jj] = st[l];
      v[2 * jj + 1] = st[l + 1];
    }
  }
}

template <typename R, int RB, int FEAT>
__global__ void __launch_bounds__(TPB, 2) k_tile2(void* __restrict__ s, const __grid_constant__ TileParams2 P) {
  extern __shared__ unsigned char smraw[];
  constexpr int NR = 1 << RB;
  // global offsets of the register part (pairs jj: slots 1..RB-1) at load / store
  uint64_t* roff_in = (uint64_t*)smraw;
  uint64_t* roff_out = roff_in + NR / 2;
  // transpose buffer, 2^b elements; between the last transpose of a tile and
  // the start of the next it stages the next tile
  Cx<R>* xb = (Cx<R>*)(smraw + NR * sizeof(uint64_t));
  Cx<R>* stg = xb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < NR / 2) {
    roff_in[threadIdx.x] = goff(lidx<RB>(P.init, 2 * threadIdx.x, 0), P.gpos, P.b);
    roff_out[threadIdx.x] = goff(lidx<RB>(P.fin, 2 * threadIdx.x, 0), P.gpos, P.b);
  }
  __syncthreads();
  const uint64_t woff_in = goff(thread_part(P.init, lane, warp), P.gpos, P.b);
  const uint64_t woff_out = goff(thread_part(P.fin, lane, warp), P.gpos, P.b);
  const uint32_t tl_in = thread_part(P.init, lane, warp);
  const uint64_t ntiles = 1ull << (P.N - P.b);
  Cx<R> v[NR];
  if (blockIdx.x < ntiles) stage_tile<R, RB>(s, stg, deposit_t(blockIdx.x, P.out_mask), roff_in, woff_in, P.init, tl_in);
  for (uint64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
    const uint64_t base = deposit_t(tau, P.out_mask);
    cp_async_wait_all();
    unstage_tile<R, RB>(stg, v, P.init, tl_in);
    const uint64_t nxt = tau + gridDim.x;
    if (P.last_xpose < 0 && nxt < ntiles)
      stage_tile<R, RB>(s, stg, deposit_t(nxt, P.out_mask), roff_in, woff_in, P.init, tl_in);
    TMap cur = P.init;
    uint32_t tl = thread_part(cur, lane, warp);
    Cx<R> fac = cx<R>((R)1, (R)0);
    int mapi = 0;
    for (int i = 0; i < P.nops; ++i) {
      const TOp& o = P.ops[i];
      if (o.type == T_XPOSE) {
        // write every register at its local index, read back under the new map
#pragma unroll
        for (int jj = 0; jj < NR / 2; ++jj) {
          const uint32_t l = lidx<RB>(cur, 2 * jj, tl);
          if constexpr (sizeof(R) == 4) {
            ((float4*)xb)[l >> 1] = make_float4(v[2 * jj].x, v[2 * jj].y, v[2 * jj + 1].x, v[2 * jj + 1].y);
          } else {
            xb[l] = v[2 * jj];
            xb[l + 1] = v[2 * jj + 1];
          }
        }
        __syncthreads();
        cur = P.maps[mapi++];
        tl = thread_part(cur, lane, warp);
#pragma unroll
        for (int jj = 0; jj < NR / 2; ++jj) {
          const uint32_t l = lidx<RB>(cur, 2 * jj, tl);
          if constexpr (sizeof(R) == 4) {
            float4 x = ((const float4*)xb)[l >> 1];
            v[2 * jj] = cx<float>(x.x, x.y);
            v[2 * jj + 1] = cx<float>(x.z, x.w);
          } else {
            v[2 * jj] = xb[l];
            v[2 * jj + 1] = xb[l + 1];
          }
        }
        __syncthreads();
        if (i == P.last_xpose && nxt < ntiles)
          stage_tile<R, RB>(s, stg, deposit_t(nxt, P.out_mask), roff_in, woff_in, P.init, tl_in);
        continue;
      }
      const bool gok = (base & o.gmask) == o.gmask;       // outer controls
      const bool tok = (tl & o.tmask) == o.tmask;         // lane / warp controls
      if (o.pad[0] != 0) {
        // folded run of per-thread diagonals: multiply the factor, apply at the end
        if (gok && tok) {
          const bool one = (o.type == T_DIAG_THR) ? ((tl >> o.a) & 1) : ((base & o.gtbit) != 0);
          if ((one ? o.c1 : o.c0) != 0) fac = cmul_code(fac, ucx<R>(o, one ? 3 : 0), 4);
        }
        if (o.pad[0] == 2) {
          if (fac.x != (R)1 || fac.y != (R)0) {
#pragma unroll
            for (int j = 0; j < NR; ++j) v[j] = cmul_code(v[j], fac, 4);
          }
          fac = cx<R>((R)1, (R)0);
        }
        continue;
      }
      if (!gok) continue;
      switch (o.type) {
        case T_REG: {
          if (!tok) break;
          if constexpr (sizeof(R) == 4) {
            // complex64: Hadamard-shaped or dense (exact for the unit entries
            // of X, Y, CNOT, TOFFOLI)
            // (a register-slot swap as renames makes the register allocation
            // spill at 128 registers; swaps on register slots stay dense)
            if ((FEAT & FEAT_HAD) && o.kind == GK_REAL) {
              OpRealF f;
              f.u00 = make_float2(o.uf[0], o.uf[0]); f.u01 = make_float2(o.uf[2], o.uf[2]);
              f.u10 = make_float2(o.uf[4], o.uf[4]); f.u11 = make_float2(o.uf[6], o.uf[6]);
              reg_op<R, RB>(v, o.a, o.smask, f);
            } else {
              OpDense<R> f; f.u00 = ucx<R>(o, 0); f.u01 = ucx<R>(o, 1); f.u10 = ucx<R>(o, 2); f.u11 = ucx<R>(o, 3);
              reg_op<R, RB>(v, o.a, o.smask, f);
            }
          } else {
            // complex128: the FP64 pipe is the bound, so keep the cheaper forms
            switch (o.kind) {
              case GK_HAD: { OpHad<R> f; f.s = uscal<R>(o); reg_op<R, RB>(v, o.a, o.smask, f); break; }
              case GK_ANTI: { OpAnti<R> f; f.f01 = ucx<R>(o, 1); f.f10 = ucx<R>(o, 2); f.c0 = o.c0; f.c1 = o.c1; reg_op<R, RB>(v, o.a, o.smask, f); break; }
              default: {
                OpDense<R> f; f.u00 = ucx<R>(o, 0); f.u01 = ucx<R>(o, 1); f.u10 = ucx<R>(o, 2); f.u11 = ucx<R>(o, 3);
                reg_op<R, RB>(v, o.a, o.smask, f);
              }
            }
          }
          break;
        }
        case T_LANE:
          lane_op<R, RB, (FEAT & FEAT_SWAP) != 0>(v, o, lane, tok);
          break;
        case T_DIAG_REG:
        case T_DIAG_THR:
        case T_DIAG_OUT: {
          if (!tok) break;
          const Cx<R> d0 = ucx<R>(o, 0), d1 = ucx<R>(o, 3);
          if (o.type == T_DIAG_REG) {
            if constexpr (sizeof(R) == 4) {
              reg_diag_rt<R, RB>(v, o.a, o.smask, d0, d1, o.c0 == 0, o.c1 == 0);
            } else {
              const int sl = o.a;
#pragma unroll
              for (int j = 0; j < NR; ++j) {
                if ((j & (int)o.smask) != (int)o.smask) continue;
                const bool one = (j >> sl) & 1;
                v[j] = one ? cmul_code(v[j], d1, o.c1) : cmul_code(v[j], d0, o.c0);
              }
            }
          } else {
            const bool one = (o.type == T_DIAG_THR) ? ((tl >> o.a) & 1) : ((base & o.gtbit) != 0);
            const int code = one ? o.c1 : o.c0;
            if (code == 0) break;
            const Cx<R> d = one ? d1 : d0;
            if (o.smask == 0) {
#pragma unroll
              for (int j = 0; j < NR; ++j) v[j] = cmul_code(v[j], d, sizeof(R) == 4 ? 4 : code);
            } else {
#pragma unroll
              for (int j = 0; j < NR; ++j)
                if ((j & (int)o.smask) == (int)o.smask) v[j] = cmul_code(v[j], d, sizeof(R) == 4 ? 4 : code);
            }
          }
          break;
        }
        default: break;
      }
    }
    store_tile<R, RB>(s, v, base, roff_out, woff_out, lane);
  }
}

}  // namespace

// ---------------------------------------------------------------------------------
// planner
// ---------------------------------------------------------------------------------
struct PassPlan {
  TileParams2 P;
};

static void fill_u(TOp& o, const double* u) {
  for (int k = 0; k < 8; ++k) { o.ud[k] = u[k]; o.uf[k] = (float)u[k]; }
}

// ---- gate-sequence rewriting inside a pass (exact up to rounding) ----------------
static bool same_controls(const qs_gate& a, const qs_gate& b) {
  if (a.nc != b.nc) return false;
  if (a.nc == 0) return true;
  if (a.nc == 1) return a.controls[0] == b.controls[0];
  return (a.controls[0] == b.controls[0] && a.controls[1] == b.controls[1]) ||
         (a.controls[0] == b.controls[1] && a.controls[1] == b.controls[0]);
}
static bool is_diag_gate(const qs_gate& g) { return classify_u2(g.u).kind == GK_DIAG; }
// u = b * a (apply a first), 2x2 complex row-major (re, im)
static void mat_mul2(const double* b, const double* a, double* u) {
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      double re = 0, im = 0;
      for (int k = 0; k < 2; ++k) {
        const double br = b[2 * (2 * r + k)], bi = b[2 * (2 * r + k) + 1];
        const double ar = a[2 * (2 * k + c)], ai = a[2 * (2 * k + c) + 1];
        re += br * ar - bi * ai;
        im += br * ai + bi * ar;
      }
      u[2 * (2 * r + c)] = re;
      u[2 * (2 * r + c) + 1] = im;
    }
}
// Diagonal gates commute with each other and with every gate whose target is
// none of their qubits (a control acts diagonally too), so each diagonal gate
// is delayed until a non-diagonal gate targets its target or one of its
// controls, or the pass ends; the delayed gates are emitted together.  Then neighbouring gates with the same
// target and the same controls are multiplied into one 2x2 (FP64, host).
static int rewrite_pass(const qs_gate* gates, const int* gidx, int ng, qs_gate* out) {
  int n = 0;
  int pend[MAX_TOPS * 2];
  int np = 0;
  for (int i = 0; i < ng; ++i) {
    const qs_gate& g = gates[gidx[i]];
    if (is_diag_gate(g)) { pend[np++] = gidx[i]; continue; }
    // a delayed diagonal must not pass a gate whose target is one of its
    // qubits (its target or one of its controls)
    bool conflict = false;
    for (int k = 0; k < np; ++k) {
      const qs_gate& d = gates[pend[k]];
      conflict |= (d.target == g.target);
      for (int c = 0; c < d.nc; ++c) conflict |= (d.controls[c] == g.target);
    }
    if (conflict) {
      for (int k = 0; k < np; ++k) out[n++] = gates[pend[k]];
      np = 0;
    }
    out[n++] = g;
  }
  for (int k = 0; k < np; ++k) out[n++] = gates[pend[k]];
  // compose neighbours with equal (target, controls)
  int m = 0;
  for (int i = 0; i < n; ++i) {
    if (m > 0 && out[m - 1].target == out[i].target && same_controls(out[m - 1], out[i])) {
      double u[8];
      mat_mul2(out[i].u, out[m - 1].u, u);
      memcpy(out[m - 1].u, u, sizeof u);
      continue;
    }
    out[m++] = out[i];
  }
  return m;
}

// Build the op list of one pass.  tile: bitmask of the tile's global bits
// (contains bits 0..5), gidx: the gates in order.  Returns false if the op
// list overflows (caller splits the pass).
static bool build_pass(const qs_gate* gates_in, const int* gidx_in, int ng_in, int N, int b, int RB, uint64_t tile,
                       TileParams2* P, bool real_kinds) {
  static thread_local qs_gate seq[MAX_TOPS * 2];
  static thread_local int seq_idx[MAX_TOPS * 2];
  if (ng_in > MAX_TOPS * 2) return false;
  const int ng = rewrite_pass(gates_in, gidx_in, ng_in, seq);
  for (int i = 0; i < ng; ++i) seq_idx[i] = i;
  const qs_gate* gates = seq;
  const int* gidx = seq_idx;
  memset(P, 0, sizeof *P);
  P->N = N;
  P->b = b;
  // local bits: 0..3 = index bits 0..3 (runs of 16 amplitudes), 4..5 = the
  // two high tile qubits with the fewest non-diagonal gates in the pass
  // (lane qubits, updated by shuffles), 6..b-1 = the other tile qubits
  // Lane score: a swap (X, CNOT, TOFFOLI) on a lane qubit costs two shuffles
  // and no arithmetic, a dense gate there costs the shuffles on top of the
  // arithmetic it costs anyway; prefer swap-heavy, dense-light lane qubits.
  int local[64];
  int uses[64];
  for (int q = 0; q < 64; ++q) { local[q] = -1; uses[q] = 0; }
  for (int i = 0; i < ng; ++i) {
    const qs_gate& g = gates[gidx[i]];
    GateClass gc = classify_u2(g.u);
    if (gc.kind == GK_DIAG) continue;
    const bool swap = (gc.kind == GK_ANTI && gc.c0 == 0 && gc.c1 == 0);
    uses[g.target] += swap ? -4 : 1;
  }
  for (int q = 0; q < LOW_BITS; ++q) { P->gpos[q] = (uint8_t)q; local[q] = q; }
  int k = LOW_BITS;
  int is_target[64];
  for (int q = 0; q < 64; ++q) is_target[q] = 0;
  for (int i = 0; i < ng; ++i)
    if (classify_u2(gates[gidx[i]].u).kind != GK_DIAG) is_target[gates[gidx[i]].target] = 1;
  // Lane qubits: high targets go to the register slots while they fit
  // (no shuffles); only the targets beyond RB-1 take lanes (best lane score
  // first), and the remaining lanes take non-target tile qubits.
  int nhigh_targets = 0;
  for (int q = LOW_BITS; q < N; ++q)
    if (((tile >> q) & 1) && is_target[q]) ++nhigh_targets;
  int lane_targets = nhigh_targets - (RB - 1);
  if (lane_targets < 0) lane_targets = 0;
  for (int pick = 0; pick < 2; ++pick) {
    const bool want_target = pick < lane_targets;
    int best = -1;
    for (int q = LOW_BITS; q < N; ++q) {
      if (!((tile >> q) & 1) || local[q] >= 0) continue;
      if (is_target[q] != (want_target ? 1 : 0)) continue;
      if (best < 0 || uses[q] < uses[best]) best = q;
    }
    if (best < 0)   // fall back to any tile qubit
      for (int q = LOW_BITS; q < N && best < 0; ++q)
        if (((tile >> q) & 1) && local[q] < 0) best = q;
    P->gpos[k] = (uint8_t)best;
    local[best] = k++;
  }
  for (int q = LOW_BITS; q < N; ++q)
    if (((tile >> q) & 1) && local[q] < 0) { P->gpos[k] = (uint8_t)q; local[q] = k++; }
  const uint64_t all = (N >= 64) ? ~0ull : ((1ull << N) - 1);
  P->out_mask = all & ~tile;
  // high local bits 6..b-1: RB-1 register slots + WARP_BITS warp bits
  const int nhigh = b - 6;
  // next use of each high local bit as a non-diagonal target, for eviction
  // choices; initial registers = the first RB-1 distinct high targets
  int slot_of[32];
  for (int i = 0; i < 32; ++i) slot_of[i] = -1;
  TMap cur;
  memset(&cur, 0, sizeof cur);
  cur.reg[0] = 0;
  int nreg = 1;
  for (int i = 0; i < ng && nreg < RB; ++i) {
    const qs_gate& g = gates[gidx[i]];
    if (classify_u2(g.u).kind == GK_DIAG) continue;
    int p = local[g.target];
    if (p >= 6 && slot_of[p] < 0) { slot_of[p] = nreg; cur.reg[nreg++] = (uint8_t)p; }
  }
  for (int p = 6; p < b && nreg < RB; ++p)
    if (slot_of[p] < 0) { slot_of[p] = nreg; cur.reg[nreg++] = (uint8_t)p; }
  int nw = 0;
  for (int p = 6; p < b; ++p)
    if (slot_of[p] < 0) cur.warp[nw++] = (uint8_t)p;
  (void)nhigh;
  P->init = cur;
  int nops = 0, nmaps = 0;
  auto reg_slot = [&](int p) -> int {
    if (p == 0) return 0;
    for (int s = 1; s < RB; ++s) if (cur.reg[s] == p) return s;
    return -1;
  };
  for (int i = 0; i < ng; ++i) {
    const qs_gate& g = gates[gidx[i]];
    GateClass gc = classify_u2(g.u);
    int p = local[g.target];
    const bool diag = (gc.kind == GK_DIAG);
    if (!diag && p >= 6 && reg_slot(p) < 0) {
      // transpose: bring p into the register slot whose next use is farthest
      if (nops >= MAX_TOPS || nmaps >= 16) return false;
      int best = 1, bestd = -1;
      for (int s = 1; s < RB; ++s) {
        int d = ng + 1;
        for (int j = i; j < ng; ++j) {
          const qs_gate& h = gates[gidx[j]];
          if (classify_u2(h.u).kind != GK_DIAG && local[h.target] == cur.reg[s]) { d = j; break; }
        }
        if (d > bestd) { bestd = d; best = s; }
      }
      int evicted = cur.reg[best];
      cur.reg[best] = (uint8_t)p;
      for (int w = 0; w < WARP_BITS; ++w)
        if (cur.warp[w] == p) cur.warp[w] = (uint8_t)evicted;
      TOp x;
      memset(&x, 0, sizeof x);
      x.type = T_XPOSE;
      P->ops[nops++] = x;
      P->maps[nmaps++] = cur;
    }
    if (nops >= MAX_TOPS) return false;
    TOp o;
    memset(&o, 0, sizeof o);
    o.kind = (uint8_t)gc.kind;
    o.c0 = (uint8_t)gc.c0;
    o.c1 = (uint8_t)gc.c1;
    fill_u(o, g.u);
    for (int c = 0; c < g.nc; ++c) {
      int q = g.controls[c];
      int lq = local[q];
      if (lq < 0) { o.gmask |= 1ull << q; continue; }
      int s = reg_slot(lq);
      if (s >= 0) o.smask |= 1u << s;
      else o.tmask |= 1u << lq;
    }
    if (p < 0) {
      o.type = T_DIAG_OUT;
      o.gtbit = 1ull << g.target;
    } else if (diag) {
      int s = reg_slot(p);
      if (s >= 0) { o.type = T_DIAG_REG; o.a = (uint8_t)s; }
      else { o.type = T_DIAG_THR; o.a = (uint8_t)p; }
    } else if (p >= 1 && p <= 5) {
      o.type = T_LANE;
      o.a = (uint8_t)(p - 1);
    } else {
      o.type = T_REG;
      o.a = (uint8_t)reg_slot(p);
    }
    // complex64: real matrices take the packed FP32x2 path, except pure swaps
    // on lane qubits (those only exchange values)
    const bool real = (g.u[1] == 0.0 && g.u[3] == 0.0 && g.u[5] == 0.0 && g.u[7] == 0.0);
    const bool pure_swap = (gc.kind == GK_ANTI && gc.c0 == 0 && gc.c1 == 0);
    if (real_kinds && real && !diag && (o.type == T_REG || (o.type == T_LANE && !pure_swap))) o.kind = GK_REAL;
    P->ops[nops++] = o;
  }
  // diagonal ops commute: inside each run of them, put the register-slot ones
  // first so that the per-thread ones are contiguous
  for (int i = 0; i < nops;) {
    auto isd = [&](int k) {
      const int t = P->ops[k].type;
      return t == T_DIAG_REG || t == T_DIAG_THR || t == T_DIAG_OUT;
    };
    int j = i;
    while (j < nops && isd(j)) ++j;
    if (j - i >= 2) {
      TOp tmp[MAX_TOPS];
      int m = 0;
      for (int k = i; k < j; ++k)
        if (P->ops[k].type == T_DIAG_REG || P->ops[k].smask != 0) tmp[m++] = P->ops[k];
      for (int k = i; k < j; ++k)
        if (!(P->ops[k].type == T_DIAG_REG || P->ops[k].smask != 0)) tmp[m++] = P->ops[k];
      for (int k = 0; k < m; ++k) P->ops[i + k] = tmp[k];
    }
    i = (j > i) ? j : i + 1;
  }
  // runs of per-thread diagonals (target on a lane / warp bit or outside the
  // tile, no register-slot control) fold into one factor per thread
  for (int i = 0; i < nops;) {
    int j = i;
    while (j < nops && (P->ops[j].type == T_DIAG_THR || P->ops[j].type == T_DIAG_OUT) && P->ops[j].smask == 0) ++j;
    if (j - i >= 2) {
      for (int k = i; k < j - 1; ++k) P->ops[k].pad[0] = 1;  // accumulate
      P->ops[j - 1].pad[0] = 2;                              // accumulate and apply
    }
    i = (j > i) ? j : i + 1;
  }
  P->nops = nops;
  P->fin = cur;
  P->last_xpose = -1;
  for (int i = 0; i < nops; ++i)
    if (P->ops[i].type == T_XPOSE) P->last_xpose = i;
  return true;
}

int tile_register_bits(qs_encoding enc) { return enc == QS_C128 ? 4 : 5; }
int tile_bits(qs_encoding enc) { return tile_register_bits(enc) + LANE_BITS + WARP_BITS; }

// Pass packing.  Each pass takes gates in circuit order while the union of
// their non-diagonal targets fits the tile; a gate that does not fit is left
// for a later pass, and so is every later gate that does not commute with a
// gate left out.  Two gates commute when every qubit they share is one on
// which both act diagonally (a control, or the target of a diagonal gate):
// both are then block-diagonal on the shared qubits and act on disjoint
// qubits inside each block.  Every gate a pass takes therefore commutes with
// all the earlier gates it overtakes, and the product equals the circuit's.
// A pass whose op list overflows is split.
static qs_status run_pass(qs_sim* s, const qs_gate* gates, const int* gidx, int ng, uint64_t tile, int* launched,
                          PassTimer* timer);

qs_status run_tile_passes(qs_sim* s, const qs_gate* gates, int n, int* n_passes, PassTimer* timer) {
  const int b = tile_bits(s->enc);
  const int N = s->N;
  // per gate: qubits acted on non-diagonally (X) and diagonally (Z)
  int* gidx = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  int* rem = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  uint64_t* xq = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n + 1));
  uint64_t* zq = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n + 1));
  if (!gidx || !rem || !xq || !zq) {
    free(gidx); free(rem); free(xq); free(zq);
    return QS_ENOMEM;
  }
  int nrem = 0;
  for (int i = 0; i < n; ++i) {
    GateClass gc = classify_u2(gates[i].u);
    if (gc.kind == GK_IDENT) continue;
    uint64_t z = 0;
    for (int c = 0; c < gates[i].nc; ++c) z |= 1ull << gates[i].controls[c];
    if (gc.kind == GK_DIAG) { xq[i] = 0; z |= 1ull << gates[i].target; }
    else xq[i] = 1ull << gates[i].target;
    zq[i] = z;
    rem[nrem++] = i;
  }
  const uint64_t low = (1ull << LOW_BITS) - 1;
  // A transpose costs about a third of a sweep, so a pass takes only as many
  // high targets as the lanes and register slots hold (no transposes); the
  // warp bits are padding.
  const int max_targets = LOW_BITS + 2 + (tile_register_bits(s->enc) - 1);
  int launched = 0;
  qs_status st = QS_OK;
  while (nrem > 0 && st == QS_OK) {
    uint64_t S = low, bx = 0, bz = 0;
    int ng = 0, nleft = 0;
    for (int k = 0; k < nrem; ++k) {
      const int i = rem[k];
      const bool blocked = (xq[i] & (bx | bz)) != 0 || ((xq[i] | zq[i]) & bx) != 0;
      if (!blocked && __builtin_popcountll(S | xq[i]) <= max_targets && ng < MAX_TOPS / 2) {
        S |= xq[i];
        gidx[ng++] = i;
      } else {
        bx |= xq[i];
        bz |= zq[i];
        rem[nleft++] = i;
      }
    }
    nrem = nleft;
    // pad the tile to b bits with qubits the pass does not touch at all:
    // diagonal gates and controls on qubits outside the tile are per-tile
    // constants (a diagonal folds into one factor), inside it they cost
    // per-element work
    uint64_t used = 0;
    for (int k = 0; k < ng; ++k) used |= xq[gidx[k]] | zq[gidx[k]];
    uint64_t tile = S;
    for (int q = 0; q < N && __builtin_popcountll(tile) < b; ++q)
      if (!((used >> q) & 1)) tile |= 1ull << q;
    for (int q = 0; q < N && __builtin_popcountll(tile) < b; ++q) tile |= 1ull << q;
    st = run_pass(s, gates, gidx, ng, tile, &launched, timer);
  }
  free(gidx); free(rem); free(xq); free(zq);
  if (n_passes) *n_passes = launched;
  return st;
}

static qs_status launch_pass(qs_sim* s, const TileParams2& P, PassTimer* timer) {
  const bool timed = timer && timer->n < timer->max_ev;
  if (timed) QS_CUDA(cudaEventRecord(timer->ev[2 * timer->n], s->stream));
  const uint64_t ntiles = 1ull << (s->N - P.b);
  const uint64_t gmax = (uint64_t)s->num_sms * 2;   // two persistent CTAs per SM
  const unsigned grid = (unsigned)(ntiles < gmax ? ntiles : gmax);
  if (s->enc == QS_C128) {
    const size_t smem = ((size_t)16 << P.b) + 16 * sizeof(uint64_t);
    QS_CUDA(cudaFuncSetAttribute(k_tile2<double, 4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tile2<double, 4, 0><<<grid, TPB, smem, s->stream>>>(s->state, P);
  } else {
    int feat = 0;
    for (int i = 0; i < P.nops; ++i) {
      const TOp& o = P.ops[i];
      if (o.type == T_LANE && o.kind == GK_ANTI && o.c0 == 0 && o.c1 == 0) feat |= FEAT_SWAP;
      if ((o.type == T_REG || o.type == T_LANE) && o.kind == GK_REAL) feat |= FEAT_HAD;
    }
    const size_t smem = ((size_t)8 << P.b) + 32 * sizeof(uint64_t);
    auto go = [&](auto kern) -> qs_status {
      QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<grid, TPB, smem, s->stream>>>(s->state, P);
      return QS_OK;
    };
    switch (feat) {
      case 0: QS_TRY(go(k_tile2<float, 5, 0>)); break;
      case 1: QS_TRY(go(k_tile2<float, 5, 1>)); break;
      case 2: QS_TRY(go(k_tile2<float, 5, 2>)); break;
      default: QS_TRY(go(k_tile2<float, 5, 3>)); break;
    }
  }
  QS_LAUNCH_CHECK();
  if (timed) {
    QS_CUDA(cudaEventRecord(timer->ev[2 * timer->n + 1], s->stream));
    timer->n++;
  } else if (timer) {
    timer->n++;
  }
  return QS_OK;
}

static qs_status run_pass(qs_sim* s, const qs_gate* gates, const int* gidx, int ng, uint64_t tile, int* launched,
                          PassTimer* timer) {
  static thread_local TileParams2 P;
  const int b = tile_bits(s->enc);
  if (build_pass(gates, gidx, ng, s->N, b, tile_register_bits(s->enc), tile, &P, s->enc == QS_C64)) {
    QS_TRY(launch_pass(s, P, timer));
    ++*launched;
    return QS_OK;
  }
  // too many ops for one launch: split the gate run in halves (same tile)
  const int h = ng / 2;
  QS_TRY(run_pass(s, gates, gidx, h, tile, launched, timer));
  return run_pass(s, gates, gidx + h, ng - h, tile, launched, timer);
}
