// Tile passes: several gates per read and write of the state (the gate
// fusion that the end of Sec. 5.2 proposes to raise arithmetic intensity;
// every gate keeps its own 2x2 matrix, the fusion is in the data movement).
//
// A tile is the 2^b amplitudes whose index bits outside the tile bit set are
// fixed (b = 13 for complex64, 12 for complex128); the set always holds the
// low LOW_BITS = 4 index bits (16-amplitude runs: 128 B of complex64, 256 B
// of complex128) plus the targets of the pass's gates, padded with qubits the
// pass does not touch.  Inside a CTA of 256 threads the b local bits are
// split three ways:
//   local bit 0 and RB-1 more local bits  -> register slots (2^RB amplitudes
//                                             per thread, updated in registers)
//   local bits 1..5                         -> the 32 lanes (updated with one
//                                             warp shuffle per amplitude)
//   the remaining 3 local bits              -> the 8 warps
// A gate on a register bit or a lane bit runs without shared memory; a gate on
// a warp bit first swaps that bit into a register slot by one shared-memory
// transpose.  A pure swap (X, CNOT, TOFFOLI) whose controls lie outside the
// register slots and the lanes moves no data: it relabels its target bit.
// Each thread keeps the relabelled local bits in a mask xl (the element a
// thread holds at physical local index p is the tile's element p ^ xl; xl is
// the same in all lanes of a warp) and their global offset gx; conditions, the
// roles of a pair, the transposes and the store address read them, and an op
// that needs a register slot in place first exchanges it back (T_UNFLIP).  Diagonal gates run in place whatever their target (the target
// bit is known for every element), and controls may be any bit (a control
// outside the tile is a per-tile condition).  The host planner may take a
// gate ahead of earlier gates left for later passes only when it commutes
// with all of them, so the result equals the per-gate sweep up to rounding
// order.
//
// This header holds the device side: it is compiled into the library (the
// op interpreter, k_tile.cu) and, as source text, into the passes compiled at
// run time (tile_jit.cu), so it includes nothing when QS_JIT is defined.
#pragma once
#ifndef QS_JIT
#include <cuda_runtime.h>
#include <stdint.h>
#endif
#include "gatekind.h"
#include "cplx.cuh"

namespace qs_tile {

constexpr int TPB = 256;      // 8 warps
constexpr int LANE_BITS = 5;  // local bits 1..5
constexpr int WARP_BITS = 3;
constexpr int MAX_TOPS = 96;
constexpr int LOW_BITS = 4;   // index bits always in the tile (16-amplitude runs)

enum TOpType : uint8_t { T_REG = 0, T_LANE = 1, T_DIAG_REG = 2, T_DIAG_THR = 3, T_DIAG_OUT = 4, T_XPOSE = 5,
                         T_DIAG_TAB = 6, T_FLIP = 7, T_UNFLIP = 8 };
constexpr int MAX_TABS = 8;   // per-register factor tables of a pass

struct TOp {
  uint8_t type, kind, c0, c1;
  uint8_t a;           // T_REG / T_DIAG_REG / T_UNFLIP: register slot; T_LANE: lane bit;
                       // T_DIAG_THR / T_FLIP: local bit
  uint8_t pad[3];      // [0]: fold flag of per-thread diagonals; [1]: the target
                       // slot may be relabelled; [2]: local bit of the slot
  uint32_t smask;      // control bits among the register slots (bits of j)
  uint32_t tmask;      // control bits among lane / warp local bits (local-index mask)
  uint64_t gmask;      // control bits outside the tile
  uint64_t gtbit;      // T_DIAG_OUT: the target bit (global); T_FLIP / T_UNFLIP: the
                       // global offset of the relabelled local bit
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
  int from_zero;       // the state is |0..0> and not in memory: tiles start as
                       // zeros (amplitude 1 at index 0), nothing is loaded
  // with from_zero: tiles start as the product state
  // a(i) = prod_q f_q(bit q of i) instead (f_q = (1, 0) for every q is |0..0>).
  // complex64: pf[q][bit] = f_q(bit) as float2 bits; ptab[j] = the product
  // over the register slots of the load map for register j, formed in FP64.
  // complex128: the same in FP64, pfd[q][bit] = (re, im) and ptabd[j] =
  // (re, im) as double bits
  int from_product;
  uint64_t pf[64][2];
  uint64_t ptab[32];
  uint64_t pfd[64][2][2];
  uint64_t ptabd[16][2];
  TOp ops[MAX_TOPS];   // T_XPOSE ops carry their new map in the next TMap slot
  TMap maps[16];
  // T_DIAG_TAB: the factor of register j, complex64 (re, im) float bits in
  // tab[t][j]; complex128 re, im double bits in tab[t][2j], tab[t][2j+1]
  uint64_t tab[MAX_TABS][32];
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
// double-float passes: the host stores each coefficient as its (hi, lo) float
// pair in the 8 bytes of the double (df_pack), so nothing here runs on the
// FP64 units
__device__ __forceinline__ DF df_unpack(uint64_t w) {
  return DF(__uint_as_float((uint32_t)w), __uint_as_float((uint32_t)(w >> 32)));
}
template <> __device__ __forceinline__ Cx<DF> ucx<DF>(const TOp& o, int k) {
  return cx<DF>(df_unpack(__double_as_longlong(o.ud[2 * k])), df_unpack(__double_as_longlong(o.ud[2 * k + 1])));
}

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
template <> __device__ __forceinline__ DF uscal<DF>(const TOp& o) { return df_unpack(__double_as_longlong(o.ud[0])); }

// factor of register j in table t (complex64: one (re, im) word; complex128:
// two FP64 words, or two packed (hi, lo) float pairs in double-float passes)
template <typename R> __device__ __forceinline__ Cx<R> tab_factor(const TileParams2& P, int t, int j);
template <> __device__ __forceinline__ Cx<float> tab_factor<float>(const TileParams2& P, int t, int j) {
  const uint64_t w = P.tab[t][j];
  return cx<float>(__uint_as_float((uint32_t)w), __uint_as_float((uint32_t)(w >> 32)));
}
template <> __device__ __forceinline__ Cx<double> tab_factor<double>(const TileParams2& P, int t, int j) {
  return cx<double>(__longlong_as_double((long long)P.tab[t][2 * j]),
                    __longlong_as_double((long long)P.tab[t][2 * j + 1]));
}
template <> __device__ __forceinline__ Cx<DF> tab_factor<DF>(const TileParams2& P, int t, int j) {
  return cx<DF>(df_unpack(P.tab[t][2 * j]), df_unpack(P.tab[t][2 * j + 1]));
}

template <typename R> __device__ __forceinline__ R shx(R x, int m);
template <> __device__ __forceinline__ float shx<float>(float x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }
template <> __device__ __forceinline__ double shx<double>(double x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }
template <> __device__ __forceinline__ DF shx<DF>(DF x, int m) {
  return DF(__shfl_xor_sync(0xffffffffu, x.hi, m), __shfl_xor_sync(0xffffffffu, x.lo, m));
}

// lane-bit op: partner values by shuffle, each lane keeps its own output
// (GK_BFLY as the butterfly: one packed instruction per amplitude, written in
// place).  CT: the op's structure is a compile-time constant (compiled passes).
template <typename R, int RB, bool SWAP, bool CT, class OS>
__device__ __forceinline__ void lane_op(Cx<R>* v, const OS& st, const TOp& o, int lane, bool tok, uint32_t xl) {
  const int m = 1 << st.a;
  const bool hi = ((lane >> st.a) ^ (xl >> (st.a + 1))) & 1;   // the tile's bit, not the lane's
  Cx<R> u00 = ucx<R>(o, 0), u01 = ucx<R>(o, 1), u10 = ucx<R>(o, 2), u11 = ucx<R>(o, 3);
  if constexpr (sizeof(R) == 4) {
    if (SWAP && st.kind == GK_ANTI && st.c0 == 0 && st.c1 == 0) {
      // pure swap: every lane takes its partner's value
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const Cx<R> p = cx<R>(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (tok && (j & (int)st.smask) == (int)st.smask) v[j] = p;
      }
      return;
    }
    if (st.kind == GK_BFLY) {
      // butterfly: own + partner (low lane), partner - own (high lane)
      const float2 sg = hi ? make_float2(-1.f, -1.f) : make_float2(1.f, 1.f);
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const float2 p = make_float2(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (!tok || (j & (int)st.smask) != (int)st.smask) continue;
#ifdef QS_HAVE_F32X2
        const float2 r = __ffma2_rn(sg, make_float2(v[j].x, v[j].y), p);
#else
        const float2 r = make_float2(fmaf(sg.x, v[j].x, p.x), fmaf(sg.x, v[j].y, p.y));
#endif
        v[j] = cx<R>(r.x, r.y);
      }
      return;
    }
    if (st.kind == GK_REAL || st.kind == GK_BFLY) {
      // real coefficients: packed FP32x2 on (re, im)
      const float2 cs = hi ? make_float2(o.uf[6], o.uf[6]) : make_float2(o.uf[0], o.uf[0]);
      const float2 cp = hi ? make_float2(o.uf[4], o.uf[4]) : make_float2(o.uf[2], o.uf[2]);
      const bool all = tok && st.smask == 0;
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const float2 p = make_float2(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (!all && (!tok || (j & (int)st.smask) != (int)st.smask)) continue;
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
    if (st.smask == 0) {
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const Cx<R> p = cx<R>(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (tok) v[j] = cmac2(cs, v[j], cp, p);
      }
    } else {
#pragma unroll
      for (int j = 0; j < (1 << RB); ++j) {
        const Cx<R> p = cx<R>(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
        if (tok && (j & (int)st.smask) == (int)st.smask) v[j] = cmac2(cs, v[j], cp, p);
      }
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    Cx<R> p = cx<R>(shx<R>(v[j].x, m), shx<R>(v[j].y, m));
    if (!tok || (j & (int)st.smask) != (int)st.smask) continue;
    Cx<R> a0 = hi ? p : v[j], a1 = hi ? v[j] : p;
    switch (st.kind) {
      case GK_HAD: {
        const R s = uscal<R>(o);
        v[j] = hi ? cx<R>((a0.x - a1.x) * s, (a0.y - a1.y) * s) : cx<R>((a0.x + a1.x) * s, (a0.y + a1.y) * s);
        break;
      }
      case GK_BFLY:
        v[j] = hi ? cx<R>(a0.x - a1.x, a0.y - a1.y) : cx<R>(a0.x + a1.x, a0.y + a1.y);
        break;
      case GK_ANTI:
        v[j] = hi ? cmul_code(a0, u10, st.c1) : cmul_code(a1, u01, st.c0);
        break;
      case GK_DIAG:
        v[j] = hi ? cmul_code(a1, u11, st.c1) : cmul_code(a0, u00, st.c0);
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
      v[2 * jj] = from_mem<R>(x);
      v[2 * jj + 1] = from_mem<R>(y);
    }
  }
}
// gx: the global offset of the relabelled local bits (never bit 0), XORed
// into each element's offset inside the tile
template <typename R, int RB>
__device__ __forceinline__ void store_tile(void* s, const Cx<R>* v, uint64_t base, const uint64_t* roff, uint64_t woff,
                                           uint64_t gx) {
  if constexpr (sizeof(R) == 4) {
    float4* s4 = (float4*)s;
#pragma unroll
    for (int jj = 0; jj < (1 << (RB - 1)); ++jj)
      s4[(base + ((woff + roff[jj]) ^ gx)) >> 1] =
          make_float4(v[2 * jj].x, v[2 * jj].y, v[2 * jj + 1].x, v[2 * jj + 1].y);
  } else {
    double2* s2 = (double2*)s;
#pragma unroll
    for (int jj = 0; jj < (1 << (RB - 1)); ++jj) {
      const uint64_t g = base + woff + roff[jj];
      s2[g] = to_mem<R>(v[2 * jj]);
      s2[g + 1] = to_mem<R>(v[2 * jj + 1]);
    }
  }
}

// Bytes of the shared-memory header of a tile pass (before the 16-byte
// aligned tile buffer): 2^RB uint64 global offsets and 2^(RB-1) uint32 local
// indices.
__host__ __device__ constexpr unsigned tile_smem_header(int RB) {
  return (unsigned)(((8u << RB) + (4u << (RB - 1)) + 15u) & ~15u);
}

// FEAT: which specialised complex64 paths the pass needs (bit 0: swaps, bit 1:
// Hadamard-shaped); passes without them run a smaller kernel.
constexpr int FEAT_SWAP = 1, FEAT_HAD = 2;   // FEAT_SWAP: lane exchanges; FEAT_HAD: real-matrix path (packed FP32x2)

// 16-byte global -> shared copies that bypass registers (LDGSTS), so the next
// tile's loads are in flight while the current tile is computed and stored.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// complex64 product-start helpers
__device__ __forceinline__ Cx<float> f2_bits(uint64_t u) {
  return cx<float>(__uint_as_float((unsigned)(u & 0xFFFFFFFFu)), __uint_as_float((unsigned)(u >> 32)));
}
__device__ __forceinline__ Cx<float> pf_at(const TileParams2& P, int q, int bit) { return f2_bits(P.pf[q][bit]); }
// complex128 product-start helpers (FP64)
__device__ __forceinline__ double2 pfd_at(const TileParams2& P, int q, int bit) {
  return make_double2(__longlong_as_double((long long)P.pfd[q][bit][0]),
                      __longlong_as_double((long long)P.pfd[q][bit][1]));
}
__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ Cx<float> cmul_f(Cx<float> a, Cx<float> b) {
  return cx<float>(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Each thread stages exactly the 16-byte chunks it will read back, so the
// stage buffer needs no barrier: the thread's own wait_group orders it.
// lreg[jj]: the local index of register 2 jj under the load map with the
// thread part 0 (tile-invariant, formed once per CTA), so a register's local
// index is tl | lreg[jj].
template <typename R, int RB>
__device__ __forceinline__ void stage_tile(const void* s, Cx<R>* st, uint64_t base, const uint64_t* roff, uint64_t woff,
                                           const uint32_t* lreg, uint32_t tl) {
#pragma unroll
  for (int jj = 0; jj < (1 << (RB - 1)); ++jj) {
    const uint32_t l = tl | lreg[jj];
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
__device__ __forceinline__ void unstage_tile(const Cx<R>* st, Cx<R>* v, const uint32_t* lreg, uint32_t tl) {
#pragma unroll
  for (int jj = 0; jj < (1 << (RB - 1)); ++jj) {
    const uint32_t l = tl | lreg[jj];
    if constexpr (sizeof(R) == 4) {
      const float4 x = ((const float4*)st)[l >> 1];
      v[2 * jj] = cx<float>(x.x, x.y);
      v[2 * jj + 1] = cx<float>(x.z, x.w);
    } else {   // the stage holds the FP64 pairs as they were in memory
      v[2 * jj] = from_mem<R>(((const double2*)st)[l]);
      v[2 * jj + 1] = from_mem<R>(((const double2*)st)[l + 1]);
    }
  }
}

// The body of a tile pass.  Prog gives the structure of op i (type, kind,
// slot, control masks, fold flag): read from the parameters at run time
// (ProgRT), or compile-time constants in a pass compiled at run time, where
// the op loop unrolls completely and every branch on the structure folds.
// The coefficients always come from P.ops[i].
template <typename R, int RB, int FEAT, class Prog>
__device__ __forceinline__ void tile_pass(void* __restrict__ s, const TileParams2& P) {
  extern __shared__ unsigned char smraw[];
  constexpr int NR = 1 << RB;
  // global offsets of the register part (pairs jj: slots 1..RB-1) at load /
  // store, and the local indices of the register part at load
  uint64_t* roff_in = (uint64_t*)smraw;
  uint64_t* roff_out = roff_in + NR / 2;
  uint32_t* lreg_in = (uint32_t*)(roff_out + NR / 2);
  // transpose buffer, 2^b elements; between the last transpose of a tile and
  // the start of the next it stages the next tile
  Cx<R>* xb = (Cx<R>*)(smraw + tile_smem_header(RB));
  Cx<R>* stg = xb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < NR / 2) {
    lreg_in[threadIdx.x] = lidx<RB>(P.init, 2 * threadIdx.x, 0);
    roff_in[threadIdx.x] = goff(lidx<RB>(P.init, 2 * threadIdx.x, 0), P.gpos, P.b);
    roff_out[threadIdx.x] = goff(lidx<RB>(P.fin, 2 * threadIdx.x, 0), P.gpos, P.b);
  }
  __syncthreads();
  const uint64_t woff_in = goff(thread_part(P.init, lane, warp), P.gpos, P.b);
  const uint64_t woff_out = goff(thread_part(P.fin, lane, warp), P.gpos, P.b);
  const uint32_t tl_in = thread_part(P.init, lane, warp);
  const uint64_t ntiles = 1ull << (P.N - P.b);
  Cx<R> v[NR];
  const bool load = !P.from_zero;
  // product start: the factor of this thread's lane and warp bits
  Cx<float> fthr = cx<float>(1.f, 0.f);
  double2 fthr_d = make_double2(1.0, 0.0);
  if (P.from_product) {
    for (int k = 1; k < P.b; ++k) {
      bool is_reg = false;
#pragma unroll
      for (int sl = 0; sl < RB; ++sl) is_reg |= (P.init.reg[sl] == k);
      if (is_reg) continue;
      const int q = k < 4 ? k : P.gpos[k];
      if constexpr (sizeof(R) == 4) fthr = cmul_f(fthr, pf_at(P, q, (tl_in >> k) & 1));
      else fthr_d = cmul_d(fthr_d, pfd_at(P, q, (tl_in >> k) & 1));
    }
  }
  // tile tau starts at base = deposit(tau) (its bits spread over the bits
  // outside the tile); the next tile of this CTA, tau + gridDim.x, starts at
  // deposit(tau) + deposit(gridDim.x) added in the deposited domain: the
  // gaps set to ones carry across them
  const uint64_t dstep = deposit_t(gridDim.x, P.out_mask);
  const uint64_t gaps = ~P.out_mask;
  uint64_t base = deposit_t(blockIdx.x, P.out_mask);
  if (load && blockIdx.x < ntiles) stage_tile<R, RB>(s, stg, base, roff_in, woff_in, lreg_in, tl_in);
  for (uint64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
    const uint64_t base_nxt = ((base | gaps) + dstep) & P.out_mask;
    if (load) {
      cp_async_wait_all();
      unstage_tile<R, RB>(stg, v, lreg_in, tl_in);
    } else if (P.from_product) {
      // product state: thread factor x the factors of the qubits outside the
      // tile x the register table
      if constexpr (sizeof(R) == 4) {
        Cx<float> f = fthr;
        for (uint64_t m = P.out_mask; m; m &= m - 1) {
          const int q = __ffsll((long long)m) - 1;
          f = cmul_f(f, pf_at(P, q, (int)((base >> q) & 1)));
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          const Cx<float> t = cmul_f(f, f2_bits(P.ptab[j]));
          v[j] = cx<R>((R)t.x, (R)t.y);
        }
      } else {
        double2 f = fthr_d;
        for (uint64_t m = P.out_mask; m; m &= m - 1) {
          const int q = __ffsll((long long)m) - 1;
          f = cmul_d(f, pfd_at(P, q, (int)((base >> q) & 1)));
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          const double2 t = cmul_d(f, make_double2(__longlong_as_double((long long)P.ptabd[j][0]),
                                                   __longlong_as_double((long long)P.ptabd[j][1])));
          v[j] = from_mem<R>(t);
        }
      }
    } else {
      // |0..0>: register 0 of thread 0 of the tile at base 0 is index 0
#pragma unroll
      for (int j = 0; j < NR; ++j) v[j] = cx<R>((R)0, (R)0);
      if (base == 0 && woff_in == 0) v[0] = cx<R>((R)1, (R)0);
    }
    const uint64_t nxt = tau + gridDim.x;
    if (load && P.last_xpose < 0 && nxt < ntiles)
      stage_tile<R, RB>(s, stg, base_nxt, roff_in, woff_in, lreg_in, tl_in);
    TMap cur = P.init;
    uint32_t tl = thread_part(cur, lane, warp);
    uint32_t xl = 0;   // relabelled local bits of this tile (the same in every lane of a warp)
    uint64_t gx = 0;   // their global offset (for the store)
    Cx<R> fac = cx<R>((R)1, (R)0);
    int mapi = 0;
    const int nops = Prog::kN >= 0 ? Prog::kN : P.nops;
#pragma unroll
    for (int i = 0; i < nops; ++i) {
      const TOp& o = P.ops[i];
      decltype(auto) st = Prog::s(P, i);
      // a compiled long pass may keep the CTA's warps within a few ops of each
      // other, so that they share the instruction lines they fetch
      if constexpr (Prog::kSync > 0)
        if (i > 0 && i % Prog::kSync == 0) __syncthreads();
      if (st.type == T_XPOSE) {
        // write every register at its local index, read back under the new map
#pragma unroll
        for (int jj = 0; jj < NR / 2; ++jj) {
          const uint32_t l = lidx<RB>(cur, 2 * jj, tl) ^ xl;   // the element's place in the tile
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
        xl = 0;
        gx = 0;
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
        if (load && i == P.last_xpose && nxt < ntiles)
          stage_tile<R, RB>(s, stg, base_nxt, roff_in, woff_in, lreg_in, tl_in);
        continue;
      }
      const bool gok = (base & st.gmask) == st.gmask;       // outer controls
      const bool tok = ((tl ^ xl) & st.tmask) == st.tmask;  // lane / warp controls
      if (st.pad[0] != 0) {
        // folded run of per-thread diagonals: multiply the factor, apply at the end
        if (gok && tok) {
          const bool one = (st.type == T_DIAG_THR) ? (((tl ^ xl) >> st.a) & 1) : ((base & st.gtbit) != 0);
          if ((one ? st.c1 : st.c0) != 0) fac = cmul_code(fac, ucx<R>(o, one ? 3 : 0), 4);
        }
        if (st.pad[0] == 2) {
          if (fac.x != (R)1 || fac.y != (R)0) {
#pragma unroll
            for (int j = 0; j < NR; ++j) v[j] = cmul_code(v[j], fac, 4);
          }
          fac = cx<R>((R)1, (R)0);
        }
        continue;
      }
      if (!gok) continue;
      switch (st.type) {
        case T_FLIP:   // gtbit: the global offset of local bit a
          if (tok) {
            xl ^= 1u << st.a;
            gx ^= st.gtbit;
          }
          break;
        case T_UNFLIP:
          // the exchange as the real matrix [[0, 1], [1, 0]] (the code shape of
          // the other real ops: plain register exchanges made the interpreter
          // spill)
          if ((xl >> st.pad[2]) & 1) {
            if constexpr (sizeof(R) == 4) {
              OpRealF f;
              f.u00 = f.u11 = make_float2(0.f, 0.f);
              f.u01 = f.u10 = make_float2(1.f, 1.f);
              reg_op<R, RB>(v, st.a, 0u, f);
            } else {
              OpAnti<R> f;
              f.f01 = f.f10 = cx<R>((R)1, (R)0);
              f.c0 = f.c1 = 0;
              reg_op<R, RB>(v, st.a, 0u, f);
            }
            xl ^= 1u << st.pad[2];
            gx ^= st.gtbit;
          }
          break;
        case T_REG: {
          if (!tok) break;
          if constexpr (sizeof(R) == 4) {
            // complex64: Hadamard-shaped or dense (exact for the unit entries
            // of X, Y, CNOT, TOFFOLI)
            // (a register-slot swap as renames makes the register allocation
            // spill at 128 registers; swaps on register slots stay dense)
            // X-type swaps (X, CNOT, TOFFOLI) take the packed real-matrix
            // path: as register exchanges they measured slower (renames under
            // per-tile conditions become moves, and the interpreter spilled
            // 2.6-3.2 KB; in compiled passes the renames doubled the time of
            // the bench circuit's passes)
            // (a relabelled target slot exchanges the roles of the pair's
            // two amplitudes: the matrix is taken as X U X)
            const bool pure_swap = st.kind == GK_ANTI && st.c0 == 0 && st.c1 == 0;
            const bool fl = st.pad[1] != 0 && ((xl >> st.pad[2]) & 1);
            if ((FEAT & FEAT_HAD) && Prog::kN >= 0 && st.kind == GK_BFLY) {
              if (st.pad[1] != 0) {
                OpBflyS f;
                f.s0 = fl ? make_float2(-1.f, -1.f) : make_float2(1.f, 1.f);
                f.s1 = fl ? make_float2(1.f, 1.f) : make_float2(-1.f, -1.f);
                reg_op<R, RB>(v, st.a, st.smask, f);
              } else {
                OpBflyF f;
                reg_op<R, RB>(v, st.a, st.smask, f);
              }
            } else if ((FEAT & FEAT_HAD) && Prog::kN < 0 && st.kind == GK_BFLY) {
              // the interpreter: in place, no register moves
              if (fl) {
                OpBflyIP<true> f;
                reg_op<R, RB>(v, st.a, st.smask, f);
              } else {
                OpBflyIP<false> f;
                reg_op<R, RB>(v, st.a, st.smask, f);
              }
            } else if ((FEAT & FEAT_HAD) && (st.kind == GK_REAL || st.kind == GK_BFLY || pure_swap)) {
              OpRealF f;
              const int k00 = fl ? 6 : 0, k01 = fl ? 4 : 2, k10 = fl ? 2 : 4, k11 = fl ? 0 : 6;
              f.u00 = make_float2(o.uf[k00], o.uf[k00]); f.u01 = make_float2(o.uf[k01], o.uf[k01]);
              f.u10 = make_float2(o.uf[k10], o.uf[k10]); f.u11 = make_float2(o.uf[k11], o.uf[k11]);
              reg_op<R, RB>(v, st.a, st.smask, f);
            } else {
              OpDense<R> f;
              f.u00 = ucx<R>(o, fl ? 3 : 0); f.u01 = ucx<R>(o, fl ? 2 : 1);
              f.u10 = ucx<R>(o, fl ? 1 : 2); f.u11 = ucx<R>(o, fl ? 0 : 3);
              reg_op<R, RB>(v, st.a, st.smask, f);
            }
          } else {
            // complex128: the FP64 pipe is the bound, so keep the cheaper forms
            switch (st.kind) {
              case GK_HAD: { OpHad<R> f; f.s = uscal<R>(o); reg_op<R, RB>(v, st.a, st.smask, f); break; }
              case GK_BFLY: { OpBfly<R> f; reg_op<R, RB>(v, st.a, st.smask, f); break; }
              case GK_ANTI: { OpAnti<R> f; f.f01 = ucx<R>(o, 1); f.f10 = ucx<R>(o, 2); f.c0 = st.c0; f.c1 = st.c1; reg_op<R, RB>(v, st.a, st.smask, f); break; }
              default: {
                OpDense<R> f; f.u00 = ucx<R>(o, 0); f.u01 = ucx<R>(o, 1); f.u10 = ucx<R>(o, 2); f.u11 = ucx<R>(o, 3);
                reg_op<R, RB>(v, st.a, st.smask, f);
              }
            }
          }
          break;
        }
        case T_LANE:
          lane_op<R, RB, (FEAT & FEAT_SWAP) != 0, (Prog::kN >= 0)>(v, st, o, lane, tok, xl);
          break;
        case T_DIAG_TAB: {
          // a run of register-slot diagonals multiplied out on the host
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            v[j] = cmul_code(v[j], tab_factor<R>(P, st.a, j), 4);
          }
          break;
        }
        case T_DIAG_REG:
        case T_DIAG_THR:
        case T_DIAG_OUT: {
          if (!tok) break;
          const Cx<R> d0 = ucx<R>(o, 0), d1 = ucx<R>(o, 3);
          if (st.type == T_DIAG_REG) {
            if constexpr (sizeof(R) == 4) {
              if (st.pad[1] != 0 && ((xl >> st.pad[2]) & 1))   // relabelled slot: the factors swap sides
                reg_diag_rt<R, RB>(v, st.a, st.smask, d1, d0, st.c1 == 0, st.c0 == 0);
              else
                reg_diag_rt<R, RB>(v, st.a, st.smask, d0, d1, st.c0 == 0, st.c1 == 0);
            } else {
              const int sl = st.a;
#pragma unroll
              for (int j = 0; j < NR; ++j) {
                if ((j & (int)st.smask) != (int)st.smask) continue;
                const bool one = (j >> sl) & 1;
                v[j] = one ? cmul_code(v[j], d1, st.c1) : cmul_code(v[j], d0, st.c0);
              }
            }
          } else {
            const bool one = (st.type == T_DIAG_THR) ? (((tl ^ xl) >> st.a) & 1) : ((base & st.gtbit) != 0);
            const int code = one ? st.c1 : st.c0;
            if (code == 0) break;
            const Cx<R> d = one ? d1 : d0;
            if (st.smask == 0) {
#pragma unroll
              for (int j = 0; j < NR; ++j) v[j] = cmul_code(v[j], d, sizeof(R) == 4 ? 4 : code);
            } else {
#pragma unroll
              for (int j = 0; j < NR; ++j)
                if ((j & (int)st.smask) == (int)st.smask) v[j] = cmul_code(v[j], d, sizeof(R) == 4 ? 4 : code);
            }
          }
          break;
        }
        default: break;
      }
    }
    store_tile<R, RB>(s, v, base, roff_out, woff_out, gx);
    base = base_nxt;
  }
}


// Op structure as compile-time constants (passes compiled at run time).
struct OpS {
  uint8_t type, kind, c0, c1, a;
  uint8_t pad[3];      // as TOp::pad
  uint32_t smask, tmask;
  uint64_t gmask, gtbit;
};

// Op structure read from the parameters (the interpreter).
struct ProgRT {
  static constexpr int kN = -1;
  static constexpr int kSync = 0;
  static __device__ __forceinline__ const TOp& s(const TileParams2& P, int i) { return P.ops[i]; }
};

}  // namespace qs_tile
