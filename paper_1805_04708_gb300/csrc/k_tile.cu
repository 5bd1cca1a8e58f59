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
#include "tile_core.cuh"
#include "tile_jit.h"
#include <string.h>
#include <stdlib.h>
#include <vector>

using namespace qs_tile;

namespace {

template <typename R, int RB, int FEAT>
__global__ void __launch_bounds__(TPB, 2) k_tile2(void* __restrict__ s, const __grid_constant__ TileParams2 P) {
  tile_pass<R, RB, FEAT, ProgRT>(s, P);
}

}  // namespace

// ---------------------------------------------------------------------------------
// planner
// ---------------------------------------------------------------------------------
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
// target and the same controls, both diagonal or both not, are multiplied
// into one 2x2 (FP64, host).
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
  // compose neighbours with equal (target, controls), both diagonal or both
  // not: a diagonal times a real or Hadamard-shaped gate is a general complex
  // matrix, dearer than the two (the diagonal folds or costs one multiply)
  int m = 0;
  for (int i = 0; i < n; ++i) {
    if (m > 0 && out[m - 1].target == out[i].target && same_controls(out[m - 1], out[i]) &&
        is_diag_gate(out[m - 1]) == is_diag_gate(out[i])) {
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
// Relabelled swaps (complex64 passes).  A pure swap (X, CNOT, TOFFOLI) whose
// controls lie outside the register slots and the lanes exchanges the two
// halves of its target bit wherever the controls hold, and the same in every
// lane of a warp: the pass then records the bit as relabelled (T_FLIP, a
// per-thread XOR mask on the local index) instead of moving data.  Later ops
// that meet a relabelled bit: an op on that register slot swaps the roles of
// its pair (flag pad[1]; pad[2] holds the slot's local bit), lane ops and
// conditions read the mask, a transpose writes every element to its own
// place (and clears the mask), the store XORs the bits' global offset into
// the address; an op that needs a register slot in place (a control on it, a
// factor table) first exchanges it back (T_UNFLIP), and so does slot 0
// (inside a 16-byte access) before a transpose and before the store.
// Returns false when the inserted ops do not fit (the pass keeps its ops).
static bool relabel_swaps(TileParams2* P, int nops, int RB, int* nops_out) {
  static thread_local TOp out[MAX_TOPS];
  int m = 0;
  TMap cur = P->init;
  int mi = 0;
  uint32_t M = 0;                    // local bits that may be relabelled
  const uint32_t lane_bits = 0x3Eu;  // local bits 1..5
  bool any = false, fits = true;
  auto gbit = [&](int lb) { return 1ull << (lb < LOW_BITS ? lb : P->gpos[lb]); };
  auto push = [&](const TOp& o) {
    if (m >= MAX_TOPS) { fits = false; return; }
    out[m++] = o;
  };
  auto unflip = [&](int slot) {
    TOp u;
    memset(&u, 0, sizeof u);
    u.type = T_UNFLIP;
    u.a = (uint8_t)slot;
    u.pad[2] = cur.reg[slot];
    u.gtbit = gbit(cur.reg[slot]);
    M &= ~(1u << cur.reg[slot]);
    push(u);
  };
  for (int i = 0; i < nops && fits; ++i) {
    TOp o = P->ops[i];
    const bool swap = (o.type == T_REG || o.type == T_LANE) && o.kind == GK_ANTI && o.c0 == 0 && o.c1 == 0 &&
                      o.smask == 0 && (o.tmask & lane_bits) == 0 && o.pad[0] == 0;
    if (swap) {
      const int lb = o.type == T_REG ? cur.reg[o.a] : o.a + 1;
      o.type = T_FLIP;
      o.a = (uint8_t)lb;
      o.gtbit = gbit(lb);
      M |= 1u << lb;
      any = true;
      push(o);
      continue;
    }
    if (o.type == T_XPOSE) {
      if (M & 1u) unflip(0);
      push(o);
      cur = P->maps[mi++];
      M = 0;
      continue;
    }
    for (int sl = 0; sl < RB; ++sl) {
      const bool needed = (o.type == T_DIAG_TAB) || ((o.smask >> sl) & 1u);
      if (needed && ((M >> cur.reg[sl]) & 1u)) unflip(sl);
    }
    if (o.type == T_REG || o.type == T_DIAG_REG) {
      o.pad[2] = cur.reg[o.a];
      if ((M >> cur.reg[o.a]) & 1u) o.pad[1] = 1;
    }
    push(o);
  }
  if (fits && (M & 1u)) unflip(0);
  if (!fits || !any) return false;
  for (int i = 0; i < m; ++i) P->ops[i] = out[i];
  *nops_out = m;
  return true;
}

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
    // (X, CNOT, TOFFOLI: those only exchange values)
    const bool real = (g.u[1] == 0.0 && g.u[3] == 0.0 && g.u[5] == 0.0 && g.u[7] == 0.0);
    const bool pure_swap = (gc.kind == GK_ANTI && gc.c0 == 0 && gc.c1 == 0);
    if (real_kinds && real && !diag && !pure_swap && (o.type == T_REG || o.type == T_LANE)) o.kind = GK_REAL;
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
  // runs of register-slot diagonals without lane, warp or outer controls
  // become one multiplication by a table of per-register factors, the
  // products formed in FP64 on the host (a control on a register slot gives
  // factor 1 to the registers where it is 0)
  const int NRj = 1 << RB;
  static thread_local double tabd[MAX_TABS][32][2];
  int ntab = 0;
  {
    int m = 0;
    auto tabbable = [&](int k) {
      const TOp& o = P->ops[k];
      return o.type == T_DIAG_REG && o.tmask == 0 && o.gmask == 0;
    };
    for (int i = 0; i < nops;) {
      int j = i;
      while (j < nops && tabbable(j)) ++j;
      if (j - i >= 2 && ntab < MAX_TABS) {
        double tr[32], ti[32];
        for (int r = 0; r < NRj; ++r) { tr[r] = 1.0; ti[r] = 0.0; }
        for (int k = i; k < j; ++k) {
          const TOp& o = P->ops[k];
          for (int r = 0; r < NRj; ++r) {
            if ((r & (int)o.smask) != (int)o.smask) continue;
            const int bit = (r >> o.a) & 1;
            const double dr = o.ud[bit ? 6 : 0], di = o.ud[bit ? 7 : 1];
            const double xr = tr[r] * dr - ti[r] * di, xi = tr[r] * di + ti[r] * dr;
            tr[r] = xr; ti[r] = xi;
          }
        }
        for (int r = 0; r < NRj; ++r) { tabd[ntab][r][0] = tr[r]; tabd[ntab][r][1] = ti[r]; }
        TOp t;
        memset(&t, 0, sizeof t);
        t.type = T_DIAG_TAB;
        t.a = (uint8_t)ntab++;
        P->ops[m++] = t;
        i = j;
      } else if (j > i) {
        for (int k = i; k < j; ++k) P->ops[m++] = P->ops[k];
        i = j;
      } else {
        P->ops[m++] = P->ops[i++];
      }
    }
    nops = m;
  }
  // uncontrolled ops of the form s [[1, 1], [1, -1]] (Hadamards) become
  // unscaled butterflies (coefficients [[1, 1], [1, -1]]); the product of
  // their scales, a scalar that commutes with every op, goes into the first
  // factor table of the pass, else into an uncontrolled real or dense op,
  // else stays with one of the Hadamards
  {
    auto unc = [&](const TOp& o) {
      return (o.type == T_REG || o.type == T_LANE) && o.smask == 0 && o.tmask == 0 && o.gmask == 0;
    };
    auto had_scale = [&](const TOp& o) -> double {
      const double* u = o.ud;
      if (o.kind != (real_kinds ? GK_REAL : GK_HAD) || u[1] != 0.0 || u[3] != 0.0 || u[5] != 0.0 || u[7] != 0.0)
        return 0.0;
      if (!(u[0] > 0.0) || u[2] != u[0] || u[4] != u[0] || u[6] != -u[0]) return 0.0;
      return u[0];
    };
    int nh = 0, first_h = -1, carrier = -1;
    for (int i = 0; i < nops; ++i) {
      const TOp& o = P->ops[i];
      if (!unc(o)) continue;
      if (had_scale(o) > 0.0) {
        if (first_h < 0) first_h = i;
        ++nh;
      } else if (carrier < 0 && (o.kind == GK_REAL || o.kind == GK_DENSE)) {
        carrier = i;
      }
    }
    if (nh >= 2 || (nh == 1 && (ntab > 0 || carrier >= 0))) {
      double scale = 1.0;
      const double bf[8] = {1, 0, 1, 0, 1, 0, -1, 0};
      for (int i = 0; i < nops; ++i) {
        TOp& o = P->ops[i];
        if (!unc(o)) continue;
        const double sc = had_scale(o);
        if (sc > 0.0) {
          scale *= sc;
          o.kind = GK_BFLY;
          fill_u(o, bf);
        }
      }
      if (ntab > 0) {
        for (int r = 0; r < NRj; ++r) { tabd[0][r][0] *= scale; tabd[0][r][1] *= scale; }
      } else {
        if (carrier < 0) {   // one of the Hadamards keeps the whole scale
          carrier = first_h;
          P->ops[carrier].kind = real_kinds ? GK_REAL : GK_HAD;
        }
        TOp& c = P->ops[carrier];
        double u[8];
        for (int k = 0; k < 8; ++k) u[k] = c.ud[k] * scale;
        fill_u(c, u);
      }
    }
  }
  // the factor tables in the state's precision
  for (int t = 0; t < ntab; ++t)
    for (int r = 0; r < NRj; ++r) {
      if (real_kinds) {
        const float fr = (float)tabd[t][r][0], fi = (float)tabd[t][r][1];
        uint32_t br, bi;
        memcpy(&br, &fr, 4); memcpy(&bi, &fi, 4);
        P->tab[t][r] = (uint64_t)br | ((uint64_t)bi << 32);
      } else {
        memcpy(&P->tab[t][2 * r], &tabd[t][r][0], 8);
        memcpy(&P->tab[t][2 * r + 1], &tabd[t][r][1], 8);
      }
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
  if (real_kinds) relabel_swaps(P, nops, RB, &nops);
  P->nops = nops;
  P->fin = cur;
  P->last_xpose = -1;
  for (int i = 0; i < nops; ++i)
    if (P->ops[i].type == T_XPOSE) P->last_xpose = i;
  return true;
}

int tile_register_bits(qs_encoding enc) { return enc == QS_C128 ? 4 : 5; }
int tile_bits(qs_encoding enc) { return tile_register_bits(enc) + LANE_BITS + WARP_BITS; }

// Where planned passes go: launched on a handle's stream (interpreter or
// compiled kernel), or only compiled (no device work).
struct PassSink {
  qs_sim* s;            // null: compile only
  int N;
  qs_encoding enc;
  int jit;              // 0: interpreter; 1: per pass structure, the fastest of
                        // the interpreter and the compiled variants (timed
                        // online); 2: compiled, no barriers (complex64)
  PassTimer* timer;
  int emitted;
  std::vector<JitJob>* collect;   // compile only: the kernels to compile
  std::vector<int>* plan;         // plan only: gate indices in run order
  std::vector<int>* plan_start;   // plan only: first index of each pass
  const double (*prod)[2][2];     // a run from a pending |0..0>: the
                                  // product start f[q][bit] = (re, im), or null
};

// Product start.  From |0..0>, a single-qubit gate that comes before every
// multi-qubit gate on its qubit acts on an unentangled qubit: it commutes
// with every earlier gate of other qubits, so these gates can all run first,
// and together they make the product state prod_q (U_q |0>)_(bit q), U_q the
// product of qubit q's gates in order.  Returns their number; f[q][bit] gets
// (U_q |0>)(bit) (FP64), rest the other gates in order.
static int product_prefix(int N, const qs_gate* g, int n, double (*f)[2][2], std::vector<qs_gate>* rest) {
  for (int q = 0; q < N; ++q) {
    f[q][0][0] = 1.0; f[q][0][1] = 0.0;
    f[q][1][0] = 0.0; f[q][1][1] = 0.0;
  }
  rest->clear();
  uint64_t entangled = 0;
  int np = 0;
  for (int i = 0; i < n; ++i) {
    const qs_gate& x = g[i];
    if (x.nc == 0 && !((entangled >> x.target) & 1)) {
      double* v = &f[x.target][0][0];   // v[0..1] = f(0), v[2..3] = f(1)
      const double* u = x.u;            // u00, u01, u10, u11
      const double a0r = v[0], a0i = v[1], a1r = v[2], a1i = v[3];
      v[0] = u[0] * a0r - u[1] * a0i + u[2] * a1r - u[3] * a1i;
      v[1] = u[0] * a0i + u[1] * a0r + u[2] * a1i + u[3] * a1r;
      v[2] = u[4] * a0r - u[5] * a0i + u[6] * a1r - u[7] * a1i;
      v[3] = u[4] * a0i + u[5] * a0r + u[6] * a1i + u[7] * a1r;
      ++np;
      continue;
    }
    entangled |= 1ull << x.target;
    for (int c = 0; c < x.nc; ++c) entangled |= 1ull << x.controls[c];
    rest->push_back(x);
  }
  return np;
}

int product_start_factors(int N, const qs_gate* gates, int n, double* factors) {
  static thread_local double f[64][2][2];
  std::vector<qs_gate> rest;
  const int np = product_prefix(N, gates, n, f, &rest);
  if (factors)
    for (int q = 0; q < N; ++q)
      for (int bit = 0; bit < 2; ++bit) {
        factors[4 * q + 2 * bit] = f[q][bit][0];
        factors[4 * q + 2 * bit + 1] = f[q][bit][1];
      }
  return np;
}

static uint64_t f2_bits_host(double re, double im) {
  const float fr = (float)re, fi = (float)im;
  uint32_t br, bi;
  memcpy(&br, &fr, 4);
  memcpy(&bi, &fi, 4);
  return (uint64_t)br | ((uint64_t)bi << 32);
}

// The product start of a pass: per-qubit factors and the register table of
// the load map (products in FP64, rounded once for complex64; kept in FP64,
// pfd and ptabd, for complex128).
static void fill_product(TileParams2& P, const double (*f)[2][2], int RB, bool fp64) {
  P.from_product = 1;
  for (int q = 0; q < P.N; ++q)
    for (int bit = 0; bit < 2; ++bit) {
      P.pf[q][bit] = f2_bits_host(f[q][bit][0], f[q][bit][1]);
      if (fp64) {
        memcpy(&P.pfd[q][bit][0], &f[q][bit][0], 8);
        memcpy(&P.pfd[q][bit][1], &f[q][bit][1], 8);
      }
    }
  for (int j = 0; j < (1 << RB); ++j) {
    double tr = 1.0, ti = 0.0;
    for (int sl = 0; sl < RB; ++sl) {
      const int l = P.init.reg[sl];
      const int q = l < LOW_BITS ? l : P.gpos[l];
      const double* c = f[q][(j >> sl) & 1];
      const double r = tr * c[0] - ti * c[1];
      ti = tr * c[1] + ti * c[0];
      tr = r;
    }
    P.ptab[j] = f2_bits_host(tr, ti);
    if (fp64 && j < 16) {
      memcpy(&P.ptabd[j][0], &tr, 8);
      memcpy(&P.ptabd[j][1], &ti, 8);
    }
  }
}

static qs_status emit_pass(PassSink& k, const TileParams2& P);

// Pass packing.  Each pass takes gates in circuit order while the union of
// their non-diagonal targets fits the tile; a gate that does not fit is left
// for a later pass, and so is every later gate that does not commute with a
// gate left out.  Two gates commute when every qubit they share is one on
// which both act diagonally (a control, or the target of a diagonal gate):
// both are then block-diagonal on the shared qubits and act on disjoint
// qubits inside each block.  Every gate a pass takes therefore commutes with
// all the earlier gates it overtakes, and the product equals the circuit's.
// A pass whose op list overflows is split.  Complex128 passes move gates
// ahead the same way: in double-float arithmetic (the default) the N = 30
// circuit takes 1.02 s against 1.06 s in circuit order; on the FP64 units
// fuller passes turn more per-tile constants into per-element work (1.17 s
// against 1.11 s in order).
static qs_status run_pass(PassSink& k, const qs_gate* gates, const int* gidx, int ng, uint64_t tile);

static qs_status plan_tile_passes(PassSink& k, const qs_gate* gates, int n) {
  const int b = tile_bits(k.enc);
  const int N = k.N;
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
  const int max_targets = LOW_BITS + 2 + (tile_register_bits(k.enc) - 1);
  // tile of a pass: its targets, padded to b bits with qubits the pass does
  // not touch at all (diagonal gates and controls on qubits outside the tile
  // are per-tile constants, a diagonal folds into one factor; inside it they
  // cost per-element work)
  auto tile_of = [&](const std::vector<int>& g) {
    uint64_t S = low, used = 0;
    for (int i : g) { S |= xq[i]; used |= xq[i] | zq[i]; }
    uint64_t tile = S;
    for (int q = 0; q < N && __builtin_popcountll(tile) < b; ++q)
      if (!((used >> q) & 1)) tile |= 1ull << q;
    for (int q = 0; q < N && __builtin_popcountll(tile) < b; ++q) tile |= 1ull << q;
    return tile;
  };
  auto targets_of = [&](const std::vector<int>& g) {
    uint64_t S = low;
    for (int i : g) S |= xq[i];
    return S;
  };
  std::vector<std::vector<int>> passes;
  qs_status st = QS_OK;
  while (nrem > 0 && st == QS_OK) {
    uint64_t S = low, bx = 0, bz = 0;
    int ng = 0, nleft = 0;
    const bool reorder = k.enc == QS_C64 || k.enc == QS_C128;
    for (int j = 0; j < nrem; ++j) {
      const int i = rem[j];
      const bool blocked = (xq[i] & (bx | bz)) != 0 || ((xq[i] | zq[i]) & bx) != 0 || (!reorder && (bx | bz) != 0);
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
    passes.emplace_back(gidx, gidx + ng);
  }
  // A last pass of a few gates costs a whole sweep; when its targets and the
  // previous pass's fit the tile, the previous pass takes its gates after
  // its own (the same order) and reaches the extra targets through the warp
  // bits by shared-memory transposes (about a third of a sweep each).
  const size_t np = passes.size();
  if (k.enc == QS_C64 && np >= 2 && passes[np - 1].size() <= 4 &&
      passes[np - 2].size() + passes[np - 1].size() <= MAX_TOPS / 2 &&
      __builtin_popcountll(targets_of(passes[np - 2]) | targets_of(passes[np - 1])) <= b) {
    passes[np - 2].insert(passes[np - 2].end(), passes[np - 1].begin(), passes[np - 1].end());
    passes.pop_back();
  }
  for (size_t p = 0; p < passes.size() && st == QS_OK; ++p)
    st = run_pass(k, gates, passes[p].data(), (int)passes[p].size(), tile_of(passes[p]));
  free(gidx); free(rem); free(xq); free(zq);
  return st;
}

// A circuit that is all product start still needs one pass to write it.
static qs_status run_empty_pass(PassSink& k) {
  const int b = tile_bits(k.enc);
  return run_pass(k, nullptr, nullptr, 0, (1ull << b) - 1);
}

qs_status run_tile_passes(qs_sim* s, const qs_gate* gates, int n, int* n_passes, PassTimer* timer, int jit) {
  PassSink k = {s, s->N, s->enc, 0, timer, 0, nullptr, nullptr, nullptr, nullptr};
  if (s->enc == QS_C64 && jit != 0) {
    if (!tile_jit_available()) {
      qs_set_error("circuit_run: compiled tile passes need NVRTC, which could not be loaded");
      return QS_EUNSUPPORTED;
    }
    k.jit = jit;
  }
  qs_status st;
  static thread_local double prod[64][2][2];
  static thread_local std::vector<qs_gate> rest;
  if ((s->enc == QS_C64 || s->enc == QS_C128) && s->zero_pending && s->product_start &&
      product_prefix(s->N, gates, n, prod, &rest) > 0) {
    k.prod = prod;
    // the gates after the prefix may all be identities, which the planner
    // drops: the product state is still written by one pass
    st = rest.empty() ? QS_OK : plan_tile_passes(k, rest.data(), (int)rest.size());
    if (st == QS_OK && k.emitted == 0) st = run_empty_pass(k);
  } else {
    st = plan_tile_passes(k, gates, n);
  }
  if (n_passes) *n_passes = k.emitted;
  return st;
}

qs_status compile_tile_passes(int N, const qs_gate* gates, int n, int* n_passes, bool all_passes) {
  std::vector<JitJob> passes;
  PassSink k = {nullptr, N, QS_C64, all_passes ? 2 : 1, nullptr, 0, &passes, nullptr, nullptr, nullptr};
  QS_TRY(plan_tile_passes(k, gates, n));
  if (n_passes) *n_passes = k.emitted;
  // the passes of a run from a pending |0..0> (the gates after the product start)
  std::vector<qs_gate> rest;
  static thread_local double prod[64][2][2];
  if (product_prefix(N, gates, n, prod, &rest) > 0) {
    PassSink kz = {nullptr, N, QS_C64, all_passes ? 2 : 1, nullptr, 0, &passes, nullptr, nullptr, nullptr};
    if (!rest.empty()) QS_TRY(plan_tile_passes(kz, rest.data(), (int)rest.size()));
    if (kz.emitted == 0) QS_TRY(run_empty_pass(kz));
  }
  return tile_jit_compile_all(passes);
}

qs_status plan_tile_pass_order(int N, qs_encoding enc, const qs_gate* gates, int n, int* order, int* pass_start,
                               int* n_passes) {
  std::vector<int> plan, start;
  PassSink k = {nullptr, N, enc, 0, nullptr, 0, nullptr, &plan, &start, nullptr};
  QS_TRY(plan_tile_passes(k, gates, n));
  for (size_t i = 0; i < plan.size(); ++i) order[i] = plan[i];
  for (size_t i = 0; i < start.size(); ++i) pass_start[i] = start[i];
  *n_passes = (int)start.size();
  return QS_OK;
}

static qs_status launch_pass(PassSink& k, const TileParams2& P) {
  qs_sim* s = k.s;
  // kernel of this launch: interpreter (cand 0) or a compiled variant
  int cand = 0;
  cudaEvent_t tune_end = nullptr;
  if (s->enc == QS_C64 && k.jit == 2) cand = 1;
  if (s->enc == QS_C64 && k.jit == 1) {
    for (;;) {
      QS_TRY(tile_tune_pick(s, P, &cand, &tune_end));
      // a variant that fails to compile is never picked again
      if (cand == 0 || tile_jit_compile(P, kTileCandSync[cand]) == QS_OK) break;
      tile_tune_fail(P, cand);
      if (tune_end) QS_CUDA(cudaEventRecord(tune_end, s->stream));
      tune_end = nullptr;
    }
  }
  PassTimer* timer = k.timer;
  const bool timed = timer && timer->n < timer->max_ev;
  if (timed) QS_CUDA(cudaEventRecord(timer->ev[2 * timer->n], s->stream));
  const uint64_t ntiles = 1ull << (s->N - P.b);
  const uint64_t gmax = (uint64_t)s->num_sms * 2;   // two persistent CTAs per SM
  const unsigned grid = (unsigned)(ntiles < gmax ? ntiles : gmax);
  if (s->enc == QS_C128) {
    const size_t smem = ((size_t)16 << P.b) + tile_smem_header(4);
    // double-float arithmetic on the FP32 pipes, except for passes that only
    // move amplitudes or multiply them by +-1, +-i: those stay exact in FP64
    // (double-float holds 48 significant bits)
    bool moves = true;
    for (int i = 0; i < P.nops && moves; ++i) {
      const TOp& o = P.ops[i];
      if (o.type == T_XPOSE) continue;
      if (o.type == T_DIAG_TAB) { moves = false; break; }
      moves = (o.kind == GK_ANTI || o.kind == GK_DIAG) && o.c0 < 4 && o.c1 < 4;
    }
    if (s->c128_df == 1 && !moves) {
      // the coefficients and factor tables as packed (hi, lo) float pairs
      static thread_local TileParams2 PD;
      PD = P;
      auto pack = [](double x) {
        const float hi = (float)x, lo = (float)(x - (double)hi);
        uint32_t bh, bl;
        memcpy(&bh, &hi, 4);
        memcpy(&bl, &lo, 4);
        const uint64_t w = (uint64_t)bh | ((uint64_t)bl << 32);
        double d;
        memcpy(&d, &w, 8);
        return d;
      };
      for (int i = 0; i < PD.nops; ++i)
        for (int k = 0; k < 8; ++k) PD.ops[i].ud[k] = pack(P.ops[i].ud[k]);
      for (int t = 0; t < MAX_TABS; ++t)
        for (int j = 0; j < 32; ++j) {
          double x;
          memcpy(&x, &P.tab[t][j], 8);
          const double w = pack(x);
          memcpy(&PD.tab[t][j], &w, 8);
        }
      QS_CUDA(cudaFuncSetAttribute(k_tile2<DF, 4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_tile2<DF, 4, 0><<<grid, TPB, smem, s->stream>>>(s->state, PD);
    } else {
      QS_CUDA(cudaFuncSetAttribute(k_tile2<double, 4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_tile2<double, 4, 0><<<grid, TPB, smem, s->stream>>>(s->state, P);
    }
  } else if (cand > 0) {
    const size_t smem = ((size_t)8 << P.b) + tile_smem_header(5);
    QS_TRY(tile_jit_launch(s, P, kTileCandSync[cand], grid, smem));
  } else {
    int feat = 0;
    for (int i = 0; i < P.nops; ++i) {
      const TOp& o = P.ops[i];
      const bool swap = o.kind == GK_ANTI && o.c0 == 0 && o.c1 == 0;
      if (o.type == T_LANE && swap) feat |= FEAT_SWAP;
      if ((o.type == T_REG && swap) || ((o.type == T_REG || o.type == T_LANE) && (o.kind == GK_REAL || o.kind == GK_BFLY)))
        feat |= FEAT_HAD;
    }
    const size_t smem = ((size_t)8 << P.b) + tile_smem_header(5);
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
  if (tune_end) QS_CUDA(cudaEventRecord(tune_end, s->stream));
  if (timed) {
    QS_CUDA(cudaEventRecord(timer->ev[2 * timer->n + 1], s->stream));
    timer->n++;
  } else if (timer) {
    timer->n++;
  }
  return QS_OK;
}

static qs_status emit_pass(PassSink& k, const TileParams2& P) {
  ++k.emitted;
  if (!k.s) {
    if (k.jit == 2) {
      k.collect->push_back(JitJob{P, 0});
    } else {
      for (int c = 1; c < kTileCands; ++c) k.collect->push_back(JitJob{P, kTileCandSync[c]});
    }
    return QS_OK;
  }
  return launch_pass(k, P);
}

static qs_status run_pass(PassSink& k, const qs_gate* gates, const int* gidx, int ng, uint64_t tile) {
  static thread_local TileParams2 P;
  const int b = tile_bits(k.enc);
  if (k.plan) {   // plan only: the pass's gates in the order it takes them
    k.plan_start->push_back((int)k.plan->size());
    for (int j = 0; j < ng; ++j) k.plan->push_back(gidx[j]);
    ++k.emitted;
    return QS_OK;
  }
  if (build_pass(gates, gidx, ng, k.N, b, tile_register_bits(k.enc), tile, &P, k.enc == QS_C64)) {
    // a pending |0..0> (or the product start) is made by the first pass
    // instead of being loaded
    P.from_zero = (k.s && k.s->zero_pending) ? 1 : 0;
    P.from_product = 0;
    if (P.from_zero && k.prod) fill_product(P, k.prod, tile_register_bits(k.enc), k.enc == QS_C128);
    QS_TRY(emit_pass(k, P));
    if (P.from_zero) k.s->zero_pending = false;
    return QS_OK;
  }
  // too many ops for one launch: split the gate run in halves (same tile)
  const int h = ng / 2;
  QS_TRY(run_pass(k, gates, gidx, h, tile));
  return run_pass(k, gates, gidx + h, ng - h, tile);
}
