// Gate records and the shared-memory gate loop used by the batched and the
// serving kernels: the pair update of Eq. (NUM2) with a general controlled
// 2x2, on a state held in shared memory.
#pragma once
#include "internal.cuh"
#include "cplx.cuh"

template <typename R> struct BGate {
  int32_t nc, c0, c1, t;
  R u[8];
};

template <typename R>
__device__ __forceinline__ void apply_gate_range(Cx<R>* st, int N, const BGate<R>& g, int tid, int nthr) {
  const uint32_t cm = (g.nc > 0 ? (1u << g.c0) : 0u) | (g.nc > 1 ? (1u << g.c1) : 0u);
  const Cx<R> u00 = cx<R>(g.u[0], g.u[1]), u01 = cx<R>(g.u[2], g.u[3]);
  const Cx<R> u10 = cx<R>(g.u[4], g.u[5]), u11 = cx<R>(g.u[6], g.u[7]);
  const int np = 1 << (N - 1);
  for (int p = tid; p < np; p += nthr) {
    const uint32_t i0 = (uint32_t)ins0((uint64_t)p, g.t), i1 = i0 | (1u << g.t);
    if ((i0 & cm) != cm) continue;
    const Cx<R> a0 = st[i0], a1 = st[i1];
    st[i0] = cmac2(u00, a0, u01, a1);
    st[i1] = cmac2(u10, a0, u11, a1);
  }
}

