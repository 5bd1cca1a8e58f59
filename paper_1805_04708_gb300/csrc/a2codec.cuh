// Device codec of the adaptive 2-byte encoding (Sec. 4.1), shared by the
// gate kernels (k_adapt2.cu) and the reductions (k_reduce.cu).
#pragma once
#include "internal.cuh"
#include "cplx.cuh"

struct Luts {
  float r[256];     // magnitude for b0 + 128
  float2 cs[256];   // (cos, sin)(pi b1 / 128) for b1 + 128: one 8-byte lookup
};

// Every thread of the block must call this (it synchronises).
static __device__ void build_luts(Luts& L, double r0, double r1) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    const int b = i - 128;
    float r;
    if (b == -128) r = 0.f;
    else if (b == 127) r = 1.f;
    else r = (float)((double)(b + 127) * (r1 - r0) / 253.0 + r0);
    L.r[i] = r;
    // theta = pi b / 128: the first quarter turn directly, the rest by exact
    // quarter turns (c, s) -> (-s, c), so opposite angles cancel exactly
    const int k = b & 63;
    const int turns = ((b - k) / 64) & 3;
    double sn, cs;
    sincospi((double)k / 128.0, &sn, &cs);
    for (int q = 0; q < turns; ++q) { const double t = cs; cs = -sn; sn = t; }
    L.cs[i] = make_float2((float)cs, (float)sn);
  }
  __syncthreads();
}

static __device__ __forceinline__ Cx<float> a2_dec(const Luts& L, unsigned int w) {
  const int b0 = (int)(w & 0xFFu) ^ 0x80;         // b0 + 128
  const int b1 = (int)((w >> 8) & 0xFFu) ^ 0x80;  // b1 + 128
  const float r = L.r[b0];
  const float2 t = L.cs[b1];
  return cx<float>(r * t.x, r * t.y);
}

