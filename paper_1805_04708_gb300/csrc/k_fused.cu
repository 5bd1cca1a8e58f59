// Dense k-qubit gates (1 <= k <= 5) on the dense encodings: every group of
// 2^k amplitudes that differ only in the qubits `qubits` is multiplied by the
// 2^k x 2^k matrix (Eq. (AQS0) for n-qubit gates; the fused multi-qubit gates
// proposed at the end of Sec. 5.2).  CUDA-core version: one thread per group,
// the group staged in shared memory, the matrix in shared memory.  complex128
// computes in double-float on the FP32 pipes unless the handle asks for the
// FP64 units (sim_set_fp64_emulation 0).
#include "internal.cuh"
#include "cplx.cuh"
#include <string.h>

namespace {

constexpr int TPB = 128;

struct FusedGeo {
  int N, k;
  int ins[5];        // qubits sorted ascending (zero bits inserted into the group index)
  int qpos[5];       // qubits in local-bit order: local bit m <-> qubits[m]
};

// an amplitude from memory in the arithmetic type R, and back
template <typename R> __device__ __forceinline__ Cx<R> ld_amp(float2 v) { return cx<R>(v.x, v.y); }
template <typename R> __device__ __forceinline__ Cx<R> ld_amp(double2 v) { return from_mem<R>(v); }
template <typename R> __device__ __forceinline__ void st_amp(float2* p, Cx<R> a) { *p = make_float2(a.x, a.y); }
template <typename R> __device__ __forceinline__ void st_amp(double2* p, Cx<R> a) { *p = to_mem<R>(a); }

template <typename R, typename A>
__global__ void __launch_bounds__(TPB) k_fused(A* __restrict__ s, FusedGeo g, const double* __restrict__ U) {
  extern __shared__ unsigned char smraw[];
  const int d = 1 << g.k;
  Cx<R>* M = (Cx<R>*)smraw;                       // d*d
  // this thread's group: element c at buf[c * TPB], so that the lanes of a
  // warp read neighbouring words (no bank conflicts)
  Cx<R>* buf = M + d * d + threadIdx.x;
  for (int i = threadIdx.x; i < d * d; i += TPB) M[i] = cx<R>(R(U[2 * i]), R(U[2 * i + 1]));
  __syncthreads();
  const uint64_t ngroups = 1ull << (g.N - g.k);
  const uint64_t grp = (uint64_t)blockIdx.x * TPB + threadIdx.x;
  if (grp >= ngroups) return;
  uint64_t base = grp;
  for (int m = 0; m < g.k; ++m) base = ins0(base, g.ins[m]);
  uint64_t lofs[32];
  for (int c = 0; c < d; ++c) {
    uint64_t o = 0;
    for (int m = 0; m < g.k; ++m) o |= (uint64_t)((c >> m) & 1) << g.qpos[m];
    lofs[c] = o;
  }
  for (int c = 0; c < d; ++c) buf[c * TPB] = ld_amp<R>(s[base | lofs[c]]);
  for (int r = 0; r < d; ++r) {
    R re = R(0), im = R(0);
    for (int c = 0; c < d; ++c) {
      Cx<R> u = M[r * d + c], a = buf[c * TPB];
      re = fma(u.x, a.x, re); re = fma(-u.y, a.y, re);
      im = fma(u.x, a.y, im); im = fma(u.y, a.x, im);
    }
    st_amp<R>(&s[base | lofs[r]], cx<R>(re, im));
  }
}

}  // namespace

qs_status launch_fused_dense(qs_sim* s, const int* qubits, int k, const double* U) {
  uint64_t qmask = 0;
  for (int m = 0; m < k; ++m) qmask |= 1ull << qubits[m];
  const bool low = qmask == (1ull << k) - 1;   // the qubits are 0..k-1
  if (s->enc == QS_C64 && s->fused_engine != QS_FUSED_CUDA_CORES) {
    if (s->fused_engine == QS_FUSED_AUTO && fused_tc05_eligible(s, qubits, k))
      return launch_fused_tc05(s, qubits, k, U);
    if (k >= 2 && s->N >= k + 4 && low) return launch_fused_tc(s, qubits, k, U);
  }
  FusedGeo g;
  g.N = s->N; g.k = k;
  for (int m = 0; m < k; ++m) { g.ins[m] = qubits[m]; g.qpos[m] = qubits[m]; }
  for (int i = 0; i < k; ++i)
    for (int j = i + 1; j < k; ++j)
      if (g.ins[j] < g.ins[i]) { int t = g.ins[i]; g.ins[i] = g.ins[j]; g.ins[j] = t; }
  const int d = 1 << k;
  QS_TRY(ensure_scratch(s, sizeof(double) * 2 * d * d));
  QS_CUDA(cudaMemcpyAsync(s->scratch, U, sizeof(double) * 2 * d * d, cudaMemcpyHostToDevice, s->stream));
  const uint64_t ng = 1ull << (s->N - k);
  const unsigned blocks = (unsigned)((ng + TPB - 1) / TPB);
  if (s->enc == QS_C128 && s->c128_df != 0) {
    size_t smem = sizeof(Cx<DF>) * (size_t)(d * d + TPB * d);
    QS_CUDA(cudaFuncSetAttribute(k_fused<DF, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fused<DF, double2><<<blocks, TPB, smem, s->stream>>>((double2*)s->state, g, (const double*)s->scratch);
  } else if (s->enc == QS_C128) {
    size_t smem = sizeof(Cx<double>) * (size_t)(d * d + TPB * d);
    QS_CUDA(cudaFuncSetAttribute(k_fused<double, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fused<double, double2><<<blocks, TPB, smem, s->stream>>>((double2*)s->state, g, (const double*)s->scratch);
  } else {
    size_t smem = sizeof(Cx<float>) * (size_t)(d * d + TPB * d);
    QS_CUDA(cudaFuncSetAttribute(k_fused<float, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fused<float, float2><<<blocks, TPB, smem, s->stream>>>((float2*)s->state, g, (const double*)s->scratch);
  }
  QS_LAUNCH_CHECK();
  // U is read from the host buffer by the async copy: wait before returning
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}
