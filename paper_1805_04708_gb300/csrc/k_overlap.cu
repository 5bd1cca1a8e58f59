// Overlap of two states held by two handles (any encodings, same N):
// <a|b> = sum_i conj(a_i) b_i and ||a - b||^2 = sum_i |a_i - b_i|^2, in FP64
// with a fixed grid and a fixed-order sum of the partials (deterministic).
// One read of each state.  Used to report how far the adaptive 2-byte
// encoding (Sec. 4.1) stays from the FP64 state of the same circuit (the
// paper compares its two simulators the same way, Tables 4-6), and as the
// fidelity of any two states.
#include "internal.cuh"
#include "cplx.cuh"
#include "a2codec.cuh"

namespace {

constexpr int TPB = 256;

template <typename A> struct Amp;
template <> struct Amp<double2> {
  static __device__ __forceinline__ double2 at(const void* s, uint64_t i, const Luts&) {
    return ((const double2*)s)[i];
  }
};
template <> struct Amp<float2> {
  static __device__ __forceinline__ double2 at(const void* s, uint64_t i, const Luts&) {
    const float2 a = ((const float2*)s)[i];
    return make_double2(a.x, a.y);
  }
};
template <> struct Amp<uint16_t> {
  static __device__ __forceinline__ double2 at(const void* s, uint64_t i, const Luts& L) {
    const Cx<float> z = a2_dec(L, ((const uint16_t*)s)[i]);
    return make_double2(z.x, z.y);
  }
};

template <typename A, typename B>
__global__ void __launch_bounds__(TPB) k_overlap(const void* __restrict__ sa, const A2Dev* da,
                                                 const void* __restrict__ sb, const A2Dev* db, uint64_t n,
                                                 double* __restrict__ part) {
  __shared__ Luts La, Lb;
  if (da) build_luts(La, da->r0, da->r1);
  if (db) build_luts(Lb, db->r0, db->r1);
  double re = 0.0, im = 0.0, d2 = 0.0;
  for (uint64_t i = (uint64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB) {
    const double2 a = Amp<A>::at(sa, i, La), b = Amp<B>::at(sb, i, Lb);
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
    const double dx = a.x - b.x, dy = a.y - b.y;
    d2 = fma(dx, dx, fma(dy, dy, d2));
  }
  __shared__ double sh[3][TPB];
  sh[0][threadIdx.x] = re;
  sh[1][threadIdx.x] = im;
  sh[2][threadIdx.x] = d2;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[(uint64_t)threadIdx.x * gridDim.x + blockIdx.x] = sh[threadIdx.x][0];
}

template <typename A>
static qs_status launch_b(qs_sim* a, qs_sim* b, unsigned grid, double* part) {
  const uint64_t n = 1ull << a->N;
  const A2Dev* da = (const A2Dev*)a->a2dev;
  const A2Dev* db = (const A2Dev*)b->a2dev;
  if (b->enc == QS_C128) k_overlap<A, double2><<<grid, TPB, 0, a->stream>>>(a->state, da, b->state, db, n, part);
  else if (b->enc == QS_C64) k_overlap<A, float2><<<grid, TPB, 0, a->stream>>>(a->state, da, b->state, db, n, part);
  else k_overlap<A, uint16_t><<<grid, TPB, 0, a->stream>>>(a->state, da, b->state, db, n, part);
  QS_LAUNCH_CHECK();
  return QS_OK;
}

}  // namespace

extern "C" qs_status sim_overlap(qs_sim* a, qs_sim* b, double* ov, double* dist2) {
  if (!a || !b || !ov || !dist2) { qs_set_error("sim_overlap: null argument"); return QS_EINVAL; }
  if (a->N != b->N) { qs_set_error("sim_overlap: the states have %d and %d qubits", a->N, b->N); return QS_EINVAL; }
  if (a->device != b->device) { qs_set_error("sim_overlap: the states live on different devices"); return QS_EINVAL; }
  QS_TRY(materialize_state(a));
  QS_TRY(materialize_state(b));
  // b's pending work before a's stream reads it
  if (b->stream != a->stream) {
    cudaEvent_t ev;
    QS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    QS_CUDA(cudaEventRecord(ev, b->stream));
    QS_CUDA(cudaStreamWaitEvent(a->stream, ev, 0));
    QS_CUDA(cudaEventDestroy(ev));
  }
  const uint64_t n = 1ull << a->N;
  const uint64_t want = (n + TPB - 1) / TPB;
  const unsigned grid = (unsigned)(want < (uint64_t)a->num_sms * 8 ? want : (uint64_t)a->num_sms * 8);
  QS_TRY(ensure_scratch(a, (size_t)(3 * grid + 3) * sizeof(double)));
  double* part = (double*)a->scratch;
  if (a->enc == QS_C128) QS_TRY(launch_b<double2>(a, b, grid, part));
  else if (a->enc == QS_C64) QS_TRY(launch_b<float2>(a, b, grid, part));
  else QS_TRY(launch_b<uint16_t>(a, b, grid, part));
  for (int c = 0; c < 3; ++c) QS_TRY(sum_partials(a, part + (size_t)c * grid, (int)grid, part + 3 * grid + c));
  double h[3];
  QS_CUDA(cudaMemcpyAsync(h, part + 3 * grid, sizeof h, cudaMemcpyDeviceToHost, a->stream));
  QS_CUDA(cudaStreamSynchronize(a->stream));
  ov[0] = h[0];
  ov[1] = h[1];
  *dist2 = h[2];
  return QS_OK;
}
