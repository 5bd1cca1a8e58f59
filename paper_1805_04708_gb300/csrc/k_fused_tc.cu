// Dense fused k-qubit gates on tensor cores (complex64 states, k = 2..5, the
// gate acting on the k lowest qubits).
//
// With the k lowest qubits as the local index, the state is a row-major
// matrix S of 2^(N-k) rows, each row the 2^k amplitudes of one group stored
// as 2^(k+1) interleaved floats (re, im).  The fused gate (Eq. (AQS0) for a
// k-qubit gate; the fusion proposed at the end of Sec. 5.2) maps every row s
// to U s, i.e. S <- S U^T; in real arithmetic S (rows x 2K') times the block
// matrix B (2K' x 2K', K' = 2^k) with
//   B[2l][2r] = Re U[r][l],  B[2l+1][2r] = -Im U[r][l],
//   B[2l][2r+1] = Im U[r][l], B[2l+1][2r+1] = Re U[r][l].
// The product runs on the tensor cores with mma.sync m16n8k8 in TF32; each
// FP32 operand is split as x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) and
// D = Ahi Bhi + Ahi Blo + Alo Bhi ("3xTF32"), which keeps the error near
// FP32 rounding.  Each warp owns 16 rows at a time, staged through shared
// memory so global loads and stores stay coalesced; rows are disjoint
// between warps, so the update is in place.
#include "internal.cuh"
#include <string.h>
#include <vector>

namespace {

constexpr int WARPS = 4;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// KR = 2^(k+1) real columns per row (8, 16, 32, 64).
template <int KR>
__global__ void __launch_bounds__(WARPS * 32) k_fused_tc(float* __restrict__ st, uint64_t nrows,
                                                          const float* __restrict__ Bg) {
  extern __shared__ __align__(16) unsigned char smraw[];
  // [k][n], tf32 bits; rows padded by 8 words so the fragment loads of a
  // warp (4 rows x 8 columns) fall in 32 distinct banks
  uint32_t(*Bhi)[KR + 8] = (uint32_t(*)[KR + 8])smraw;
  uint32_t(*Blo)[KR + 8] = Bhi + KR;
  float(*tile)[16][KR + 4] = (float(*)[16][KR + 4])(Blo + KR);
  for (int i = threadIdx.x; i < KR * KR; i += blockDim.x) {
    const float x = Bg[i];
    const uint32_t h = to_tf32(x);
    Bhi[i / KR][i % KR] = h;
    Blo[i / KR][i % KR] = to_tf32(x - __uint_as_float(h));
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3;
  float(*T)[KR + 4] = tile[w];
  const uint64_t ntiles = (nrows + 15) / 16;
  for (uint64_t t = (uint64_t)blockIdx.x * WARPS + w; t < ntiles; t += (uint64_t)gridDim.x * WARPS) {
    const uint64_t r0 = t * 16;
    const int rows = (int)((nrows - r0) < 16 ? (nrows - r0) : 16);
    // stage the 16 x KR tile (coalesced float4 loads)
    constexpr int V = KR / 4;  // float4 per row
    for (int i = lane; i < 16 * V; i += 32) {
      const int r = i / V, c = (i % V) * 4;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) x = *(const float4*)(st + (r0 + r) * KR + c);
      T[r][c] = x.x; T[r][c + 1] = x.y; T[r][c + 2] = x.z; T[r][c + 3] = x.w;
    }
    __syncwarp();
    // A fragments for every k-step, split into hi and lo
    uint32_t ahi[KR / 8][4], alo[KR / 8][4];
#pragma unroll
    for (int ks = 0; ks < KR / 8; ++ks) {
      const float v[4] = {T[gid][ks * 8 + tig], T[gid + 8][ks * 8 + tig], T[gid][ks * 8 + tig + 4],
                          T[gid + 8][ks * 8 + tig + 4]};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ahi[ks][j] = to_tf32(v[j]);
        alo[ks][j] = to_tf32(v[j] - __uint_as_float(ahi[ks][j]));
      }
    }
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < KR / 8; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < KR / 8; ++ks) {
        const uint32_t bh[2] = {Bhi[ks * 8 + tig][nt * 8 + gid], Bhi[ks * 8 + tig + 4][nt * 8 + gid]};
        const uint32_t bl[2] = {Blo[ks * 8 + tig][nt * 8 + gid], Blo[ks * 8 + tig + 4][nt * 8 + gid]};
        mma_tf32(d, alo[ks], bh);
        mma_tf32(d, ahi[ks], bl);
        mma_tf32(d, ahi[ks], bh);
      }
      T[gid][nt * 8 + 2 * tig] = d[0];
      T[gid][nt * 8 + 2 * tig + 1] = d[1];
      T[gid + 8][nt * 8 + 2 * tig] = d[2];
      T[gid + 8][nt * 8 + 2 * tig + 1] = d[3];
    }
    __syncwarp();
    for (int i = lane; i < 16 * V; i += 32) {
      const int r = i / V, c = (i % V) * 4;
      if (r < rows) *(float4*)(st + (r0 + r) * KR + c) = make_float4(T[r][c], T[r][c + 1], T[r][c + 2], T[r][c + 3]);
    }
    __syncwarp();
  }
}

}  // namespace

// U: 2^k x 2^k complex, row-major (re, im), local bit m of the index = qubit
// qubits[m]; qubits is a permutation of 0..k-1.  B: KR x KR floats
// (KR = 2^(k+1)), row-major, the real block form of U^T in natural qubit
// order (natural index bit m <-> qubit m).
void fused_block_matrix(const int* qubits, int k, const double* U, float* B) {
  const int K = 1 << k, KR = 2 * K;
  auto to_api = [&](int nat) {
    int a = 0;
    for (int m = 0; m < k; ++m)
      if ((nat >> qubits[m]) & 1) a |= 1 << m;
    return a;
  };
  for (int r = 0; r < K; ++r)
    for (int l = 0; l < K; ++l) {
      const int ar = to_api(r), al = to_api(l);
      const double ur = U[2 * (ar * K + al)], ui = U[2 * (ar * K + al) + 1];
      B[(size_t)(2 * l) * KR + 2 * r] = (float)ur;
      B[(size_t)(2 * l + 1) * KR + 2 * r] = (float)-ui;
      B[(size_t)(2 * l) * KR + 2 * r + 1] = (float)ui;
      B[(size_t)(2 * l + 1) * KR + 2 * r + 1] = (float)ur;
    }
}

qs_status launch_fused_tc(qs_sim* s, const int* qubits, int k, const double* U) {
  const int KR = 2 << k;
  std::vector<float> B((size_t)KR * KR);
  fused_block_matrix(qubits, k, U, B.data());
  QS_TRY(ensure_scratch(s, sizeof(float) * B.size()));
  QS_CUDA(cudaMemcpyAsync(s->scratch, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice, s->stream));
  const uint64_t nrows = 1ull << (s->N - k);
  const uint64_t ntiles = (nrows + 15) / 16;
  const uint64_t gmax = (uint64_t)s->num_sms * 8;
  const uint64_t need = (ntiles + WARPS - 1) / WARPS;
  const unsigned grid = (unsigned)(need < gmax ? need : gmax);
  float* st = (float*)s->state;
  const float* Bd = (const float*)s->scratch;
  const size_t smem = (size_t)2 * KR * (KR + 8) * 4 + (size_t)WARPS * 16 * (KR + 4) * 4;
  auto go = [&](auto kern) -> qs_status {
    QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, WARPS * 32, smem, s->stream>>>(st, nrows, Bd);
    return QS_OK;
  };
  switch (k) {
    case 2: QS_TRY(go(k_fused_tc<8>)); break;
    case 3: QS_TRY(go(k_fused_tc<16>)); break;
    case 4: QS_TRY(go(k_fused_tc<32>)); break;
    default: QS_TRY(go(k_fused_tc<64>)); break;
  }
  QS_LAUNCH_CHECK();
  QS_CUDA(cudaStreamSynchronize(s->stream));   // B is read from a host vector by the async copy
  return QS_OK;
}
