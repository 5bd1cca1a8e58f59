// Dense fused k-qubit gates (k = 3..5, the gate on the k lowest qubits of a
// complex64 state with N >= 12) on the fifth-generation tensor cores.
//
// The product is the one of the mma.sync kernel: with the k lowest qubits as
// the local index the state is a row-major matrix S (2^(N-k) rows of
// KR = 2^(k+1) floats) and the fused gate (Eq. (AQS0) for a k-qubit gate;
// the fusion proposed at the end of Sec. 5.2) is S <- S B, B the real block
// form of U^T, each operand split as x = hi + lo in TF32 and
// D = lo*hi + hi*lo + hi*hi ("3xTF32").
//
// Here the state streams through shared memory in stages of 2^12 amplitudes
// (32 KB, ROWS = 8192 / KR rows), one persistent CTA per SM:
//  - a bulk copy (cp.async.bulk, completion counted on an mbarrier) brings
//    stage i+1 into one of two raw buffers while stage i is processed;
//  - all threads split the raw stage into hi / lo TF32 planes in the
//    canonical K-major, no-swizzle operand layout: core matrices of 8 rows x
//    16 bytes, stored 128 bytes apart along the rows (SBO) and 2048 bytes
//    apart along K (LBO);
//  - one thread issues 24 tcgen05.mma (kind::tf32, M = 128, N = KR, K = 8):
//    for each 128-row sub-tile and each K step the products lo*hi, hi*lo,
//    hi*hi accumulate into columns [s*KR, s*KR + KR) of a 64-column tensor
//    memory allocation; tcgen05.commit arrives on an mbarrier;
//  - the warps read the accumulators back (tcgen05.ld 32x32b: lane = row),
//    write them into the consumed raw buffer (16-byte chunks XOR-swizzled per
//    row against bank conflicts) and store them, coalesced, where the stage
//    came from.  Stages are disjoint, so the update is in place.
// Every wait is bounded: one that runs out makes the CTA wait (again
// bounded) for the copies and products it has in flight, free its tensor
// memory and exit, and sets the error word the host reads.
#include "internal.cuh"
#include <vector>

namespace {

constexpr int TPB = 256;
constexpr int STAGE_FLOATS = 8192;             // 2^12 complex64 amplitudes
constexpr int STAGE_BYTES = STAGE_FLOATS * 4;  // 32 KB
constexpr int APLANE = STAGE_BYTES;            // one TF32 plane of a stage
constexpr int LBO_A = 2048;                    // 16 row groups x 128 B
constexpr int TMEM_COLS = 64;
constexpr uint32_t WAIT_SPINS = 1u << 20;      // about a second with the back-off below

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// generic-proxy writes of shared memory made visible to the async proxy
// (tensor cores, bulk copies)
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase of parity `parity` to complete; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < WAIT_SPINS; ++it) {
    if (mbar_test(bar, parity)) return true;
    if (it >= 64) __nanosleep(it < 4096 ? 64 : 1024);
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::tf32: F32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int n, int m) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Swizzle of the 16-byte chunk j of row r in the staging buffer (V chunks
// per row): 8 consecutive rows writing the same chunk hit 8 distinct bank
// groups.
template <int V>
__device__ __forceinline__ int swz(int r, int j) {
  return V >= 8 ? (j ^ (r & 7)) : (j ^ ((r >> 1) & 3));
}

template <int KR>
__global__ void __launch_bounds__(TPB, 1)
    k_fused_tc05(float* __restrict__ st, uint64_t nstages, const float* __restrict__ Bg, int* __restrict__ err) {
  constexpr int V = KR / 4;                  // 16-byte chunks per row
  constexpr int ROWS = STAGE_FLOATS / KR;    // rows per stage
  constexpr int S = ROWS / 128;              // 128-row sub-tiles per stage
  constexpr int BPLANE = 4 * KR * KR;        // one TF32 plane of B
  constexpr int LBO_B = (KR / 8) * 128;      // KR/8 column groups x 128 B
  constexpr int SUB_A = V * LBO_A;           // bytes of one 128-row sub-tile of A
  constexpr uint32_t IDESC = idesc_tf32(KR, 128);
  static_assert(S * KR == TMEM_COLS, "one stage fills the accumulator columns");
  static_assert(S * SUB_A == APLANE, "A plane layout");

  extern __shared__ __align__(128) unsigned char smraw[];
  const uint32_t raw_base = smem_u32(smraw);
  const uint32_t pad = (128u - (raw_base & 127u)) & 127u;
  unsigned char* sm = smraw + pad;
  const uint32_t sb = raw_base + pad;
  // layout: B hi | B lo | A hi | A lo | raw 0 | raw 1 | 3 mbarriers | tmem slot
  const uint32_t sBhi = sb, sBlo = sb + BPLANE, sAhi = sb + 2 * BPLANE, sAlo = sAhi + APLANE;
  const uint32_t sRaw = sAlo + APLANE;
  const uint32_t sBar = sRaw + 2 * STAGE_BYTES;          // full[0], full[1], mma
  unsigned char* pBhi = sm;
  unsigned char* pBlo = sm + BPLANE;
  unsigned char* pAhi = sm + 2 * BPLANE;
  unsigned char* pAlo = pAhi + APLANE;
  unsigned char* pRaw = pAlo + APLANE;
  uint32_t* tslot = (uint32_t*)(pRaw + 2 * STAGE_BYTES + 24);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(sBar, 1);
    mbar_init(sBar + 8, 1);
    mbar_init(sBar + 16, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  // B planes: element (row k, column n) of the KR x KR block matrix is the
  // K-major operand's (n, k)
  for (int i = tid; i < KR * KR; i += TPB) {
    const int kk = i / KR, n = i % KR;
    const float x = Bg[i];
    const uint32_t h = to_tf32(x), l = to_tf32(x - __uint_as_float(h));
    const int off = (kk >> 2) * LBO_B + (n >> 3) * 128 + (n & 7) * 16 + (kk & 3) * 4;
    *(uint32_t*)(pBhi + off) = h;
    *(uint32_t*)(pBlo + off) = l;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const uint64_t first = blockIdx.x, step = gridDim.x;
  // outstanding work, tracked by thread 0 for the bounded drain after a timeout
  uint32_t issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0, committed = 0, mma_waited = 0;
  if (tid == 0 && first < nstages) {
    mbar_expect_tx(sBar, STAGE_BYTES);
    bulk_g2s(sRaw, st + first * STAGE_FLOATS, STAGE_BYTES, sBar);
    issued0 = 1;
  }
  bool failed = false;
  uint32_t it = 0;
  for (uint64_t g = first; g < nstages; g += step, ++it) {
    const int b = it & 1;
    const uint32_t fullb = sBar + 8 * b;
    unsigned char* praw = pRaw + b * STAGE_BYTES;
    if (tid == 0 && g + step < nstages) {
      // the other raw buffer was last read (as staging) before the barrier
      // that closed the previous iteration
      fence_async_smem();
      mbar_expect_tx(sBar + 8 * (b ^ 1), STAGE_BYTES);
      bulk_g2s(sRaw + (b ^ 1) * STAGE_BYTES, st + (g + step) * STAGE_FLOATS, STAGE_BYTES, sBar + 8 * (b ^ 1));
      if (b) ++issued0; else ++issued1;
    }
    const bool ok_load = mbar_wait(fullb, (it >> 1) & 1);
    if (__syncthreads_or(!ok_load)) { failed = true; break; }
    if (tid == 0) { if (b) ++waited1; else ++waited0; }

    // split into TF32 hi / lo planes: a warp covers 8 rows x 4 chunks, the
    // chunk index rotated by the row so reads and writes spread over the banks
#pragma unroll 4
    for (int q = tid; q < ROWS * V; q += TPB) {
      const int rlo = q & 7, cq = (q >> 3) % V, oct = (q >> 3) / V;
      const int r = oct * 8 + rlo, c = (cq + rlo) & (V - 1);
      const float4 x = *(const float4*)(praw + r * (KR * 4) + c * 16);
      uint4 h, l;
      h.x = to_tf32(x.x); l.x = to_tf32(x.x - __uint_as_float(h.x));
      h.y = to_tf32(x.y); l.y = to_tf32(x.y - __uint_as_float(h.y));
      h.z = to_tf32(x.z); l.z = to_tf32(x.z - __uint_as_float(h.z));
      h.w = to_tf32(x.w); l.w = to_tf32(x.w - __uint_as_float(h.w));
      const int rr = r & 127;
      const int off = (r >> 7) * SUB_A + c * LBO_A + (rr >> 3) * 128 + (rr & 7) * 16;
      *(uint4*)(pAhi + off) = h;
      *(uint4*)(pAlo + off) = l;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const uint32_t d = tmem + s * KR;
#pragma unroll
        for (int ks = 0; ks < KR / 8; ++ks) {
          const uint32_t ao = s * SUB_A + 2 * ks * LBO_A, bo = 2 * ks * LBO_B;
          const uint64_t ahi = sdesc(sAhi + ao, LBO_A, 128), alo = sdesc(sAlo + ao, LBO_A, 128);
          const uint64_t bhi = sdesc(sBhi + bo, LBO_B, 128), blo = sdesc(sBlo + bo, LBO_B, 128);
          mma_tf32(d, alo, bhi, IDESC, ks > 0);
          mma_tf32(d, ahi, blo, IDESC, 1);
          mma_tf32(d, ahi, bhi, IDESC, 1);
        }
      }
      mma_commit(sBar + 16);
      ++committed;
    }
    const bool ok_mma = mbar_wait(sBar + 16, it & 1);
    if (__syncthreads_or(!ok_mma)) { failed = true; break; }
    if (tid == 0) ++mma_waited;
    tc_fence_after();

    // accumulators -> staging (the consumed raw buffer): warp w reads lanes
    // 32*(w%4).. and column chunks 2*(w/4), 2*(w/4)+1 (16 columns each)
    {
      const int q4 = warp & 3, half = warp >> 2;
      uint32_t v[2][16];
#pragma unroll
      for (int jc = 0; jc < 2; ++jc) {
        const int col0 = 16 * (2 * half + jc);
        tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + col0, v[jc]);
      }
      tmem_wait_ld();
#pragma unroll
      for (int jc = 0; jc < 2; ++jc) {
        const int col0 = 16 * (2 * half + jc);
        const int s = col0 / KR, cc = col0 % KR;
        const int r = s * 128 + 32 * q4 + lane;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int j = cc / 4 + t;
          *(uint4*)(praw + r * (KR * 4) + swz<V>(r, j) * 16) =
              make_uint4(v[jc][4 * t], v[jc][4 * t + 1], v[jc][4 * t + 2], v[jc][4 * t + 3]);
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    float* dst = st + g * STAGE_FLOATS;
#pragma unroll 4
    for (int q = tid; q < ROWS * V; q += TPB) {
      const int r = q / V, j = q % V;
      *(float4*)(dst + 4 * q) = *(const float4*)(praw + r * (KR * 4) + swz<V>(r, j) * 16);
    }
    __syncthreads();
  }

  if (failed) {
    if (tid == 0) {
      atomicExch(err, 1);
      if (issued0 > waited0) mbar_wait(sBar, (issued0 - 1) & 1);
      if (issued1 > waited1) mbar_wait(sBar + 8, (issued1 - 1) & 1);
      if (committed > mma_waited) mbar_wait(sBar + 16, (committed - 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
  }
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int KR>
constexpr size_t smem_bytes() {
  return (size_t)2 * 4 * KR * KR + 4 * (size_t)STAGE_BYTES + 32 + 128;
}

}  // namespace

bool fused_tc05_eligible(const qs_sim* s, const int* qubits, int k) {
  if (s->enc != QS_C64 || k < 3 || k > 5 || s->N < 12) return false;
  int mask = 0;
  for (int m = 0; m < k; ++m) mask |= 1 << qubits[m];
  return mask == (1 << k) - 1;
}

qs_status launch_fused_tc05(qs_sim* s, const int* qubits, int k, const double* U) {
  const int KR = 2 << k;
  std::vector<float> B((size_t)KR * KR);
  fused_block_matrix(qubits, k, U, B.data());
  const size_t bbytes = sizeof(float) * B.size();
  QS_TRY(ensure_scratch(s, bbytes + 256));
  int* err = (int*)((char*)s->scratch + bbytes);
  QS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s->stream));
  QS_CUDA(cudaMemcpyAsync(s->scratch, B.data(), bbytes, cudaMemcpyHostToDevice, s->stream));
  const uint64_t nstages = 1ull << (s->N - 12);
  const unsigned grid = (unsigned)(nstages < (uint64_t)s->num_sms ? nstages : (uint64_t)s->num_sms);
  float* st = (float*)s->state;
  const float* Bd = (const float*)s->scratch;
  auto go = [&](auto kern, size_t smem) -> qs_status {
    QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, TPB, smem, s->stream>>>(st, nstages, Bd, err);
    return QS_OK;
  };
  switch (k) {
    case 3: QS_TRY(go(k_fused_tc05<16>, smem_bytes<16>())); break;
    case 4: QS_TRY(go(k_fused_tc05<32>, smem_bytes<32>())); break;
    default: QS_TRY(go(k_fused_tc05<64>, smem_bytes<64>())); break;
  }
  QS_LAUNCH_CHECK();
  int herr = 0;
  QS_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  if (herr) {
    qs_set_error("apply_fused: a tensor-core wait ran out of time");
    return QS_ETIMEOUT;
  }
  return QS_OK;
}
