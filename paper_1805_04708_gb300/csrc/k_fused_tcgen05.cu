// Dense fused k-qubit gates (k = 3..5 on any qubits of a complex64 state
// with N >= 12) on the fifth-generation tensor cores.
//
// The product is the one of the mma.sync kernel: with the k lowest qubits as
// the local index the state is a row-major matrix S (2^(N-k) rows of
// KR = 2^(k+1) floats) and the fused gate (Eq. (AQS0) for a k-qubit gate;
// the fusion proposed at the end of Sec. 5.2) is S <- S B, B the real block
// form of U^T, each operand split as x = hi + lo in TF32 and
// D = lo*hi + hi*lo + hi*hi ("3xTF32").
//
// One persistent CTA per SM streams "stages" of 2^12 amplitudes (32 KB,
// 8192 / KR rows) through a ring of NBH stage buffers (plus a ring of NBL
// planes for the lo parts), with warp-specialised roles connected by
// mbarriers:
//  - producer (one thread): TMA tensor loads (cp.async.bulk.tensor, 128- or
//    64-byte swizzle) of boxes of 128 rows x 128 (or 64) bytes, which land
//    in the canonical K-major swizzled operand layout;
//  - converters (4 warps): split each element into the TF32 hi part (in
//    place) and the lo part (into a lo plane);
//  - MMA issuer (one thread): per 128-row sub-tile and K step of 8, the
//    three tcgen05.mma (kind::tf32, M = 128, N = KR) into one of two
//    64-column accumulators in tensor memory; tcgen05.commit signals the
//    epilogue;
//  - epilogue (4 warps, one per TMEM lane quarter): tcgen05.ld of the
//    accumulators, written back into the stage buffer in the same swizzled
//    layout, then TMA tensor stores to where the stage came from; the
//    buffer goes back to the producer once the store has read it.
// Stages are disjoint, so the update is in place.
//
// Gates on other qubits (the gather variant): a stage is every amplitude
// whose index varies only in the gate's qubits S and in the 12 - k lowest
// index bits outside S (the set L), so it holds 2^(12-k) whole groups.  Those
// 12 bits start with a contiguous run of at least 2^(12-k) amplitudes from
// bit 0, so the producer warp loads the stage with at most 32 untiled bulk
// copies of whole runs (cp.async.bulk, >= 1 KB each) in index order; the
// converters read each row (group) out of that order into registers, and
// after a barrier write its hi and lo parts in the swizzled operand layout;
// the epilogue stores the results from registers straight to their
// addresses (runs of 2^(lowest qubit of S) amplitudes across a warp), and the
// stage buffer goes back to the producer as soon as the products are done.
// Every wait is bounded; a
// wait that runs out raises a CTA-wide abort flag, every role leaves its
// loop, the producer and the MMA issuer wait (bounded) for what they still
// have in flight, the tensor memory is freed and the error word is set.
#include "internal.cuh"
#include "tma.cuh"
#include <vector>
#include <string.h>

namespace {

using namespace qs_tma;

constexpr int NWARPS = 10;          // producer, MMA, 4 converters, 4 epilogue
constexpr int TPB = NWARPS * 32;
constexpr int STAGE_FLOATS = 8192;  // 2^12 complex64 amplitudes
constexpr int STAGE_BYTES = STAGE_FLOATS * 4;
constexpr int NBH = 4;              // stage buffers (data, then hi part, then result)
constexpr int NBL = 2;              // lo planes
constexpr int TMEM_COLS = 128;      // two 64-column accumulators
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major swizzled operand: start
// address, stride between 8-row groups (SBO) in 16-byte units, descriptor
// version 1 (bits 46-47), layout type at bits 61-63 (2 = 128-byte swizzle,
// 4 = 64-byte swizzle).  The leading offset is unused by swizzled K-major
// layouts whose K step stays inside one swizzle row; it is set to 1.
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t addr, uint32_t sbo, uint64_t layout) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46) |
         (layout << 61);
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


// Geometry of one stage for KR floats per row.
template <int KR>
struct Geo {
  static constexpr int BOXW = KR >= 32 ? 32 : 16;   // floats per box row
  static constexpr int ROWB = BOXW * 4;             // bytes per box row = swizzle span
  static constexpr int BOXB = 128 * ROWB;           // bytes per box (128 rows)
  static constexpr int QX = KR / BOXW;              // boxes across a row
  static constexpr int S = 64 / KR;                 // 128-row sub-tiles per stage
  static constexpr int Q = S * QX;                  // boxes per stage
  static constexpr int SBO = 8 * ROWB;              // stride of 8-row groups
  static constexpr uint64_t LAYOUT = KR >= 32 ? 2 : 4;
  static constexpr int BPLANE = 4 * KR * KR;        // one TF32 plane of B
  static_assert(Q * BOXB == STAGE_BYTES, "stage = boxes");
  static_assert(S * KR == 64, "one stage fills one accumulator");
};

// Swizzled position of the 16-byte chunk j of row r inside a box: the chunk
// index XOR address bits 7.. (128-byte rows: r mod 8; 64-byte rows:
// (r / 2) mod 4), as written by the TMA swizzle modes.
template <int ROWB>
__device__ __forceinline__ int swz(int r, int j) {
  return ROWB == 128 ? (j ^ (r & 7)) : (j ^ ((r >> 1) & 3));
}

// Index geometry of the gather variant.
struct GatherGeo {
  float2* st;         // the state
  uint64_t nons;      // index bits outside the gate's qubits
  uint64_t smask;     // the gate's qubits S
  uint64_t lmask;     // L: the 12 - k lowest bits of nons
  uint64_t vmask;     // S | L, the 12 bits one stage spans
  int run_log;        // a stage is 2^(12 - run_log) runs of 2^run_log amplitudes
};
// x's bits, lowest first, placed at the set bits of mask (and the inverse)
__device__ __forceinline__ uint64_t dep_bits(uint64_t x, uint64_t mask) {
  uint64_t r = 0;
  for (uint64_t m = mask; m && x; m &= m - 1, x >>= 1)
    if (x & 1) r |= m & (~m + 1);
  return r;
}
__device__ __forceinline__ uint64_t ext_bits(uint64_t x, uint64_t mask) {
  uint64_t r = 0;
  int i = 0;
  for (uint64_t m = mask; m; m &= m - 1, ++i)
    if (x & m & (~m + 1)) r |= 1ull << i;
  return r;
}

template <int KR, bool GATHER>
__global__ void __launch_bounds__(TPB, 1)
    k_fused_tc05(const __grid_constant__ CUtensorMap tmap, GatherGeo gg, uint64_t nstages,
                 const float* __restrict__ Bg, int* __restrict__ err, uint32_t spins) {
  using G = Geo<KR>;
  constexpr int K = KR / 2;                           // amplitudes per group
  constexpr int LOGK = KR == 16 ? 3 : (KR == 32 ? 4 : 5);
  constexpr int KH = K / 8;                           // column c = 8 a + m: tables per a and per m
  constexpr uint32_t IDESC = idesc_tf32(KR, 128);
  extern __shared__ __align__(1024) unsigned char smraw[];
  const uint32_t base0 = smem_u32(smraw);
  const uint32_t pad = (1024u - (base0 & 1023u)) & 1023u;
  unsigned char* sm = smraw + pad;
  const uint32_t sb = base0 + pad;
  // layout: B hi | B lo | NBH stage buffers | NBL lo planes | mbarriers |
  // tmem slot, abort flag
  const uint32_t sBhi = sb, sBlo = sb + G::BPLANE, sA = sb + 2 * G::BPLANE;
  const uint32_t sLo = sA + NBH * STAGE_BYTES;
  const uint32_t sBar = sLo + NBL * STAGE_BYTES;
  auto FULL = [&](int b) { return sBar + 8 * b; };                  // stage landed
  auto EMPTY = [&](int b) { return sBar + 8 * (NBH + b); };         // buffer free
  auto MMAD = [&](int b) { return sBar + 8 * (2 * NBH + b); };      // products done
  auto CONV = [&](int l) { return sBar + 8 * (3 * NBH + l); };      // split done
  auto LOFREE = [&](int l) { return sBar + 8 * (3 * NBH + NBL + l); };   // lo plane read
  auto TFREE = [&](int t) { return sBar + 8 * (3 * NBH + 2 * NBL + t); };  // accumulator read
  uint32_t* tslot = (uint32_t*)(sm + (sBar - sb) + 8 * (3 * NBH + 2 * NBL + 2));
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < NBH; ++b) {
      mbar_init(FULL(b), 1);
      mbar_init(EMPTY(b), 1);
      mbar_init(MMAD(b), 1);
    }
    for (int l = 0; l < NBL; ++l) {
      mbar_init(CONV(l), 4);
      mbar_init(LOFREE(l), 1);
    }
    mbar_init(TFREE(0), 4);
    mbar_init(TFREE(1), 4);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  // B planes: element (row k, column n) of the KR x KR block matrix is the
  // K-major operand's (n, k), stored in the swizzled layout of the A boxes
  for (int i = tid; i < KR * KR; i += TPB) {
    const int kk = i / KR, n = i % KR;
    const float x = Bg[i];
    const uint32_t h = to_tf32(x), l = to_tf32(x - __uint_as_float(h));
    const int hb = kk / G::BOXW, kc = kk % G::BOXW;
    const int off = hb * (KR * G::ROWB) + n * G::ROWB + swz<G::ROWB>(n, kc >> 2) * 16 + (kc & 3) * 4;
    *(uint32_t*)(sm + off) = h;
    *(uint32_t*)(sm + G::BPLANE + off) = l;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t nloc =
      nstages > blockIdx.x ? (uint32_t)((nstages - 1 - blockIdx.x) / gridDim.x + 1) : 0u;   // stages of this CTA

  if (GATHER && warp == 0) {
    // ---- producer (gather): one bulk copy per run, lanes in parallel ----
    const int nruns = 1 << (12 - gg.run_log);
    const uint32_t run_bytes = 8u << gg.run_log;
    uint32_t n_issued = 0;
    for (uint32_t i = 0; i < nloc; ++i) {
      const int b = i % NBH;
      int ok = 1;
      if (lane == 0) {
        ok = mbar_wait_or_abort(EMPTY(b), ((i / NBH) & 1) ^ 1, abort_flag, spins);
        if (ok) mbar_expect_tx(FULL(b), STAGE_BYTES);
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      const uint64_t g = blockIdx.x + (uint64_t)i * gridDim.x;
      const uint64_t base = dep_bits(g << (12 - LOGK), gg.nons);
      if (lane < nruns)
        bulk_load(sA + b * STAGE_BYTES + lane * run_bytes,
                  gg.st + base + dep_bits((uint64_t)lane << gg.run_log, gg.vmask), run_bytes, FULL(b));
      ++n_issued;
    }
    if (lane == 0 && *abort_flag)
      for (uint32_t i = (n_issued > NBH ? n_issued - NBH : 0); i < n_issued; ++i)
        mbar_wait(FULL(i % NBH), (i / NBH) & 1);
    __syncwarp();
  } else if (warp == 0) {
    // ---- producer ----
    if (lane == 0) {
      uint32_t n_issued = 0;
      for (uint32_t i = 0; i < nloc; ++i) {
        const int b = i % NBH;
        if (!mbar_wait_or_abort(EMPTY(b), ((i / NBH) & 1) ^ 1, abort_flag, spins)) break;
        const uint64_t g = blockIdx.x + (uint64_t)i * gridDim.x;
        const uint32_t hi = sA + b * STAGE_BYTES;
        mbar_expect_tx(FULL(b), STAGE_BYTES);
#pragma unroll
        for (int q = 0; q < G::Q; ++q)
          tma_load_3d(hi + q * G::BOXB, &tmap, (q % G::QX) * G::BOXW, 0, (int)(g * G::S + q / G::QX), FULL(b));
        ++n_issued;
      }
      if (*abort_flag)
        for (uint32_t i = (n_issued > NBH ? n_issued - NBH : 0); i < n_issued; ++i)
          mbar_wait(FULL(i % NBH), (i / NBH) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      uint32_t n_commit = 0;
      for (uint32_t i = 0; i < nloc; ++i) {
        const int b = i % NBH, l = i % NBL, t = i & 1;
        if (!mbar_wait_or_abort(CONV(l), (i / NBL) & 1, abort_flag, spins)) break;
        if (!mbar_wait_or_abort(TFREE(t), ((i >> 1) & 1) ^ 1, abort_flag, spins)) break;
        tc_fence_after();
        const uint32_t ahi = sA + b * STAGE_BYTES, alo = sLo + l * STAGE_BYTES;
#pragma unroll
        for (int s = 0; s < G::S; ++s) {
          const uint32_t d = tmem + t * 64 + s * KR;
#pragma unroll
          for (int ks = 0; ks < KR / 8; ++ks) {
            const int k0 = 8 * ks, hb = k0 / G::BOXW, wb = (k0 % G::BOXW) * 4;
            const uint32_t ao = (s * G::QX + hb) * G::BOXB + wb, bo = hb * (KR * G::ROWB) + wb;
            const uint64_t dah = sdesc_sw(ahi + ao, G::SBO, G::LAYOUT), dal = sdesc_sw(alo + ao, G::SBO, G::LAYOUT);
            const uint64_t dbh = sdesc_sw(sBhi + bo, G::SBO, G::LAYOUT), dbl = sdesc_sw(sBlo + bo, G::SBO, G::LAYOUT);
            mma_tf32(d, dal, dbh, IDESC, ks > 0);
            mma_tf32(d, dah, dbl, IDESC, 1);
            mma_tf32(d, dah, dbh, IDESC, 1);
          }
        }
        mma_commit(MMAD(b));
        mma_commit(LOFREE(l));
        ++n_commit;
      }
      if (*abort_flag && n_commit) mbar_wait(MMAD((n_commit - 1) % NBH), ((n_commit - 1) / NBH) & 1);
    }
    __syncwarp();
  } else if (GATHER && warp < 6) {
    // ---- converters (gather): rows out of index order -> hi (same buffer) + lo ----
    const int ct = tid - 64;                       // the row of every sub-tile this thread converts
    // stage positions (bytes) of row ct of each sub-tile and of column
    // c = 8 a + m (the parts add: they come from disjoint index bits)
    uint32_t rpos[G::S], cph[KH], cpl[8];
#pragma unroll
    for (int sub = 0; sub < G::S; ++sub)
      rpos[sub] = 8u * (uint32_t)ext_bits(dep_bits((uint64_t)(sub * 128 + ct), gg.lmask), gg.vmask);
#pragma unroll
    for (int a = 0; a < KH; ++a) cph[a] = 8u * (uint32_t)ext_bits(dep_bits((uint64_t)(8 * a), gg.smask), gg.vmask);
#pragma unroll
    for (int m = 0; m < 8; ++m) cpl[m] = 8u * (uint32_t)ext_bits(dep_bits((uint64_t)m, gg.smask), gg.vmask);
    for (uint32_t i = 0; i < nloc; ++i) {
      const int b = i % NBH, l = i % NBL;
      bool ok = mbar_wait_or_abort(FULL(b), (i / NBH) & 1, abort_flag, spins);
      ok = ok && mbar_wait_or_abort(LOFREE(l), ((i / NBL) & 1) ^ 1, abort_flag, spins);
      if (!bar_and(2, 128, ok)) break;
      unsigned char* hi = sm + (sA - sb) + b * STAGE_BYTES;
      unsigned char* lo = sm + (sLo - sb) + l * STAGE_BYTES;
      float2 x[G::S][K];
#pragma unroll
      for (int sub = 0; sub < G::S; ++sub)
#pragma unroll
        for (int a = 0; a < KH; ++a) {
          const unsigned char* rb = hi + rpos[sub] + cph[a];
#pragma unroll
          for (int m = 0; m < 8; ++m) x[sub][8 * a + m] = *(const float2*)(rb + cpl[m]);
        }
      bar_sync(3, 128);                            // the whole stage is in registers
#pragma unroll
      for (int sub = 0; sub < G::S; ++sub)
#pragma unroll
        for (int j = 0; j < KR / 4; ++j) {
          const int col = 4 * j, hb = col / G::BOXW, jj = (col % G::BOXW) / 4;
          const int off = (sub * G::QX + hb) * G::BOXB + ct * G::ROWB + swz<G::ROWB>(ct, jj) * 16;
          const float v[4] = {x[sub][2 * j].x, x[sub][2 * j].y, x[sub][2 * j + 1].x, x[sub][2 * j + 1].y};
          uint32_t h[4], w[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            h[e] = to_tf32(v[e]);
            w[e] = to_tf32(v[e] - __uint_as_float(h[e]));
          }
          *(uint4*)(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
          *(uint4*)(lo + off) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(CONV(l));
    }
  } else if (warp < 6) {
    // ---- converters: x -> hi (in place) + lo ----
    const int ct = tid - 64;
    for (uint32_t i = 0; i < nloc; ++i) {
      const int b = i % NBH, l = i % NBL;
      bool ok = mbar_wait_or_abort(FULL(b), (i / NBH) & 1, abort_flag, spins);
      ok = ok && mbar_wait_or_abort(LOFREE(l), ((i / NBL) & 1) ^ 1, abort_flag, spins);
      if (!__all_sync(0xffffffffu, ok)) break;
      unsigned char* hi = sm + (sA - sb) + b * STAGE_BYTES;
      unsigned char* lo = sm + (sLo - sb) + l * STAGE_BYTES;
#pragma unroll 4
      for (int q = ct; q < STAGE_BYTES / 16; q += 128) {
        const float4 x = *(const float4*)(hi + 16 * q);
        uint4 h, l;
        h.x = to_tf32(x.x); l.x = to_tf32(x.x - __uint_as_float(h.x));
        h.y = to_tf32(x.y); l.y = to_tf32(x.y - __uint_as_float(h.y));
        h.z = to_tf32(x.z); l.z = to_tf32(x.z - __uint_as_float(h.z));
        h.w = to_tf32(x.w); l.w = to_tf32(x.w - __uint_as_float(h.w));
        *(uint4*)(hi + 16 * q) = h;
        *(uint4*)(lo + 16 * q) = l;
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(CONV(l));
    }
  } else if (GATHER) {
    // ---- epilogue (gather): accumulators -> their addresses in the state ----
    const int q4 = warp & 3;
    const bool leader = (warp == 6 && lane == 0);
    const int r = 32 * q4 + lane;
    // index offsets of row r of each sub-tile and of column c = 8 a + m
    uint64_t rofs[G::S], coh[KH], col[8];
#pragma unroll
    for (int sub = 0; sub < G::S; ++sub) rofs[sub] = dep_bits((uint64_t)(sub * 128 + r), gg.lmask);
#pragma unroll
    for (int a = 0; a < KH; ++a) coh[a] = dep_bits((uint64_t)(8 * a), gg.smask);
#pragma unroll
    for (int m = 0; m < 8; ++m) col[m] = dep_bits((uint64_t)m, gg.smask);
    for (uint32_t i = 0; i < nloc; ++i) {
      const int b = i % NBH, t = i & 1;
      const bool ok = bar_and(1, 128, mbar_wait_or_abort(MMAD(b), (i / NBH) & 1, abort_flag, spins));
      if (!ok) break;
      if (leader) mbar_arrive(EMPTY(b));         // the products have read the stage buffer
      tc_fence_after();
      uint32_t v[4][16];
#pragma unroll
      for (int c = 0; c < 4; ++c) tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + t * 64 + 16 * c, v[c]);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(TFREE(t));
      const uint64_t g = blockIdx.x + (uint64_t)i * gridDim.x;
      const uint64_t base = dep_bits(g << (12 - LOGK), gg.nons);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int sub = (16 * c) / KR, a = ((16 * c) % KR) / 16;   // columns 8 a .. 8 a + 7
        float2* row = gg.st + (base + rofs[sub] + coh[a]);
#pragma unroll
        for (int m = 0; m < 8; ++m)
          row[col[m]] = make_float2(__uint_as_float(v[c][2 * m]), __uint_as_float(v[c][2 * m + 1]));
      }
    }
  } else {
    // ---- epilogue: accumulators -> stage buffer -> TMA store ----
    const int q4 = warp & 3;                     // TMEM lane quarter of this warp
    const bool leader = (warp == 6 && lane == 0);
    for (uint32_t i = 0; i < nloc; ++i) {
      const int b = i % NBH, t = i & 1;
      const bool ok = bar_and(1, 128, mbar_wait_or_abort(MMAD(b), (i / NBH) & 1, abort_flag, spins));
      if (!ok) break;
      tc_fence_after();
      uint32_t v[4][16];
#pragma unroll
      for (int c = 0; c < 4; ++c) tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + t * 64 + 16 * c, v[c]);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(TFREE(t));
      unsigned char* out = sm + (sA - sb) + b * STAGE_BYTES;   // the hi part, consumed by the MMA
      const int r = 32 * q4 + lane;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int s = (16 * c) / KR, c0 = (16 * c) % KR;
#pragma unroll
        for (int tq = 0; tq < 4; ++tq) {
          const int col = c0 + 4 * tq, hb = col / G::BOXW, j = (col % G::BOXW) / 4;
          *(uint4*)(out + (s * G::QX + hb) * G::BOXB + r * G::ROWB + swz<G::ROWB>(r, j) * 16) =
              make_uint4(v[c][4 * tq], v[c][4 * tq + 1], v[c][4 * tq + 2], v[c][4 * tq + 3]);
        }
      }
      fence_async_smem();
      bar_sync(1, 128);
      if (leader) {
        const uint64_t g = blockIdx.x + (uint64_t)i * gridDim.x;
        const uint32_t so = sA + b * STAGE_BYTES;
#pragma unroll
        for (int q = 0; q < G::Q; ++q)
          tma_store_3d(&tmap, so + q * G::BOXB, (q % G::QX) * G::BOXW, 0, (int)(g * G::S + q / G::QX));
        bulk_commit();
        bulk_wait_read0();
        mbar_arrive(EMPTY(b));
      }
    }
    if (leader) bulk_wait0();
  }

  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(err, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int KR>
constexpr size_t smem_bytes() {
  return (size_t)2 * Geo<KR>::BPLANE + (size_t)(NBH + NBL) * STAGE_BYTES + 8 * (3 * NBH + 2 * NBL + 2) + 8 + 1024;
}

}  // namespace

bool fused_tc05_eligible(const qs_sim* s, const int* qubits, int k) {
  if (s->enc != QS_C64 || k < 3 || k > 5 || s->N < 12 || s->N >= 64) return false;
  uint64_t mask = 0;
  for (int m = 0; m < k; ++m) mask |= 1ull << qubits[m];
  return __builtin_popcountll(mask) == k;
}

qs_status launch_fused_tc05(qs_sim* s, const int* qubits, int k, const double* U) {
  const int KR = 2 << k;
  uint64_t smask = 0;
  for (int m = 0; m < k; ++m) smask |= 1ull << qubits[m];
  const bool gather = smask != (1ull << k) - 1;
  // the block matrix's columns follow the group's own index order: the m-th
  // qubit of the gate is bit (its rank among the gate's qubits)
  int local[5];
  for (int m = 0; m < k; ++m) local[m] = __builtin_popcountll(smask & ((1ull << qubits[m]) - 1));
  std::vector<float> B((size_t)KR * KR);
  fused_block_matrix(local, k, U, B.data());
  CUtensorMap map;
  memset(&map, 0, sizeof map);
  GatherGeo gg;
  memset(&gg, 0, sizeof gg);
  if (gather) {
    gg.st = (float2*)s->state;
    gg.smask = smask;
    gg.nons = ((1ull << s->N) - 1) & ~smask;
    uint64_t m = gg.nons;
    for (int i = 0; i < 12 - k; ++i) {
      gg.lmask |= m & (~m + 1);
      m &= m - 1;
    }
    gg.vmask = smask | gg.lmask;
    gg.run_log = __builtin_ctzll(~gg.vmask);   // >= 12 - k: bits 0 .. 11-k all lie in S or L
  } else {
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
      qs_set_error("apply_fused: cuTensorMapEncodeTiled is not available from the driver");
      return QS_ECUDA;
    }
    // the state as a 3-D tensor: KR floats x 128 rows x 2^(N-k-7) blocks
    const int boxw = KR >= 32 ? 32 : 16;
    const cuuint64_t dims[3] = {(cuuint64_t)KR, 128, 1ull << (s->N - k - 7)};
    const cuuint64_t strides[2] = {(cuuint64_t)KR * 4, (cuuint64_t)128 * KR * 4};
    const cuuint32_t box[3] = {(cuuint32_t)boxw, 128, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, s->state, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE,
                      KR >= 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
      qs_set_error("apply_fused: cuTensorMapEncodeTiled failed (%d)", (int)cr);
      return QS_ECUDA;
    }
  }
  const size_t bbytes = sizeof(float) * B.size();
  QS_TRY(ensure_scratch(s, bbytes + 256));
  int* err = (int*)((char*)s->scratch + bbytes);
  QS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s->stream));
  QS_CUDA(cudaMemcpyAsync(s->scratch, B.data(), bbytes, cudaMemcpyHostToDevice, s->stream));
  const uint64_t nstages = 1ull << (s->N - 12);
  const unsigned grid = (unsigned)(nstages < (uint64_t)s->num_sms ? nstages : (uint64_t)s->num_sms);
  const float* Bd = (const float*)s->scratch;
  auto go = [&](auto kern, size_t smem) -> qs_status {
    QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, TPB, smem, s->stream>>>(map, gg, nstages, Bd, err, pipeline_wait_spins());
    return QS_OK;
  };
  switch (k * 2 + (gather ? 1 : 0)) {
    case 6: QS_TRY(go(k_fused_tc05<16, false>, smem_bytes<16>())); break;
    case 7: QS_TRY(go(k_fused_tc05<16, true>, smem_bytes<16>())); break;
    case 8: QS_TRY(go(k_fused_tc05<32, false>, smem_bytes<32>())); break;
    case 9: QS_TRY(go(k_fused_tc05<32, true>, smem_bytes<32>())); break;
    case 10: QS_TRY(go(k_fused_tc05<64, false>, smem_bytes<64>())); break;
    default: QS_TRY(go(k_fused_tc05<64, true>, smem_bytes<64>())); break;
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
