// The adaptive 2-byte encoding of JUQCS-A (Sec. 4.1) on the device.
//
// One 16-bit word per amplitude: low byte b0 (magnitude code), high byte b1
// (angle code, theta = pi b1 / 128).  b0 = -128 is r = 0, b0 = 127 is r = 1,
// and -127 <= b0 <= 126 is r = (b0 + 127)(r1 - r0)/253 + r0, where r0 and r1
// are the minimum and maximum of |z| over the amplitudes with 0 < |z| < 1.
//
// Gates fall into three classes:
//  * X-type permutations (X, CNOT, TOFFOLI, and the register permutations in
//    k_perm.cu) move words; nothing is decoded.
//  * Diagonal and anti-diagonal unitaries (Z, S, T, R, U(k), RZ, Y, ...) keep
//    every |z|, hence b0 and (r0, r1): they only add the phase to b1 (an exact
//    integer for multiples of pi/128, else rounded in code units) and, for
//    anti-diagonal ones, swap the pair.
//  * Every other gate (H, +X, U2, U3, Haar U(2), ...) is arithmetic and takes
//    two passes: the range pass decodes, applies the gate in FP32 and gathers
//    min / max |z| over 0 < |z| < 1 of the whole post-gate state; the encode
//    pass decodes, applies the gate again and encodes every amplitude with the
//    new (r0, r1).  A one-thread kernel then makes the new range current.
//    All of this stays on the stream: no host synchronisation per gate.
#include "internal.cuh"
#include "cplx.cuh"
#include "a2codec.cuh"
#include <math.h>

namespace {

constexpr int TPB = 256;
constexpr unsigned int INF_BITS = 0x7f800000u;

struct EncP {
  float r0, r1, scale;
};
// |z| below about 1e-18 has a square that is denormal or zero in FP32; such
// magnitudes are taken from the scaled components instead, so that the range
// and the codes of tiny amplitudes follow |z| as the FP64 definition does
constexpr float TINY2 = 1e-36f;
// |z| < 1e-18: scaled by 2^100 (exact) the square is a normal number for
// every nonzero FP32 input, so no division is needed
__device__ __forceinline__ float tiny_mag(Cx<float> z) {
  const float xs = z.x * 1.2676506002282294e30f, ys = z.y * 1.2676506002282294e30f;   // 2^100
  return sqrtf(fmaf(xs, xs, ys * ys)) * 7.888609052210118e-31f;                        // 2^-100
}
__device__ __forceinline__ float a2_mag(Cx<float> z) {
  const float m2 = fmaf(z.x, z.x, z.y * z.y);
  return (m2 < TINY2 && (z.x != 0.f || z.y != 0.f)) ? tiny_mag(z) : sqrtf(m2);
}

__device__ __forceinline__ unsigned int a2_enc(Cx<float> z, const EncP& e) {
  if (z.x == 0.f && z.y == 0.f) return 0x0080u;
  const float m = a2_mag(z);
  int b0;
  if (m >= 1.f) {
    b0 = 127;
  } else if (e.r1 > e.r0) {
    float q = rintf((m - e.r0) * e.scale);
    q = fminf(fmaxf(q, 0.f), 253.f);
    b0 = (int)q - 127;
  } else {
    b0 = -127;
  }
  int b1 = (int)rintf(atan2f(z.y, z.x) * 40.74366543152521f);  // 128 / pi
  if (b1 >= 128) b1 -= 256;
  return ((unsigned int)(b0 & 0xFF)) | ((unsigned int)(b1 & 0xFF) << 8);
}

__device__ EncP enc_params(const A2Dev* d) {
  EncP e;
  if (d->mn == INF_BITS) {
    e.r0 = e.r1 = 0.f;
    e.scale = 0.f;
  } else {
    e.r0 = __uint_as_float(d->mn);
    e.r1 = __uint_as_float(d->mx);
    e.scale = (e.r1 > e.r0) ? (float)(253.0 / ((double)e.r1 - (double)e.r0)) : 0.f;
  }
  return e;
}

// Range tracking on squared magnitudes: sqrtf is monotonic, so the min / max
// of sqrtf(m2) is sqrtf of the min / max of m2 (taken once per thread in
// block_minmax), and for a float m2, sqrtf(m2) < 1 exactly when m2 < 1 (the
// float below 1 has its root below the midpoint of 1 - 2^-24 and 1) and
// sqrtf(m2) > 0 exactly when m2 > 0.
// A nonzero amplitude whose square is below TINY2 goes to mn as its
// magnitude (tiny_mag); mn2 / mx2 track the others' squares.
__device__ __forceinline__ void track(Cx<float> z, float& mn2, float& mx2, float& mnt) {
  const float m2 = fmaf(z.x, z.x, z.y * z.y);
  if (m2 >= TINY2 && m2 < 1.f) { mn2 = fminf(mn2, m2); mx2 = fmaxf(mx2, m2); }
  else if (m2 < TINY2 && (z.x != 0.f || z.y != 0.f)) mnt = fminf(mnt, tiny_mag(z));
}

// mn2 / mx2: the thread's min / max of squared magnitudes (INF / 0 if none);
// mnt: its smallest tiny magnitude (INF if none)
__device__ void block_minmax(float mn2, float mx2, float mnt, A2Dev* d) {
  __shared__ float smn[32], smx[32];
  float mn = (mn2 < __uint_as_float(INF_BITS)) ? sqrtf(mn2) : mn2;
  mn = fminf(mn, mnt);
  float mx = sqrtf(mx2);
  if (mx2 == 0.f && mnt < __uint_as_float(INF_BITS)) mx = mnt;   // only tiny values seen
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { smn[w] = mn; smx[w] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { mn = fminf(mn, smn[i]); mx = fmaxf(mx, smx[i]); }
    if (mn < __uint_as_float(INF_BITS)) atomicMin(&d->mn, __float_as_uint(mn));
    if (mx > 0.f) atomicMax(&d->mx, __float_as_uint(mx));
  }
}

// ---- word access in 16-byte chunks (8 amplitudes) -------------------------------------
__device__ __forceinline__ unsigned int wget(const uint4& c, int k) {
  const unsigned int v = (k < 2) ? c.x : (k < 4) ? c.y : (k < 6) ? c.z : c.w;
  return (k & 1) ? (v >> 16) : (v & 0xFFFFu);
}
__device__ __forceinline__ void wset(uint4& c, int k, unsigned int w) {
  unsigned int* p = (k < 2) ? &c.x : (k < 4) ? &c.y : (k < 6) ? &c.z : &c.w;
  *p = (k & 1) ? ((*p & 0xFFFFu) | (w << 16)) : ((*p & 0xFFFF0000u) | (w & 0xFFFFu));
}

struct Geo {
  int N, t;
  uint64_t cmask;   // control bits (global index)
};

// Arithmetic gate, PASS 0 = range, PASS 1 = encode.  A unit is a pair of
// chunks (t >= 3) or one chunk holding four pairs (t < 3).
template <int PASS, typename Op>
__global__ void __launch_bounds__(TPB) k_a2_arith(uint16_t* __restrict__ st, Geo g, Op op, A2Dev* d) {
  __shared__ Luts L;
  build_luts(L, d->r0, d->r1);
  EncP e;
  if (PASS == 1) e = enc_params(d);
  float mn = __uint_as_float(INF_BITS), mx = 0.f, mnt = __uint_as_float(INF_BITS);
  uint4* s4 = (uint4*)st;
  const uint64_t nchunks = 1ull << (g.N - 3);
  const uint64_t nunits = (g.t >= 3) ? (nchunks >> 1) : nchunks;
  for (uint64_t u = (uint64_t)blockIdx.x * TPB + threadIdx.x; u < nunits; u += (uint64_t)gridDim.x * TPB) {
    if (g.t >= 3) {
      const uint64_t c0 = ins0(u, g.t - 3), c1 = c0 | (1ull << (g.t - 3));
      uint4 w0 = s4[c0], w1 = s4[c1];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        Cx<float> a = a2_dec(L, wget(w0, k)), b = a2_dec(L, wget(w1, k));
        const uint64_t i0 = c0 * 8 + k;
        if ((i0 & g.cmask) == g.cmask) op.pair(a, b);
        if (PASS == 0) { track(a, mn, mx, mnt); track(b, mn, mx, mnt); }
        else { wset(w0, k, a2_enc(a, e)); wset(w1, k, a2_enc(b, e)); }
      }
      if (PASS == 1) { s4[c0] = w0; s4[c1] = w1; }
    } else {
      uint4 w = s4[u];
      const int m = 1 << g.t;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k & m) continue;
        Cx<float> a = a2_dec(L, wget(w, k)), b = a2_dec(L, wget(w, k | m));
        const uint64_t i0 = u * 8 + k;
        if ((i0 & g.cmask) == g.cmask) op.pair(a, b);
        if (PASS == 0) { track(a, mn, mx, mnt); track(b, mn, mx, mnt); }
        else { wset(w, k, a2_enc(a, e)); wset(w, k | m, a2_enc(b, e)); }
      }
      if (PASS == 1) s4[u] = w;
    }
  }
  if (PASS == 0) block_minmax(mn, mx, mnt, d);
}

// Small states (N < 4): one thread per pair, plain word accesses.
template <int PASS, typename Op>
__global__ void k_a2_arith_small(uint16_t* __restrict__ st, Geo g, Op op, A2Dev* d) {
  __shared__ Luts L;
  build_luts(L, d->r0, d->r1);
  EncP e;
  if (PASS == 1) e = enc_params(d);
  float mn = __uint_as_float(INF_BITS), mx = 0.f, mnt = __uint_as_float(INF_BITS);
  const uint64_t npairs = 1ull << (g.N - 1);
  for (uint64_t p = threadIdx.x; p < npairs; p += blockDim.x) {
    const uint64_t i0 = ins0(p, g.t), i1 = i0 | (1ull << g.t);
    Cx<float> a = a2_dec(L, st[i0]), b = a2_dec(L, st[i1]);
    if ((i0 & g.cmask) == g.cmask) op.pair(a, b);
    if (PASS == 0) { track(a, mn, mx, mnt); track(b, mn, mx, mnt); }
    else { st[i0] = (uint16_t)a2_enc(a, e); st[i1] = (uint16_t)a2_enc(b, e); }
  }
  if (PASS == 0) block_minmax(mn, mx, mnt, d);
}

__global__ void k_a2_begin(A2Dev* d) { d->mn = INF_BITS; d->mx = 0u; }
__global__ void k_a2_commit(A2Dev* d) {
  if (d->mn == INF_BITS) { d->r0 = 0.0; d->r1 = 0.0; }
  else { d->r0 = (double)__uint_as_float(d->mn); d->r1 = (double)__uint_as_float(d->mx); }
}
__global__ void k_a2_set(A2Dev* d, double r0, double r1) { d->r0 = r0; d->r1 = r1; d->mn = INF_BITS; d->mx = 0u; }

// ---- code-only gates: word swaps and angle-code shifts -----------------------------------
// new word of the bit-0 element = (anti ? w1 : w0) with b1 += sh0, of the bit-1
// element = (anti ? w0 : w1) with b1 += sh1, where the controls hold.
__device__ __forceinline__ unsigned int shift_b1(unsigned int w, float sh, int ish, bool exact) {
  if ((w & 0xFFu) == 0x80u) return w;  // r = 0: the angle code stays 0
  const int b1 = (int)(signed char)(w >> 8);
  const int nb = exact ? (b1 + ish) : (int)rintf((float)b1 + sh);
  return (w & 0xFFu) | ((unsigned int)(nb & 0xFF) << 8);
}
struct CodeOp {
  int anti;
  float sh0, sh1;
  int ish0, ish1;
  int exact;
  int touch0, touch1;   // element needs a change (shift or swap)
  __device__ __forceinline__ void pair(unsigned int& w0, unsigned int& w1) const {
    unsigned int a = anti ? w1 : w0, b = anti ? w0 : w1;
    if (touch0) a = shift_b1(a, sh0, ish0, exact);
    if (touch1) b = shift_b1(b, sh1, ish1, exact);
    w0 = a; w1 = b;
  }
};

__global__ void __launch_bounds__(TPB) k_a2_codes(uint16_t* __restrict__ st, Geo g, CodeOp op) {
  uint4* s4 = (uint4*)st;
  const uint64_t nchunks = 1ull << (g.N - 3);
  const uint64_t nunits = (g.t >= 3) ? (nchunks >> 1) : nchunks;
  for (uint64_t u = (uint64_t)blockIdx.x * TPB + threadIdx.x; u < nunits; u += (uint64_t)gridDim.x * TPB) {
    if (g.t >= 3) {
      const uint64_t c0 = ins0(u, g.t - 3), c1 = c0 | (1ull << (g.t - 3));
      uint4 w0 = s4[c0], w1 = s4[c1];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (((c0 * 8 + k) & g.cmask) != g.cmask) continue;
        unsigned int a = wget(w0, k), b = wget(w1, k);
        op.pair(a, b);
        wset(w0, k, a);
        wset(w1, k, b);
      }
      s4[c0] = w0;
      s4[c1] = w1;
    } else {
      uint4 w = s4[u];
      const int m = 1 << g.t;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if ((k & m) || (((u * 8 + k) & g.cmask) != g.cmask)) continue;
        unsigned int a = wget(w, k), b = wget(w, k | m);
        op.pair(a, b);
        wset(w, k, a);
        wset(w, k | m, b);
      }
      s4[u] = w;
    }
  }
}
__global__ void k_a2_codes_small(uint16_t* __restrict__ st, Geo g, CodeOp op) {
  const uint64_t npairs = 1ull << (g.N - 1);
  for (uint64_t p = threadIdx.x; p < npairs; p += blockDim.x) {
    const uint64_t i0 = ins0(p, g.t), i1 = i0 | (1ull << g.t);
    if ((i0 & g.cmask) != g.cmask) continue;
    unsigned int a = st[i0], b = st[i1];
    op.pair(a, b);
    st[i0] = (uint16_t)a;
    st[i1] = (uint16_t)b;
  }
}

// ---- reductions: sum of r^2 (norm) --------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_a2_norm(const uint16_t* __restrict__ st, uint64_t nchunks, const A2Dev* d,
                                                 double* part) {
  __shared__ Luts L;
  build_luts(L, d->r0, d->r1);
  __shared__ double sh[32];
  const uint4* s4 = (const uint4*)st;
  double acc = 0.0;
  float hi = 0.f, lo = 0.f;   // float-float sum of exact r^2 = p + e
  int cnt = 0;
  for (uint64_t c = (uint64_t)blockIdx.x * TPB + threadIdx.x; c < nchunks; c += (uint64_t)gridDim.x * TPB) {
    const uint4 w = s4[c];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float r = L.r[(int)(wget(w, k) & 0xFFu) ^ 0x80];
      const float p = r * r, e = fmaf(r, r, -p);
      const float t = hi + p, bp = t - hi;
      lo += ((hi - (t - bp)) + (p - bp)) + e;
      hi = t;
    }
    if (++cnt == 8) { acc += (double)hi + (double)lo; hi = lo = 0.f; cnt = 0; }
  }
  acc += (double)hi + (double)lo;
  // block sum, fixed order
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < TPB / 32; ++i) r += sh[i];
    part[blockIdx.x] = r;
  }
}

__global__ void k_a2_norm_small(const uint16_t* __restrict__ st, int N, const A2Dev* d, double* out) {
  __shared__ Luts L;
  build_luts(L, d->r0, d->r1);
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int i = 0; i < (1 << N); ++i) {
      const float r = L.r[(int)(st[i] & 0xFFu) ^ 0x80];
      acc = fma((double)r, (double)r, acc);
    }
    out[0] = acc;
  }
}

}  // namespace

// =========================================================================================
static unsigned a2_grid(const qs_sim* s, uint64_t units) {
  const uint64_t g = (uint64_t)s->num_sms * 8;
  const uint64_t need = (units + TPB - 1) / TPB;
  return (unsigned)(need < g ? (need ? need : 1) : g);
}

qs_status a2_set_range(qs_sim* s, double r0, double r1) {
  k_a2_set<<<1, 1, 0, s->stream>>>((A2Dev*)s->a2dev, r0, r1);
  QS_LAUNCH_CHECK();
  return QS_OK;
}

qs_status a2_get_range(qs_sim* s, double* r0, double* r1) {
  A2Dev h;
  QS_CUDA(cudaMemcpyAsync(&h, s->a2dev, sizeof h, cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  *r0 = h.r0;
  *r1 = h.r1;
  return QS_OK;
}

template <typename Op>
static qs_status a2_arith(qs_sim* s, const Geo& g, const Op& op) {
  A2Dev* d = (A2Dev*)s->a2dev;
  k_a2_begin<<<1, 1, 0, s->stream>>>(d);
  QS_LAUNCH_CHECK();
  if (s->N >= 4) {
    const uint64_t nchunks = 1ull << (s->N - 3);
    const uint64_t units = (g.t >= 3) ? nchunks / 2 : nchunks;
    const unsigned grid = a2_grid(s, units);
    k_a2_arith<0, Op><<<grid, TPB, 0, s->stream>>>((uint16_t*)s->state, g, op, d);
    QS_LAUNCH_CHECK();
    k_a2_arith<1, Op><<<grid, TPB, 0, s->stream>>>((uint16_t*)s->state, g, op, d);
    QS_LAUNCH_CHECK();
  } else {
    k_a2_arith_small<0, Op><<<1, 32, 0, s->stream>>>((uint16_t*)s->state, g, op, d);
    QS_LAUNCH_CHECK();
    k_a2_arith_small<1, Op><<<1, 32, 0, s->stream>>>((uint16_t*)s->state, g, op, d);
    QS_LAUNCH_CHECK();
  }
  k_a2_commit<<<1, 1, 0, s->stream>>>(d);
  QS_LAUNCH_CHECK();
  return QS_OK;
}

// Phase angle of a unit-modulus factor in code units (128/pi rad), and
// whether it is an integer.
static void phase_code(double re, double im, float* sh, int* ish, int* exact) {
  const double m = atan2(im, re) * 128.0 / M_PI;
  const double r = nearbyint(m);
  *sh = (float)m;
  *ish = (int)r;
  *exact = fabs(m - r) <= 1e-9;
}

qs_status a2_apply_u2(qs_sim* s, const int* controls, int nc, int target, const double u[8]) {
  GateClass gc = classify_u2(u);
  if (gc.kind == GK_IDENT) return QS_OK;
  Geo g;
  g.N = s->N;
  g.t = target;
  g.cmask = 0;
  for (int i = 0; i < nc; ++i) g.cmask |= 1ull << controls[i];
  if (gc.kind == GK_DIAG || gc.kind == GK_ANTI) {
    CodeOp op;
    op.anti = (gc.kind == GK_ANTI);
    const double* f0 = op.anti ? u + 2 : u;      // factor landing on the bit-0 element
    const double* f1 = op.anti ? u + 4 : u + 6;  // factor landing on the bit-1 element
    int e0, e1;
    phase_code(f0[0], f0[1], &op.sh0, &op.ish0, &e0);
    phase_code(f1[0], f1[1], &op.sh1, &op.ish1, &e1);
    op.exact = e0 && e1;
    op.touch0 = !(e0 && op.ish0 == 0);
    op.touch1 = !(e1 && op.ish1 == 0);
    if (s->N >= 4) {
      const uint64_t nchunks = 1ull << (s->N - 3);
      const uint64_t units = (g.t >= 3) ? nchunks / 2 : nchunks;
      k_a2_codes<<<a2_grid(s, units), TPB, 0, s->stream>>>((uint16_t*)s->state, g, op);
    } else {
      k_a2_codes_small<<<1, 32, 0, s->stream>>>((uint16_t*)s->state, g, op);
    }
    QS_LAUNCH_CHECK();
    return QS_OK;
  }
  auto fcx = [&](int k) { Cx<float> c; c.x = (float)u[2 * k]; c.y = (float)u[2 * k + 1]; return c; };
  if (gc.kind == GK_HAD) {
    OpHad<float> op;
    op.s = (float)u[0];
    return a2_arith(s, g, op);
  }
  OpDense<float> op;
  op.u00 = fcx(0); op.u01 = fcx(1); op.u10 = fcx(2); op.u11 = fcx(3);
  return a2_arith(s, g, op);
}

qs_status a2_apply_arith(qs_sim* s, const int* controls, int nc, int target, const double u[8]) {
  Geo g;
  g.N = s->N;
  g.t = target;
  g.cmask = 0;
  for (int i = 0; i < nc; ++i) g.cmask |= 1ull << controls[i];
  auto fcx = [&](int k) { Cx<float> c; c.x = (float)u[2 * k]; c.y = (float)u[2 * k + 1]; return c; };
  OpDense<float> op;
  op.u00 = fcx(0); op.u01 = fcx(1); op.u10 = fcx(2); op.u11 = fcx(3);
  return a2_arith(s, g, op);
}

qs_status a2_norm(qs_sim* s, double* out) {
  const A2Dev* d = (const A2Dev*)s->a2dev;
  if (s->N < 4) {
    QS_TRY(ensure_scratch(s, sizeof(double)));
    k_a2_norm_small<<<1, 256, 0, s->stream>>>((const uint16_t*)s->state, s->N, d, (double*)s->scratch);
    QS_LAUNCH_CHECK();
    QS_CUDA(cudaMemcpyAsync(out, s->scratch, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA(cudaStreamSynchronize(s->stream));
    return QS_OK;
  }
  const uint64_t nchunks = 1ull << (s->N - 3);
  const unsigned grid = a2_grid(s, nchunks);
  QS_TRY(ensure_scratch(s, sizeof(double) * (grid + 1)));
  double* part = (double*)s->scratch;
  k_a2_norm<<<grid, TPB, 0, s->stream>>>((const uint16_t*)s->state, nchunks, d, part);
  QS_LAUNCH_CHECK();
  QS_TRY(sum_partials(s, part, grid, part + grid));
  QS_TRY(ensure_hbuf(s, sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(s->hbuf, part + grid, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  *out = *(double*)s->hbuf;
  return QS_OK;
}

qs_status a2_shorbox(qs_sim* s, int nx, uint64_t G, uint64_t y) { return launch_shorbox(s, nx, G, y); }
qs_status a2_reset(qs_sim* s) { return launch_reset(s); }
