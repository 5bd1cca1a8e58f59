// The auxiliary-variable method of Sec. 4.2: a few amplitudes of the output
// of a circuit of single-qubit gates, controlled phase shifts, CNOT and
// TOFFOLI gates, without the 2^N state.
//
// Host: every entangling gate becomes controlled phase shifts U_ct(a) =
// diag(1, 1, 1, e^{ia}) (Eq. (appa4)) and single-qubit gates: CNOT c t =
// H_t U_ct(pi) H_t; a controlled diagonal unitary diag(d0, d1) = diag(1, d0)
// on c times U_ct(arg(d1 / d0)); TOFFOLI through the standard decomposition
// into H, T, T^dagger and six CNOTs.  Each U_ct(a) is the sum over one
// auxiliary variable s = +-1 of diag(e^{i th}, e^{-i th}) on c and on t, th =
// x s - a/4, cos 2x = e^{ia/2} (the discrete Hubbard-Stratonovich
// transformation, Eqs. (appa5), (appa6)).  Per qubit the single-qubit gates
// between two auxiliary factors are multiplied into one 2x2 matrix (FP64);
// qubits that carry no auxiliary factor contribute a constant per amplitude.
//
// Device: one configuration (s_1..s_P) per thread and loop step; for every
// qubit with auxiliary factors the 2-vector W_j(s)|0> is formed by its chain
// of 2x2 products, and each requested amplitude <z| accumulates
// prod_j (W_j(s)|0>)(z_j) (Eq. (appa7)).  Sums in FP64 in a fixed order (per
// thread, then a block tree, then the blocks on the host), so results repeat
// bit for bit.  Work: O(2^P (P + N_active M)) complex operations; the FP64
// pipe bounds it.
#include "internal.cuh"
#include <complex>
#include <math.h>
#include <string.h>
#include <vector>

namespace {

constexpr int TPB = 256;
constexpr int MC = 8;          // amplitudes per kernel pass
constexpr int MAX_P = 40;

// a chain element of one qubit: kind 0 = 2x2 matrix m (8 doubles), kind 1 =
// auxiliary factor p: f[s](bit) for s = +1 (f[0..3]) and s = -1 (f[4..7])
struct AuxOp {
  int kind, p;
  double m[8];
};
struct AuxQubit {
  int q, first, count;   // chain ops[first .. first + count)
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__global__ void __launch_bounds__(TPB) k_aux(const AuxOp* __restrict__ ops, const AuxQubit* __restrict__ aq,
                                             int nact, uint64_t ncfg, const uint64_t* __restrict__ basis, int m0,
                                             int mc, double* __restrict__ part) {
  double2 acc[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) acc[m] = make_double2(0.0, 0.0);
  uint64_t zz[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) zz[m] = m < mc ? basis[m0 + m] : 0;
  for (uint64_t cfg = (uint64_t)blockIdx.x * TPB + threadIdx.x; cfg < ncfg; cfg += (uint64_t)gridDim.x * TPB) {
    double2 term[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) term[m] = make_double2(1.0, 0.0);
    for (int a = 0; a < nact; ++a) {
      const AuxQubit Q = aq[a];
      double2 w0 = make_double2(1.0, 0.0), w1 = make_double2(0.0, 0.0);
      for (int k = 0; k < Q.count; ++k) {
        const AuxOp& o = ops[Q.first + k];
        if (o.kind == 0) {
          const double2 u00 = make_double2(o.m[0], o.m[1]), u01 = make_double2(o.m[2], o.m[3]);
          const double2 u10 = make_double2(o.m[4], o.m[5]), u11 = make_double2(o.m[6], o.m[7]);
          const double2 n0 = cmul(u00, w0), n1 = cmul(u10, w0);
          const double2 n0b = cmul(u01, w1), n1b = cmul(u11, w1);
          w0 = make_double2(n0.x + n0b.x, n0.y + n0b.y);
          w1 = make_double2(n1.x + n1b.x, n1.y + n1b.y);
        } else {
          const int off = ((cfg >> o.p) & 1) ? 4 : 0;   // bit 0: s = +1, bit 1: s = -1
          w0 = cmul(w0, make_double2(o.m[off], o.m[off + 1]));
          w1 = cmul(w1, make_double2(o.m[off + 2], o.m[off + 3]));
        }
      }
#pragma unroll
      for (int m = 0; m < MC; ++m)
        if (m < mc) term[m] = cmul(term[m], ((zz[m] >> Q.q) & 1) ? w1 : w0);
    }
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      acc[m].x += term[m].x;
      acc[m].y += term[m].y;
    }
  }
  // block tree in shared memory, fixed order
  __shared__ double sh[TPB];
  for (int m = 0; m < mc; ++m) {
    for (int c = 0; c < 2; ++c) {
      sh[threadIdx.x] = c ? acc[m].y : acc[m].x;
      __syncthreads();
      for (int o = TPB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
      }
      if (threadIdx.x == 0) part[((uint64_t)blockIdx.x * MC + m) * 2 + c] = sh[0];
      __syncthreads();
    }
  }
}

using cd = std::complex<double>;

struct Rewriter {
  int N;
  // per qubit: the chain of 2x2 matrices and auxiliary factors, in the order
  // they act on |0>
  std::vector<std::vector<AuxOp>> chain;
  int P = 0;

  explicit Rewriter(int n) : N(n), chain(n) {
    for (int q = 0; q < n; ++q) chain[q].push_back(ident());
  }
  static AuxOp ident() {
    AuxOp o;
    o.kind = 0; o.p = -1;
    double id[8] = {1, 0, 0, 0, 0, 0, 1, 0};
    memcpy(o.m, id, sizeof id);
    return o;
  }
  // left-multiply the qubit's trailing matrix by u
  void one(int q, const double* u) {
    if (chain[q].back().kind != 0) chain[q].push_back(ident());
    AuxOp& b = chain[q].back();
    const cd u00(u[0], u[1]), u01(u[2], u[3]), u10(u[4], u[5]), u11(u[6], u[7]);
    const cd m00(b.m[0], b.m[1]), m01(b.m[2], b.m[3]), m10(b.m[4], b.m[5]), m11(b.m[6], b.m[7]);
    const cd r[4] = {u00 * m00 + u01 * m10, u00 * m01 + u01 * m11, u10 * m00 + u11 * m10, u10 * m01 + u11 * m11};
    for (int k = 0; k < 4; ++k) { b.m[2 * k] = r[k].real(); b.m[2 * k + 1] = r[k].imag(); }
  }
  void one_named(int q, const char* which) {
    const double h = 1.0 / sqrt(2.0), c = cos(M_PI / 4), s = sin(M_PI / 4);
    if (!strcmp(which, "H")) { double u[8] = {h, 0, h, 0, h, 0, -h, 0}; one(q, u); }
    else if (!strcmp(which, "T")) { double u[8] = {1, 0, 0, 0, 0, 0, c, s}; one(q, u); }
    else { double u[8] = {1, 0, 0, 0, 0, 0, c, -s}; one(q, u); }
  }
  // U_ct(a): one auxiliary variable, a factor on each of c and t
  void cphase(int c, int t, double a) {
    const cd x = 0.5 * std::acos(std::exp(cd(0.0, 0.5 * a)));
    AuxOp o;
    o.kind = 1;
    o.p = P++;
    for (int si = 0; si < 2; ++si) {
      const double sg = si == 0 ? 1.0 : -1.0;
      const cd th = x * sg - a / 4.0;
      const cd f0 = std::exp(cd(0.0, 1.0) * th), f1 = std::exp(cd(0.0, -1.0) * th);
      o.m[4 * si + 0] = f0.real(); o.m[4 * si + 1] = f0.imag();
      o.m[4 * si + 2] = f1.real(); o.m[4 * si + 3] = f1.imag();
    }
    chain[c].push_back(o);
    chain[t].push_back(o);
  }
  void cnot(int c, int t) {
    one_named(t, "H");
    cphase(c, t, M_PI);
    one_named(t, "H");
  }
  void toffoli(int a, int b, int t) {
    one_named(t, "H"); cnot(b, t); one_named(t, "TD"); cnot(a, t); one_named(t, "T"); cnot(b, t);
    one_named(t, "TD"); cnot(a, t); one_named(b, "T"); one_named(t, "T"); one_named(t, "H"); cnot(a, b);
    one_named(a, "T"); one_named(b, "TD"); cnot(a, b);
  }
  qs_status add(const qs_gate& g) {
    const double* u = g.u;
    const bool diag = u[2] == 0 && u[3] == 0 && u[4] == 0 && u[5] == 0;
    const bool isx = u[0] == 0 && u[1] == 0 && u[6] == 0 && u[7] == 0 && u[2] == 1 && u[3] == 0 && u[4] == 1 &&
                     u[5] == 0;
    if (g.nc == 0) { one(g.target, u); return QS_OK; }
    if (g.nc == 1 && isx) { cnot(g.controls[0], g.target); return QS_OK; }
    if (g.nc == 1 && diag) {
      const cd d0(u[0], u[1]), d1(u[6], u[7]);
      if (d0 == cd(1, 0) && d1 == cd(1, 0)) return QS_OK;
      double cu[8] = {1, 0, 0, 0, 0, 0, d0.real(), d0.imag()};
      one(g.controls[0], cu);
      cphase(g.controls[0], g.target, std::arg(d1 / d0));
      return QS_OK;
    }
    if (g.nc == 2 && isx) { toffoli(g.controls[0], g.controls[1], g.target); return QS_OK; }
    qs_set_error("aux_amplitudes: the auxiliary-variable method covers single-qubit gates, controlled "
                 "phases, CNOT and TOFFOLI (gate with %d controls on qubit %d is none of these)", g.nc, g.target);
    return QS_EUNSUPPORTED;
  }
};

}  // namespace

static qs_status aux_rewrite(int N, const qs_gate* gates, int n, Rewriter& R) {
  for (int i = 0; i < n; ++i) {
    const qs_gate& g = gates[i];
    if (g.target < 0 || g.target >= N || g.nc < 0 || g.nc > 2) {
      qs_set_error("aux_amplitudes: gate %d has a qubit out of range", i);
      return QS_EINVAL;
    }
    for (int c = 0; c < g.nc; ++c)
      if (g.controls[c] < 0 || g.controls[c] >= N || g.controls[c] == g.target ||
          (c == 1 && g.controls[1] == g.controls[0])) {
        qs_set_error("aux_amplitudes: gate %d has bad controls", i);
        return QS_EINVAL;
      }
    QS_TRY(R.add(g));
    if (R.P > MAX_P) {
      qs_set_error("aux_amplitudes: more than %d auxiliary variables", MAX_P);
      return QS_EINVAL;
    }
  }
  return QS_OK;
}

extern "C" qs_status aux_count(int N, const qs_gate* gates, int n, int* P) {
  if (N < 1 || N > 63 || n < 0 || (n && !gates) || !P) { qs_set_error("aux_count: bad arguments"); return QS_EINVAL; }
  Rewriter R(N);
  QS_TRY(aux_rewrite(N, gates, n, R));
  *P = R.P;
  return QS_OK;
}

extern "C" qs_status aux_amplitudes(int N, const qs_gate* gates, int n, const uint64_t* basis, int M, double* out,
                                    int* P_out, void* cuda_stream) {
  if (N < 1 || N > 63 || n < 0 || (n && !gates) || !basis || !out || M < 1 || M > 4096) {
    qs_set_error("aux_amplitudes: bad arguments (1 <= N <= 63, 1 <= M <= 4096)");
    return QS_EINVAL;
  }
  for (int m = 0; m < M; ++m)
    if (N < 64 && (basis[m] >> N) != 0) { qs_set_error("aux_amplitudes: basis index %d out of range", m); return QS_EINVAL; }
  Rewriter R(N);
  QS_TRY(aux_rewrite(N, gates, n, R));
  if (P_out) *P_out = R.P;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // qubits with auxiliary factors go to the device; the others give a
  // constant factor per amplitude (their whole chain is one matrix)
  std::vector<AuxOp> ops;
  std::vector<AuxQubit> act;
  std::vector<std::complex<double>> cst(M, 1.0);
  for (int q = 0; q < N; ++q) {
    const auto& ch = R.chain[q];
    bool has_aux = false;
    for (const auto& o : ch) has_aux |= (o.kind == 1);
    if (!has_aux) {
      const AuxOp& mtx = ch[0];   // a single matrix
      const cd w0(mtx.m[0], mtx.m[1]), w1(mtx.m[4], mtx.m[5]);
      for (int m = 0; m < M; ++m) cst[m] *= ((basis[m] >> q) & 1) ? w1 : w0;
      continue;
    }
    AuxQubit a;
    a.q = q;
    a.first = (int)ops.size();
    a.count = (int)ch.size();
    for (const auto& o : ch) ops.push_back(o);
    act.push_back(a);
  }
  const uint64_t ncfg = 1ull << R.P;
  int dev = 0, sms = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const uint64_t want = (ncfg + TPB - 1) / TPB;
  const unsigned grid = (unsigned)(want < (uint64_t)sms * 4 ? want : (uint64_t)sms * 4);
  std::vector<double> sums(2 * (size_t)M, 0.0);
  if (!act.empty()) {
    AuxOp* d_ops = nullptr;
    AuxQubit* d_aq = nullptr;
    uint64_t* d_basis = nullptr;
    double* d_part = nullptr;
    const size_t part_n = (size_t)grid * MC * 2;
    qs_status rc = QS_OK;
    auto cu = [&](cudaError_t e, const char* what) {
      if (e != cudaSuccess && rc == QS_OK) {
        qs_set_error("aux_amplitudes: %s: %s", what, cudaGetErrorString(e));
        rc = QS_ECUDA;
      }
    };
    cu(cudaMallocAsync(&d_ops, ops.size() * sizeof(AuxOp), st), "alloc");
    cu(cudaMallocAsync(&d_aq, act.size() * sizeof(AuxQubit), st), "alloc");
    cu(cudaMallocAsync(&d_basis, M * sizeof(uint64_t), st), "alloc");
    cu(cudaMallocAsync(&d_part, part_n * sizeof(double), st), "alloc");
    std::vector<double> part(part_n);
    if (rc == QS_OK) {
      cu(cudaMemcpyAsync(d_ops, ops.data(), ops.size() * sizeof(AuxOp), cudaMemcpyHostToDevice, st), "copy");
      cu(cudaMemcpyAsync(d_aq, act.data(), act.size() * sizeof(AuxQubit), cudaMemcpyHostToDevice, st), "copy");
      cu(cudaMemcpyAsync(d_basis, basis, M * sizeof(uint64_t), cudaMemcpyHostToDevice, st), "copy");
    }
    for (int m0 = 0; m0 < M && rc == QS_OK; m0 += MC) {
      const int mc = (M - m0) < MC ? (M - m0) : MC;
      k_aux<<<grid, TPB, 0, st>>>(d_ops, d_aq, (int)act.size(), ncfg, d_basis, m0, mc, d_part);
      qs_count_launch();
      cu(cudaGetLastError(), "launch");
      if (rc != QS_OK) break;
      cu(cudaMemcpyAsync(part.data(), d_part, part_n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
      cu(cudaStreamSynchronize(st), "sync");
      // blocks in order, compensated (Neumaier)
      for (int m = 0; m < mc && rc == QS_OK; ++m)
        for (int c = 0; c < 2; ++c) {
          double sum = 0.0, comp = 0.0;
          for (unsigned b = 0; b < grid; ++b) {
            const double x = part[((size_t)b * MC + m) * 2 + c];
            const double t = sum + x;
            comp += fabs(sum) >= fabs(x) ? (sum - t) + x : (x - t) + sum;
            sum = t;
          }
          sums[2 * (m0 + m) + c] = sum + comp;
        }
    }
    cudaFreeAsync(d_ops, st);
    cudaFreeAsync(d_aq, st);
    cudaFreeAsync(d_basis, st);
    cudaFreeAsync(d_part, st);
    if (rc != QS_OK) return rc;
    QS_CUDA(cudaStreamSynchronize(st));
  } else {
    for (int m = 0; m < M; ++m) sums[2 * m] = 1.0;   // no configuration sum (P = 0)
  }
  const double scale = ldexp(1.0, -R.P);
  for (int m = 0; m < M; ++m) {
    const cd v = cst[m] * cd(sums[2 * m], sums[2 * m + 1]) * scale;
    out[2 * m] = v.real();
    out[2 * m + 1] = v.imag();
  }
  return QS_OK;
}
