// Host-side gate library: the instruction-set matrices (Appendix A), gate
// classification for the specialised kernels, unitarity checks and
// composition of fused k-qubit matrices in FP64.
#include "internal.cuh"
#include <math.h>
#include <string.h>
#include <ctype.h>

int unit_code(double re, double im) {
  if (re == 1.0 && im == 0.0) return 0;
  if (re == 0.0 && im == 1.0) return 1;
  if (re == -1.0 && im == 0.0) return 2;
  if (re == 0.0 && im == -1.0) return 3;
  return 4;
}

static bool is_zero(const double* u, int k) { return u[2 * k] == 0.0 && u[2 * k + 1] == 0.0; }

GateClass classify_u2(const double u[8]) {
  GateClass g;
  g.c0 = g.c1 = 4;
  if (is_zero(u, 1) && is_zero(u, 2)) {
    g.kind = GK_DIAG;
    g.c0 = unit_code(u[0], u[1]);
    g.c1 = unit_code(u[6], u[7]);
    if (g.c0 == 0 && g.c1 == 0) g.kind = GK_IDENT;
    return g;
  }
  if (is_zero(u, 0) && is_zero(u, 3)) {
    g.kind = GK_ANTI;
    g.c0 = unit_code(u[2], u[3]);
    g.c1 = unit_code(u[4], u[5]);
    return g;
  }
  if (u[1] == 0.0 && u[3] == 0.0 && u[5] == 0.0 && u[7] == 0.0 && u[0] == u[2] && u[0] == u[4] &&
      u[0] == -u[6]) {
    g.kind = GK_HAD;
    return g;
  }
  g.kind = GK_DENSE;
  return g;
}

double unitarity_defect(const double* U, int d) {
  double worst = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double re = 0.0, im = 0.0;  // (U U^dagger)_{ij} = sum_k U_ik conj(U_jk)
      for (int k = 0; k < d; ++k) {
        double ar = U[2 * (i * d + k)], ai = U[2 * (i * d + k) + 1];
        double br = U[2 * (j * d + k)], bi = -U[2 * (j * d + k) + 1];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      double e = fabs(re - (i == j ? 1.0 : 0.0)) + fabs(im);
      if (!(e <= worst)) worst = e;  // NaN propagates as "not unitary"
    }
  return worst;
}

// ---------------------------------------------------------------------------
// gate_std: instruction-set mnemonics -> controlled-U(2) records
// ---------------------------------------------------------------------------
static void set2(double* u, double a, double b, double c, double d, double e, double f, double g,
                 double h) {
  u[0] = a; u[1] = b; u[2] = c; u[3] = d; u[4] = e; u[5] = f; u[6] = g; u[7] = h;
}

static bool ieq(const char* a, const char* b) {
  while (*a && *b) {
    if (toupper((unsigned char)*a) != toupper((unsigned char)*b)) return false;
    ++a; ++b;
  }
  return *a == 0 && *b == 0;
}

// Phase e^{i*ang} with exact values for the angles that have them.
static void phase(double ang_num_pi_over, int k, int sign, double* re, double* im) {
  (void)ang_num_pi_over;
  // angle = sign * 2 pi / 2^k
  if (k == 0) { *re = 1.0; *im = 0.0; return; }
  if (k == 1) { *re = -1.0; *im = 0.0; return; }
  if (k == 2) { *re = 0.0; *im = (double)sign; return; }
  double a = sign * 2.0 * M_PI / ldexp(1.0, k);
  if (k == 3) { double s = 1.0 / sqrt(2.0); *re = s; *im = sign * s; return; }
  *re = cos(a); *im = sin(a);
}

extern "C" qs_status gate_std(const char* m, const int* q, int nq, const double* p, int np,
                              qs_gate* out) {
  if (!m || !out || (nq > 0 && !q) || (np > 0 && !p)) { qs_set_error("gate_std: null argument"); return QS_EINVAL; }
  qs_gate g;
  memset(&g, 0, sizeof g);
  const double s2 = 1.0 / sqrt(2.0);
  double* u = g.u;
  int need_q = 1;
  if (ieq(m, "I")) set2(u, 1, 0, 0, 0, 0, 0, 1, 0);
  else if (ieq(m, "H")) set2(u, s2, 0, s2, 0, s2, 0, -s2, 0);
  else if (ieq(m, "X")) set2(u, 0, 0, 1, 0, 1, 0, 0, 0);
  else if (ieq(m, "Y")) set2(u, 0, 0, 0, -1, 0, 1, 0, 0);
  else if (ieq(m, "Z")) set2(u, 1, 0, 0, 0, 0, 0, -1, 0);
  else if (ieq(m, "S")) set2(u, 1, 0, 0, 0, 0, 0, 0, 1);
  else if (ieq(m, "S+")) set2(u, 1, 0, 0, 0, 0, 0, 0, -1);
  else if (ieq(m, "T")) set2(u, 1, 0, 0, 0, 0, 0, s2, s2);
  else if (ieq(m, "T+")) set2(u, 1, 0, 0, 0, 0, 0, s2, -s2);
  else if (ieq(m, "+X")) set2(u, s2, 0, 0, s2, 0, s2, s2, 0);
  else if (ieq(m, "-X")) set2(u, s2, 0, 0, -s2, 0, -s2, s2, 0);
  else if (ieq(m, "+Y")) set2(u, s2, 0, s2, 0, -s2, 0, s2, 0);
  else if (ieq(m, "-Y")) set2(u, s2, 0, -s2, 0, s2, 0, s2, 0);
  else if (ieq(m, "U1")) {
    if (np < 1) goto badp;
    set2(u, 1, 0, 0, 0, 0, 0, cos(p[0]), sin(p[0]));
  } else if (ieq(m, "U2")) {
    if (np < 2) goto badp;
    double ph = p[0], la = p[1];
    set2(u, s2, 0, -s2 * cos(la), -s2 * sin(la), s2 * cos(ph), s2 * sin(ph), s2 * cos(ph + la),
         s2 * sin(ph + la));
  } else if (ieq(m, "U3")) {
    if (np < 3) goto badp;
    double c = cos(p[0] / 2), s = sin(p[0] / 2), ph = p[1], la = p[2];
    set2(u, c, 0, -s * cos(la), -s * sin(la), s * cos(ph), s * sin(ph), c * cos(ph + la),
         c * sin(ph + la));
  } else if (ieq(m, "R")) {
    if (np < 1) goto badp;
    int k = (int)p[0];
    double re, im;
    phase(0, k < 0 ? -k : k, k < 0 ? -1 : 1, &re, &im);
    set2(u, 1, 0, 0, 0, 0, 0, re, im);
  } else if (ieq(m, "RZ")) {
    if (np < 1) goto badp;
    double h = 0.5 * p[0];
    set2(u, cos(h), -sin(h), 0, 0, 0, 0, cos(h), sin(h));
  } else if (ieq(m, "MAT")) {
    if (np < 8) goto badp;
    memcpy(u, p, 8 * sizeof(double));
  } else if (ieq(m, "CNOT")) {
    need_q = 2;
    set2(u, 0, 0, 1, 0, 1, 0, 0, 0);
  } else if (ieq(m, "U")) {
    need_q = 2; if (np < 1) goto badp;
    int k = (int)p[0];
    double re, im;
    phase(0, k < 0 ? -k : k, k < 0 ? -1 : 1, &re, &im);
    set2(u, 1, 0, 0, 0, 0, 0, re, im);
  } else if (ieq(m, "TOFFOLI") || ieq(m, "CCX")) {
    need_q = 3;
    set2(u, 0, 0, 1, 0, 1, 0, 0, 0);
  } else if (ieq(m, "CMAT")) {
    if (np < 8) goto badp;
    if (nq < 1 || nq > 3) { qs_set_error("gate_std: CMAT takes 1..3 qubits"); return QS_EINVAL; }
    need_q = nq;
    memcpy(u, p, 8 * sizeof(double));
  } else {
    qs_set_error("gate_std: unknown mnemonic '%s'", m);
    return QS_EINVAL;
  }
  if (nq != need_q) { qs_set_error("gate_std: '%s' takes %d qubit(s), got %d", m, need_q, nq); return QS_EINVAL; }
  g.nc = need_q - 1;
  for (int i = 0; i < g.nc; ++i) g.controls[i] = q[i];
  g.target = q[need_q - 1];
  *out = g;
  return QS_OK;
badp:
  qs_set_error("gate_std: '%s' needs more parameters", m);
  return QS_EINVAL;
}
