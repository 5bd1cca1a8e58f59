// Adaptive 2-byte encoding (Sec. 4.1) -- kernels.
#include "internal.cuh"

qs_status a2_apply_u2(qs_sim* s, const int* controls, int nc, int target, const double u[8]) {
  (void)s; (void)controls; (void)nc; (void)target; (void)u;
  qs_set_error("ADAPT2 gates not built yet");
  return QS_EUNSUPPORTED;
}
qs_status a2_norm(qs_sim* s, double* out) { (void)s; (void)out; return QS_EUNSUPPORTED; }
qs_status a2_expect(qs_sim* s, double* qx, double* qy, double* qz) { (void)s; (void)qx; (void)qy; (void)qz; return QS_EUNSUPPORTED; }
qs_status a2_marginal(qs_sim* s, const int* q, int nq, double* out) { (void)s; (void)q; (void)nq; (void)out; return QS_EUNSUPPORTED; }
qs_status a2_shorbox(qs_sim* s, int nx, uint64_t G, uint64_t y) { return launch_shorbox(s, nx, G, y); }
qs_status a2_reset(qs_sim* s) { return launch_reset(s); }
