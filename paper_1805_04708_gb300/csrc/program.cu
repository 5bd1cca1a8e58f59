// Front-end for the instruction language of Appendix A: parses a program
// (QUBITS, BIT ASSIGNMENT, the gate mnemonics, BEGIN MEASUREMENT, M, CLEAR,
// SET, SHORBOX, DEPOLARIZING CHANNEL, GENERATE EVENTS, EXIT) and runs it on a
// state handle through the library's own calls.  Host code only: every step
// that touches the amplitudes is one of the library's kernels.
//
// Consecutive gate instructions are collected and run as one circuit_run, so
// the tile planner sees whole gate runs.  BIT ASSIGNMENT renumbers where the
// qubits are stored: logical qubit k lives in index bit perm[k] from then on;
// every result is reported per logical qubit.  Before any gate the
// renumbering moves nothing (the state is |0..0>); later it permutes the
// stored amplitudes (permute_qubits).  GENERATE EVENTS first moves the qubits
// back to their own bits, so that the inverse CDF walks the logical index
// order and the events do not depend on the renumbering.
//
// Seeds (the paper takes the system's value for a seed <= 0; here the run's
// seed stands in, so runs repeat): M number m draws qs_uniforms(run_seed, m);
// GENERATE EVENTS e s draws qs_uniforms(s > 0 ? s : run_seed + 1, k) for event
// k; DEPOLARIZING CHANNEL ... SEED = s draws with seed s > 0 ? s : run_seed + 2
// and counter g N + q for gate operation g (counted from the start of the
// program) and logical qubit q.
#include "internal.cuh"
#include <ctype.h>
#include <stdlib.h>
#include <string.h>
#include <string>
#include <vector>

struct ProgInstr {
  int op;                 // PI_*
  qs_gate gate;           // PI_GATE (logical qubits)
  int q;                  // M / CLEAR / SET
  int perm[64];           // BIT ASSIGNMENT
  double px, py, pz;      // DEPOLARIZING CHANNEL
  long long seed;         // DEPOLARIZING CHANNEL / GENERATE EVENTS
  long long nev;          // GENERATE EVENTS
  int nx;                 // SHORBOX
  unsigned long long G, y;
  int line;
};
enum { PI_GATE, PI_BITASSIGN, PI_BEGIN, PI_M, PI_CLEAR, PI_SET, PI_SHORBOX, PI_DEPOL, PI_EVENTS, PI_EXIT };

struct qs_program {
  int N;
  std::vector<ProgInstr> ins;
  // results of the last run
  std::vector<double> expect;           // 3N per BEGIN MEASUREMENT: qx, qy, qz
  std::vector<int> m_qubit, m_outcome;  // per M (logical qubit)
  std::vector<double> m_probs;          // p0, p1 per M
  std::vector<uint64_t> events;
  std::vector<double> proj_prob;        // per CLEAR / SET
};

namespace {

std::string upper(const std::string& s) {
  std::string r = s;
  for (auto& c : r) c = (char)toupper((unsigned char)c);
  return r;
}
std::vector<std::string> split(const std::string& s) {
  std::vector<std::string> t;
  size_t i = 0;
  while (i < s.size()) {
    while (i < s.size() && (isspace((unsigned char)s[i]) || s[i] == ',')) ++i;
    size_t j = i;
    while (j < s.size() && !isspace((unsigned char)s[j]) && s[j] != ',') ++j;
    if (j > i) t.push_back(s.substr(i, j - i));
    i = j;
  }
  return t;
}
bool to_int(const std::string& s, long long* v) {
  if (s.empty()) return false;
  char* e = nullptr;
  *v = strtoll(s.c_str(), &e, 10);
  return *e == 0;
}
bool to_num(const std::string& s, double* v) {
  if (s.empty()) return false;
  char* e = nullptr;
  *v = strtod(s.c_str(), &e);
  return *e == 0;
}

struct GateSpec { const char* name; int nq, np; };
const GateSpec kGates[] = {
    {"I", 1, 0}, {"H", 1, 0}, {"X", 1, 0}, {"Y", 1, 0}, {"Z", 1, 0}, {"S", 1, 0}, {"S+", 1, 0},
    {"T", 1, 0}, {"T+", 1, 0}, {"U1", 1, 1}, {"U2", 1, 2}, {"U3", 1, 3}, {"+X", 1, 0}, {"-X", 1, 0},
    {"+Y", 1, 0}, {"-Y", 1, 0}, {"R", 1, 1}, {"RZ", 1, 1}, {"CNOT", 2, 0}, {"U", 2, 1}, {"TOFFOLI", 3, 0}};

qs_status fail(int line, const char* what, const std::string& text) {
  qs_set_error("program line %d: %s (%s)", line, what, text.c_str());
  return QS_EINVAL;
}

// DEPOLARIZING CHANNEL arguments: KEY = value pairs in any order
bool parse_depol(const std::string& up, ProgInstr* in) {
  in->px = in->py = in->pz = 0.0;
  in->seed = 0;
  const char* keys[4] = {"P_X", "P_Y", "P_Z", "SEED"};
  std::string rest = up.substr(strlen("DEPOLARIZING CHANNEL"));
  for (auto& c : rest)
    if (c == '=' || c == ',') c = ' ';
  auto t = split(rest);
  if (t.size() % 2) return false;
  for (size_t i = 0; i < t.size(); i += 2) {
    int k = -1;
    for (int j = 0; j < 4; ++j)
      if (t[i] == keys[j]) k = j;
    if (k < 0) return false;
    if (k == 3) {
      double d;
      if (!to_num(t[i + 1], &d)) return false;
      in->seed = (long long)d;
    } else {
      double d;
      if (!to_num(t[i + 1], &d)) return false;
      (k == 0 ? in->px : k == 1 ? in->py : in->pz) = d;
    }
  }
  return in->px >= 0 && in->py >= 0 && in->pz >= 0 && in->px + in->py + in->pz <= 1.0;
}

}  // namespace

extern "C" qs_status program_parse(const char* text, qs_program** out) {
  if (!text || !out) { qs_set_error("program_parse: null argument"); return QS_EINVAL; }
  *out = nullptr;
  qs_program* p = new qs_program();
  p->N = 0;
  std::string src(text);
  size_t pos = 0;
  int line = 0;
  qs_status st = QS_OK;
  while (pos <= src.size() && st == QS_OK) {
    size_t nl = src.find('\n', pos);
    if (nl == std::string::npos) nl = src.size();
    std::string raw = src.substr(pos, nl - pos);
    pos = nl + 1;
    ++line;
    std::string body = raw.substr(0, raw.find('!'));
    std::string up = upper(body);
    auto t = split(up);
    if (t.empty()) continue;
    ProgInstr in;
    memset(&in, 0, sizeof in);
    in.line = line;
    if (t[0] == "QUBITS") {
      long long n;
      if (p->N != 0 || t.size() != 2 || !to_int(t[1], &n) || n <= 1 || n >= 64) {
        st = fail(line, "QUBITS N must come first, once, with 1 < N < 64", raw);
        break;
      }
      p->N = (int)n;
      continue;
    }
    if (p->N == 0) { st = fail(line, "QUBITS must be the first instruction", raw); break; }
    const int N = p->N;
    auto qubit = [&](const std::string& s, int* q) {
      long long v;
      if (!to_int(s, &v) || v < 0 || v >= N) return false;
      *q = (int)v;
      return true;
    };
    if (t.size() >= 2 && t[0] == "BIT" && t[1] == "ASSIGNMENT") {
      if ((int)t.size() != 2 + N) { st = fail(line, "BIT ASSIGNMENT needs N qubit numbers", raw); break; }
      uint64_t seen = 0;
      for (int k = 0; k < N && st == QS_OK; ++k) {
        if (!qubit(t[2 + k], &in.perm[k]) || ((seen >> in.perm[k]) & 1)) st = fail(line, "not a permutation", raw);
        seen |= 1ull << in.perm[k];
      }
      in.op = PI_BITASSIGN;
    } else if (t.size() == 2 && t[0] == "BEGIN" && t[1] == "MEASUREMENT") {
      in.op = PI_BEGIN;
    } else if (t.size() >= 3 && t[0] == "GENERATE" && t[1] == "EVENTS") {
      if (t.size() > 4 || !to_int(t[2], &in.nev) || in.nev < 1 || in.nev > (1ll << 31) ||
          (t.size() == 4 && !to_int(t[3], &in.seed))) {
        st = fail(line, "GENERATE EVENTS events [seed]", raw);
        break;
      }
      in.op = PI_EVENTS;
    } else if (t.size() >= 2 && t[0] == "DEPOLARIZING" && t[1] == "CHANNEL") {
      if (!parse_depol(up, &in)) { st = fail(line, "bad DEPOLARIZING CHANNEL arguments", raw); break; }
      in.op = PI_DEPOL;
    } else if (t[0] == "M" || t[0] == "CLEAR" || t[0] == "SET") {
      if (t.size() != 2 || !qubit(t[1], &in.q)) { st = fail(line, "needs one qubit in range", raw); break; }
      in.op = t[0] == "M" ? PI_M : (t[0] == "CLEAR" ? PI_CLEAR : PI_SET);
    } else if (t[0] == "SHORBOX") {
      long long nx, G, y;
      if (t.size() != 4 || !to_int(t[1], &nx) || !to_int(t[2], &G) || !to_int(t[3], &y) || nx < 1 || nx >= N ||
          G < 2 || y < 1 || y >= G || (unsigned long long)G > (1ull << (N - nx))) {
        st = fail(line, "SHORBOX n_x G y", raw);
        break;
      }
      in.op = PI_SHORBOX;
      in.nx = (int)nx; in.G = (unsigned long long)G; in.y = (unsigned long long)y;
    } else if (t[0] == "EXIT") {
      in.op = PI_EXIT;
    } else {
      const GateSpec* g = nullptr;
      for (const auto& k : kGates)
        if (t[0] == k.name) g = &k;
      if (!g) { st = fail(line, "unknown instruction", raw); break; }
      if ((int)t.size() != 1 + g->nq + g->np) { st = fail(line, "wrong number of operands", raw); break; }
      int qs[3];
      double ps[3];
      for (int k = 0; k < g->nq && st == QS_OK; ++k) {
        if (!qubit(t[1 + k], &qs[k])) st = fail(line, "qubit out of range", raw);
        for (int j = 0; j < k && st == QS_OK; ++j)
          if (qs[j] == qs[k]) st = fail(line, "qubit repeated", raw);
      }
      for (int k = 0; k < g->np && st == QS_OK; ++k)
        if (!to_num(t[1 + g->nq + k], &ps[k])) st = fail(line, "bad number", raw);
      if (st != QS_OK) break;
      if (gate_std(g->name, qs, g->nq, ps, g->np, &in.gate) != QS_OK) {
        st = fail(line, qs_last_error_string(), raw);
        break;
      }
      in.op = PI_GATE;
    }
    if (st == QS_OK) p->ins.push_back(in);
  }
  if (st == QS_OK && p->N == 0) {
    qs_set_error("program_parse: no QUBITS instruction");
    st = QS_EINVAL;
  }
  if (st != QS_OK) {
    delete p;
    return st;
  }
  *out = p;
  return QS_OK;
}

extern "C" qs_status program_destroy(qs_program* p) {
  delete p;
  return QS_OK;
}

extern "C" qs_status program_info(const qs_program* p, int* N, int* n_instr) {
  if (!p) { qs_set_error("program_info: null program"); return QS_EINVAL; }
  if (N) *N = p->N;
  if (n_instr) *n_instr = (int)p->ins.size();
  return QS_OK;
}

// ---- qubit permutation of the stored state ------------------------------------------------
extern "C" qs_status permute_qubits(qs_sim* s, const int* perm) {
  if (!s || !perm) { qs_set_error("permute_qubits: null argument"); return QS_EINVAL; }
  const int N = s->N;
  uint64_t seen = 0;
  for (int k = 0; k < N; ++k) {
    if (perm[k] < 0 || perm[k] >= N || ((seen >> perm[k]) & 1)) {
      qs_set_error("permute_qubits: not a permutation of 0..%d", N - 1);
      return QS_EINVAL;
    }
    seen |= 1ull << perm[k];
  }
  // the content of bit k moves to bit perm[k]: follow each cycle with
  // transpositions, each a SWAP = three CNOTs (pure amplitude moves)
  std::vector<qs_gate> g;
  int cur[64];   // cur[b]: which original bit's content is now at bit b
  int where[64]; // where[k]: current bit of original bit k
  for (int k = 0; k < N; ++k) { cur[k] = k; where[k] = k; }
  auto cnot = [&](int c, int t) {
    qs_gate x;
    memset(&x, 0, sizeof x);
    x.nc = 1; x.controls[0] = c; x.target = t;
    x.u[2] = 1.0; x.u[4] = 1.0;
    g.push_back(x);
  };
  for (int k = 0; k < N; ++k) {
    const int a = where[k], b = perm[k];
    if (a == b) continue;
    cnot(a, b); cnot(b, a); cnot(a, b);
    const int ob = cur[b];
    cur[b] = k; where[k] = b;
    cur[a] = ob; where[ob] = a;
  }
  if (g.empty()) return QS_OK;
  return circuit_run(s, g.data(), (int)g.size(), s->enc == QS_ADAPT2 ? 0 : 1, nullptr);
}

extern "C" qs_status program_run(qs_program* p, qs_sim* s, uint64_t run_seed, int mode) {
  if (!p || !s) { qs_set_error("program_run: null argument"); return QS_EINVAL; }
  if (s->N != p->N) { qs_set_error("program_run: the program needs %d qubits, the state has %d", p->N, s->N); return QS_EINVAL; }
  if (mode < 0 || mode > 3) { qs_set_error("program_run: mode %d not in 0..3", mode); return QS_EINVAL; }
  if (s->enc == QS_ADAPT2) mode = 0;
  const int N = p->N;
  p->expect.clear(); p->m_qubit.clear(); p->m_outcome.clear(); p->m_probs.clear();
  p->events.clear(); p->proj_prob.clear();
  QS_TRY(sim_reset(s));
  int map[64];                   // logical qubit -> index bit
  for (int k = 0; k < N; ++k) map[k] = k;
  bool any_gate = false;
  bool noisy = false;
  double px = 0, py = 0, pz = 0;
  uint64_t nseed = 0;
  long long ngate = 0;           // gate operations executed
  uint64_t nmeas = 0;
  std::vector<qs_gate> pending;  // logical gate records waiting to run
  std::vector<qs_gate> buf;

  auto relabel = [&](qs_gate g) {
    for (int i = 0; i < g.nc; ++i) g.controls[i] = map[g.controls[i]];
    g.target = map[g.target];
    return g;
  };
  auto flush = [&]() -> qs_status {
    if (pending.empty()) return QS_OK;
    const qs_gate* src = pending.data();
    int n = (int)pending.size();
    if (noisy) {
      int need = 0;
      QS_TRY(depolarize_circuit(N, pending.data(), n, px, py, pz, nseed, ngate, nullptr, 0, &need));
      buf.resize(need);
      QS_TRY(depolarize_circuit(N, pending.data(), n, px, py, pz, nseed, ngate, buf.data(), need, &need));
      src = buf.data();
      n = need;
    }
    std::vector<qs_gate> phys(n);
    for (int i = 0; i < n; ++i) phys[i] = relabel(src[i]);
    ngate += (long long)pending.size();
    pending.clear();
    any_gate = true;
    return circuit_run(s, phys.data(), n, mode, nullptr);
  };
  auto measure_all = [&]() -> qs_status {
    std::vector<double> x(N), y(N), z(N);
    QS_TRY(expect_xyz(s, x.data(), y.data(), z.data()));
    for (int k = 0; k < N; ++k) p->expect.push_back(x[map[k]]);
    for (int k = 0; k < N; ++k) p->expect.push_back(y[map[k]]);
    for (int k = 0; k < N; ++k) p->expect.push_back(z[map[k]]);
    return QS_OK;
  };

  for (const ProgInstr& in : p->ins) {
    if (in.op == PI_GATE) {
      pending.push_back(in.gate);
      continue;
    }
    QS_TRY(flush());
    switch (in.op) {
      case PI_BITASSIGN: {
        if (any_gate) {   // move the stored qubits to their new bits
          int sigma[64];
          for (int k = 0; k < N; ++k) sigma[map[k]] = in.perm[k];
          QS_TRY(permute_qubits(s, sigma));
        }
        for (int k = 0; k < N; ++k) map[k] = in.perm[k];
        break;
      }
      case PI_DEPOL:
        noisy = in.px + in.py + in.pz > 0;
        px = in.px; py = in.py; pz = in.pz;
        nseed = in.seed > 0 ? (uint64_t)in.seed : run_seed + 2;
        break;
      case PI_BEGIN:
        QS_TRY(measure_all());
        break;
      case PI_M: {
        double u, pr[2];
        int o;
        QS_TRY(qs_uniforms(run_seed, nmeas++, 1, &u));
        QS_TRY(measure_qubit(s, map[in.q], u, &o, pr));
        p->m_qubit.push_back(in.q);
        p->m_outcome.push_back(o);
        p->m_probs.push_back(pr[0]);
        p->m_probs.push_back(pr[1]);
        any_gate = true;
        break;
      }
      case PI_CLEAR:
      case PI_SET: {
        double pr;
        qs_status st = project_qubit(s, map[in.q], in.op == PI_SET ? 1 : 0, &pr);
        if (st != QS_OK) {
          qs_set_error("program line %d: %s", in.line, qs_last_error_string());
          return st;
        }
        p->proj_prob.push_back(pr);
        any_gate = true;
        break;
      }
      case PI_SHORBOX: {
        QS_TRY(shorbox_init(s, in.nx, in.G, in.y));
        bool ident = true;
        for (int k = 0; k < N; ++k) ident &= (map[k] == k);
        if (!ident) QS_TRY(permute_qubits(s, map));
        any_gate = true;
        break;
      }
      case PI_EVENTS: {
        // the inverse CDF walks the index order: sample with the qubits back
        // in their logical bits, so the events do not depend on the
        // renumbering (the run ends here)
        bool ident = true;
        for (int k = 0; k < N; ++k) ident &= (map[k] == k);
        if (!ident) {
          int sigma[64];
          for (int k = 0; k < N; ++k) sigma[map[k]] = k;
          QS_TRY(permute_qubits(s, sigma));
          for (int k = 0; k < N; ++k) map[k] = k;
        }
        const uint64_t es = in.seed > 0 ? (uint64_t)in.seed : run_seed + 1;
        p->events.assign(in.nev, 0);
        return generate_events_seeded(s, es, in.nev, p->events.data());
      }
      case PI_EXIT:
        return measure_all();
      default:
        break;
    }
  }
  return flush();
}

extern "C" qs_status program_results(const qs_program* p, int* n_measurements, int* n_m, int* n_proj,
                                     int64_t* n_events) {
  if (!p) { qs_set_error("program_results: null program"); return QS_EINVAL; }
  if (n_measurements) *n_measurements = p->N ? (int)(p->expect.size() / (3 * (size_t)p->N)) : 0;
  if (n_m) *n_m = (int)p->m_qubit.size();
  if (n_proj) *n_proj = (int)p->proj_prob.size();
  if (n_events) *n_events = (int64_t)p->events.size();
  return QS_OK;
}

extern "C" qs_status program_expectations(const qs_program* p, int k, double* qx, double* qy, double* qz) {
  if (!p || !qx || !qy || !qz) { qs_set_error("program_expectations: null argument"); return QS_EINVAL; }
  const size_t per = 3 * (size_t)p->N;
  if (k < 0 || (size_t)(k + 1) * per > p->expect.size()) {
    qs_set_error("program_expectations: no measurement %d", k);
    return QS_EINVAL;
  }
  const double* e = p->expect.data() + k * per;
  memcpy(qx, e, p->N * sizeof(double));
  memcpy(qy, e + p->N, p->N * sizeof(double));
  memcpy(qz, e + 2 * p->N, p->N * sizeof(double));
  return QS_OK;
}

extern "C" qs_status program_outcomes(const qs_program* p, int* qubits, int* outcomes, double* probs,
                                      double* proj_probs) {
  if (!p) { qs_set_error("program_outcomes: null program"); return QS_EINVAL; }
  for (size_t i = 0; i < p->m_qubit.size(); ++i) {
    if (qubits) qubits[i] = p->m_qubit[i];
    if (outcomes) outcomes[i] = p->m_outcome[i];
    if (probs) { probs[2 * i] = p->m_probs[2 * i]; probs[2 * i + 1] = p->m_probs[2 * i + 1]; }
  }
  if (proj_probs)
    for (size_t i = 0; i < p->proj_prob.size(); ++i) proj_probs[i] = p->proj_prob[i];
  return QS_OK;
}

extern "C" qs_status program_events(const qs_program* p, uint64_t* events) {
  if (!p || (!events && !p->events.empty())) { qs_set_error("program_events: null argument"); return QS_EINVAL; }
  if (!p->events.empty()) memcpy(events, p->events.data(), p->events.size() * sizeof(uint64_t));
  return QS_OK;
}
