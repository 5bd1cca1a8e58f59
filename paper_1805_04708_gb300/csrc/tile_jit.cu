// Tile passes compiled at run time.
//
// The interpreter (k_tile2) reads the structure of every op of a pass (its
// type, kind, register slot or lane bit, control masks, fold flag) from the
// kernel parameters and dispatches on it for every tile.  Here the structure
// of a complex64 pass is written into the source of a kernel as constants
// and compiled with NVRTC for sm_103a: the op loop of the same device code
// (tile_core.cuh) unrolls completely and every branch on the structure folds
// away, leaving straight-line arithmetic.  The coefficients stay in the
// parameters, so passes of the same structure share one compiled kernel.
// A variant adds a CTA barrier every few ops (long passes outgrow the
// instruction cache; warps kept together share the lines they fetch).
//
// circuit_run mode 2 picks, per pass structure, among the interpreter and
// three compiled variants by timing each once with CUDA events (a pass's
// duration does not depend on the amplitudes, only on its structure) and
// then keeps the fastest.
//
// NVRTC is loaded with dlopen on first use; without it the compiled path
// reports itself unavailable and the interpreter runs the passes.
#include "internal.cuh"
#include "tile_core.cuh"
#include "tile_jit.h"
#include <nvrtc.h>
#include <dlfcn.h>
#include <stdio.h>
#include <string.h>
#include <atomic>
#include <mutex>
#include <thread>
#include <string>
#include <unordered_map>
#include <vector>

#include "jit_core.inc"   // kJitCore: gatekind.h, cplx.cuh and tile_core.cuh as text

using namespace qs_tile;

namespace {

struct Nvrtc {
  bool ok = false;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*log_size)(nvrtcProgram, size_t*);
  nvrtcResult (*log)(nvrtcProgram, char*);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
  nvrtcResult (*cubin)(nvrtcProgram, char*);
  nvrtcResult (*destroy)(nvrtcProgram*);
};

Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
    void* h = nullptr;
    for (const char* nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) return;
    n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
    n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
    n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
    n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
    n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
    n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
    n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
  });
  return n;
}

struct Entry {
  std::vector<char> cubin;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  size_t smem_set = 0;
};

std::mutex g_mu;   // guards the cache, the compile count and kernel loading
std::unordered_map<std::string, Entry>& cache() {
  static std::unordered_map<std::string, Entry> c;
  return c;
}
long g_compiles = 0;

// The structure of the pass as a compile-time program (sync: barrier every
// `sync` ops, 0 for none).
std::string program_of(const TileParams2& P, int sync) {
  std::string s;
  char buf[256];
  snprintf(buf, sizeof buf, "struct ProgJ {\n  static constexpr int kN = %d;\n  static constexpr int kSync = %d;\n",
           P.nops, sync);
  s += buf;
  s += "  static __device__ __forceinline__ OpS s(const TileParams2&, int i) {\n    switch (i) {\n";
  for (int i = 0; i < P.nops; ++i) {
    const TOp& o = P.ops[i];
    snprintf(buf, sizeof buf,
             "      case %d: return OpS{%u, %u, %u, %u, %u, {%u, %u, %u}, %uu, %uu, %lluull, %lluull};\n", i,
             (unsigned)o.type, (unsigned)o.kind, (unsigned)o.c0, (unsigned)o.c1, (unsigned)o.a, (unsigned)o.pad[0],
             (unsigned)o.pad[1], (unsigned)o.pad[2],
             (unsigned)o.smask, (unsigned)o.tmask, (unsigned long long)o.gmask, (unsigned long long)o.gtbit);
    s += buf;
  }
  s += "      default: return OpS{};\n    }\n  }\n};\n";
  return s;
}

std::string source_of(const std::string& prog) {
  std::string s =
      "#define QS_JIT 1\n"
      "typedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\n"
      "typedef unsigned int uint32_t;\ntypedef unsigned long long uint64_t;\n";
  s += kJitCore;
  s += "\nnamespace qs_tile {\n";
  s += prog;
  s += "}  // namespace qs_tile\n"
       "extern \"C\" __global__ void __launch_bounds__(256, 2)\n"
       "qs_tile_pass_c64(void* s, const __grid_constant__ qs_tile::TileParams2 P) {\n"
       "  qs_tile::tile_pass<float, 5, 3, qs_tile::ProgJ>(s, P);\n"
       "}\n";
  return s;
}

qs_status compile_prog(const std::string& prog, Entry& e) {
  Nvrtc& n = nvrtc();
  if (!n.ok) {
    qs_set_error("compiled tile passes: NVRTC is not available");
    return QS_EUNSUPPORTED;
  }
  const std::string src = source_of(prog);
  nvrtcProgram p;
  if (n.create(&p, src.c_str(), "qs_tile_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    qs_set_error("compiled tile passes: nvrtcCreateProgram failed");
    return QS_ECUDA;
  }
  const char* opts[] = {"-arch=sm_103a", "-std=c++17"};
  const nvrtcResult r = n.compile(p, 2, opts);
  if (r != NVRTC_SUCCESS) {
    size_t ls = 0;
    n.log_size(p, &ls);
    std::string log(ls + 1, '\0');
    n.log(p, &log[0]);
    n.destroy(&p);
    qs_set_error("compiled tile passes: NVRTC failed: %.900s", log.c_str());
    return QS_ECUDA;
  }
  size_t cs = 0;
  n.cubin_size(p, &cs);
  e.cubin.resize(cs);
  n.cubin(p, e.cubin.data());
  n.destroy(&p);
  std::lock_guard<std::mutex> g(g_mu);
  ++g_compiles;
  return QS_OK;
}

// The cache entry of a pass's structure, compiled if new.  The compile runs
// outside the lock, so several passes can compile at once; if two threads
// compile the same structure, the first result is kept.
qs_status entry_of(const TileParams2& P, int sync, Entry** out) {
  const std::string prog = program_of(P, sync);
  {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = cache().find(prog);
    if (it != cache().end()) {
      *out = &it->second;
      return QS_OK;
    }
  }
  Entry e;
  QS_TRY(compile_prog(prog, e));
  std::lock_guard<std::mutex> g(g_mu);
  auto it = cache().emplace(prog, std::move(e)).first;   // unordered_map: references stay valid
  *out = &it->second;
  return QS_OK;
}

}  // namespace

bool tile_jit_available() { return nvrtc().ok; }

long tile_jit_compiles() {
  std::lock_guard<std::mutex> g(g_mu);
  return g_compiles;
}

qs_status tile_jit_compile(const TileParams2& P, int sync) {
  Entry* e;
  return entry_of(P, sync, &e);
}

qs_status tile_jit_compile_all(const std::vector<JitJob>& passes) {
  const size_t n = passes.size();
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 4;
  if (nt > 16) nt = 16;
  if (nt > n) nt = (unsigned)n;
  std::atomic<size_t> next(0);
  std::atomic<int> status((int)QS_OK);
  auto work = [&] {
    for (size_t i; (i = next.fetch_add(1)) < n;) {
      const qs_status st = tile_jit_compile(passes[i].P, passes[i].sync);
      if (st != QS_OK) status.store((int)st);
    }
  };
  std::vector<std::thread> th;
  for (unsigned t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return (qs_status)status.load();
}

qs_status tile_jit_launch(qs_sim* s, const TileParams2& P, int sync, unsigned grid, size_t smem) {
  Entry* e;
  QS_TRY(entry_of(P, sync, &e));
  cudaKernel_t k;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!e->lib) {
      QS_CUDA(cudaLibraryLoadData(&e->lib, e->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
      QS_CUDA(cudaLibraryGetKernel(&e->kern, e->lib, "qs_tile_pass_c64"));
    }
    if (e->smem_set < smem) {
      QS_CUDA(cudaFuncSetAttribute((const void*)e->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      e->smem_set = smem;
    }
    k = e->kern;
  }
  void* state = s->state;
  void* args[] = {&state, (void*)&P};
  QS_CUDA(cudaLaunchKernel((const void*)k, dim3(grid), dim3(TPB), args, smem, s->stream));
  return QS_OK;
}

// ---- online choice of the pass kernel (circuit_run mode 2) --------------------
namespace {
// Every candidate is timed in kTuneRounds launches (slot n runs candidate
// n % kTileCands); a candidate's time is the fastest of its launches, so one
// slow sample (a cold instruction cache, a clock step) does not decide.
constexpr int kTuneRounds = 2;
constexpr int kTuneSlots = kTileCands * kTuneRounds;
struct Tune {
  int next = 0, best = -1;
  bool launched[kTuneSlots] = {}, done[kTuneSlots] = {}, failed[kTileCands] = {};
  float ms[kTuneSlots] = {};
  cudaEvent_t ev[kTuneSlots][2] = {};
};
std::unordered_map<std::string, Tune>& tunes() {
  static std::unordered_map<std::string, Tune> t;
  return t;
}
// fastest sample of candidate c so far, or a huge time
float cand_ms(const Tune& t, int c) {
  float m = 3.0e38f;
  if (t.failed[c]) return m;
  for (int n = c; n < kTuneSlots; n += kTileCands)
    if (t.done[n] && t.ms[n] < m) m = t.ms[n];
  return m;
}
}  // namespace

const int kTileCandSync[kTileCands] = {0, 0, 2, 8};

qs_status tile_tune_pick(qs_sim* s, const TileParams2& P, int* cand, cudaEvent_t* end_ev) {
  *end_ev = nullptr;
  std::lock_guard<std::mutex> g(g_mu);
  Tune& t = tunes()[program_of(P, -1)];
  if (t.best < 0) {
    bool all = true;
    for (int n = 0; n < kTuneSlots; ++n) {
      if (t.launched[n] && !t.done[n] && cudaEventQuery(t.ev[n][1]) == cudaSuccess) {
        QS_CUDA(cudaEventElapsedTime(&t.ms[n], t.ev[n][0], t.ev[n][1]));
        t.done[n] = true;
      }
      all = all && (t.done[n] || t.failed[n % kTileCands]);
    }
    if (all) {
      t.best = 0;
      for (int c = 1; c < kTileCands; ++c)
        if (cand_ms(t, c) < cand_ms(t, t.best)) t.best = c;
    }
  }
  if (t.best >= 0) {
    *cand = t.best;
    return QS_OK;
  }
  while (t.next < kTuneSlots && t.failed[t.next % kTileCands]) ++t.next;
  if (t.next < kTuneSlots) {
    const int n = t.next++;
    if (!t.ev[n][0]) {
      QS_CUDA(cudaEventCreate(&t.ev[n][0]));
      QS_CUDA(cudaEventCreate(&t.ev[n][1]));
    }
    QS_CUDA(cudaEventRecord(t.ev[n][0], s->stream));
    t.launched[n] = true;
    *cand = n % kTileCands;
    *end_ev = t.ev[n][1];
    return QS_OK;
  }
  // every slot launched, some still running: the fastest measured so far
  int best = 0;
  for (int c = 1; c < kTileCands; ++c)
    if (cand_ms(t, c) < cand_ms(t, best)) best = c;
  *cand = best;
  return QS_OK;
}

void tile_tune_fail(const TileParams2& P, int cand) {
  std::lock_guard<std::mutex> g(g_mu);
  Tune& t = tunes()[program_of(P, -1)];
  t.failed[cand] = true;
}
