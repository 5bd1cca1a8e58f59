// Serving loop with continuous batching (native scheduler).
//
// Requests (circuits of mixed qubit counts) arrive over time.  The loop
//  * admits the oldest waiting request once its state fits the device-memory
//    budget (first-fit allocator over one pooled allocation: admission by HBM
//    footprint), so requests join while others are in flight;
//  * advances every admitted request by up to `quantum` gates per tick:
//    small states (N <= small_max_n) all together in ONE launch that holds
//    each state in shared memory for its gate chunk (a new request starts
//    from |0..0> inside that launch, a finishing one computes its norm and
//    P(qubit = 1) there too); larger states run their chunk through the tile
//    planner on their own streams, so their work overlaps on the device;
//  * retires finished requests, frees their memory and records times.
// Each gate is the pair update of Eq. (NUM2); serving itself has no
// counterpart in the paper.
#include "internal.cuh"
#include "cplx.cuh"
#include "batch_common.cuh"
#include <chrono>
#include <map>
#include <vector>
#include <algorithm>
#include <stdlib.h>
#include <string.h>
#include <thread>

namespace {

constexpr int STPB = 256;

struct SmallEntry {
  float2* state;          // device
  const BGate<float>* gates;  // device, the request's whole gate list
  int N, g0, g1;          // gate range for this tick
  int fresh;              // start from |0..0>
  int final_;             // compute results after the chunk
  double* out;            // device: [norm, P1(0..N-1)]
};

__global__ void __launch_bounds__(STPB) k_serve_small(const SmallEntry* __restrict__ tab) {
  extern __shared__ unsigned char smraw[];
  Cx<float>* st = (Cx<float>*)smraw;
  __shared__ double red[32];
  const SmallEntry e = tab[blockIdx.x];
  const int n = 1 << e.N;
  if (e.fresh) {
    for (int i = threadIdx.x; i < n; i += STPB) st[i] = cx<float>(i == 0 ? 1.f : 0.f, 0.f);
  } else {
    for (int i = threadIdx.x; i < n; i += STPB) { float2 a = e.state[i]; st[i] = cx<float>(a.x, a.y); }
  }
  __syncthreads();
  for (int k = e.g0; k < e.g1; ++k) {
    apply_gate_range<float>(st, e.N, e.gates[k], threadIdx.x, STPB);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += STPB) e.state[i] = make_float2(st[i].x, st[i].y);
  if (!e.final_) return;
  // results: norm and P(qubit q = 1), FP64, fixed order
  for (int q = -1; q < e.N; ++q) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += STPB)
      if (q < 0 || ((i >> q) & 1)) acc += (double)st[i].x * st[i].x + (double)st[i].y * st[i].y;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (int w = 0; w < STPB / 32; ++w) r += red[w];
      e.out[q + 1] = r;
    }
    __syncthreads();
  }
}

// ---- persistent mode -------------------------------------------------------------------
// A work item: one small state and its next gate chunk.  Items live in a ring
// in host-mapped memory; the host fills an item, then publishes it by
// raising `tail` (release); a CTA claims the oldest published item with a
// CAS on the device counter `head`, runs it with the state in shared memory,
// writes the results (for a final chunk) and marks the ring slot done with
// the item's number (release, system scope).
struct __align__(128) WorkItem {   // one cache line per item, never shared
  float2* state;
  const BGate<float>* gates;
  double* res;                 // host-mapped: [norm, P1(0..N-1)] for a final chunk
  int N, g0, g1, fresh, final_;
  int pad[21];
};
struct QueueCtl {              // host-mapped
  unsigned long long tail;     // items published
  unsigned long long stop;     // nonzero: CTAs end at their next wait
  unsigned long long done[1];  // [ring]: number + 1 of the item finished in the slot
};

__device__ __forceinline__ unsigned long long ld_acq_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A persistent CTA may take chunk k + 1 of a state whose chunk k another SM
// wrote, and a pool region may hold a new request's gates: everything such a
// CTA reads that others wrote during the kernel's lifetime is loaded through
// L2 (ld.global.cg), never from this SM's L1, which is not coherent with the
// other SMs' writes.
__device__ __forceinline__ BGate<float> gate_cg(const BGate<float>* p) {
  static_assert(sizeof(BGate<float>) == 48, "gate record layout");
  const int4* q = (const int4*)p;
  int4 w[3] = {__ldcg(q), __ldcg(q + 1), __ldcg(q + 2)};
  BGate<float> g;
  memcpy(&g, w, sizeof g);
  return g;
}
// A work item lives in host memory the host rewrites: its words are read
// with system-scope strong loads, which observe the host's latest writes (a
// weak load may be served by a line an earlier read left in the GPU's
// caches).  The first 48 bytes hold the fields.
__device__ __forceinline__ WorkItem item_sys(const WorkItem* p) {
  static_assert(sizeof(WorkItem) == 128, "work item layout");
  WorkItem it;
  unsigned long long w[6];
  const unsigned long long* q = (const unsigned long long*)p;
#pragma unroll
  for (int i = 0; i < 6; ++i)
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(w[i]) : "l"(q + i) : "memory");
  memcpy(&it, w, sizeof w);
  return it;
}

__global__ void __launch_bounds__(STPB) k_serve_persist(const WorkItem* ring, unsigned ring_n, QueueCtl* ctl,
                                                        unsigned long long* head, unsigned long long wait_ns,
                                                        unsigned int* idle_exits, unsigned long long* taken) {
  extern __shared__ unsigned char smraw[];
  Cx<float>* st = (Cx<float>*)smraw;
  __shared__ double red[32];
  __shared__ long long my;
  __shared__ WorkItem it;
  for (;;) {
    if (threadIdx.x == 0) {
      // claim the oldest published item; wait at most wait_ns for one
      long long got = -1;
      const unsigned long long t0 = gtimer();
      for (;;) {
        const unsigned long long h = atomicAdd(head, 0ull);
        const unsigned long long t = ld_acq_sys(&ctl->tail);
        if (h < t) {
          if (atomicCAS(head, h, h + 1) == h) { got = (long long)h; break; }
          continue;
        }
        if (ld_acq_sys(&ctl->stop) || gtimer() - t0 > wait_ns) break;
        __nanosleep(1000);
      }
      my = got;
      if (got >= 0) {
        it = item_sys(ring + got % ring_n);
        atomicAdd(taken, 1ull);
      } else {
        atomicAdd(idle_exits, 1u);
      }
    }
    __syncthreads();
    if (my < 0) return;
    const int n = 1 << it.N;
    if (it.fresh) {
      for (int i = threadIdx.x; i < n; i += STPB) st[i] = cx<float>(i == 0 ? 1.f : 0.f, 0.f);
    } else {
      for (int i = threadIdx.x; i < n; i += STPB) { float2 a = __ldcg(it.state + i); st[i] = cx<float>(a.x, a.y); }
    }
    __syncthreads();
    for (int k = it.g0; k < it.g1; ++k) {
      apply_gate_range<float>(st, it.N, gate_cg(it.gates + k), threadIdx.x, STPB);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += STPB) __stcg(it.state + i, make_float2(st[i].x, st[i].y));
    if (it.final_) {
      for (int q = -1; q < it.N; ++q) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < n; i += STPB)
          if (q < 0 || ((i >> q) & 1)) acc += (double)st[i].x * st[i].x + (double)st[i].y * st[i].y;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
          double r = 0.0;
          for (int w = 0; w < STPB / 32; ++w) r += red[w];
          it.res[q + 1] = r;
        }
        __syncthreads();
      }
    }
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) st_rel_sys(&ctl->done[my % ring_n], (unsigned long long)my + 1);
    __syncthreads();
  }
}

// first-fit allocator over [0, size) with 256-byte granules
class Pool {
 public:
  explicit Pool(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
    }
  }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

struct Active {
  int id;
  bool small;
  size_t off, bytes;          // pool region of the state
  size_t goff, gbytes;        // pool region of the device gate list (small)
  int next;                   // next gate
  bool fresh;
  qs_sim* sim;                // large: handle over the pool region
  int stream;
};

}  // namespace

static qs_status serve_persistent(qs_request* reqs, int n, const qs_serve_config* cfg, qs_serve_stats* stats,
                                  int small_max, int quantum, int nstreams, size_t budget);

extern "C" qs_status serve_run(qs_request* reqs, int n, const qs_serve_config* cfg, qs_serve_stats* stats) {
  if (!reqs || n < 0 || !cfg) { qs_set_error("serve_run: null argument"); return QS_EINVAL; }
  const int small_max = cfg->small_max_n > 0 ? (cfg->small_max_n < 14 ? cfg->small_max_n : 14) : 14;
  const int quantum = cfg->quantum > 0 ? cfg->quantum : 64;
  const int nstreams = cfg->nstreams > 0 ? (cfg->nstreams < 16 ? cfg->nstreams : 16) : 4;
  const size_t budget = cfg->mem_budget;
  for (int i = 0; i < n; ++i) {
    const qs_request& r = reqs[i];
    if (r.N < 2 || r.N > 34 || r.ngates < 0 || (r.ngates > 0 && !r.gates) || !r.qz) {
      qs_set_error("serve_run: request %d malformed", i);
      return QS_EINVAL;
    }
    if (((size_t)8 << r.N) + (size_t)r.ngates * sizeof(BGate<float>) + 1024 > budget) {
      qs_set_error("serve_run: request %d (N = %d) does not fit the memory budget", i, r.N);
      return QS_ENOMEM;
    }
    if (i > 0 && r.arrival_s < reqs[i - 1].arrival_s) { qs_set_error("serve_run: arrivals must be sorted"); return QS_EINVAL; }
    for (int k = 0; k < r.ngates; ++k) {
      const qs_gate& g = r.gates[k];
      if (g.nc < 0 || g.nc > 2 || g.target < 0 || g.target >= r.N) { qs_set_error("serve_run: request %d gate %d", i, k); return QS_EINVAL; }
      for (int c = 0; c < g.nc; ++c)
        if (g.controls[c] < 0 || g.controls[c] >= r.N || g.controls[c] == g.target ||
            (c == 1 && g.controls[1] == g.controls[0])) {
          qs_set_error("serve_run: request %d gate %d: bad controls", i, k);
          return QS_EINVAL;
        }
      if (!(unitarity_defect(g.u, 2) <= 1e-10)) { qs_set_error("serve_run: request %d gate %d not unitary", i, k); return QS_ENOTUNITARY; }
    }
  }
  if (stats) memset(stats, 0, sizeof *stats);
  if (cfg->persistent) return serve_persistent(reqs, n, cfg, stats, small_max, quantum, nstreams, budget);
  // resources
  unsigned char* pool_base = nullptr;
  QS_CUDA(cudaMalloc(&pool_base, budget));
  Pool pool(budget);
  std::vector<cudaStream_t> streams(nstreams + 1);
  for (auto& s : streams) QS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  const int max_small = cfg->max_small > 0 ? cfg->max_small : 4096;
  SmallEntry* htab = nullptr;
  SmallEntry* dtab = nullptr;
  double* hres = nullptr;
  double* dres = nullptr;
  const size_t res_stride = 40;
  QS_CUDA(cudaMallocHost(&htab, sizeof(SmallEntry) * max_small));
  QS_CUDA(cudaMalloc(&dtab, sizeof(SmallEntry) * max_small));
  QS_CUDA(cudaMallocHost(&hres, sizeof(double) * res_stride * max_small));
  QS_CUDA(cudaMalloc(&dres, sizeof(double) * res_stride * max_small));
  QS_CUDA(cudaFuncSetAttribute(k_serve_small, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 << 14));

  std::vector<Active> active;
  std::vector<BGate<float>> hg;
  int next_arrival = 0, completed = 0, ticks = 0, max_active = 0;
  const uint64_t launches0 = qs_kernel_launches();
  const auto t0 = std::chrono::steady_clock::now();
  auto now_s = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  qs_status st = QS_OK;
  double busy = 0.0;
  while (completed < n && st == QS_OK) {
    // admission: oldest first, while the state and its gate list fit
    while (next_arrival < n && reqs[next_arrival].arrival_s <= now_s()) {
      qs_request& r = reqs[next_arrival];
      Active a;
      memset(&a, 0, sizeof a);
      a.id = next_arrival;
      a.small = r.N <= small_max;
      a.bytes = (size_t)8 << r.N;
      a.gbytes = a.small ? (size_t)r.ngates * sizeof(BGate<float>) : 0;
      if (!pool.alloc(a.bytes, &a.off)) break;
      if (a.small && a.gbytes && !pool.alloc(a.gbytes, &a.goff)) { pool.release(a.off, a.bytes); break; }
      a.fresh = true;
      a.stream = (int)(active.size() % nstreams) + 1;
      if (a.small && r.ngates) {
        hg.resize(r.ngates);
        for (int k = 0; k < r.ngates; ++k) {
          const qs_gate& g = r.gates[k];
          BGate<float>& o = hg[k];
          o.nc = g.nc; o.c0 = g.controls[0]; o.c1 = g.controls[1]; o.t = g.target;
          for (int j = 0; j < 8; ++j) o.u[j] = (float)g.u[j];
        }
        // on the stream of the small-state kernel, so the copy is ordered before
        // the launch that reads it (a pageable cudaMemcpy may return before
        // its DMA reaches the device)
        if (cudaMemcpyAsync(pool_base + a.goff, hg.data(), a.gbytes, cudaMemcpyHostToDevice, streams[0]) !=
            cudaSuccess) {
          qs_set_error("serve_run: gate upload failed");
          st = QS_ECUDA;
          break;
        }
      }
      if (!a.small) {
        st = sim_create_in(r.N, QS_C64, pool_base + a.off, a.bytes, (void*)streams[a.stream], &a.sim);
        if (st != QS_OK) break;
      }
      r.admit_s = now_s();
      active.push_back(a);
      ++next_arrival;
    }
    if (st != QS_OK) break;
    max_active = std::max(max_active, (int)active.size());
    if (active.empty()) {
      // idle until the next arrival
      const double wait = reqs[next_arrival].arrival_s - now_s();
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait < 1e-3 ? wait : 1e-3));
      continue;
    }
    const double tick_start = now_s();
    ++ticks;
    // small states: one launch for all
    int ns = 0, maxn = 2;
    std::vector<int> small_ids;
    for (auto& a : active) {
      if (!a.small || ns >= max_small) continue;
      const qs_request& r = reqs[a.id];
      SmallEntry& e = htab[ns];
      e.state = (float2*)(pool_base + a.off);
      e.gates = (const BGate<float>*)(pool_base + a.goff);
      e.N = r.N;
      e.g0 = a.next;
      e.g1 = std::min(r.ngates, a.next + quantum);
      e.fresh = a.fresh ? 1 : 0;
      e.final_ = (e.g1 == r.ngates) ? 1 : 0;
      e.out = dres + res_stride * ns;
      maxn = std::max(maxn, r.N);
      small_ids.push_back((int)(&a - active.data()));
      ++ns;
    }
    if (ns > 0) {
      QS_CUDA(cudaMemcpyAsync(dtab, htab, sizeof(SmallEntry) * ns, cudaMemcpyHostToDevice, streams[0]));
      k_serve_small<<<ns, STPB, (size_t)8 << maxn, streams[0]>>>(dtab);
      qs_count_launch();
      QS_CUDA(cudaGetLastError());
      QS_CUDA(cudaMemcpyAsync(hres, dres, sizeof(double) * res_stride * ns, cudaMemcpyDeviceToHost, streams[0]));
    }
    // large states: their chunk on their own streams
    for (auto& a : active) {
      if (a.small) continue;
      const qs_request& r = reqs[a.id];
      const int g1 = std::min(r.ngates, a.next + quantum);
      if (g1 > a.next) {
        st = circuit_run(a.sim, r.gates + a.next, g1 - a.next, 1, nullptr);
        if (st != QS_OK) break;
      }
    }
    if (st != QS_OK) break;
    for (auto& s : streams) QS_CUDA(cudaStreamSynchronize(s));
    // bookkeeping and retirement
    for (int k = 0; k < ns; ++k) {
      Active& a = active[small_ids[k]];
      const SmallEntry& e = htab[k];
      a.fresh = false;
      a.next = e.g1;
      if (e.final_) {
        qs_request& r = reqs[a.id];
        r.norm = hres[res_stride * k];
        for (int q = 0; q < r.N; ++q) r.qz[q] = hres[res_stride * k + 1 + q];
      }
    }
    for (auto& a : active) {
      if (a.small) continue;
      const qs_request& r = reqs[a.id];
      a.next = std::min(r.ngates, a.next + quantum);
    }
    std::vector<Active> keep;
    for (auto& a : active) {
      qs_request& r = reqs[a.id];
      if (a.next < r.ngates || (a.small && a.fresh)) { keep.push_back(a); continue; }
      if (!a.small) {
        std::vector<double> qx(r.N), qy(r.N);
        st = expect_xyz(a.sim, qx.data(), qy.data(), r.qz);
        if (st == QS_OK) st = sim_norm(a.sim, &r.norm);
        sim_destroy(a.sim);
        if (st != QS_OK) break;
      }
      r.finish_s = now_s();
      pool.release(a.off, a.bytes);
      if (a.gbytes) pool.release(a.goff, a.gbytes);
      ++completed;
    }
    active.swap(keep);
    busy += now_s() - tick_start;
  }
  const double wall = now_s();
  for (auto& a : active)
    if (a.sim) sim_destroy(a.sim);
  for (auto& s : streams) cudaStreamDestroy(s);
  cudaFree(pool_base);
  cudaFree(dtab);
  cudaFree(dres);
  cudaFreeHost(htab);
  cudaFreeHost(hres);
  if (stats) {
    stats->completed = completed;
    stats->ticks = ticks;
    stats->wall_s = wall;
    stats->busy_s = busy;
    stats->launches = qs_kernel_launches() - launches0;
    stats->peak_bytes = pool.peak();
    stats->max_active = max_active;
  }
  return st;
}

// =========================================================================================
// persistent mode: event-driven host loop around the persistent kernel
// =========================================================================================
namespace {
struct PActive {
  int id;
  bool small;
  size_t off, bytes, goff, gbytes;
  int next;                 // next gate to enqueue
  bool fresh;
  long long item;           // small: number of the item in flight, -1 if none
  int pending_g1;           // small: end of the chunk in flight
  qs_sim* sim;              // large
  int stream;
  cudaEvent_t ev;           // large: end of the chunk in flight
  bool in_flight;
};
}  // namespace

static qs_status serve_persistent(qs_request* reqs, int n, const qs_serve_config* cfg, qs_serve_stats* stats,
                                  int small_max, int quantum, int nstreams, size_t budget) {
  const unsigned R = 4096;                      // ring slots: at most R small states in flight
  const int res_stride = 16;                    // doubles per result slot (N <= 14: 1 + 14)
  const int lq = cfg->large_quantum > 0 ? cfg->large_quantum : quantum;
  const double wait_ms = cfg->device_wait_ms > 0 ? cfg->device_wait_ms : 200.0;
  int dev = 0, sms = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int ctas = cfg->persistent_ctas > 0 ? cfg->persistent_ctas : (sms / 2 > 0 ? sms / 2 : 1);
  // resources (released at the end whatever happens)
  unsigned char* pool_base = nullptr;
  WorkItem* ring_h = nullptr;
  QueueCtl* ctl_h = nullptr;
  double* res_h = nullptr;
  unsigned long long* dcount = nullptr;   // head, taken
  unsigned int* didle = nullptr;
  // streams[0]: the persistent kernel; 1..nstreams: larger states (and
  // streams[nstreams] the gate uploads too)
  std::vector<cudaStream_t> streams(nstreams + 1, nullptr);
  cudaEvent_t kev = nullptr;
  std::vector<PActive> active;
  qs_status st = QS_OK;
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == QS_OK) {
      qs_set_error("serve_run: %s: %s", what, cudaGetErrorString(e));
      st = QS_ECUDA;
    }
    return st == QS_OK;
  };
  cu(cudaMalloc(&pool_base, budget), "pool");
  cu(cudaHostAlloc(&ring_h, sizeof(WorkItem) * R, cudaHostAllocMapped), "ring");
  cu(cudaHostAlloc(&ctl_h, sizeof(QueueCtl) + sizeof(unsigned long long) * (R - 1), cudaHostAllocMapped), "queue");
  cu(cudaHostAlloc(&res_h, sizeof(double) * res_stride * R, cudaHostAllocMapped), "results");
  cu(cudaMalloc(&dcount, 2 * sizeof(unsigned long long)), "counters");
  cu(cudaMalloc(&didle, sizeof(unsigned int)), "counters");
  for (auto& x : streams) cu(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "stream");
  cu(cudaEventCreateWithFlags(&kev, cudaEventDisableTiming), "event");
  WorkItem* ring_d = nullptr;
  QueueCtl* ctl_d = nullptr;
  double* res_d = nullptr;
  if (st == QS_OK) {
    memset(ctl_h, 0, sizeof(QueueCtl) + sizeof(unsigned long long) * (R - 1));
    memset(ring_h, 0, sizeof(WorkItem) * R);
    memset(res_h, 0, sizeof(double) * res_stride * R);
    cu(cudaHostGetDevicePointer((void**)&ring_d, ring_h, 0), "mapping");
    cu(cudaHostGetDevicePointer((void**)&ctl_d, ctl_h, 0), "mapping");
    cu(cudaHostGetDevicePointer((void**)&res_d, res_h, 0), "mapping");
    cu(cudaMemsetAsync(dcount, 0, 2 * sizeof(unsigned long long), streams[0]), "memset");
    cu(cudaMemsetAsync(didle, 0, sizeof(unsigned int), streams[0]), "memset");
    cu(cudaFuncSetAttribute(k_serve_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 << 14), "attribute");
    cu(cudaStreamSynchronize(streams[0]), "sync");
  }
  Pool pool(budget);
  const uint64_t launches0 = qs_kernel_launches();
  const auto t0 = std::chrono::steady_clock::now();
  auto now_s = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  unsigned long long published = 0, finished_items = 0;
  bool kernel_live = false;
  int relaunches = 0, completed = 0, max_active = 0, nsmall = 0, next_arrival = 0;
  double busy = 0.0, last_progress = 0.0, busy_from = -1.0;
  std::vector<BGate<float>> hg;
  auto launch_kernel = [&]() {
    k_serve_persist<<<ctas, STPB, 8 << 14, streams[0]>>>(ring_d, R, ctl_d, dcount, (unsigned long long)(wait_ms * 1e6),
                                                        didle, dcount + 1);
    qs_count_launch();
    cu(cudaGetLastError(), "persistent launch");
    cu(cudaEventRecord(kev, streams[0]), "event");
    kernel_live = true;
    ++relaunches;
  };
  auto publish = [&](PActive& a) {
    const qs_request& r = reqs[a.id];
    const unsigned long long k = published;
    WorkItem& w = ring_h[k % R];
    w.state = (float2*)(pool_base + a.off);
    w.gates = (const BGate<float>*)(pool_base + a.goff);
    w.res = res_d + (size_t)res_stride * (k % R);
    w.N = r.N;
    w.g0 = a.next;
    w.g1 = std::min(r.ngates, a.next + quantum);
    w.fresh = a.fresh ? 1 : 0;
    w.final_ = (w.g1 == r.ngates) ? 1 : 0;
    a.item = (long long)k;
    a.pending_g1 = w.g1;
    published = k + 1;
    __atomic_store_n(&ctl_h->tail, published, __ATOMIC_RELEASE);
  };
  while (st == QS_OK && completed < n) {
    bool progress = false;
    const double tnow = now_s();
    // admission, oldest first, while the state and its gate list fit
    while (st == QS_OK && next_arrival < n && reqs[next_arrival].arrival_s <= tnow) {
      qs_request& r = reqs[next_arrival];
      PActive a;
      memset(&a, 0, sizeof a);
      a.id = next_arrival;
      a.small = r.N <= small_max;
      if (a.small && nsmall >= (int)R) break;
      a.bytes = (size_t)8 << r.N;
      a.gbytes = a.small ? (size_t)r.ngates * sizeof(BGate<float>) : 0;
      if (!pool.alloc(a.bytes, &a.off)) break;
      if (a.small && a.gbytes && !pool.alloc(a.gbytes, &a.goff)) { pool.release(a.off, a.bytes); break; }
      a.fresh = true;
      a.item = -1;
      a.stream = (int)(next_arrival % nstreams) + 1;
      if (a.small) {
        hg.resize(r.ngates);
        for (int k = 0; k < r.ngates; ++k) {
          const qs_gate& g = r.gates[k];
          BGate<float>& o = hg[k];
          o.nc = g.nc; o.c0 = g.controls[0]; o.c1 = g.controls[1]; o.t = g.target;
          for (int j = 0; j < 8; ++j) o.u[j] = (float)g.u[j];
        }
        // the copy must have reached device memory before the item is
        // published: a pageable cudaMemcpy may return earlier, so copy on a
        // stream of its own and wait for that stream
        if (r.ngates) {
          cu(cudaMemcpyAsync(pool_base + a.goff, hg.data(), a.gbytes, cudaMemcpyHostToDevice, streams[nstreams]),
             "gate upload");
          cu(cudaStreamSynchronize(streams[nstreams]), "gate upload");
        }
        ++nsmall;
      } else {
        qs_status s2 = sim_create_in(r.N, QS_C64, pool_base + a.off, a.bytes, (void*)streams[a.stream], &a.sim);
        if (s2 != QS_OK) { st = s2; break; }
        cu(cudaEventCreateWithFlags(&a.ev, cudaEventDisableTiming), "event");
      }
      r.admit_s = tnow;
      active.push_back(a);
      ++next_arrival;
      progress = true;
    }
    if (st != QS_OK) break;
    max_active = std::max(max_active, (int)active.size());
    if (!active.empty() && busy_from < 0) busy_from = tnow;
    // advance every request whose previous work finished
    std::vector<PActive> keep;
    keep.reserve(active.size());
    for (auto& a : active) {
      qs_request& r = reqs[a.id];
      bool done_req = false;
      if (a.small) {
        if (a.item >= 0) {
          const unsigned long long d = __atomic_load_n(&ctl_h->done[a.item % R], __ATOMIC_ACQUIRE);
          if (d == (unsigned long long)a.item + 1) {
            ++finished_items;
            progress = true;
            a.fresh = false;
            a.next = a.pending_g1;
            if (a.next == r.ngates) {
              const double* res = res_h + (size_t)res_stride * (a.item % R);
              r.norm = res[0];
              for (int q = 0; q < r.N; ++q) r.qz[q] = res[1 + q];
              done_req = true;
            }
            a.item = -1;
          }
        }
        if (!done_req && a.item < 0) {
          publish(a);
          progress = true;
        }
      } else {
        if (a.in_flight) {
          const cudaError_t q = cudaEventQuery(a.ev);
          if (q == cudaErrorNotReady) { keep.push_back(a); continue; }
          if (!cu(q, "large chunk")) break;
          a.in_flight = false;
          progress = true;
        }
        if (a.next < r.ngates) {
          const int g1 = std::min(r.ngates, a.next + lq);
          qs_status s2 = circuit_run(a.sim, r.gates + a.next, g1 - a.next, 1, nullptr);
          if (s2 != QS_OK) { st = s2; break; }
          a.next = g1;
          cu(cudaEventRecord(a.ev, streams[a.stream]), "event");
          a.in_flight = true;
        } else {
          std::vector<double> qx(r.N), qy(r.N);
          qs_status s2 = expect_xyz(a.sim, qx.data(), qy.data(), r.qz);
          if (s2 == QS_OK) s2 = sim_norm(a.sim, &r.norm);
          if (s2 != QS_OK) { st = s2; break; }
          sim_destroy(a.sim);
          a.sim = nullptr;
          cudaEventDestroy(a.ev);
          done_req = true;
        }
      }
      if (done_req) {
        r.finish_s = now_s();
        pool.release(a.off, a.bytes);
        if (a.gbytes) pool.release(a.goff, a.gbytes);
        if (a.small) --nsmall;
        ++completed;
        progress = true;
      } else {
        keep.push_back(a);
      }
    }
    if (st != QS_OK) break;
    active.swap(keep);
    if (active.empty() && busy_from >= 0) { busy += now_s() - busy_from; busy_from = -1.0; }
    // the persistent kernel: (re)launch when items wait and its CTAs have ended
    if (kernel_live) {
      const cudaError_t q = cudaEventQuery(kev);
      if (q == cudaSuccess) kernel_live = false;
      else if (q != cudaErrorNotReady) { cu(q, "persistent kernel"); break; }
    }
    if (!kernel_live && published > finished_items) launch_kernel();
    if (progress) {
      last_progress = now_s();
    } else {
      if (now_s() - last_progress > 60.0) {
        qs_set_error("serve_run: no progress for 60 s");
        st = QS_ETIMEOUT;
        break;
      }
      if (active.empty() && next_arrival < n) {
        const double w = reqs[next_arrival].arrival_s - now_s();
        if (w > 0) std::this_thread::sleep_for(std::chrono::duration<double>(w < 1e-3 ? w : 1e-3));
      } else {
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
    }
  }
  if (busy_from >= 0) busy += now_s() - busy_from;
  const double wall = now_s();
  // stop the persistent CTAs (they see the flag within one poll) and wait,
  // bounded, for the kernel and the streams
  if (ctl_h) __atomic_store_n(&ctl_h->stop, 1ull, __ATOMIC_RELEASE);
  if (kernel_live) {
    const auto ts = std::chrono::steady_clock::now();
    while (cudaEventQuery(kev) == cudaErrorNotReady &&
           std::chrono::steady_clock::now() - ts < std::chrono::seconds(30))
      std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  unsigned long long taken = 0;
  unsigned int idle = 0;
  if (dcount) cudaMemcpy(&taken, dcount + 1, sizeof taken, cudaMemcpyDeviceToHost);
  if (didle) cudaMemcpy(&idle, didle, sizeof idle, cudaMemcpyDeviceToHost);
  for (auto& x : streams)
    if (x) cudaStreamSynchronize(x);
  for (auto& a : active) {
    if (a.sim) sim_destroy(a.sim);
    if (!a.small && a.ev) cudaEventDestroy(a.ev);
  }
  for (auto& x : streams)
    if (x) cudaStreamDestroy(x);
  if (kev) cudaEventDestroy(kev);
  cudaFree(pool_base);
  cudaFree(dcount);
  cudaFree(didle);
  cudaFreeHost(ring_h);
  cudaFreeHost(ctl_h);
  cudaFreeHost(res_h);
  if (stats) {
    stats->completed = completed;
    stats->ticks = 0;
    stats->wall_s = wall;
    stats->busy_s = busy;
    stats->launches = qs_kernel_launches() - launches0;
    stats->peak_bytes = pool.peak();
    stats->max_active = max_active;
    stats->work_items = taken;
    stats->idle_exits = (int)idle;
    stats->relaunches = relaunches;
  }
  return st;
}
