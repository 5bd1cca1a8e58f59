// Tile passes compiled at run time (tile_jit.cu).
#pragma once
#include "internal.cuh"
#include "tile_core.cuh"
#include <vector>

// NVRTC could be loaded.
bool tile_jit_available();
// Number of passes compiled so far in this process (the rest came from the
// cache of compiled structures).
long tile_jit_compiles();
// Compile the pass (or find it in the cache); host only, no device work.
// sync: a CTA barrier every `sync` ops (0: none).
qs_status tile_jit_compile(const qs_tile::TileParams2& P, int sync);
// The same for several passes, on up to 16 host threads.
struct JitJob {
  qs_tile::TileParams2 P;
  int sync;
};
qs_status tile_jit_compile_all(const std::vector<JitJob>& passes);
// Compile if needed, load and launch the pass on the handle's stream.
qs_status tile_jit_launch(qs_sim* s, const qs_tile::TileParams2& P, int sync, unsigned grid, size_t smem);

// Kernel candidates of a pass in circuit_run mode 2: 0 the interpreter, 1..3
// compiled with a barrier every kTileCandSync[c] ops (0: none).
constexpr int kTileCands = 4;
extern const int kTileCandSync[kTileCands];
// Pick the candidate for this launch of the pass's structure.  While the
// structure is being tuned, the start event is recorded on the handle's
// stream and *end_ev receives the event to record after the launch (else
// null).
qs_status tile_tune_pick(qs_sim* s, const qs_tile::TileParams2& P, int* cand, cudaEvent_t* end_ev);
// Mark a candidate that failed to compile as never faster.
void tile_tune_fail(const qs_tile::TileParams2& P, int cand);
