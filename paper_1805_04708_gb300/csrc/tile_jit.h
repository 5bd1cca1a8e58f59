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
qs_status tile_jit_compile(const qs_tile::TileParams2& P);
// The same for several passes, on up to 16 host threads.
qs_status tile_jit_compile_all(const std::vector<qs_tile::TileParams2>& passes);
// Compile if needed, load and launch the pass on the handle's stream.
qs_status tile_jit_launch(qs_sim* s, const qs_tile::TileParams2& P, unsigned grid, size_t smem);
