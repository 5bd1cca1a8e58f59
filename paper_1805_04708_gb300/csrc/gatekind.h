// Kinds of 2x2 update, each giving the same result as the dense product.
// Plain C++ with no includes: compiled into the library and into the tile
// passes that are compiled at run time.
#pragma once
enum GateKind : int {
  GK_DENSE = 0,   // general u
  GK_HAD = 1,     // s * [[1, 1], [1, -1]], s real
  GK_DIAG = 2,    // diag(d0, d1)
  GK_ANTI = 3,    // [[0, f01], [f10, 0]]
  GK_IDENT = 4,   // identity (no-op)
  GK_REAL = 5,    // real dense u (tile passes of complex64 states only)
  GK_BFLY = 6     // (a0 + a1, a0 - a1): a Hadamard without its scale (idem)
};
