// Instantiations of the fused LAST + FIRST kernel of the GD and power-iteration
// loops for every tile shape, and the 2D-grid variants for square grids (see passes.cuh).
#include "passes.cuh"

namespace sr {

const void* pick_last_first(int ell, int T, int nl, int map) {
  if (map) {
    if (SR_NL_SPECIAL(ell, T, nl)) return reinterpret_cast<const void*>(&k_last_first<256, 16, 256, 1>);
#define SR_PICK_LF_2D(E_, T_) \
  if (ell == E_ && T == T_) return reinterpret_cast<const void*>(&k_last_first<E_, T_, 0, 1>);
    SR_SQUARE_SHAPES(SR_PICK_LF_2D)
#undef SR_PICK_LF_2D
    return nullptr;
  }
  if (SR_NL_SPECIAL(ell, T, nl)) return reinterpret_cast<const void*>(&k_last_first<256, 16, 256>);
#define SR_PICK_LF(E_, T_) \
  if (ell == E_ && T == T_) return reinterpret_cast<const void*>(&k_last_first<E_, T_>);
  SR_TILE_SHAPES(SR_PICK_LF)
#undef SR_PICK_LF
  return nullptr;
}

}  // namespace sr
