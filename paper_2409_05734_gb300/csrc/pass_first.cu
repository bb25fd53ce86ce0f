// Instantiations of the FIRST pass kernel for every tile shape and
// transform direction, and the 2D-grid variants for square grids (see passes.cuh).
#include "passes.cuh"

namespace sr {

const void* pick_first(int ell, int T, int db, int map) {
#define SR_PICK_FIRST(E_, T_)                                                   \
  if (ell == E_ && T == T_) {                                                   \
    if (db < 0) return reinterpret_cast<const void*>(&k_first<E_, T_, -1>);     \
    return reinterpret_cast<const void*>(&k_first<E_, T_, 1>);                  \
  }
#define SR_PICK_FIRST_2D(E_, T_)                                                \
  if (ell == E_ && T == T_) {                                                   \
    if (db < 0) return reinterpret_cast<const void*>(&k_first<E_, T_, -1, 1>);  \
    return reinterpret_cast<const void*>(&k_first<E_, T_, 1, 1>);               \
  }
  if (map) {
    SR_SQUARE_SHAPES(SR_PICK_FIRST_2D)
    return nullptr;
  }
  SR_TILE_SHAPES(SR_PICK_FIRST)
#undef SR_PICK_FIRST
#undef SR_PICK_FIRST_2D
  return nullptr;
}

}  // namespace sr
