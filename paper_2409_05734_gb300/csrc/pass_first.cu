// Instantiations of the FIRST pass kernel for every tile shape and
// transform direction (see passes.cuh).
#include "passes.cuh"

namespace sr {

const void* pick_first(int ell, int T, int db) {
#define SR_PICK_FIRST(E_, T_)                                                   \
  if (ell == E_ && T == T_) {                                                   \
    if (db < 0) return reinterpret_cast<const void*>(&k_first<E_, T_, -1>);     \
    return reinterpret_cast<const void*>(&k_first<E_, T_, 1>);                  \
  }
  SR_TILE_SHAPES(SR_PICK_FIRST)
#undef SR_PICK_FIRST
  return nullptr;
}

}  // namespace sr
