// Instantiations of the LAST pass kernel for every tile shape and
// transform direction, and the 2D-grid variants for square grids (see passes.cuh).
#include "passes.cuh"

namespace sr {

const void* pick_last(int ell, int T, int da, int nl, int map) {
  if (map) {
    if (SR_NL_SPECIAL(ell, T, nl)) {
      if (da < 0) return reinterpret_cast<const void*>(&k_last<256, 16, -1, 256, 1>);
      return reinterpret_cast<const void*>(&k_last<256, 16, 1, 256, 1>);
    }
#define SR_PICK_LAST_2D(E_, T_)                                                  \
  if (ell == E_ && T == T_) {                                                    \
    if (da < 0) return reinterpret_cast<const void*>(&k_last<E_, T_, -1, 0, 1>); \
    return reinterpret_cast<const void*>(&k_last<E_, T_, 1, 0, 1>);              \
  }
    SR_SQUARE_SHAPES(SR_PICK_LAST_2D)
#undef SR_PICK_LAST_2D
    return nullptr;
  }
  if (SR_NL_SPECIAL(ell, T, nl)) {
    if (da < 0) return reinterpret_cast<const void*>(&k_last<256, 16, -1, 256>);
    return reinterpret_cast<const void*>(&k_last<256, 16, 1, 256>);
  }
#define SR_PICK_LAST(E_, T_)                                                  \
  if (ell == E_ && T == T_) {                                                 \
    if (da < 0) return reinterpret_cast<const void*>(&k_last<E_, T_, -1>);    \
    return reinterpret_cast<const void*>(&k_last<E_, T_, 1>);                 \
  }
  SR_TILE_SHAPES(SR_PICK_LAST)
#undef SR_PICK_LAST
  return nullptr;
}

}  // namespace sr
