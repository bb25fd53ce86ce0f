// Instantiations of the MID pass kernel for every tile shape and
// transform direction (see passes.cuh).
#include "passes.cuh"

namespace sr {

// Direction pairs that occur in the chains: forward-forward (inside A),
// forward-inverse (the epilogue between A and A^H), inverse-inverse (inside A^H).
const void* pick_mid(int ell, int T, int da, int db, int nl) {
  if (SR_NL_SPECIAL(ell, T, nl)) {
    if (da < 0 && db < 0) return reinterpret_cast<const void*>(&k_mid<256, 16, -1, -1, 256>);
    if (da < 0 && db > 0) return reinterpret_cast<const void*>(&k_mid<256, 16, -1, 1, 256>);
    if (da > 0 && db > 0) return reinterpret_cast<const void*>(&k_mid<256, 16, 1, 1, 256>);
    return nullptr;
  }
#define SR_PICK_MID(E_, T_)                                                       \
  if (ell == E_ && T == T_) {                                                     \
    if (da < 0 && db < 0) return reinterpret_cast<const void*>(&k_mid<E_, T_, -1, -1>); \
    if (da < 0 && db > 0) return reinterpret_cast<const void*>(&k_mid<E_, T_, -1, 1>);  \
    if (da > 0 && db > 0) return reinterpret_cast<const void*>(&k_mid<E_, T_, 1, 1>);   \
    return nullptr;                                                               \
  }
  SR_TILE_SHAPES(SR_PICK_MID)
#undef SR_PICK_MID
  return nullptr;
}

}  // namespace sr
