// bl_slot.cuh -- the slot decode of the blocked layout's symmetric storage (internal).
//
// The factorisation writes H_k of the blocked layout slot by slot; this gives, for a slot, the
// block and element it holds (the inverse of bl_sym_index in pimpc_internal.cuh). Host-callable,
// so that the layout test checks it against bl_sym_index on the CPU.
#pragma once

#include "pimpc_internal.cuh"

namespace pimpc {

// The inverse of bl_sym_index: the block (d, I) and element (a, b) held by slot w of the
// symmetric storage (0 <= w < bl_sym_words); false for the padding of the diagonal region.
__host__ __device__ inline bool bl_sym_slot(int nb, int w, int &d, int &I, int &a, int &b) {
  const int Df = bl_full_diags(nb), D0 = bl_diag_words(nb), full = 16 * nb * (Df - 1);
  if (w < D0) {  // slot t of the upper triangle of diagonal block I
    I = w / 10;
    const int t = w - 10 * I;
    a = t < 4 ? 0 : (t < 7 ? 1 : (t < 9 ? 2 : 3));
    b = a + t - bl_tri(a, a);
    d = 0;
    return I < nb;
  }
  if (w < D0 + full) {
    const int q = (w - D0) >> 2;
    b = (w - D0) & 3;
    I = q % nb;
    d = 1 + (q / nb) % (Df - 1);
    a = q / (nb * (Df - 1));
    return true;
  }
  const int q = (w - D0 - full) >> 2, hb = nb >> 1;  // the middle diagonal, block rows < nb/2
  b = (w - D0 - full) & 3;
  I = q % hb;
  d = hb;
  a = q / hb;
  return true;
}

}  // namespace pimpc
