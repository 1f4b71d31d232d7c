// Instantiations of the lazy-box gridder for P = 1 and P = 2.
#include "lazy.cuh"
#include "internal.h"

namespace gbg {

#define GB_LAZY(BU, BV, P) {BU, BV, P, (const void*)&grid_lazy_kernel<BU, BV, P>, &lazy_smem_bytes<BU, BV, P>}

const LazyEntry* lazy_kernels_p1(int* n) {
  static const LazyEntry t[] = {
      GB_LAZY(2, 2, 1), GB_LAZY(4, 2, 1), GB_LAZY(2, 4, 1), GB_LAZY(4, 4, 1), GB_LAZY(8, 2, 1), GB_LAZY(2, 8, 1),
      GB_LAZY(8, 4, 1), GB_LAZY(4, 8, 1), GB_LAZY(8, 8, 1),
  };
  *n = (int)(sizeof(t) / sizeof(t[0]));
  return t;
}

const LazyEntry* lazy_kernels_p2(int* n) {
  static const LazyEntry t[] = {
      GB_LAZY(2, 2, 2), GB_LAZY(4, 2, 2), GB_LAZY(2, 4, 2), GB_LAZY(4, 4, 2), GB_LAZY(8, 2, 2), GB_LAZY(2, 8, 2),
  };
  *n = (int)(sizeof(t) / sizeof(t[0]));
  return t;
}

}  // namespace gbg
