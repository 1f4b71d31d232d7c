// Instantiations of the lazy-box gridder for P = 4 (block shapes whose
// accumulators fit in registers: Bu*Bv*P <= 32 complex values).
#include "lazy.cuh"
#include "internal.h"

namespace gbg {

#define GB_LAZY(BU, BV, P) {BU, BV, P, (const void*)&grid_lazy_kernel<BU, BV, P>, &lazy_smem_bytes<BU, BV, P>}

const LazyEntry* lazy_kernels_p4(int* n) {
  static const LazyEntry t[] = {
      GB_LAZY(2, 1, 4), GB_LAZY(2, 2, 4), GB_LAZY(4, 1, 4), GB_LAZY(4, 2, 4), GB_LAZY(2, 4, 4), GB_LAZY(8, 1, 4),
  };
  *n = (int)(sizeof(t) / sizeof(t[0]));
  return t;
}

}  // namespace gbg
