// Instantiations of the gridding and degridding kernels for P = 1.
#include "kernels.cuh"
#include "internal.h"

namespace gbg {

#define GB_ENTRY(BU, BV)                                                                                  \
  {BU, BV, 1, TapForm<BU, BV, 1>::value, (const void*)&grid_kernel<BU, BV, 1, false>, (const void*)&grid_kernel<BU, BV, 1, true>, \
   (const void*)&degrid_kernel<BU, BV, 1>, &grid_smem_bytes<BU, BV, 1>, \
   &degrid_smem_bytes<BU, BV, 1>}

const KernelEntry* kernels_p1(int* n) {
  static const KernelEntry t[] = {
      GB_ENTRY(1, 1), GB_ENTRY(2, 1), GB_ENTRY(1, 2), GB_ENTRY(2, 2), GB_ENTRY(4, 1), GB_ENTRY(1, 4), GB_ENTRY(4, 2),
      GB_ENTRY(2, 4), GB_ENTRY(3, 3), GB_ENTRY(4, 4), GB_ENTRY(8, 1), GB_ENTRY(1, 8), GB_ENTRY(8, 2), GB_ENTRY(2, 8),
  };
  *n = (int)(sizeof(t) / sizeof(t[0]));
  return t;
}

}  // namespace gbg
