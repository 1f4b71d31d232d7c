// Instantiations of the gridding and degridding kernels for P = 4.
#include "kernels.cuh"
#include "internal.h"

namespace gbg {

#define GB_ENTRY(BU, BV)                                                                                  \
  {BU, BV, 4, TapForm<BU, BV, 4>::value, (const void*)&grid_kernel<BU, BV, 4, false>, (const void*)&grid_kernel<BU, BV, 4, true>, \
   (const void*)&degrid_kernel<BU, BV, 4>, &grid_smem_bytes<BU, BV, 4>, \
   &degrid_smem_bytes<BU, BV, 4>}

const KernelEntry* kernels_p4(int* n) {
  static const KernelEntry t[] = {
      GB_ENTRY(1, 1), GB_ENTRY(2, 1), GB_ENTRY(1, 2), GB_ENTRY(2, 2), GB_ENTRY(4, 1), GB_ENTRY(1, 4), GB_ENTRY(4, 2),
      GB_ENTRY(2, 4), GB_ENTRY(3, 3), GB_ENTRY(4, 4), GB_ENTRY(8, 1), GB_ENTRY(1, 8), GB_ENTRY(8, 2), GB_ENTRY(2, 8),
  };
  *n = (int)(sizeof(t) / sizeof(t[0]));
  return t;
}

}  // namespace gbg
