// Instantiations of the rotated-table chunked gridder for P = 2.
#include "internal.h"
#include "rotated.cuh"

namespace gbg {

#define GB_ROT(BU, BV) \
  {BU, BV, 2, (const void*)&grid_rot_kernel<BU, BV, 2, false>, (const void*)&grid_rot_kernel<BU, BV, 2, true>, &rot_smem_bytes<2>, &rot_smem_bytes_wide<2>}

const RotEntry* rot_kernels_p2(int* n) {
  static const RotEntry t[] = {
      GB_ROT(1, 1), GB_ROT(2, 1), GB_ROT(1, 2), GB_ROT(2, 2), GB_ROT(4, 1), GB_ROT(1, 4), GB_ROT(4, 2),
      GB_ROT(2, 4), GB_ROT(3, 3), GB_ROT(4, 4), GB_ROT(8, 1), GB_ROT(1, 8), GB_ROT(8, 2), GB_ROT(2, 8),
  };
  *n = (int)(sizeof(t) / sizeof(t[0]));
  return t;
}

}  // namespace gbg
