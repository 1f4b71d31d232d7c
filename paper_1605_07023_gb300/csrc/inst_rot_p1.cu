// Instantiations of the rotated-table chunked gridder for P = 1.
#include "internal.h"
#include "rotated.cuh"

namespace gbg {

#define GB_ROT(BU, BV) \
  {BU, BV, 1, (const void*)&grid_rot_kernel<BU, BV, 1, false>, (const void*)&grid_rot_kernel<BU, BV, 1, true>, &rot_smem_bytes<1>, &rot_smem_bytes_wide<1>}

const RotEntry* rot_kernels_p1(int* n) {
  static const RotEntry t[] = {
      GB_ROT(1, 1), GB_ROT(2, 1), GB_ROT(1, 2), GB_ROT(2, 2), GB_ROT(4, 1), GB_ROT(1, 4), GB_ROT(4, 2),
      GB_ROT(2, 4), GB_ROT(3, 3), GB_ROT(4, 4), GB_ROT(8, 1), GB_ROT(1, 8), GB_ROT(8, 2), GB_ROT(2, 8),
  };
  *n = (int)(sizeof(t) / sizeof(t[0]));
  return t;
}

}  // namespace gbg
