// tile_u32_keys32.cu - tile and merge kernels for uint32_t keys without
// payload, 32 keys per thread.
#include "tile_entry.cuh"

namespace darm {

KernelEntry tile_kernel_u32_keys32(int logt, int var, bool merge) {
  if (logt == 13) return tile_pick<uint32_t, false, 5, 13>(var, merge);
  if (logt == 14) return tile_pick<uint32_t, false, 5, 14>(var, merge);
  return KernelEntry{nullptr, 0};
}

}  // namespace darm
