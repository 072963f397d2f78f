// tile_u32_pairs.cu - tile and merge kernels for uint32_t keys with a
// uint32_t payload, 16 pairs per thread.
#include "tile_entry.cuh"

namespace darm {

KernelEntry tile_kernel_u32_pairs(int loge, int logt, int var, bool merge) {
  if (loge == 4 && logt == 12) return tile_pick<uint32_t, true, 4, 12>(var, merge);
  if (loge == 4 && logt == 13) return tile_pick<uint32_t, true, 4, 13>(var, merge);
  return KernelEntry{nullptr, 0};
}

}  // namespace darm
