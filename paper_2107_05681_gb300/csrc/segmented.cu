// segmented.cu - batched sort of independent power-of-two segments.
#include "darm.h"
#include "darm_internal.h"

namespace darm {
void segmented_release_all() {}
}  // namespace darm

extern "C" int darm_segmented_sort(uint32_t*, uint32_t*, const uint64_t*, const uint32_t*,
                                   uint32_t, int, int, const uint8_t*, void*) {
  return DARM_ERR_NOT_FOUND;
}
