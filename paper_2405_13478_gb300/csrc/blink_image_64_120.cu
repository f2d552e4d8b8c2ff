// Image kernels instantiated for sizes 64, 96, 120.
#include "blink_image_impl.cuh"

namespace blink {
template struct SizeOps<64>;
template struct SizeOps<96>;
template struct SizeOps<120>;
}  // namespace blink
