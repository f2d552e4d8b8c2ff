// Image kernels instantiated for sizes 128, 160.
#include "blink_image_impl.cuh"

namespace blink {
template struct SizeOps<128>;
template struct SizeOps<160>;
}  // namespace blink
