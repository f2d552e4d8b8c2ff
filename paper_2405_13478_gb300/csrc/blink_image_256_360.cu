// Image kernels instantiated for sizes 256, 360.
#include "blink_image_impl.cuh"

namespace blink {
template struct SizeOps<256>;
template struct SizeOps<360>;
}  // namespace blink
