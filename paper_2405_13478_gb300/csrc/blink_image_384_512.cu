// Image kernels instantiated for sizes 384, 512.
#include "blink_image_impl.cuh"

namespace blink {
template struct SizeOps<384>;
template struct SizeOps<512>;
}  // namespace blink
