// Image kernels instantiated for sizes 768, 1024.
#include "blink_image_impl.cuh"

namespace blink {
template struct SizeOps<768>;
template struct SizeOps<1024>;
}  // namespace blink
