// Image kernels instantiated for sizes 180, 192.
#include "blink_image_impl.cuh"

namespace blink {
template struct SizeOps<180>;
template struct SizeOps<192>;
}  // namespace blink
