// Image kernels instantiated for sizes 16, 20, 24, 32, 36, 48.
#include "blink_image_impl.cuh"

namespace blink {
template struct SizeOps<16>;
template struct SizeOps<20>;
template struct SizeOps<24>;
template struct SizeOps<32>;
template struct SizeOps<36>;
template struct SizeOps<48>;
}  // namespace blink
