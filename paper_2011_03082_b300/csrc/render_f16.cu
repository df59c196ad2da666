// Render kernel instantiations with FP16 decoders (see render_kernel.cuh), one per
// scheduling variant; a translation unit of their own so that the precisions compile in parallel.
#include "render_kernel.cuh"

namespace ms {
namespace render {

const void* variant_kernel_fp16(int i) { return variant_kernel<kDecFP16>(i); }

}  // namespace render
}  // namespace ms
