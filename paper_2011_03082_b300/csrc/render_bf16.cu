// Render kernel instantiations with BF16 decoders (see render_kernel.cuh), one per
// scheduling variant; a translation unit of their own so that the precisions compile in parallel.
#include "render_kernel.cuh"

namespace ms {
namespace render {

const void* variant_kernel_bf16(int i) { return variant_kernel<kDecBF16>(i); }

}  // namespace render
}  // namespace ms
