// Bit-reproducible double-precision walk.  This translation unit is compiled with --fmad=false: every
// product and sum is rounded separately, as in any other implementation of the same steps.
#include "walk_impl.cuh"

namespace ms {
namespace walk {

cudaError_t launch_f64(const Job& J, cudaStream_t stream) { return launch<F64>(J, stream); }

}  // namespace walk
}  // namespace ms
