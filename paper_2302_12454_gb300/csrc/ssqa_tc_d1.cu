// Shuffle-exchange variants of the persistent tensor-core kernel with replica delay d = 1
// (Eq. 6a, sigma_{i,k+1}(t - d)).
#include "ssqa_tc_kernel.cuh"

namespace ssqa {
namespace tc {
SSQA_TC_DEFINE_PICK_SHFL(1)
}  // namespace tc
}  // namespace ssqa
