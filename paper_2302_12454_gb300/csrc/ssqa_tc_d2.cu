// Shuffle-exchange variants of the persistent tensor-core kernel with replica delay d = 2
// (Eq. 6a, sigma_{i,k+1}(t - d)).
#include "ssqa_tc_kernel.cuh"

namespace ssqa {
namespace tc {
SSQA_TC_DEFINE_PICK_SHFL(2)
}  // namespace tc
}  // namespace ssqa
