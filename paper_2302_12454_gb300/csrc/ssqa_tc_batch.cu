// Batched launches of the persistent tensor-core kernel: the shuffle-exchange
// variants with replica delay d = 1, several problems per launch (the serving
// path batches queued requests this way).
#include "ssqa_tc_kernel.cuh"

namespace ssqa {
namespace tc {

#define SSQA_TC_BATCH(B, T, F) ssqa_tc_batch_kernel<1, B, T, true, F, true>

BatchFn pick_batch(int d, bool both, bool track, bool bytes, bool f16, bool shfl) {
    if (d != 1 || !bytes || !shfl) return nullptr;
    if (both) return track ? (f16 ? SSQA_TC_BATCH(true, true, true) : SSQA_TC_BATCH(true, true, false))
                           : (f16 ? SSQA_TC_BATCH(true, false, true) : SSQA_TC_BATCH(true, false, false));
    return track ? (f16 ? SSQA_TC_BATCH(false, true, true) : SSQA_TC_BATCH(false, true, false))
                 : (f16 ? SSQA_TC_BATCH(false, false, true) : SSQA_TC_BATCH(false, false, false));
}

}  // namespace tc
}  // namespace ssqa
