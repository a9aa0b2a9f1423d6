// hs_k_85x16_f32_batch.cu -- batched kernels of the 85 x 16 FP32 shape (descriptor-carrying
// launches and the packed plane).
#include "hs_staged.cuh"

namespace hs {

int batch_shapes_85x16_f32(const BatchEntry **out)
{
    static const BatchEntry e[] = {batch_entry<85, 16, 128, float, HS_F32>()};
    *out = e;
    return 1;
}

} // namespace hs
