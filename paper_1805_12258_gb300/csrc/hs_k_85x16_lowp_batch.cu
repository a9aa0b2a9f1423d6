// hs_k_85x16_lowp_batch.cu -- batched kernels of the 85 x 16 shape stored as BF16.
#include "hs_staged.cuh"

namespace hs {

int batch_shapes_85x16_lowp(const BatchEntry **out)
{
    static const BatchEntry e[] = {batch_entry<85, 16, 128, __nv_bfloat16, HS_BF16>()};
    *out = e;
    return 1;
}

} // namespace hs
