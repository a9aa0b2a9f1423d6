// hs_k_21x8.cu -- the small plane shape: 21 templates, 8 levels (FP32, BF16, FP16),
// and its batched FP32 kernels.
#include "hs_staged.cuh"

namespace hs {

int plane_shapes_21x8(const ShapeEntry **out)
{
    static const ShapeEntry e[] = {plane_entry<21, 8, 128, float, HS_F32, true>(),
                                   plane_entry<21, 8, 128, __nv_bfloat16, HS_BF16, false>(),
                                   plane_entry<21, 8, 128, __half, HS_F16, false>()};
    *out = e;
    return 3;
}

int batch_shapes_21x8(const BatchEntry **out)
{
    static const BatchEntry e[] = {batch_entry<21, 8, 128, float, HS_F32>()};
    *out = e;
    return 1;
}

} // namespace hs
