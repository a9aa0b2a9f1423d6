// hs_k_85x16_lowp.cu -- the 85 x 16 shape stored as BF16 or FP16 (FP32 accumulation).
#include "hs_staged.cuh"

namespace hs {

int plane_shapes_85x16_lowp(const ShapeEntry **out)
{
    static const ShapeEntry e[] = {plane_entry<85, 16, 128, __nv_bfloat16, HS_BF16, true>(),
                                   plane_entry<85, 16, 128, __half, HS_F16, true>()};
    *out = e;
    return 2;
}

} // namespace hs
