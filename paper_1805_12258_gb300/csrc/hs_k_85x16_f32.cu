// hs_k_85x16_f32.cu -- the SKA plane shape: 85 templates, 16 levels, FP32, 128-bin tiles (the
// sign-checked kernel and the one for planes declared non-negative).
#include "hs_staged.cuh"

namespace hs {

int plane_shapes_85x16_f32(const ShapeEntry **out)
{
    static const ShapeEntry e[] = {plane_entry<85, 16, 128, float, HS_F32, true>()};
    *out = e;
    return 1;
}

} // namespace hs
