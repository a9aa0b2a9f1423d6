// hs_k_85x16_f32_alt.cu -- other forms of the 85 x 16 FP32 shape: tile widths 64 and 96
// (autotuner choices) and the pipelined ring variants.
#include "hs_staged.cuh"

namespace hs {

int plane_shapes_85x16_f32_widths(const ShapeEntry **out)
{
    static const ShapeEntry e[] = {plane_entry<85, 16, 64, float, HS_F32, false>(),
                                   plane_entry<85, 16, 96, float, HS_F32, false>()};
    *out = e;
    return 2;
}

// (templates, levels, tile bins, consumer groups, stages, type)
int ring_shapes_85x16_f32(const RingEntry **out)
{
    static const RingEntry e[] = {ring_entry<85, 16, 128, 2, 3, float, HS_F32>(),
                                  ring_entry<85, 16, 128, 3, 3, float, HS_F32>(),
                                  ring_entry<85, 16, 96, 2, 4, float, HS_F32>(),
                                  ring_entry<85, 16, 96, 4, 4, float, HS_F32>()};
    *out = e;
    return 4;
}

} // namespace hs
