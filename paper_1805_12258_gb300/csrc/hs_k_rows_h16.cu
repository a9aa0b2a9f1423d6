// hs_k_rows_h16.cu -- runtime-row families at 16 levels (FP32, 128-bin
// tiles): one kernel for every odd template count up to 85, one up to 127.
#include "hs_staged.cuh"

namespace hs {

int plane_shapes_rows_h16(const ShapeEntry **out)
{
    static const ShapeEntry e[] = {plane_entry_rt<85, 16, 128, float, HS_F32>(),
                                   plane_entry_rt<127, 16, 128, float, HS_F32>()};
    *out = e;
    return 2;
}

} // namespace hs
