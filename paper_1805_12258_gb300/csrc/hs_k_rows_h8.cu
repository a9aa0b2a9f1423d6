// hs_k_rows_h8.cu -- the runtime-row family at 8 levels (FP32, 128-bin
// tiles): every odd template count up to 85, e.g. the paper's 85 templates
// with N_hp = 8 harmonic planes (Section VI-A).
#include "hs_staged.cuh"

namespace hs {

int plane_shapes_rows_h8(const ShapeEntry **out)
{
    static const ShapeEntry e[] = {plane_entry_rt<85, 8, 128, float, HS_F32>()};
    *out = e;
    return 1;
}

} // namespace hs
