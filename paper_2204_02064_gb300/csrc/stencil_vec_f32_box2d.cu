// Instantiations of the vectorised persistent stencil kernel: the 2-D box and radius-2 kernels (2d9pt, 2d25pt, 2ds9pt),
// f32 storage (4 bytes: V = 4 cells per thread, prefetch depth 12 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_f32_box2d(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<float, S2d9, 256, 4, 0, 12, false>(PERKS_F32, SH_2D9));
    out.push_back(vec_entry<float, S2d9, 256, 4, 0, 12, true>(PERKS_F32, SH_2D9));
    out.push_back(vec_entry<float, S2d25, 256, 4, 0, 12, false>(PERKS_F32, SH_2D25));
    out.push_back(vec_entry<float, S2d25, 256, 4, 0, 12, true>(PERKS_F32, SH_2D25));
    out.push_back(vec_entry<float, S2ds9, 256, 4, 0, 12, false>(PERKS_F32, SH_2DS9));
}

}  // namespace perks
