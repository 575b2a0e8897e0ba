// Instantiations of the vectorised persistent stencil kernel: the 2-D box and radius-2 kernels (2d9pt, 2d25pt, 2ds9pt),
// f64 storage (8 bytes: V = 2 cells per thread, prefetch depth 8 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_f64_box2d(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<double, S2d9, 256, 2, 0, 8, false>(PERKS_F64, SH_2D9));
    out.push_back(vec_entry<double, S2d9, 256, 2, 0, 8, true>(PERKS_F64, SH_2D9));
    out.push_back(vec_entry<double, S2d25, 256, 2, 0, 8, false>(PERKS_F64, SH_2D25));
    out.push_back(vec_entry<double, S2d25, 256, 2, 0, 8, true>(PERKS_F64, SH_2D25));
    out.push_back(vec_entry<double, S2ds9, 256, 2, 0, 8, false>(PERKS_F64, SH_2DS9));
}

}  // namespace perks
