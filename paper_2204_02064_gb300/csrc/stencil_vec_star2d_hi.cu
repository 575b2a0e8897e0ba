// Instantiations of the vectorised stencil kernel for the high-order 2-D
// stars (2d13pt: radius 3, 2d17pt: radius 4), cache-free body only: run one
// launch per step or, as a persistent plan, all steps in one cooperative
// launch with the grid barrier between steps.  x-neighbours up to 4 cells
// away come from up to two lanes back / forward; row-edge lanes read a
// 4-cell x-halo staged in the ring.
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_star2d_hi(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<double, S2d13, 256, 2, 0, 8, true>(PERKS_F64, SH_2D13));
    out.push_back(vec_entry<double, S2d17, 256, 2, 0, 8, true>(PERKS_F64, SH_2D17));
    out.push_back(vec_entry<float, S2d13, 256, 4, 0, 12, true>(PERKS_F32, SH_2D13));
    out.push_back(vec_entry<float, S2d17, 256, 4, 0, 12, true>(PERKS_F32, SH_2D17));
    out.push_back(vec_entry<__nv_bfloat16, S2d13, 256, 8, 0, 16, true>(PERKS_BF16, SH_2D13));
    out.push_back(vec_entry<__nv_bfloat16, S2d17, 256, 8, 0, 16, true>(PERKS_BF16, SH_2D17));
}

}  // namespace perks
