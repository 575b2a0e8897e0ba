// Instantiations of the vectorised persistent stencil kernel: the 3-D 19-point
// "poisson" stencil (centre, faces, edges), f32 storage (4 bytes: V = 4 cells per thread, prefetch depth 12 planes;
// 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_f32_poisson(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<float, S3d19, 512, 4, 0, 12, false>(PERKS_F32, SH_3D19));
    out.push_back(vec_entry<float, S3d19, 512, 4, 0, 12, true>(PERKS_F32, SH_3D19));
}

}  // namespace perks
