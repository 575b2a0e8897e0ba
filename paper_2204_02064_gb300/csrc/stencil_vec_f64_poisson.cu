// Instantiations of the vectorised persistent stencil kernel: the 3-D 19-point
// "poisson" stencil (centre, faces, edges), f64 storage (8 bytes: V = 2 cells per thread, prefetch depth 8 planes;
// 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_f64_poisson(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<double, S3d19, 512, 2, 0, 8, false>(PERKS_F64, SH_3D19));
    out.push_back(vec_entry<double, S3d19, 512, 2, 0, 8, true>(PERKS_F64, SH_3D19));
}

}  // namespace perks
