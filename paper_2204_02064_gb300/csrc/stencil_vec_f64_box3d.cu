// Instantiations of the vectorised persistent stencil kernel: the 3-D wide kernels (3d27pt, 3d13pt),
// f64 storage (8 bytes: V = 2 cells per thread, prefetch depth 8 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_f64_box3d(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<double, S3d27, 512, 2, 0, 8, false>(PERKS_F64, SH_3D27));
    out.push_back(vec_entry<double, S3d13, 512, 2, 0, 8, false>(PERKS_F64, SH_3D13));
}

}  // namespace perks
