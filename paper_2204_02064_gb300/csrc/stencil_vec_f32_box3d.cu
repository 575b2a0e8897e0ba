// Instantiations of the vectorised persistent stencil kernel: the 3-D wide kernels (3d27pt, 3d13pt),
// f32 storage (4 bytes: V = 4 cells per thread, prefetch depth 12 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_f32_box3d(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<float, S3d27, 512, 4, 0, 12, false>(PERKS_F32, SH_3D27));
    out.push_back(vec_entry<float, S3d13, 512, 4, 0, 12, false>(PERKS_F32, SH_3D13));
}

}  // namespace perks
