// Instantiations of the vectorised persistent stencil kernel: the 3d7pt and 2d5pt kernels,
// f32 storage (4 bytes: V = 4 cells per thread, prefetch depth 12 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_f32_core(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<float, S3d7, 512, 4, 0, 12, false>(PERKS_F32, SH_3D7));
    out.push_back(vec_entry<float, S3d7, 512, 4, 0, 12, false, 4>(PERKS_F32, SH_3D7));
    out.push_back(vec_entry<float, S3d7, 512, 4, 8, 12, false>(PERKS_F32, SH_3D7));
    out.push_back(vec_entry<float, S3d7, 512, 4, 8, 12, false, 4>(PERKS_F32, SH_3D7));
    out.push_back(vec_entry<float, S3d7, 512, 4, 0, 12, true>(PERKS_F32, SH_3D7));
    out.push_back(vec_entry<float, S3d7, 512, 4, 0, 12, true, 4>(PERKS_F32, SH_3D7));
    out.push_back(vec_entry<float, S2d5, 256, 4, 0, 12, false>(PERKS_F32, SH_2D5));
    out.push_back(vec_entry<float, S2d5, 256, 4, 0, 12, false, 4>(PERKS_F32, SH_2D5));
    out.push_back(vec_entry<float, S2d5, 256, 4, 16, 12, false>(PERKS_F32, SH_2D5));
    out.push_back(vec_entry<float, S2d5, 256, 4, 16, 12, false, 4>(PERKS_F32, SH_2D5));
    out.push_back(vec_entry<float, S2d5, 256, 4, 0, 12, true>(PERKS_F32, SH_2D5));
    out.push_back(vec_entry<float, S2d5, 256, 4, 0, 12, true, 4>(PERKS_F32, SH_2D5));
}

}  // namespace perks
