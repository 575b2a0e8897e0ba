// Instantiations of the vectorised persistent stencil kernel: the 3d7pt and 2d5pt kernels,
// f64 storage (8 bytes: V = 2 cells per thread, prefetch depth 8 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_f64_core(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<double, S3d7, 512, 2, 0, 8, false>(PERKS_F64, SH_3D7));
    out.push_back(vec_entry<double, S3d7, 512, 2, 0, 8, false, 4>(PERKS_F64, SH_3D7));
    out.push_back(vec_entry<double, S3d7, 512, 2, 8, 8, false>(PERKS_F64, SH_3D7));
    out.push_back(vec_entry<double, S3d7, 512, 2, 8, 8, false, 4>(PERKS_F64, SH_3D7));
    out.push_back(vec_entry<double, S3d7, 512, 2, 0, 8, true>(PERKS_F64, SH_3D7));
    out.push_back(vec_entry<double, S3d7, 512, 2, 0, 8, true, 4>(PERKS_F64, SH_3D7));
    // cache-free body with 256 threads and at most 128 registers: two blocks per SM, so that
    // one block's FP64 work overlaps the other's block barriers
    out.push_back(vec_entry<double, S3d7, 256, 2, 0, 8, true, 2, 2>(PERKS_F64, SH_3D7));
    out.push_back(vec_entry<double, S3d7, 256, 2, 0, 8, true, 4, 2>(PERKS_F64, SH_3D7));
    out.push_back(vec_entry<double, S2d5, 256, 2, 0, 8, false>(PERKS_F64, SH_2D5));
    out.push_back(vec_entry<double, S2d5, 256, 2, 0, 8, false, 4>(PERKS_F64, SH_2D5));
    out.push_back(vec_entry<double, S2d5, 256, 2, 16, 8, false>(PERKS_F64, SH_2D5));
    out.push_back(vec_entry<double, S2d5, 256, 2, 16, 8, false, 4>(PERKS_F64, SH_2D5));
    out.push_back(vec_entry<double, S2d5, 256, 2, 0, 8, true>(PERKS_F64, SH_2D5));
    out.push_back(vec_entry<double, S2d5, 256, 2, 0, 8, true, 4>(PERKS_F64, SH_2D5));
}

}  // namespace perks
