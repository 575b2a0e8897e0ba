// Instantiations of the vectorised persistent stencil kernel: the 3-D wide kernels (3d27pt, 3d13pt),
// bf16 storage (2 bytes: V = 8 cells per thread, prefetch depth 16 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_bf16_box3d(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<__nv_bfloat16, S3d27, 512, 8, 0, 16, false>(PERKS_BF16, SH_3D27));
    out.push_back(vec_entry<__nv_bfloat16, S3d13, 512, 8, 0, 16, false>(PERKS_BF16, SH_3D13));
}

}  // namespace perks
