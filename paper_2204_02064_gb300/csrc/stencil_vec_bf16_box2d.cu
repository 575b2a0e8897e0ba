// Instantiations of the vectorised persistent stencil kernel: the 2-D box and radius-2 kernels (2d9pt, 2d25pt, 2ds9pt),
// bf16 storage (2 bytes: V = 8 cells per thread, prefetch depth 16 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_bf16_box2d(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<__nv_bfloat16, S2d9, 256, 8, 0, 16, false>(PERKS_BF16, SH_2D9));
    out.push_back(vec_entry<__nv_bfloat16, S2d9, 256, 8, 0, 16, true>(PERKS_BF16, SH_2D9));
    out.push_back(vec_entry<__nv_bfloat16, S2d25, 256, 8, 0, 16, false>(PERKS_BF16, SH_2D25));
    out.push_back(vec_entry<__nv_bfloat16, S2d25, 256, 8, 0, 16, true>(PERKS_BF16, SH_2D25));
    out.push_back(vec_entry<__nv_bfloat16, S2ds9, 256, 8, 0, 16, false>(PERKS_BF16, SH_2DS9));
}

}  // namespace perks
