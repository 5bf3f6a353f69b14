// Instantiations of the packed double-float Gray walk for real matrices, orders 1..32.
#include "glynn_walk_xr.cuh"

namespace perm {

cudaError_t walk_launch_pdf_r64_lo(const WalkArgs& a) { return xr_dispatch<1, 32>(a); }

int walk_blocks_pdf_r64_lo(int n) { return xr_blocks_dispatch<1, 32>(n); }

}  // namespace perm
