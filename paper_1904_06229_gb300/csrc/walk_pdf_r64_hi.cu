// Instantiations of the packed double-float Gray walk for real matrices, orders 33..64.
#include "glynn_walk_xr.cuh"

namespace perm {

cudaError_t walk_launch_pdf_r64_hi(const WalkArgs& a) { return xr_dispatch<33, 64>(a); }

int walk_blocks_pdf_r64_hi(int n) { return xr_blocks_dispatch<33, 64>(n); }

}  // namespace perm
