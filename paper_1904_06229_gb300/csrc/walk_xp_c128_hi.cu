// Instantiations of the packed double-float Gray walk with exact float-pair rows (complex matrices), orders 33..64.
#include "glynn_walk_xp.cuh"

namespace perm {

cudaError_t walk_launch_xp_c128_hi(const WalkArgs& a) { return xp_dispatch<true, 33, 64>(a); }

int walk_blocks_xp_c128_hi(int n) { return xp_blocks_dispatch<true, 33, 64>(n); }

}  // namespace perm
