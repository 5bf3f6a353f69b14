// Instantiations of the packed double-float Gray walk with exact float-pair rows (complex matrices), orders 1..32.
#include "glynn_walk_xp.cuh"

namespace perm {

cudaError_t walk_launch_xp_c128_lo(const WalkArgs& a) { return xp_dispatch<true, 1, 32>(a); }

int walk_blocks_xp_c128_lo(int n) { return xp_blocks_dispatch<true, 1, 32>(n); }

}  // namespace perm
