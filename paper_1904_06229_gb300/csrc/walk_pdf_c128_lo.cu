// Instantiations of the packed double-float Gray walk with double-float rows re-seeded from exact int64 (complex matrices), orders 1..32.
#include "glynn_walk_xp.cuh"

namespace perm {

cudaError_t walk_launch_pdf_c128_lo(const WalkArgs& a) { return xp_dispatch<false, 1, 32>(a); }

int walk_blocks_pdf_c128_lo(int n) { return xp_blocks_dispatch<false, 1, 32>(n); }

}  // namespace perm
