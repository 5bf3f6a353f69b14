// Instantiations of the packed double-float Gray walk with double-float rows re-seeded from exact int64 (complex matrices), orders 33..64.
#include "glynn_walk_xp.cuh"

namespace perm {

cudaError_t walk_launch_pdf_c128_hi(const WalkArgs& a) { return xp_dispatch<false, 33, 64>(a); }

int walk_blocks_pdf_c128_hi(int n) { return xp_blocks_dispatch<false, 33, 64>(n); }

}  // namespace perm
