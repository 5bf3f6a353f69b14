// Instantiations of the double-float Gray walk (complex matrices), orders 1..64.
#include "glynn_walk_df.cuh"

namespace perm {

cudaError_t walk_launch_df_c128(const WalkArgs& a) { return df_dispatch<1, 64>(a); }

int walk_blocks_df_c128(int n) { return df_blocks_dispatch<1, 64>(n); }

}  // namespace perm
