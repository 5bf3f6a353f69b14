// Instantiations of the Gray-walk kernel: real matrices, FP32-significand products, orders 1..64.
#include "glynn_walk.cuh"

namespace perm {

cudaError_t walk_launch_r64_f32(const WalkArgs& a) { return walk_dispatch<false, kProdF32, 1, 64>(a); }

int walk_blocks_r64_f32(int n) { return walk_blocks_dispatch<false, kProdF32, 1, 64>(n); }

}  // namespace perm
