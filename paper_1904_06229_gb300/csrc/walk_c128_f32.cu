// Instantiations of the Gray-walk kernel: complex matrices, FP32-significand products, orders 1..64.
#include "glynn_walk.cuh"

namespace perm {

cudaError_t walk_launch_c128_f32(const WalkArgs& a) { return walk_dispatch<true, kProdF32, 1, 64>(a); }

int walk_blocks_c128_f32(int n) { return walk_blocks_dispatch<true, kProdF32, 1, 64>(n); }

}  // namespace perm
