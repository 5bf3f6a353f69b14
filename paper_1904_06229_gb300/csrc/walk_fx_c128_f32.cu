// Instantiations of the fixed-point-row Gray walk: complex matrices, FP32-significand products, orders 1..64.
#include "glynn_walk_fx.cuh"

namespace perm {

cudaError_t walk_launch_fx_c128_f32(const WalkArgs& a) { return fx_dispatch<true, kProdF32, 1, 64>(a); }

int walk_blocks_fx_c128_f32(int n) { return fx_blocks_dispatch<true, kProdF32, 1, 64>(n); }

}  // namespace perm
