// Instantiations of the Gray-walk kernel: complex matrices, FP64 products, orders 1..32.
#include "glynn_walk.cuh"

namespace perm {

cudaError_t walk_launch_c128_f64_lo(const WalkArgs& a) { return walk_dispatch<true, kProdF64, 1, 32>(a); }

int walk_blocks_c128_f64_lo(int n) { return walk_blocks_dispatch<true, kProdF64, 1, 32>(n); }

}  // namespace perm
