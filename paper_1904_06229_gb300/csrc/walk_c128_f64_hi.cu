// Instantiations of the Gray-walk kernel: complex matrices, FP64 products, orders 33..64.
#include "glynn_walk.cuh"

namespace perm {

cudaError_t walk_launch_c128_f64_hi(const WalkArgs& a) { return walk_dispatch<true, kProdF64, 33, 64>(a); }

int walk_blocks_c128_f64_hi(int n) { return walk_blocks_dispatch<true, kProdF64, 33, 64>(n); }

}  // namespace perm
