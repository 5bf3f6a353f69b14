// Instantiations of the fixed-point-row Gray walk: real matrices, FP64 products, orders 1..64.
#include "glynn_walk_fx.cuh"

namespace perm {

cudaError_t walk_launch_fx_r64_f64(const WalkArgs& a) { return fx_dispatch<false, kProdF64, 1, 64>(a); }

int walk_blocks_fx_r64_f64(int n) { return fx_blocks_dispatch<false, kProdF64, 1, 64>(n); }

}  // namespace perm
