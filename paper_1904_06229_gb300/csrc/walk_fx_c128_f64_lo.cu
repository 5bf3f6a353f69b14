// Instantiations of the fixed-point-row Gray walk: complex matrices, products mostly in integer block floating point, orders 1..32.
#include "glynn_walk_fx.cuh"

namespace perm {

cudaError_t walk_launch_fx_c128_f64_lo(const WalkArgs& a) { return fx_dispatch<true, kProdF64, 1, 32>(a); }

int walk_blocks_fx_c128_f64_lo(int n) { return fx_blocks_dispatch<true, kProdF64, 1, 32>(n); }

}  // namespace perm
