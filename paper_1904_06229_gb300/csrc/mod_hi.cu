// Instantiations of the exact-integer / modular walk, orders 49..64.
#include "glynn_mod.cuh"

namespace perm {

int mod_resident_hi(int n) { return mod_resident_dispatch<49, 64>(n); }

cudaError_t mod_launch_hi(int n, const int8_t* A, const ModConsts& c, uint64_t count, uint64_t* partials, int blocks,
                          cudaStream_t s) {
  return mod_launch_dispatch<49, 64>(n, A, c, count, partials, blocks, s);
}

}  // namespace perm
