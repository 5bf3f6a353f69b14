// Instantiations of the exact-integer / modular walk, orders 33..48.
#include "glynn_mod.cuh"

namespace perm {

int mod_resident_mid(int n) { return mod_resident_dispatch<33, 48>(n); }

cudaError_t mod_launch_mid(int n, const int8_t* A, const ModConsts& c, uint64_t count, uint64_t* partials, int blocks,
                           cudaStream_t s) {
  return mod_launch_dispatch<33, 48>(n, A, c, count, partials, blocks, s);
}

}  // namespace perm
