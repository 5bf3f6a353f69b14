// Block-per-item batch kernel, variant with 256 threads per block, one block per SM (batch_cta.cuh).
#include "batch_cta.cuh"

namespace perm {

cudaError_t batch_launch_cta256(const BatchArgs* ba, const int* perm, const BatchTable& tab, int kind,
                                double* partials, unsigned long long* ticket, int* status, cudaStream_t s) {
  return CtaKernel<1, 256>::launch(ba, perm, tab, kind, partials, ticket, status, s);
}

int batch_resident_cta256() { return CtaKernel<1, 256>::resident(); }

}  // namespace perm
