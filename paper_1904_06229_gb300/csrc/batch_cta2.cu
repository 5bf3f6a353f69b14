// Block-per-item batch kernel, variant allowing 2 blocks per SM (batch_cta.cuh).
#include "batch_cta.cuh"

namespace perm {

cudaError_t batch_launch_cta_minb2(const BatchArgs* ba, const int* perm, const BatchTable& tab, int kind,
                                   double* partials, unsigned long long* ticket, int* status, cudaStream_t s) {
  return CtaKernel<2, kBatchCtaThreads>::launch(ba, perm, tab, kind, partials, ticket, status, s);
}

int batch_resident_cta_minb2() { return CtaKernel<2, kBatchCtaThreads>::resident(); }

}  // namespace perm
