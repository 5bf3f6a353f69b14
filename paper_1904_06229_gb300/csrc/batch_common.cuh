// Device side of the batch layout shared by the batch kernels (batch.cu,
// batch_cta.cu): decoding a ticket of one kernel kind into its item.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "perm_internal.h"

namespace perm {

struct BatchItemRef {
  int n;             // order
  int matrix;        // matrix index (into the pointer array)
  uint64_t first;    // first code of the item
  uint64_t count;    // codes of the item
  uint64_t partial;  // index of its partial (4 doubles)
};

// Ticket t of kernel kind `kind` -> item.  Orders are scanned largest first,
// as the tickets were laid out.  Returns false past the kernel's last item.
__device__ __forceinline__ bool batch_decode(const BatchTable& tab, int kind, const int* __restrict__ perm,
                                             uint64_t t, BatchItemRef& it) {
  if (t >= tab.kitems[kind]) return false;
  for (int m = kBatchNMax; m >= 1; --m) {
    if (tab.kind[m] != kind) continue;
    const uint64_t ipm = tab.items_per_matrix[m];
    const uint64_t cnt = (uint64_t)tab.mcount[m] * ipm;
    if (t < tab.kbase[m] + cnt) {
      const uint64_t local = t - tab.kbase[m];
      const uint64_t slot = local / ipm, sub = local - slot * ipm;
      const uint64_t total = 1ull << (m - 1);
      it.n = m;
      it.matrix = perm[tab.mstart[m] + slot];
      it.first = sub * tab.per_item[m];
      it.count = total - it.first < tab.per_item[m] ? total - it.first : tab.per_item[m];
      it.partial = tab.gbase[m] + local;
      return true;
    }
  }
  return false;
}

}  // namespace perm
