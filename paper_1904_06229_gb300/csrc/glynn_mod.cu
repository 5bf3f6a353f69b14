// Exact permanents of small-integer matrices modulo four odd moduli < 2^62:
// the host entry point perm_mod01 and the final reduction.  The walk kernel
// and its arithmetic are in glynn_mod.cuh (instantiated in mod_lo.cu and
// mod_hi.cu).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "glynn_mod.cuh"
#include "modular_host.h"
#include "perm.h"
#include "perm_internal.h"

namespace perm {

// Sum the block residues and multiply by scale_R[q] / R = (-1)^(n-1) 2^-(n-1).
__global__ void k_mod_finalize(const uint64_t* __restrict__ partials, int nparts, ModConsts c, const uint64_t scaleR0,
                               const uint64_t scaleR1, const uint64_t scaleR2, const uint64_t scaleR3,
                               uint64_t* __restrict__ residues) {
  const int q = threadIdx.x;
  if (q >= 4) return;
  const uint64_t p = c.p[q];
  uint64_t s = 0;
  for (int k = 0; k < nparts; ++k) {
    s += partials[(size_t)k * 4 + q];
    if (s >= p) s -= p;
  }
  const uint64_t sr[4] = {scaleR0, scaleR1, scaleR2, scaleR3};
  residues[q] = mont_mul(s, sr[q], p, c.pinv[q]);
}

void preload_mod_kernels() { load_kernel(k_mod_finalize); }

}  // namespace perm

namespace {

bool is_device_ptr_mod(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

uint64_t pow_r_mod(uint64_t p, int k) {  // R^k mod p, R = 2^64
  uint64_t r = perm::mont_r_mod(p), out = 1 % p;
  for (int i = 0; i < k; ++i) out = perm::mulmod_u64(out, r, p);
  return out;
}

}  // namespace

extern "C" int perm_mod01(const int8_t* A, int n, const uint64_t* primes, uint64_t* residues, void* stream) {
  using namespace perm;
  TraceRange trace("perm_mod01");
  if (n < 1 || n > PERM_NMAX) return PERM_EINVAL;
  if (!A || !primes || !residues) return PERM_ENULL;
  int rc = check_moduli(primes, 4);
  if (rc) return rc;
  int count_dev = 0, dev = 0;
  if (cudaGetDeviceCount(&count_dev) != cudaSuccess || count_dev < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
  ensure_kernels_loaded();
  cudaStream_t s = (cudaStream_t)stream;

  ModConsts c;
  uint64_t scaleR[4];
  const int groups[3] = {(n + 11) / 12, (n + 7) / 8, (n + 3) / 4};  // G = 12, 8, 4
  c.pmin = primes[0];
  const char* sum_env = std::getenv("PERM_MOD_SUM");
  c.exact_ok = (sum_env && std::strcmp(sum_env, "modular") == 0) ? 0 : 1;
  for (int q = 0; q < 4; ++q) {
    const uint64_t p = primes[q];
    c.p[q] = p;
    c.pinv[q] = mont_neg_inv(p);
    c.r2[q] = pow_r_mod(p, 2);
    for (int gi = 0; gi < 3; ++gi)
      for (int k = 0; k < 2; ++k) c.fix[gi][k][q] = pow_r_mod(p, groups[gi] - 1 + k);
    for (int w = 0; w < 4; ++w) c.rpow[w][q] = pow_r_mod(p, w);
    if (p < c.pmin) c.pmin = p;
    // (-1)^(n-1) / 2^(n-1) mod p, times R for the Montgomery product
    uint64_t inv2 = (p + 1) / 2;
    uint64_t sc = powmod_u64(inv2, (uint64_t)(n - 1), p);
    if (((n - 1) & 1) && sc) sc = p - sc;
    scaleR[q] = mulmod_u64(sc, mont_r_mod(p), p);
  }

  const uint64_t total = 1ull << (n - 1);
  int resident = n <= 32 ? mod_resident_lo(n) : (n <= 48 ? mod_resident_mid(n) : mod_resident_hi(n));
  if (resident < 1) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  const uint64_t per_block = 16ull * kModThreads;
  uint64_t want = (total + per_block - 1) / per_block;
  int blocks = (int)(want < 1 ? 1 : (want > (uint64_t)resident ? (uint64_t)resident : want));

  const bool a_dev = is_device_ptr_mod(A);
  const bool o_dev = is_device_ptr_mod(residues);
  const size_t szA = a_dev ? 0 : (((size_t)n * n + 255) & ~(size_t)255);
  const size_t szP = (((size_t)blocks * 4 * sizeof(uint64_t)) + 255) & ~(size_t)255;
  const size_t szO = o_dev ? 0 : 256;
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, szA + szP + szO, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA;
  }
  const int8_t* dA = A;
  if (!a_dev) {
    e = cudaMemcpyAsync(base, A, (size_t)n * n, cudaMemcpyHostToDevice, s);
    dA = (const int8_t*)base;
  }
  uint64_t* partials = (uint64_t*)(base + szA);
  uint64_t* dOut = o_dev ? residues : (uint64_t*)(base + szA + szP);
  if (e == cudaSuccess)
    e = n <= 32   ? mod_launch_lo(n, dA, c, total, partials, blocks, s)
        : n <= 48 ? mod_launch_mid(n, dA, c, total, partials, blocks, s)
                  : mod_launch_hi(n, dA, c, total, partials, blocks, s);
  if (e == cudaSuccess) {
    k_mod_finalize<<<1, 32, 0, s>>>(partials, blocks, c, scaleR[0], scaleR[1], scaleR[2], scaleR[3], dOut);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !o_dev) e = cudaMemcpyAsync(residues, dOut, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}
