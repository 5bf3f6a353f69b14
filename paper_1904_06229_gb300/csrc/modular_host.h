// Host-side modular arithmetic helpers (host_modular.cpp).
#pragma once

#include <cstdint>

namespace perm {

uint64_t mulmod_u64(uint64_t a, uint64_t b, uint64_t m);
uint64_t powmod_u64(uint64_t a, uint64_t e, uint64_t m);
uint64_t invmod_u64(uint64_t a, uint64_t m);
bool is_prime_u64(uint64_t n);
uint64_t mont_neg_inv(uint64_t p);
uint64_t mont_r_mod(uint64_t p);
uint64_t mont_r2_mod(uint64_t p);
int check_moduli(const uint64_t* primes, int k);

}  // namespace perm
