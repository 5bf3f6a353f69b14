// Host-side modular helpers of the exact path: prime search, Montgomery
// constants and Chinese remaindering (Garner's mixed-radix method).
// 64-bit products are reduced through unsigned __int128.
#include <cstdint>
#include <cstring>

#include "modular_host.h"
#include "perm.h"

namespace perm {

uint64_t mulmod_u64(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }

uint64_t powmod_u64(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod_u64(r, a, m);
    a = mulmod_u64(a, a, m);
    e >>= 1;
  }
  return r;
}

// Inverse of a modulo m by the extended Euclidean algorithm; 0 if none.
uint64_t invmod_u64(uint64_t a, uint64_t m) {
  __int128 t = 0, nt = 1, r = m, nr = a % m;
  while (nr != 0) {
    __int128 q = r / nr;
    __int128 tmp = t - q * nt;
    t = nt;
    nt = tmp;
    tmp = r - q * nr;
    r = nr;
    nr = tmp;
  }
  if (r != 1) return 0;
  if (t < 0) t += m;
  return (uint64_t)t;
}

// Miller-Rabin with the first twelve prime bases: exact below 3.3e24.
bool is_prime_u64(uint64_t n) {
  static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (uint64_t p : bases) {
    if (n % p == 0) return n == p;
  }
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) d >>= 1, ++s;
  for (uint64_t a : bases) {
    uint64_t x = powmod_u64(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int k = 1; k < s; ++k) {
      x = mulmod_u64(x, x, n);
      if (x == n - 1) {
        witness = false;
        break;
      }
    }
    if (witness) return false;
  }
  return true;
}

// -p^{-1} mod 2^64 for odd p (Newton iteration on the 2-adic inverse).
uint64_t mont_neg_inv(uint64_t p) {
  uint64_t inv = p;  // correct to 3 bits for odd p
  for (int i = 0; i < 6; ++i) inv *= 2 - p * inv;
  return (uint64_t)0 - inv;
}

uint64_t mont_r_mod(uint64_t p) {  // 2^64 mod p
  return (uint64_t)(((unsigned __int128)1 << 64) % p);
}

uint64_t mont_r2_mod(uint64_t p) {  // 2^128 mod p
  uint64_t r = mont_r_mod(p);
  return mulmod_u64(r, r, p);
}

int check_moduli(const uint64_t* primes, int k) {
  for (int i = 0; i < k; ++i) {
    uint64_t p = primes[i];
    if (p < 3 || (p & 1) == 0 || p >= (1ull << 62)) return PERM_EPRIME;
    for (int j = 0; j < i; ++j)
      if (primes[j] == p) return PERM_EPRIME;
  }
  return PERM_OK;
}

}  // namespace perm

namespace {

// 256-bit little-endian unsigned helpers
void u256_muladd(uint64_t* x, uint64_t m, uint64_t a) {  // x = x*m + a
  unsigned __int128 carry = a;
  for (int i = 0; i < 4; ++i) {
    unsigned __int128 t = (unsigned __int128)x[i] * m + carry;
    x[i] = (uint64_t)t;
    carry = t >> 64;
  }
}

int u256_cmp(const uint64_t* a, const uint64_t* b) {
  for (int i = 3; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  }
  return 0;
}

void u256_sub(uint64_t* a, const uint64_t* b) {  // a -= b (mod 2^256)
  unsigned __int128 borrow = 0;
  for (int i = 0; i < 4; ++i) {
    unsigned __int128 t = (unsigned __int128)a[i] - b[i] - borrow;
    a[i] = (uint64_t)t;
    borrow = (t >> 64) ? 1 : 0;
  }
}

}  // namespace

extern "C" {

int perm_default_primes(uint64_t* out4) {
  if (!out4) return PERM_ENULL;
  int found = 0;
  for (uint64_t c = (1ull << 62) - 1; found < 4 && c > 2; c -= 2) {
    if (perm::is_prime_u64(c)) out4[found++] = c;
  }
  return found == 4 ? PERM_OK : PERM_EPRIME;
}

int perm_crt(const uint64_t* residues, const uint64_t* primes, int k, uint64_t* out_limbs) {
  using namespace perm;
  if (!residues || !primes || !out_limbs) return PERM_ENULL;
  if (k < 1 || k > 4) return PERM_EINVAL;
  for (int i = 0; i < k; ++i) {
    if (primes[i] < 2) return PERM_EPRIME;
    if (residues[i] >= primes[i]) return PERM_EINVAL;
  }
  // Garner: x = v0 + v1 p0 + v2 p0 p1 + ... with 0 <= v_i < p_i
  uint64_t v[4];
  for (int i = 0; i < k; ++i) {
    const uint64_t p = primes[i];
    // value of the first i digits modulo p (Horner), and prod_{j<i} p_j mod p
    uint64_t t = 0, prod = 1 % p;
    for (int j = i - 1; j >= 0; --j) t = (uint64_t)(((unsigned __int128)t * (primes[j] % p) + v[j]) % p);
    for (int j = 0; j < i; ++j) prod = mulmod_u64(prod, primes[j] % p, p);
    uint64_t inv = (i == 0) ? 1 : invmod_u64(prod, p);
    if (i > 0 && inv == 0) return PERM_EPRIME;  // not coprime
    uint64_t diff = (residues[i] % p + p - t) % p;
    v[i] = mulmod_u64(diff, inv, p);
  }
  // rebuild by Horner from the top digit: x = (((v_{k-1}) p_{k-2} + v_{k-2}) p_{k-3} + ...) p_0 + v_0
  uint64_t x[4] = {0, 0, 0, 0};
  x[0] = v[k - 1];
  for (int i = k - 2; i >= 0; --i) u256_muladd(x, primes[i], v[i]);
  // centre: if x > P/2 then x - P
  uint64_t P[4] = {1, 0, 0, 0};
  for (int i = 0; i < k; ++i) u256_muladd(P, primes[i], 0);
  uint64_t half[4];
  std::memcpy(half, P, sizeof(half));
  for (int i = 0; i < 4; ++i) half[i] = (half[i] >> 1) | (i + 1 < 4 ? (half[i + 1] << 63) : 0);
  if (u256_cmp(x, half) > 0) u256_sub(x, P);
  std::memcpy(out_limbs, x, sizeof(x));
  return PERM_OK;
}

}  // extern "C"
