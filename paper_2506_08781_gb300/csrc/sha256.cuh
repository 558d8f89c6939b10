// SHA-256 compression for the POSLO instantiation "POSLO" (Sec. 7.2, Table 2): both the
// PRF of the seed tree and the message hash H are SHA-256.  Written from FIPS 180-4
// Sec. 6.2.2; fully unrolled so the 16-word schedule window stays in registers and the
// round constants become immediates.  Rotations are funnel shifts (SHF), the choice and
// majority functions compile to LOP3.
#pragma once
#include <cstdint>

namespace poslo {

// FIPS 180-4 Sec. 4.2.2: first 32 bits of the fractional parts of the cube roots of the
// first 64 primes.
__device__ __constant__ static const uint32_t kSha256K[64] = {
    0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u, 0x923f82a4u, 0xab1c5ed5u,
    0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u, 0x72be5d74u, 0x80deb1feu, 0x9bdc06a7u, 0xc19bf174u,
    0xe49b69c1u, 0xefbe4786u, 0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu, 0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau,
    0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u, 0xc6e00bf3u, 0xd5a79147u, 0x06ca6351u, 0x14292967u,
    0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu, 0x53380d13u, 0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u,
    0xa2bfe8a1u, 0xa81a664bu, 0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u,
    0x19a4c116u, 0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au, 0x5b9cca4fu, 0x682e6ff3u,
    0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u, 0x90befffau, 0xa4506cebu, 0xbef9a3f7u, 0xc67178f2u};

// FIPS 180-4 Sec. 5.3.3: initial hash value.
#define POSLO_SHA256_IV0 0x6a09e667u
#define POSLO_SHA256_IV1 0xbb67ae85u
#define POSLO_SHA256_IV2 0x3c6ef372u
#define POSLO_SHA256_IV3 0xa54ff53au
#define POSLO_SHA256_IV4 0x510e527fu
#define POSLO_SHA256_IV5 0x9b05688cu
#define POSLO_SHA256_IV6 0x1f83d9abu
#define POSLO_SHA256_IV7 0x5be0cd19u

__device__ __forceinline__ void sha256_init(uint32_t st[8]) {
  st[0] = POSLO_SHA256_IV0; st[1] = POSLO_SHA256_IV1; st[2] = POSLO_SHA256_IV2; st[3] = POSLO_SHA256_IV3;
  st[4] = POSLO_SHA256_IV4; st[5] = POSLO_SHA256_IV5; st[6] = POSLO_SHA256_IV6; st[7] = POSLO_SHA256_IV7;
}

__device__ __forceinline__ uint32_t rotr32(uint32_t x, uint32_t n) { return __funnelshift_r(x, x, n); }

// Big-endian load helper: byte-swap a little-endian 32-bit word.
__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// One compression of the 16 big-endian message words w (clobbered) into state st.
__device__ __forceinline__ void sha256_compress(uint32_t st[8], uint32_t w[16]) {
  uint32_t a = st[0], b = st[1], c = st[2], d = st[3], e = st[4], f = st[5], g = st[6], h = st[7];
#pragma unroll
  for (int i = 0; i < 64; ++i) {
    uint32_t wi;
    if (i < 16) {
      wi = w[i];
    } else {
      const uint32_t x = w[(i + 1) & 15], y = w[(i + 14) & 15];
      const uint32_t s0 = rotr32(x, 7) ^ rotr32(x, 18) ^ (x >> 3);
      const uint32_t s1 = rotr32(y, 17) ^ rotr32(y, 19) ^ (y >> 10);
      wi = w[i & 15] + s0 + w[(i + 9) & 15] + s1;
      w[i & 15] = wi;
    }
    const uint32_t S1 = rotr32(e, 6) ^ rotr32(e, 11) ^ rotr32(e, 25);
    const uint32_t ch = (e & f) ^ (~e & g);
    const uint32_t t1 = h + S1 + ch + kSha256K[i] + wi;
    const uint32_t S0 = rotr32(a, 2) ^ rotr32(a, 13) ^ rotr32(a, 22);
    const uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
    h = g; g = f; f = e; e = d + t1;
    d = c; c = b; b = a; a = t1 + S0 + maj;
  }
  st[0] += a; st[1] += b; st[2] += c; st[3] += d; st[4] += e; st[5] += f; st[6] += g; st[7] += h;
}

// PRF_bit(z) for a 16-byte node z given as 4 big-endian words: one block holding
// z || bit || 0x80 || 0... || bitlen(17 bytes).  The 16-byte output is the first four
// state words (big-endian), returned in out[0..3].
__device__ __forceinline__ void prf_node(const uint32_t z[4], uint32_t bit, uint32_t out[4]) {
  uint32_t w[16];
  w[0] = z[0]; w[1] = z[1]; w[2] = z[2]; w[3] = z[3];
  w[4] = (bit << 24) | 0x00800000u;
#pragma unroll
  for (int k = 5; k < 15; ++k) w[k] = 0;
  w[15] = 17 * 8;
  uint32_t st[8];
  sha256_init(st);
  sha256_compress(st, w);
  out[0] = st[0]; out[1] = st[1]; out[2] = st[2]; out[3] = st[3];
}

// x_i^j = PRF_0(x_0[i] || le32(j)): one block holding x0 || le32(j) || 0x00 || 0x80 ...
// || bitlen(21 bytes).
__device__ __forceinline__ void prf_entry(const uint32_t x0[4], uint32_t j, uint32_t out[4]) {
  uint32_t w[16];
  w[0] = x0[0]; w[1] = x0[1]; w[2] = x0[2]; w[3] = x0[3];
  w[4] = bswap32(j);
  w[5] = 0x00800000u;
#pragma unroll
  for (int k = 6; k < 15; ++k) w[k] = 0;
  w[15] = 21 * 8;
  uint32_t st[8];
  sha256_init(st);
  sha256_compress(st, w);
  out[0] = st[0]; out[1] = st[1]; out[2] = st[2]; out[3] = st[3];
}

}  // namespace poslo
