// AES-128 (FIPS-197) and the two constructions of the POSLO+ instantiation (Sec. 7.2):
// the PRF is MMO-AES-128 with kappa = 127 (Def. MMO), H is MDC-2 over AES-128 (Def. MDC-2).
//
// Round function.  After SubBytes and ShiftRows, output column j takes row r from input
// column j + r; MixColumns then multiplies each substituted byte a by one column of the
// circulant matrix (2 3 1 1 / 1 2 3 1 / 1 1 2 3 / 3 1 1 2).  The table T[a] holds
// (2 S(a), S(a), S(a), 3 S(a)) as a big-endian word (rows 0..3); the contributions of rows
// 1, 2, 3 are T rotated right by 8, 16, 24 bits.  S(a) itself is byte 2 (and byte 1) of T[a].
//
// Shared memory.  The table has 32 copies, entry a of copy c at word 32 a + c, i.e. in bank
// c: lane c of a warp reads only copy c, so data-dependent lookups never conflict (32 KiB
// per block).  Each block builds it at start from the S-box definition (the inverse in
// GF(2^8) followed by the affine map of FIPS-197 Sec. 5.1.1); no table is stored anywhere.
//
// Words are big-endian columns: state column c is bytes 4c..4c+3 of the block, row 0 in the
// most significant byte, which is how the message stream hands out words.  Round keys are
// derived on the fly, one per round (FIPS-197 Sec. 5.2 with Nk = 4), because in MMO and
// MDC-2 every block is enciphered under a new key (the chaining value).
#pragma once
#include <cstdint>

namespace poslo {

constexpr int kAesCopies = 32;
struct AesShared {
  uint32_t t[256][kAesCopies];
};

// x * {02} in GF(2^8) (FIPS-197 Sec. 4.2.1), on a byte held in the low 8 bits.
__device__ __forceinline__ uint32_t gf8_xtime(uint32_t a) { return ((a << 1) ^ ((a & 0x80u) ? 0x1bu : 0u)) & 0xffu; }

__device__ __forceinline__ uint32_t gf8_mul(uint32_t a, uint32_t b) {
  uint32_t r = 0;
  for (int i = 0; i < 8; ++i) {
    if (b & 1u) r ^= a;
    b >>= 1;
    a = gf8_xtime(a);
  }
  return r;
}

// S(x) = affine(x^-1), with 0 mapped through the affine map alone (x^254 = x^-1 for x != 0).
__device__ __forceinline__ uint32_t aes_sbox_entry(uint32_t x) {
  uint32_t inv = 1, base = x;
  for (uint32_t e = 254; e; e >>= 1) {
    if (e & 1u) inv = gf8_mul(inv, base);
    base = gf8_mul(base, base);
  }
  if (x == 0) inv = 0;
  // b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i, c = 0x63 (indices mod 8)
  uint32_t out = 0;
  for (int i = 0; i < 8; ++i) {
    uint32_t bit = 0;
    for (int k = 0; k < 8; k += (k == 0 ? 4 : 1)) bit ^= (inv >> ((i + k) & 7)) & 1u;
    out |= (bit ^ ((0x63u >> i) & 1u)) << i;
  }
  return out;
}

// Every thread of the block must call this (it ends with a barrier).
__device__ __forceinline__ void aes_tables_init(AesShared& sh) {
  for (uint32_t a = threadIdx.x; a < 256; a += blockDim.x) {
    const uint32_t s = aes_sbox_entry(a), s2 = gf8_xtime(s);
    const uint32_t t = (s2 << 24) | (s << 16) | (s << 8) | (s2 ^ s);
    for (int c = 0; c < kAesCopies; ++c) sh.t[a][c] = t;
  }
  __syncthreads();
}

// Table reads: entry (byte K of w) of the lane's copy; a byte permute isolates the byte in one
// instruction (13 % faster on GB300 than shift-and-mask; the kernel is bound by the ALU pipe,
// 78 % busy, with the shared-memory pipe at 45 %).  Explicit byte-offset addressing, with or
// without ld.shared, measured no faster.
struct AesCtx {
  const AesShared* sh;
  uint32_t lane;
  template <int K>
  __device__ __forceinline__ uint32_t T(uint32_t w) const { return sh->t[__byte_perm(w, 0u, 0x4440u | K)][lane]; }
};

__device__ __forceinline__ AesCtx aes_ctx(const AesShared* sh) { return AesCtx{sh, threadIdx.x & 31u}; }

__device__ __forceinline__ uint32_t ror32(uint32_t x, uint32_t n) { return __funnelshift_r(x, x, n); }

// Four S-box values assembled into one word: bytes 3..0 from S of byte 3 of a, byte 2 of b,
// byte 1 of c, byte 0 of d (S is byte 2 of a table entry).
__device__ __forceinline__ uint32_t aes_sub4(const AesCtx& c, uint32_t a, uint32_t b, uint32_t cc, uint32_t d) {
  return (c.T<3>(a) & 0x00ff0000u) << 8 | (c.T<2>(b) & 0x00ff0000u) | (c.T<1>(cc) & 0x00ff0000u) >> 8 |
         (c.T<0>(d) & 0x00ff0000u) >> 16;
}

// State of one FIPS-197 Cipher (Nk = 4, Nr = 10) between rounds: the round key k and the
// state s, both as four big-endian column words.
struct AesState {
  uint32_t k0, k1, k2, k3, s0, s1, s2, s3;
};

__device__ __forceinline__ AesState aes_begin(const uint32_t key[4], const uint32_t in[4]) {
  return AesState{key[0], key[1], key[2], key[3], in[0] ^ key[0], in[1] ^ key[1], in[2] ^ key[2], in[3] ^ key[3]};
}

// Round r (1..10) with round constant rcon = x^(r-1).
__device__ __forceinline__ void aes_round(const AesCtx& c, AesState& a, int r, uint32_t rcon) {
  // round key r from round key r-1: SubWord(RotWord(w3)) ^ Rcon into w0, then the chain
  // (RotWord moves byte 2 of w3 to the top, so SubWord(RotWord(w3)) = S(w3 bytes 2,1,0,3))
  const uint32_t sub = aes_sub4(c, a.k3 << 8, a.k3 << 8, a.k3 << 8, a.k3 >> 24);
  a.k0 ^= sub ^ (rcon << 24);
  a.k1 ^= a.k0;
  a.k2 ^= a.k1;
  a.k3 ^= a.k2;
  uint32_t t0, t1, t2, t3;
  if (r < 10) {
    t0 = c.T<3>(a.s0) ^ ror32(c.T<2>(a.s1), 8) ^ ror32(c.T<1>(a.s2), 16) ^ ror32(c.T<0>(a.s3), 24) ^ a.k0;
    t1 = c.T<3>(a.s1) ^ ror32(c.T<2>(a.s2), 8) ^ ror32(c.T<1>(a.s3), 16) ^ ror32(c.T<0>(a.s0), 24) ^ a.k1;
    t2 = c.T<3>(a.s2) ^ ror32(c.T<2>(a.s3), 8) ^ ror32(c.T<1>(a.s0), 16) ^ ror32(c.T<0>(a.s1), 24) ^ a.k2;
    t3 = c.T<3>(a.s3) ^ ror32(c.T<2>(a.s0), 8) ^ ror32(c.T<1>(a.s1), 16) ^ ror32(c.T<0>(a.s2), 24) ^ a.k3;
  } else {   // last round: no MixColumns
    t0 = aes_sub4(c, a.s0, a.s1, a.s2, a.s3) ^ a.k0;
    t1 = aes_sub4(c, a.s1, a.s2, a.s3, a.s0) ^ a.k1;
    t2 = aes_sub4(c, a.s2, a.s3, a.s0, a.s1) ^ a.k2;
    t3 = aes_sub4(c, a.s3, a.s0, a.s1, a.s2) ^ a.k3;
  }
  a.s0 = t0; a.s1 = t1; a.s2 = t2; a.s3 = t3;
}

// E_key(in): FIPS-197 Cipher with Nk = 4, Nr = 10.
__device__ __forceinline__ void aes128_encrypt(const AesCtx& c, const uint32_t key[4], const uint32_t in[4],
                                               uint32_t out[4]) {
  AesState a = aes_begin(key, in);
  uint32_t rcon = 0x01u;
#pragma unroll 1
  for (int r = 1; r <= 10; ++r) {
    aes_round(c, a, r, rcon);
    rcon = gf8_xtime(rcon);
  }
  out[0] = a.s0; out[1] = a.s1; out[2] = a.s2; out[3] = a.s3;
}

// E_keyA(in) and E_keyB(in) with their rounds interleaved: two independent chains in one
// loop, so each one's table reads and XORs fill the other's dependency gaps.
__device__ __forceinline__ void aes128_encrypt2(const AesCtx& c, const uint32_t keyA[4], const uint32_t keyB[4],
                                                const uint32_t in[4], uint32_t outA[4], uint32_t outB[4]) {
  AesState a = aes_begin(keyA, in), b = aes_begin(keyB, in);
  uint32_t rcon = 0x01u;
#pragma unroll 1
  for (int r = 1; r <= 10; ++r) {
    aes_round(c, a, r, rcon);
    aes_round(c, b, r, rcon);
    rcon = gf8_xtime(rcon);
  }
  outA[0] = a.s0; outA[1] = a.s1; outA[2] = a.s2; outA[3] = a.s3;
  outB[0] = b.s0; outB[1] = b.s1; outB[2] = b.s2; outB[3] = b.s3;
}

// Initial values (the MDC-2 constants 0x52.. and 0x25.. widened to 16 bytes): MMO and the
// first MDC-2 chain start from kIvA, the second MDC-2 chain from kIvB.
constexpr uint32_t kIvA = 0x52525252u, kIvB = 0x25252525u;

// One MMO step: h <- E_h(m) ^ m.
__device__ __forceinline__ void mmo_step(const AesCtx& c, uint32_t h[4], const uint32_t m[4]) {
  uint32_t o[4];
  aes128_encrypt(c, h, m, o);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = o[i] ^ m[i];
}

// PRF_bit(z) with kappa = 127: the seed's first 127 bits and the bit fill one block, one
// AES call; the output keeps 127 bits (bit 0 of byte 15 cleared).
__device__ __forceinline__ void prf_node_aes(const AesCtx& c, const uint32_t z[4], uint32_t bit, uint32_t out[4]) {
  const uint32_t m[4] = {z[0], z[1], z[2], (z[3] & ~1u) | bit};
  uint32_t h[4] = {kIvA, kIvA, kIvA, kIvA};
  mmo_step(c, h, m);
  out[0] = h[0]; out[1] = h[1]; out[2] = h[2]; out[3] = h[3] & ~1u;
}

// x_i^j = PRF_0(x_0[i] || j): MMO over seed (PRF bit 0) || le32(j), 20 bytes padded with
// 0x80 and zeros to two blocks; truncated to 127 bits.
__device__ __forceinline__ void prf_entry_aes(const AesCtx& c, const uint32_t x0[4], uint32_t j, uint32_t out[4]) {
  const uint32_t m1[4] = {x0[0], x0[1], x0[2], x0[3] & ~1u};
  const uint32_t m2[4] = {__byte_perm(j, 0, 0x0123), 0x80000000u, 0u, 0u};
  uint32_t h[4] = {kIvA, kIvA, kIvA, kIvA};
  mmo_step(c, h, m1);
  mmo_step(c, h, m2);
  out[0] = h[0]; out[1] = h[1]; out[2] = h[2]; out[3] = h[3] & ~1u;
}

// One MDC-2 step on block m: both chains take an MMO step, then exchange their right
// halves (words 2 and 3).
__device__ __forceinline__ void mdc2_step(const AesCtx& c, uint32_t h[4], uint32_t g[4], const uint32_t m[4]) {
  uint32_t a[4], b[4];
  aes128_encrypt2(c, h, g, m, a, b);
#pragma unroll
  for (int i = 0; i < 4; ++i) { a[i] ^= m[i]; b[i] ^= m[i]; }
  h[0] = a[0]; h[1] = a[1]; h[2] = b[2]; h[3] = b[3];
  g[0] = b[0]; g[1] = b[1]; g[2] = a[2]; g[3] = a[3];
}

}  // namespace poslo
