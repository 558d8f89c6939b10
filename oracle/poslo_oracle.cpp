// Plain C++ statement of the POSLO verification definitions (test infrastructure only).
//
// This file is the CPU oracle in a compiled language, used as the timed CPU baseline and
// checked against the Python oracle (oracle/poslo_oracle.py) by the CPU tests.  Only tests,
// the package smoke check and the benchmark's CPU-baseline leg load it; the verification
// library never links or calls it, and it shares no code with the CUDA path.
//
// It follows the same readings as the Python oracle, for the SHA-256 instantiation "POSLO"
// of Sec. 7.2 (Nouma and Yavuz, arXiv 2506.08781):
//   * group: the prime-order subgroup of edwards25519 (p = 2^255 - 19, a = -1,
//     d = -121665/121666, q = 2^252 + 27742317777372353535851937790883648493);
//   * PRF_b(z) = SHA-256(z || byte b)[0..16) for the seed tree (Eq. 1, Fig. 2a);
//   * x_i^j = SHA-256(x_0[i] || le32(j) || 0x00)[0..16), j = t mod n2 (Fig. 3a, Fig. 6);
//   * e_t = SHA-256(m_t || x_t) read little-endian, reduced mod q;
//   * strict point decoding (RFC 8032 Sec. 5.1.3), canonical scalars (< q), and the
//     cofactored check [8](R - eY - sG) = O for every single and aggregate equation.
//
// Arithmetic is deliberately textbook: field elements are four 64-bit limbs multiplied
// schoolbook with unsigned __int128 and reduced by folding 2^256 = 38 (mod p) followed by
// subtraction of p; inversion and square roots are Fermat exponentiations; scalar
// multiplication is left-to-right double-and-add with the unified addition law of Hisil,
// Wong, Carter and Dawson ("Twisted Edwards curves revisited", 2008) also used for doubling;
// scalars mod q are reduced by repeated subtraction.  SHA-256 is written from FIPS 180-4.
// Entries are split into contiguous ranges over std::thread workers; nothing else is
// parallel or reordered.
#include <cstdint>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

namespace {

typedef unsigned __int128 u128;

// ------------------------------------------------------------------------------ SHA-256
// FIPS 180-4 Sec. 4.1.2 (functions), 4.2.2 (constants), 5.1.1 (padding), 5.3.3 (initial
// hash value), 6.2.2 (computation).

const uint32_t K256[64] = {
    0x428a2f98, 0x71374491, 0xb5c0fbcf, 0xe9b5dba5, 0x3956c25b, 0x59f111f1, 0x923f82a4, 0xab1c5ed5,
    0xd807aa98, 0x12835b01, 0x243185be, 0x550c7dc3, 0x72be5d74, 0x80deb1fe, 0x9bdc06a7, 0xc19bf174,
    0xe49b69c1, 0xefbe4786, 0x0fc19dc6, 0x240ca1cc, 0x2de92c6f, 0x4a7484aa, 0x5cb0a9dc, 0x76f988da,
    0x983e5152, 0xa831c66d, 0xb00327c8, 0xbf597fc7, 0xc6e00bf3, 0xd5a79147, 0x06ca6351, 0x14292967,
    0x27b70a85, 0x2e1b2138, 0x4d2c6dfc, 0x53380d13, 0x650a7354, 0x766a0abb, 0x81c2c92e, 0x92722c85,
    0xa2bfe8a1, 0xa81a664b, 0xc24b8b70, 0xc76c51a3, 0xd192e819, 0xd6990624, 0xf40e3585, 0x106aa070,
    0x19a4c116, 0x1e376c08, 0x2748774c, 0x34b0bcb5, 0x391c0cb3, 0x4ed8aa4a, 0x5b9cca4f, 0x682e6ff3,
    0x748f82ee, 0x78a5636f, 0x84c87814, 0x8cc70208, 0x90befffa, 0xa4506ceb, 0xbef9a3f7, 0xc67178f2};

uint32_t rotr(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

void sha256_block(uint32_t H[8], const uint8_t* blk) {
  uint32_t W[64];
  for (int t = 0; t < 16; ++t)
    W[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) | ((uint32_t)blk[4 * t + 2] << 8) |
           blk[4 * t + 3];
  for (int t = 16; t < 64; ++t) {
    uint32_t s0 = rotr(W[t - 15], 7) ^ rotr(W[t - 15], 18) ^ (W[t - 15] >> 3);
    uint32_t s1 = rotr(W[t - 2], 17) ^ rotr(W[t - 2], 19) ^ (W[t - 2] >> 10);
    W[t] = s1 + W[t - 7] + s0 + W[t - 16];
  }
  uint32_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5], g = H[6], h = H[7];
  for (int t = 0; t < 64; ++t) {
    uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
    uint32_t ch = (e & f) ^ (~e & g);
    uint32_t T1 = h + S1 + ch + K256[t] + W[t];
    uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
    uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
    uint32_t T2 = S0 + maj;
    h = g;
    g = f;
    f = e;
    e = d + T1;
    d = c;
    c = b;
    b = a;
    a = T1 + T2;
  }
  H[0] += a;
  H[1] += b;
  H[2] += c;
  H[3] += d;
  H[4] += e;
  H[5] += f;
  H[6] += g;
  H[7] += h;
}

// SHA-256 of the concatenation of two byte strings.
void sha256_2(const uint8_t* a, size_t na, const uint8_t* b, size_t nb, uint8_t out[32]) {
  uint32_t H[8] = {0x6a09e667, 0xbb67ae85, 0x3c6ef372, 0xa54ff53a, 0x510e527f, 0x9b05688c, 0x1f83d9ab, 0x5be0cd19};
  std::vector<uint8_t> msg(a, a + na);
  msg.insert(msg.end(), b, b + nb);
  const uint64_t bits = (uint64_t)msg.size() * 8;
  msg.push_back(0x80);
  while (msg.size() % 64 != 56) msg.push_back(0);
  for (int k = 7; k >= 0; --k) msg.push_back((uint8_t)(bits >> (8 * k)));
  for (size_t off = 0; off < msg.size(); off += 64) sha256_block(H, msg.data() + off);
  for (int k = 0; k < 8; ++k) {
    out[4 * k] = (uint8_t)(H[k] >> 24);
    out[4 * k + 1] = (uint8_t)(H[k] >> 16);
    out[4 * k + 2] = (uint8_t)(H[k] >> 8);
    out[4 * k + 3] = (uint8_t)H[k];
  }
}

// ------------------------------------------------------------------------------ 256-bit integers
struct U256 {
  uint64_t v[4];  // little-endian limbs
};

U256 from_le(const uint8_t b[32]) {
  U256 r;
  for (int i = 0; i < 4; ++i) {
    uint64_t w = 0;
    for (int k = 7; k >= 0; --k) w = (w << 8) | b[8 * i + k];
    r.v[i] = w;
  }
  return r;
}

void to_le(const U256& a, uint8_t b[32]) {
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 8; ++k) b[8 * i + k] = (uint8_t)(a.v[i] >> (8 * k));
}

bool geq(const U256& a, const U256& b) {
  for (int i = 3; i >= 0; --i) {
    if (a.v[i] != b.v[i]) return a.v[i] > b.v[i];
  }
  return true;
}

bool is_zero(const U256& a) { return (a.v[0] | a.v[1] | a.v[2] | a.v[3]) == 0; }

bool eq(const U256& a, const U256& b) {
  return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2] && a.v[3] == b.v[3];
}

// a + b, returning the carry out of bit 256
uint64_t add_raw(const U256& a, const U256& b, U256& r) {
  u128 c = 0;
  for (int i = 0; i < 4; ++i) {
    c += (u128)a.v[i] + b.v[i];
    r.v[i] = (uint64_t)c;
    c >>= 64;
  }
  return (uint64_t)c;
}

// a - b, returning the borrow
uint64_t sub_raw(const U256& a, const U256& b, U256& r) {
  uint64_t borrow = 0;
  for (int i = 0; i < 4; ++i) {
    u128 d = (u128)a.v[i] - b.v[i] - borrow;
    r.v[i] = (uint64_t)d;
    borrow = (uint64_t)(d >> 64) & 1;
  }
  return borrow;
}

// ------------------------------------------------------------------------------ F_p, p = 2^255 - 19
const U256 kP = {{0xffffffffffffffedull, 0xffffffffffffffffull, 0xffffffffffffffffull, 0x7fffffffffffffffull}};

typedef U256 Fe;  // always fully reduced: 0 <= value < p

Fe fe_small(uint64_t x) { return Fe{{x, 0, 0, 0}}; }

Fe fe_add(const Fe& a, const Fe& b) {
  Fe r;
  add_raw(a, b, r);  // a + b < 2p < 2^256: no carry out
  if (geq(r, kP)) sub_raw(r, kP, r);
  return r;
}

Fe fe_sub(const Fe& a, const Fe& b) {
  Fe r;
  if (sub_raw(a, b, r)) add_raw(r, kP, r);  // a - b + p, the carry out cancels the borrow
  return r;
}

Fe fe_neg(const Fe& a) { return fe_sub(fe_small(0), a); }

Fe fe_mul(const Fe& a, const Fe& b) {
  // schoolbook 4 x 4 limbs into a 512-bit product t
  uint64_t t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 4; ++i) {
    u128 c = 0;
    for (int j = 0; j < 4; ++j) {
      c += (u128)a.v[i] * b.v[j] + t[i + j];
      t[i + j] = (uint64_t)c;
      c >>= 64;
    }
    t[i + 4] = (uint64_t)c;
  }
  // t = lo + 2^256 hi = lo + 38 hi (mod p)
  uint64_t r[5];
  u128 c = 0;
  for (int i = 0; i < 4; ++i) {
    c += (u128)t[i] + (u128)t[i + 4] * 38;
    r[i] = (uint64_t)c;
    c >>= 64;
  }
  r[4] = (uint64_t)c;
  // fold the fifth limb the same way until nothing is left above 2^256
  while (r[4]) {
    u128 cc = (u128)r[0] + (u128)r[4] * 38;
    r[0] = (uint64_t)cc;
    cc >>= 64;
    for (int i = 1; i < 4; ++i) {
      cc += r[i];
      r[i] = (uint64_t)cc;
      cc >>= 64;
    }
    r[4] = (uint64_t)cc;
  }
  Fe out{{r[0], r[1], r[2], r[3]}};
  while (geq(out, kP)) sub_raw(out, kP, out);
  return out;
}

Fe fe_sq(const Fe& a) { return fe_mul(a, a); }

// a^e by left-to-right square-and-multiply over the bits of e
Fe fe_pow(const Fe& a, const U256& e) {
  Fe r = fe_small(1);
  for (int i = 255; i >= 0; --i) {
    r = fe_sq(r);
    if ((e.v[i / 64] >> (i % 64)) & 1) r = fe_mul(r, a);
  }
  return r;
}

const U256 kPm2 = {{0xffffffffffffffebull, 0xffffffffffffffffull, 0xffffffffffffffffull, 0x7fffffffffffffffull}};
const U256 kPp3d8 = {{0xfffffffffffffffeull, 0xffffffffffffffffull, 0xffffffffffffffffull, 0x0fffffffffffffffull}};
const U256 kPm1d4 = {{0xfffffffffffffffbull, 0xffffffffffffffffull, 0xffffffffffffffffull, 0x1fffffffffffffffull}};

Fe fe_inv(const Fe& a) { return fe_pow(a, kPm2); }

Fe g_d, g_d2, g_sqrtm1;  // d, 2d and sqrt(-1), set once by init_constants

// ------------------------------------------------------------------------------ edwards25519
struct Pt {
  Fe X, Y, Z, T;  // x = X/Z, y = Y/Z, xy = T/Z
};

Pt identity() { return Pt{fe_small(0), fe_small(1), fe_small(1), fe_small(0)}; }

Pt from_affine(const Fe& x, const Fe& y) { return Pt{x, y, fe_small(1), fe_mul(x, y)}; }

// unified addition, a = -1 (Hisil, Wong, Carter, Dawson 2008)
Pt add(const Pt& p, const Pt& q) {
  Fe A = fe_mul(fe_sub(p.Y, p.X), fe_sub(q.Y, q.X));
  Fe B = fe_mul(fe_add(p.Y, p.X), fe_add(q.Y, q.X));
  Fe C = fe_mul(fe_mul(p.T, g_d2), q.T);
  Fe D = fe_mul(fe_add(p.Z, p.Z), q.Z);
  Fe E = fe_sub(B, A), F = fe_sub(D, C), G = fe_add(D, C), H = fe_add(B, A);
  return Pt{fe_mul(E, F), fe_mul(G, H), fe_mul(F, G), fe_mul(E, H)};
}

Pt neg(const Pt& p) { return Pt{fe_neg(p.X), p.Y, p.Z, fe_neg(p.T)}; }

// [k]P, k a 256-bit integer, left-to-right double-and-add
Pt scalar_mult(const U256& k, const Pt& p) {
  Pt acc = identity();
  for (int i = 255; i >= 0; --i) {
    acc = add(acc, acc);
    if ((k.v[i / 64] >> (i % 64)) & 1) acc = add(acc, p);
  }
  return acc;
}

bool is_identity(const Pt& p) { return is_zero(p.X) && eq(p.Y, p.Z); }

// Strict decoding of a compressed point (RFC 8032 Sec. 5.1.3): false if y >= p, if x^2 has
// no square root, or if x = 0 with the sign bit set.
bool decode(const uint8_t b[32], Pt& out) {
  U256 y = from_le(b);
  const int sign = (int)(y.v[3] >> 63);
  y.v[3] &= 0x7fffffffffffffffull;
  if (geq(y, kP)) return false;
  Fe yy = fe_sq(y);
  Fe u = fe_sub(yy, fe_small(1));
  Fe v = fe_add(fe_mul(g_d, yy), fe_small(1));
  Fe x2 = fe_mul(u, fe_inv(v));
  Fe x;
  if (is_zero(x2)) {
    if (sign) return false;
    x = fe_small(0);
  } else {
    x = fe_pow(x2, kPp3d8);
    if (!eq(fe_sq(x), x2)) x = fe_mul(x, g_sqrtm1);
    if (!eq(fe_sq(x), x2)) return false;
    if ((int)(x.v[0] & 1) != sign) x = fe_neg(x);
  }
  out = from_affine(x, y);
  return true;
}

void encode(const Pt& p, uint8_t b[32]) {
  Fe zi = fe_inv(p.Z);
  Fe x = fe_mul(p.X, zi), y = fe_mul(p.Y, zi);
  to_le(y, b);
  b[31] |= (uint8_t)((x.v[0] & 1) << 7);
}

Pt g_base;  // G: y = 4/5, x even

void init_constants() {
  // d = -121665 / 121666
  g_d = fe_mul(fe_neg(fe_small(121665)), fe_inv(fe_small(121666)));
  g_d2 = fe_add(g_d, g_d);
  g_sqrtm1 = fe_pow(fe_small(2), kPm1d4);
  Fe y = fe_mul(fe_small(4), fe_inv(fe_small(5)));
  uint8_t enc[32];
  to_le(y, enc);  // sign bit 0: x even
  decode(enc, g_base);
}

// ------------------------------------------------------------------------------ scalars mod q
const U256 kQ = {{0x5812631a5cf5d3edull, 0x14def9dea2f79cd6ull, 0x0000000000000000ull, 0x1000000000000000ull}};

U256 mod_q(U256 k) {
  while (geq(k, kQ)) sub_raw(k, kQ, k);  // at most 15 subtractions below 2^256
  return k;
}

U256 add_q(const U256& a, const U256& b) {  // a, b < q
  U256 r;
  add_raw(a, b, r);
  return mod_q(r);
}

U256 sub_q(const U256& a, const U256& b) {  // a, b < q
  U256 r;
  if (sub_raw(a, b, r)) add_raw(r, kQ, r);
  return r;
}

// a * b mod q by double-and-add over the bits of b (a < q)
U256 mul_q(const U256& a, const U256& b) {
  U256 r{{0, 0, 0, 0}};
  for (int i = 255; i >= 0; --i) {
    r = add_q(r, r);
    if ((b.v[i / 64] >> (i % 64)) & 1) r = add_q(r, a);
  }
  return r;
}

// ------------------------------------------------------------------------------ seeds and hashing
struct Node {
  uint32_t d, i;
  uint8_t seed[16];
};

void prf(int bit, const uint8_t z[16], uint8_t out[16]) {
  uint8_t bb = (uint8_t)bit, h[32];
  sha256_2(z, 16, &bb, 1, h);
  memcpy(out, h, 16);
}

// SRet (Fig. 2a): pop nodes until one covers leaf i, then walk down from it (SC).
bool sret(const std::vector<Node>& ds, uint64_t i, uint8_t out[16]) {
  if (ds.empty()) return false;
  size_t top = ds.size();
  const Node* n = &ds[--top];
  if (i >= ((uint64_t)n->i + 1) << n->d) return false;  // not disclosed yet
  while (i < ((uint64_t)n->i << n->d)) {
    if (top == 0) return false;
    n = &ds[--top];
  }
  uint8_t x[16];
  memcpy(x, n->seed, 16);
  const uint64_t off = i - ((uint64_t)n->i << n->d);
  for (int j = (int)n->d - 1; j >= 0; --j) {
    uint8_t nx[16];
    prf((int)((off >> j) & 1), x, nx);
    memcpy(x, nx, 16);
  }
  memcpy(out, x, 16);
  return true;
}

// e_t = SHA-256(m || x_t) mod q with x_t = SHA-256(x_0[i] || le32(j) || 0x00)[0..16)
bool entry_scalar(const std::vector<Node>& ds, uint32_t n2, uint64_t t, const uint8_t* m, size_t len, U256& e) {
  uint8_t x0[16];
  if (!sret(ds, t / n2, x0)) return false;
  const uint32_t j = (uint32_t)(t % n2);
  uint8_t tail[5] = {(uint8_t)j, (uint8_t)(j >> 8), (uint8_t)(j >> 16), (uint8_t)(j >> 24), 0};
  uint8_t h[32];
  sha256_2(x0, 16, tail, 5, h);
  sha256_2(m, len, h, 16, h);
  e = mod_q(from_le(h));
  return true;
}

std::vector<Node> parse_ds(const uint8_t* ds, uint32_t nodes) {
  std::vector<Node> v(nodes);
  for (uint32_t k = 0; k < nodes; ++k) {
    const uint8_t* p = ds + 24 * (size_t)k;
    v[k].d = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
    v[k].i = (uint32_t)p[4] | ((uint32_t)p[5] << 8) | ((uint32_t)p[6] << 16) | ((uint32_t)p[7] << 24);
    memcpy(v[k].seed, p + 8, 16);
  }
  return v;
}

// [8](R - eY - sG) = O
bool cofactored_check(const Pt& R, const U256& e, const Pt& Y, const U256& s) {
  Pt diff = add(add(R, neg(scalar_mult(e, Y))), neg(scalar_mult(s, g_base)));
  for (int k = 0; k < 3; ++k) diff = add(diff, diff);
  return is_identity(diff);
}

struct Input {
  Pt Y;
  const uint8_t* msgs;
  const uint64_t* offs;
  uint64_t first_index;
  uint32_t n2;
  const uint8_t* s;
  const uint8_t* R;
  std::vector<Node> ds;
};

// One entry's own check (Fig. 4 AVer with one entry): canonical s, decodable R, the equation.
// Returns -1 when its seed is not disclosed.
int verify_entry(const Input& in, uint64_t k, U256* s_out, Pt* R_out) {
  U256 e;
  const uint64_t a = in.offs[k], b = in.offs[k + 1];
  if (!entry_scalar(in.ds, in.n2, in.first_index + k, in.msgs + a, (size_t)(b - a), e)) return -1;
  U256 s = from_le(in.s + 32 * k);
  if (geq(s, kQ)) return 0;
  Pt R;
  if (!decode(in.R + 32 * k, R)) return 0;
  *s_out = s;
  *R_out = R;
  return cofactored_check(R, e, in.Y, s) ? 1 : 0;
}

void run_threads(uint64_t n, int threads, const std::function<void(int, uint64_t, uint64_t)>& fn) {
  if (threads <= 0) threads = (int)std::thread::hardware_concurrency();
  if (threads <= 0) threads = 1;
  if ((uint64_t)threads > n) threads = (int)(n ? n : 1);
  std::vector<std::thread> pool;
  for (int w = 0; w < threads; ++w) {
    const uint64_t lo = n * (uint64_t)w / (uint64_t)threads, hi = n * (uint64_t)(w + 1) / (uint64_t)threads;
    pool.emplace_back(fn, w, lo, hi);
  }
  for (auto& th : pool) th.join();
}

struct Once {
  Once() { init_constants(); }
};
Once g_once;

}  // namespace

extern "C" {

// Return codes: 0 ok, -1 malformed argument (undecodable Y, undisclosed seed).

// e_t for every entry (32 bytes each).
int oracle_hash_entries(const uint8_t* msgs, const uint64_t* offs, uint64_t n, uint64_t first_index, uint32_t n2,
                        const uint8_t* ds, uint32_t ds_nodes, uint8_t* e_out) {
  if (n2 == 0) return -1;
  std::vector<Node> v = parse_ds(ds, ds_nodes);
  for (uint64_t k = 0; k < n; ++k) {
    U256 e;
    if (!entry_scalar(v, n2, first_index + k, msgs + offs[k], (size_t)(offs[k + 1] - offs[k]), e)) return -1;
    to_le(e, e_out + 32 * k);
  }
  return 0;
}

// SRet for epochs first .. first + count - 1 (16 bytes each).
int oracle_epoch_seeds(const uint8_t* ds, uint32_t ds_nodes, uint64_t first, uint64_t count, uint8_t* out) {
  std::vector<Node> v = parse_ds(ds, ds_nodes);
  for (uint64_t k = 0; k < count; ++k)
    if (!sret(v, first + k, out + 16 * k)) return -1;
  return 0;
}

// Point operations for the pins: decode (1 ok, 0 not a point), [k]P, P + Q.
int oracle_decode_ok(const uint8_t b[32]) {
  Pt p;
  return decode(b, p) ? 1 : 0;
}

int oracle_scalar_mult(const uint8_t k[32], const uint8_t P[32], uint8_t out[32]) {
  Pt p;
  if (!decode(P, p)) return -1;
  encode(scalar_mult(from_le(k), p), out);
  return 0;
}

int oracle_base_mult(const uint8_t k[32], uint8_t out[32]) {
  encode(scalar_mult(from_le(k), g_base), out);
  return 0;
}

// POSLO-F Distill by the per-entry definition (Sec. 4.3, Fig. 3b at entry granularity): the
// ascending global indices of the entries failing their own check, and ccd^v = (sum of the
// valid s_t mod q, sum of the valid R_t).  invalid_out needs room for n indices.
int oracle_distill_f(const uint8_t Y[32], const uint8_t* msgs, const uint64_t* offs, uint64_t n,
                     uint64_t first_index, uint32_t n2, const uint8_t* s, const uint8_t* R, const uint8_t* ds,
                     uint32_t ds_nodes, int threads, uint64_t* invalid_out, uint64_t* n_invalid,
                     uint8_t ccd_s[32], uint8_t ccd_R[32]) {
  if (n2 == 0) return -1;
  Input in;
  if (!decode(Y, in.Y)) return -1;
  in.msgs = msgs;
  in.offs = offs;
  in.first_index = first_index;
  in.n2 = n2;
  in.s = s;
  in.R = R;
  in.ds = parse_ds(ds, ds_nodes);
  std::vector<uint8_t> ok(n, 0);
  const int nt = threads <= 0 ? (int)std::thread::hardware_concurrency() : threads;
  std::vector<U256> part_s((size_t)(nt > 0 ? nt : 1) + 1, U256{{0, 0, 0, 0}});
  std::vector<Pt> part_R((size_t)(nt > 0 ? nt : 1) + 1, identity());
  std::vector<int> part_err(part_s.size(), 0);
  run_threads(n, nt, [&](int w, uint64_t lo, uint64_t hi) {
    U256 acc_s{{0, 0, 0, 0}};
    Pt acc_R = identity();
    for (uint64_t k = lo; k < hi; ++k) {
      U256 sk;
      Pt Rk;
      const int r = verify_entry(in, k, &sk, &Rk);
      if (r < 0) {
        part_err[w] = 1;
        return;
      }
      ok[k] = (uint8_t)r;
      if (r) {
        acc_s = add_q(acc_s, sk);
        acc_R = add(acc_R, Rk);
      }
    }
    part_s[w] = acc_s;
    part_R[w] = acc_R;
  });
  U256 tot_s{{0, 0, 0, 0}};
  Pt tot_R = identity();
  for (size_t w = 0; w < part_s.size(); ++w) {
    if (part_err[w]) return -1;
    tot_s = add_q(tot_s, part_s[w]);
    tot_R = add(tot_R, part_R[w]);
  }
  uint64_t c = 0;
  for (uint64_t k = 0; k < n; ++k)
    if (!ok[k]) invalid_out[c++] = first_index + k;
  *n_invalid = c;
  to_le(tot_s, ccd_s);
  encode(tot_R, ccd_R);
  return 0;
}

// POSLO-F AVer with unit coefficients (Fig. 4): every s_t canonical, every R_t decodable and
// [8](sum R_t - (sum e_t) Y - (sum s_t) G) = O.  *accept = 1 or 0.
int oracle_aver_f(const uint8_t Y[32], const uint8_t* msgs, const uint64_t* offs, uint64_t n, uint64_t first_index,
                  uint32_t n2, const uint8_t* s, const uint8_t* R, const uint8_t* ds, uint32_t ds_nodes,
                  uint8_t* accept) {
  if (n2 == 0) return -1;
  Pt Yp;
  if (!decode(Y, Yp)) return -1;
  std::vector<Node> v = parse_ds(ds, ds_nodes);
  U256 se{{0, 0, 0, 0}}, ss{{0, 0, 0, 0}};
  Pt sR = identity();
  for (uint64_t k = 0; k < n; ++k) {
    U256 sk = from_le(s + 32 * k);
    Pt Rk;
    if (geq(sk, kQ) || !decode(R + 32 * k, Rk)) {  // a malformed entry rejects the batch
      *accept = 0;
      return 0;
    }
    U256 e;
    if (!entry_scalar(v, n2, first_index + k, msgs + offs[k], (size_t)(offs[k + 1] - offs[k]), e)) return -1;
    se = add_q(se, e);
    ss = add_q(ss, sk);
    sR = add(sR, Rk);
  }
  *accept = (uint8_t)cofactored_check(sR, se, Yp, ss);
  return 0;
}

// POSLO-F.Sig (Fig. 4) with the BPV online step of Definition 3, for test data: entry t
// (global index first_index + t) takes r_t = sum of the table scalars bpv_r[k] over its
// subset (k per entry, indices into the v-entry table), R_t = sum of [bpv_r[k]]G, x_t from
// the seed tree under root (depth D), e_t = H(m_t || x_t) and s_t = r_t - e_t y mod q.
// Writes s_t and the encoded R_t (32 bytes each).
int oracle_sign_f(const uint8_t y[32], const uint8_t root[16], uint32_t D, uint32_t n2, const uint8_t* bpv_r,
                  uint32_t v, uint32_t k, const uint16_t* subsets, const uint8_t* msgs, const uint64_t* offs,
                  uint64_t n, uint64_t first_index, int threads, uint8_t* s_out, uint8_t* R_out) {
  if (n2 == 0 || v == 0) return -1;
  const U256 yy = mod_q(from_le(y));
  std::vector<U256> r(v);
  std::vector<Pt> Rt(v);
  for (uint32_t i = 0; i < v; ++i) {
    r[i] = mod_q(from_le(bpv_r + 32 * (size_t)i));
    Rt[i] = scalar_mult(r[i], g_base);
  }
  std::vector<Node> ds(1);
  ds[0].d = D;
  ds[0].i = 0;
  memcpy(ds[0].seed, root, 16);
  std::vector<int> bad(1, 0);
  std::vector<uint8_t> fail(n ? n : 1, 0);
  run_threads(n, threads, [&](int, uint64_t lo, uint64_t hi) {
    for (uint64_t t = lo; t < hi; ++t) {
      U256 rt{{0, 0, 0, 0}};
      Pt R = identity();
      for (uint32_t j = 0; j < k; ++j) {
        const uint16_t idx = subsets[t * k + j];
        if (idx >= v) {
          fail[t] = 1;
          return;
        }
        rt = add_q(rt, r[idx]);
        R = add(R, Rt[idx]);
      }
      U256 e;
      if (!entry_scalar(ds, n2, first_index + t, msgs + offs[t], (size_t)(offs[t + 1] - offs[t]), e)) {
        fail[t] = 1;
        return;
      }
      to_le(sub_q(rt, mul_q(e, yy)), s_out + 32 * t);
      encode(R, R_out + 32 * t);
    }
  });
  for (uint64_t t = 0; t < n; ++t)
    if (fail[t]) return -1;
  return 0;
}

}  // extern "C"
