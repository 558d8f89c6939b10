"""CPU oracle for POSLO batch verification (test infrastructure only).

This is the plain, slow, obviously-correct statement of what the GPU path computes.  It
is imported by the tests, by the package smoke check and by the benchmark's CPU-baseline
leg, and by nothing else: the product path never calls it.  It shares no code with the
CUDA library; the two meet only through the seeded inputs of ``synth``.

Everything is exact integer arithmetic with Python ints.  SHA-256 is hashlib (a library
primitive used as one step).  Section, figure and equation numbers refer to Nouma and
Yavuz, "Lightweight and High-Throughput Secure Logging for Internet of Things and Cold
Cloud Continuum" (arXiv 2506.08781).

Readings of points the paper leaves open:
  * group: the prime-order subgroup of edwards25519 (the paper names FourQ with
    |q| = 256, which is self-inconsistent; no FourQ constants are given);
  * PRF_b(z) = SHA-256(z || byte b)[:16] for the seed tree; the per-entry seed is
    x_i^j = PRF_0(x_0[i] || j) = SHA-256(x_0[i] || le32(j) || 0x00)[:16], j 0-based;
  * e = SHA-256(m || x) read little-endian, reduced mod q;
  * POSLO+ (``instantiation("POSLO+")``): PRF = MMO-AES-128 with kappa = 127, H = MDC-2
    over AES-128, with the initial values and padding stated beside ``mmo``;
  * POSLO-C nonces r_i^j = SHA-256(r || le32(i) || le32(j) || 0x00) mod q;
  * points are 32-byte compressed edwards25519 encodings, decoded strictly; scalars are
    32-byte little-endian and must be canonical (< q);
  * every group equation is checked with the cofactor: [8](R - eY - sG) = O.

Parity pins: see tests/test_oracle_pins.py (hashlib KATs, libsodium group operations,
the seed-tree worked example of Sec. 4.1, closed forms and brute force).
"""
from __future__ import annotations

import hashlib
import struct
from dataclasses import dataclass

# ----------------------------------------------------------------------------------
# edwards25519 (RFC 8032 Sec. 5.1 parameters)
# ----------------------------------------------------------------------------------
P = 2 ** 255 - 19
Q = 2 ** 252 + 27742317777372353535851937790883648493
D = (-121665 * pow(121666, P - 2, P)) % P
SQRT_M1 = pow(2, (P - 1) // 4, P)
COFACTOR = 8

IDENTITY = (0, 1, 1, 0)          # extended coordinates (X:Y:Z:T), x = X/Z, y = Y/Z, xy = T/Z


def _recover_x(y: int, sign: int):
    """x with x^2 = (y^2 - 1) / (d y^2 + 1) and parity `sign`, or None (RFC 8032 5.1.3)."""
    if y >= P:
        return None
    u = (y * y - 1) % P
    v = (D * y * y + 1) % P
    x2 = u * pow(v, P - 2, P) % P
    if x2 == 0:
        return None if sign else 0
    x = pow(x2, (P + 3) // 8, P)
    if (x * x - x2) % P != 0:
        x = x * SQRT_M1 % P
    if (x * x - x2) % P != 0:
        return None
    if x & 1 != sign:
        x = P - x
    return x


def point_from_affine(x: int, y: int):
    return (x % P, y % P, 1, x * y % P)


def to_affine(pt):
    X, Y, Z, _ = pt
    zi = pow(Z, P - 2, P)
    return X * zi % P, Y * zi % P


def on_curve(pt) -> bool:
    x, y = to_affine(pt)
    return (-x * x + y * y - 1 - D * x * x * y * y) % P == 0


def decode_point(b: bytes):
    """Strict decoding of a 32-byte compressed point; None if not a curve point."""
    if len(b) != 32:
        return None
    v = int.from_bytes(b, "little")
    sign = v >> 255
    y = v & ((1 << 255) - 1)
    x = _recover_x(y, sign)
    if x is None:
        return None
    return point_from_affine(x, y)


def encode_point(pt) -> bytes:
    x, y = to_affine(pt)
    return (y | ((x & 1) << 255)).to_bytes(32, "little")


def point_add(p1, p2):
    """Unified addition in extended coordinates for a = -1 (Hisil, Wong, Carter, Dawson,
    "Twisted Edwards curves revisited", 2008); complete on edwards25519 since d is a
    non-square."""
    X1, Y1, Z1, T1 = p1
    X2, Y2, Z2, T2 = p2
    A = (Y1 - X1) * (Y2 - X2) % P
    B = (Y1 + X1) * (Y2 + X2) % P
    C = T1 * 2 * D * T2 % P
    Dd = Z1 * 2 * Z2 % P
    E, F, G_, H = B - A, Dd - C, Dd + C, B + A
    return (E * F % P, G_ * H % P, F * G_ % P, E * H % P)


def point_neg(pt):
    X, Y, Z, T = pt
    return ((-X) % P, Y, Z, (-T) % P)


def point_sub(p1, p2):
    return point_add(p1, point_neg(p2))


def is_identity(pt) -> bool:
    X, Y, Z, _ = pt
    return X % P == 0 and (Y - Z) % P == 0


def point_eq(p1, p2) -> bool:
    X1, Y1, Z1, _ = p1
    X2, Y2, Z2, _ = p2
    return (X1 * Z2 - X2 * Z1) % P == 0 and (Y1 * Z2 - Y2 * Z1) % P == 0


def scalar_mult(k: int, pt):
    """Textbook left-to-right double-and-add, k >= 0."""
    acc = IDENTITY
    for bit in bin(k)[2:] if k else "":
        acc = point_add(acc, acc)
        if bit == "1":
            acc = point_add(acc, pt)
    return acc


def _base_point():
    y = 4 * pow(5, P - 2, P) % P
    return point_from_affine(_recover_x(y, 0), y)


G = _base_point()


def mul_by_cofactor(pt):
    return scalar_mult(COFACTOR, pt)


# ----------------------------------------------------------------------------------
# scalars mod q
# ----------------------------------------------------------------------------------

def scalar_to_bytes(k: int) -> bytes:
    return (k % Q).to_bytes(32, "little")


def scalar_from_bytes(b: bytes):
    """Canonical 32-byte little-endian scalar, or None if >= q."""
    k = int.from_bytes(b, "little")
    return k if k < Q else None


# ----------------------------------------------------------------------------------
# H and PRF (Sec. 7.2 instantiation "POSLO": SHA-256 for both)
# ----------------------------------------------------------------------------------

def sha256(data: bytes) -> bytes:
    return hashlib.sha256(data).digest()


def prf_sha(bit: int, z: bytes) -> bytes:
    """PRF_bit(z) = F(z || bit) with F = SHA-256 truncated to kappa = 128 bits."""
    return sha256(z + bytes([bit]))[:16]


def entry_seed_sha(x0: bytes, j: int) -> bytes:
    """x_i^j = PRF_0(x_0[i] || j) (Fig. 3a AVer, Fig. 6 Agg-eKeys)."""
    return sha256(x0 + struct.pack("<I", j) + b"\x00")[:16]


def hash_to_scalar_sha(m: bytes, x: bytes) -> int:
    """e = H(m || x) mod q."""
    return int.from_bytes(sha256(m + x), "little") % Q


# ----------------------------------------------------------------------------------
# AES-128 (FIPS-197), the block cipher E of the POSLO+ instantiation (Sec. 7.2)
# ----------------------------------------------------------------------------------

def gf_mul(a: int, b: int) -> int:
    """Product in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1 (FIPS-197 Sec. 4.2)."""
    r = 0
    for _ in range(8):
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a & 0x100:
            a ^= 0x11B
    return r


def _sbox_entry(x: int) -> int:
    """SubBytes (FIPS-197 Sec. 5.1.1): the multiplicative inverse in GF(2^8) ({00} maps
    to {00}), then the affine map b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i with
    c = {63}."""
    inv = 0
    if x:
        inv = 1
        for _ in range(254):          # x^254 = x^-1 in a field of 256 elements
            inv = gf_mul(inv, x)
    out = 0
    for i in range(8):
        bit = 0
        for k in (0, 4, 5, 6, 7):
            bit ^= (inv >> ((i + k) % 8)) & 1
        out |= (bit ^ ((0x63 >> i) & 1)) << i
    return out


SBOX = [_sbox_entry(x) for x in range(256)]


def aes128_key_expansion(key: bytes) -> list:
    """KeyExpansion (FIPS-197 Sec. 5.2): 44 words w[i], each a list of 4 bytes."""
    w = [list(key[4 * i:4 * i + 4]) for i in range(4)]
    rcon = 1
    for i in range(4, 44):
        t = list(w[i - 1])
        if i % 4 == 0:
            t = t[1:] + t[:1]                     # RotWord
            t = [SBOX[b] for b in t]              # SubWord
            t[0] ^= rcon
            rcon = gf_mul(rcon, 2)
        w.append([a ^ b for a, b in zip(w[i - 4], t)])
    return w


def aes128_encrypt(key: bytes, block: bytes) -> bytes:
    """Cipher (FIPS-197 Sec. 5.1): the state is 4x4 bytes, state[r][c] = in[r + 4c]."""
    w = aes128_key_expansion(key)
    st = [[block[r + 4 * c] for c in range(4)] for r in range(4)]

    def add_round_key(rnd):
        for c in range(4):
            for r in range(4):
                st[r][c] ^= w[4 * rnd + c][r]

    add_round_key(0)
    for rnd in range(1, 11):
        for r in range(4):                        # SubBytes
            for c in range(4):
                st[r][c] = SBOX[st[r][c]]
        for r in range(1, 4):                     # ShiftRows: row r rotates left by r
            st[r] = st[r][r:] + st[r][:r]
        if rnd < 10:                              # MixColumns
            for c in range(4):
                a = [st[r][c] for r in range(4)]
                st[0][c] = gf_mul(a[0], 2) ^ gf_mul(a[1], 3) ^ a[2] ^ a[3]
                st[1][c] = a[0] ^ gf_mul(a[1], 2) ^ gf_mul(a[2], 3) ^ a[3]
                st[2][c] = a[0] ^ a[1] ^ gf_mul(a[2], 2) ^ gf_mul(a[3], 3)
                st[3][c] = gf_mul(a[0], 3) ^ a[1] ^ a[2] ^ gf_mul(a[3], 2)
        add_round_key(rnd)
    return bytes(st[r][c] for c in range(4) for r in range(4))


def _xor(a: bytes, b: bytes) -> bytes:
    return bytes(x ^ y for x, y in zip(a, b))


# ----------------------------------------------------------------------------------
# MMO and MDC-2 over AES-128 (Def. MMO, Def. MDC-2; Sec. 7.2 instantiation "POSLO+")
# ----------------------------------------------------------------------------------
# Readings: the initial values are 16 bytes of 0x52 (MMO and the first MDC-2 chain) and 16
# bytes of 0x25 (the second MDC-2 chain), the DES-era MDC-2 values widened to the AES block;
# padding is a 1 bit then 0 bits up to a whole number of blocks, t = ceil((k+1)/128) blocks
# for MDC-2 (an input of whole blocks gains a padding block); MMO pads only an input that
# is not a whole number of blocks, so the kappa = 127 PRF input (127 + 1 bits) is one block
# and one AES call, as Sec. 7.2 states.

IV_A = b"\x52" * 16
IV_B = b"\x25" * 16


def _pad_blocks(data: bytes, always: bool) -> list:
    if always or len(data) % 16:
        data = data + b"\x80" + bytes((-len(data) - 1) % 16)
    return [data[i:i + 16] for i in range(0, len(data), 16)]


def mmo_chain(E, iv: bytes, blocks: list) -> bytes:
    """The MMO chaining of Def. MMO over already padded blocks: h_0 = iv,
    h_i = E_{h_{i-1}}(m_i) xor m_i (the chaining value keys the cipher, the block is
    enciphered); returns h_t.  E(key, block) is the block cipher."""
    h = iv
    for m in blocks:
        h = _xor(E(h, m), m)
    return h


def mdc2_chain(E, iv1: bytes, iv2: bytes, blocks: list, key1=None, key2=None) -> bytes:
    """The MDC-2 chaining of Def. MDC-2 over already padded blocks: two MMO steps on the same
    block from the two chaining values (keyed through key1/key2 when the cipher needs a key
    transform, none for AES), then the chains exchange their right halves:
    h_i = A_L || B_R and h'_i = B_L || A_R.  Returns h_t || h'_t."""
    h, h2 = iv1, iv2
    half = len(iv1) // 2
    for m in blocks:
        a = _xor(E(key1(h) if key1 else h, m), m)
        b = _xor(E(key2(h2) if key2 else h2, m), m)
        h, h2 = a[:half] + b[half:], b[:half] + a[half:]
    return h + h2


def mmo(data: bytes) -> bytes:
    """MMO over AES-128: h_0 = IV_A, padding as stated above; the digest is h_t (16 bytes)."""
    return mmo_chain(aes128_encrypt, IV_A, _pad_blocks(data, always=False))


def mdc2(data: bytes) -> bytes:
    """MDC-2 over AES-128: chains from IV_A and IV_B, exchanging bytes 8..15 after each
    block; the digest is h_t || h'_t (32 bytes)."""
    return mdc2_chain(aes128_encrypt, IV_A, IV_B, _pad_blocks(data, always=True))


def _k127(x: bytes, bit: int) -> bytes:
    """A 16-byte seed whose least significant bit (bit 0 of byte 15) carries the PRF bit:
    the kappa = 127 seed x (its first 127 bits) followed by j (Sec. 7.2)."""
    return x[:15] + bytes([(x[15] & 0xFE) | bit])


def prf_aes(bit: int, z: bytes) -> bytes:
    """PRF_bit(z) = MMO-AES-128(z || bit) with kappa = 127: one block, one AES call; the
    output is truncated to 127 bits (bit 0 of byte 15 cleared)."""
    return _k127(mmo(_k127(z, bit)), 0)


def entry_seed_aes(x0: bytes, j: int) -> bytes:
    """x_i^j = PRF_0(x_0[i] || j): MMO over the 127-bit seed, the PRF bit 0 and le32(j)
    (20 bytes, padded to two blocks), truncated to 127 bits."""
    return _k127(mmo(_k127(x0, 0) + struct.pack("<I", j)), 0)


def hash_to_scalar_aes(m: bytes, x: bytes) -> int:
    """e = H(m || x) mod q with H = MDC-2-AES-128 (32-byte digest read little-endian)."""
    return int.from_bytes(mdc2(m + x), "little") % Q


# ----------------------------------------------------------------------------------
# Instantiation in force (Table "instantiations", Sec. 7.2): POSLO = SHA-256 for PRF and H,
# POSLO+ = MMO-AES-128 for PRF and MDC-2-AES-128 for H.  The POSLO-C nonces stay SHA-256
# (a signer-side derivation the verifier never recomputes).
# ----------------------------------------------------------------------------------

INSTANTIATIONS = {
    "POSLO": (prf_sha, entry_seed_sha, hash_to_scalar_sha),
    "POSLO+": (prf_aes, entry_seed_aes, hash_to_scalar_aes),
}
_current = ["POSLO"]


def prf(bit: int, z: bytes) -> bytes:
    return INSTANTIATIONS[_current[0]][0](bit, z)


def entry_seed(x0: bytes, j: int) -> bytes:
    return INSTANTIATIONS[_current[0]][1](x0, j)


def hash_to_scalar(m: bytes, x: bytes) -> int:
    return INSTANTIATIONS[_current[0]][2](m, x)


class instantiation:
    """``with instantiation("POSLO+"): ...`` evaluates every definition below with the
    AES-based PRF and H."""

    def __init__(self, name: str):
        if name not in INSTANTIATIONS:
            raise ValueError(name)
        self.name = name

    def __enter__(self):
        self.prev = _current[0]
        _current[0] = self.name
        return self

    def __exit__(self, *exc):
        _current[0] = self.prev
        return False


def nonce_c(r: bytes, i: int, j: int) -> int:
    """POSLO-C one-time nonce r_i^j = PRF_0(r || i || j) mod q (Fig. 3a Kg)."""
    return int.from_bytes(sha256(r + struct.pack("<II", i, j) + b"\x00"), "little") % Q


# ----------------------------------------------------------------------------------
# POSLOT seed tree and seed management functions (Sec. 4.1, Eq. 1, Fig. 2a)
# ----------------------------------------------------------------------------------

def tree_node(root: bytes, D_: int, d: int, i: int) -> bytes:
    """x_d[i] by the recursive definition of Eq. 1: even children take PRF_0 of the
    parent, odd children PRF_1; x_D[0] is the root."""
    if not (0 <= d <= D_ and 0 <= i < (1 << (D_ - d))):
        raise ValueError("node out of range")
    if d == D_:
        return root
    parent = tree_node(root, D_, d + 1, i // 2)
    return prf(i % 2, parent)


def SC(x_src: bytes, d0: int, i0: int, d1: int, i1: int) -> bytes:
    """Seed computation: walk from x_{d0}[i0] down to its descendant x_{d1}[i1]; bit j of
    the relative offset (most significant first) chooses PRF_0 or PRF_1 (Fig. 2a)."""
    if not (d1 <= d0 and i0 * (1 << (d0 - d1)) <= i1 < (i0 + 1) * (1 << (d0 - d1))):
        raise ValueError("SC: target is not a descendant")
    x = x_src
    off = i1 - i0 * (1 << (d0 - d1))
    for j in range(d0 - d1 - 1, -1, -1):
        x = prf((off >> j) & 1, x)
    return x


@dataclass(frozen=True)
class Node:
    d: int
    i: int
    seed: bytes


def SSO(ds: list, root: bytes, D_: int, i: int):
    """Seed storage optimiser (Fig. 2a): returns (ds_i, x_0[i]) from ds_{i-1}.  While the
    top of the stack sits at the current depth it is merged away and we move one level
    up; then the node reached is pushed."""
    if not 0 <= i < (1 << D_):
        raise ValueError("SSO: epoch out of range")
    ds = list(ds)
    d1, i1 = 0, i
    while ds and ds[-1].d == d1:
        ds.pop()
        d1 += 1
        i1 //= 2
    node = Node(d1, i1, SC(root, D_, 0, d1, i1))
    ds.append(node)
    return ds, SC(node.seed, d1, i1, 0, i)


def SRet(ds: list, i_target: int) -> bytes:
    """Seed retrieval (Fig. 2a): pop nodes until one covers leaf i_target, then walk down
    to it.  Raises ValueError for the paper's bottom symbol."""
    stack = list(ds)
    if not stack:
        raise ValueError("SRet: empty ds")
    n = stack.pop()
    if i_target >= (n.i + 1) << n.d:
        raise ValueError("SRet: leaf not yet disclosed")
    while i_target < n.i << n.d:
        if not stack:
            raise ValueError("SRet: no ancestor in ds")
        n = stack.pop()
    return SC(n.seed, n.d, n.i, 0, i_target)


def ds_after(root: bytes, D_: int, i: int) -> list:
    """ds_i obtained by running SSO for epochs 0..i from an empty stack."""
    ds = []
    for k in range(i + 1):
        ds, _ = SSO(ds, root, D_, k)
    return ds


def ds_root(root: bytes, D_: int) -> list:
    """The final disclosure: the root alone (Sec. 4.1)."""
    return [Node(D_, 0, root)]


def ds_serialize(ds: list) -> bytes:
    """Wire form: 24 bytes per node, bottom of the stack first: le32 depth, le32 index,
    16-byte seed."""
    return b"".join(struct.pack("<II", n.d, n.i) + n.seed for n in ds)


# ----------------------------------------------------------------------------------
# POSLO-C (Fig. 3a)
# ----------------------------------------------------------------------------------

@dataclass
class SecretKeyC:
    y: int
    r: bytes
    root: bytes
    D: int
    n2: int


def kg_c(y_bytes: bytes, r: bytes, root: bytes, D_: int, n2: int):
    """POSLO-C.Kg: Y = yG and, per epoch i, R~_i = (sum_j r_i^j mod q) G."""
    y = int.from_bytes(y_bytes, "little") % Q
    if y == 0:
        raise ValueError("y must be non-zero")
    Y = scalar_mult(y, G)
    epoch_R = []
    for i in range(1 << D_):
        ri = sum(nonce_c(r, i, j) for j in range(n2)) % Q
        epoch_R.append(encode_point(scalar_mult(ri, G)))
    return SecretKeyC(y, r, root, D_, n2), encode_point(Y), epoch_R


def sig_c(sk: SecretKeyC, i: int, msgs_i: list) -> bytes:
    """POSLO-C.Sig for epoch i: s~_i = sum_j (r_i^j - e_i^j y) mod q.  The disclosed
    seeds ds_i that go with it come from SSO (ds_after)."""
    if len(msgs_i) != sk.n2:
        raise ValueError("epoch must hold n2 entries")
    x0 = SC(sk.root, sk.D, 0, 0, i)
    s = 0
    for j, m in enumerate(msgs_i):
        e = hash_to_scalar(m, entry_seed(x0, j))
        s = (s + nonce_c(sk.r, i, j) - e * sk.y) % Q
    return scalar_to_bytes(s)


def agg_scalars(scalars: list) -> bytes:
    """POSLO-C.Agg on scalar components: sum mod q."""
    return scalar_to_bytes(sum(int.from_bytes(s, "little") for s in scalars) % Q)


def agg_points(points: list) -> bytes:
    """POSLO-C.Agg on commitments: the group operation over all of them."""
    acc = IDENTITY
    for b in points:
        pt = decode_point(b)
        if pt is None:
            raise ValueError("undecodable point")
        acc = point_add(acc, pt)
    return encode_point(acc)


def cofactored_check(R, e: int, Y, s: int) -> bool:
    """[8](R - eY - sG) = O."""
    diff = point_sub(point_sub(R, scalar_mult(e % Q, Y)), scalar_mult(s % Q, G))
    return is_identity(mul_by_cofactor(diff))


def aver_c(Y_bytes: bytes, epochs: list, msgs: list, n2: int, s_agg: bytes, R_agg, ds: list):
    """POSLO-C.AVer (Fig. 3a): `epochs` lists the epoch indices I; msgs[k] holds the n2
    entries of epoch epochs[k]; R_agg is either the aggregate R~ (bytes) or the list of
    per-epoch R~_i from pk.  Returns True/False; raises ValueError for bottom."""
    if any(len(mk) != n2 for mk in msgs) or len(msgs) != len(epochs):
        raise ValueError("epoch sizes must equal n2")
    Y = decode_point(Y_bytes)
    if Y is None:
        raise ValueError("bad public key")
    if isinstance(R_agg, (bytes, bytearray)):
        R = decode_point(bytes(R_agg))
    else:
        R = IDENTITY
        for b in R_agg:
            pt = decode_point(b)
            if pt is None:
                return False
            R = point_add(R, pt)
    s = scalar_from_bytes(s_agg)
    if R is None or s is None:
        return False
    e = 0
    for i, mk in zip(epochs, msgs):
        x0 = SRet(ds, i)
        for j, m in enumerate(mk):
            e = (e + hash_to_scalar(m, entry_seed(x0, j))) % Q
    return cofactored_check(R, e, Y, s)


# ----------------------------------------------------------------------------------
# POSLO-C distillation and selective batch verification (Fig. 3b)
# ----------------------------------------------------------------------------------
# Readings: epochs are numbered from 0 and processed in order; umbrella l covers the g =
# n1 / n^u consecutive epochs [l g, (l+1) g) of the batch and is closed after the last of
# them, valid or not (the listing tests "i = 0 mod floor(n1/n^u)" inside the valid branch,
# which would merge two groups whenever a group ends with an invalid epoch, and SeBVer's U
# mode verifies exactly one group per umbrella; its range "floor(n^u/n)" is read as g); an
# umbrella collects the valid epochs of its group, so a group with none holds (0, O).

@dataclass
class CcdC:
    sv: bytes                 # s~^v: sum of the valid epochs' s~_i mod q
    Rv: bytes                 # R~^v: sum of their R~_i (encoded)
    umbrellas: list           # [(s~^u, R~^u, l)] for l = 0 .. n^u - 1
    invalid: list             # [(s~_i, R~_i, i)] for the invalid epochs, ascending i


def distill_c(Y_bytes: bytes, epochs: list, msgs: list, n2: int, s_list: list, R_list: list, ds: list,
              n_umbrella: int):
    """POSLO-C.Distill over epochs (Fig. 3b, C.Distill, one call per epoch in order):
    epoch i is verified on its own, b_i = C.AVer(pk, m_i, (s~_i, R~_i)); a valid epoch joins
    ccd^v and its group's umbrella, an invalid one is listed in ccd^i.  Returns (b, ccd)."""
    n1 = len(epochs)
    if n_umbrella <= 0 or n1 % n_umbrella:
        raise ValueError("n1 must be a multiple of n^u")
    g = n1 // n_umbrella
    b = []
    sv, Rv = 0, IDENTITY
    su, Ru = 0, IDENTITY
    umbrellas, invalid = [], []
    for k, i in enumerate(epochs):
        ok = aver_c(Y_bytes, [i], [msgs[k]], n2, s_list[k], [R_list[k]], ds)
        b.append(ok)
        if ok:
            si = int.from_bytes(s_list[k], "little")
            Ri = decode_point(R_list[k])
            sv, Rv = (sv + si) % Q, point_add(Rv, Ri)
            su, Ru = (su + si) % Q, point_add(Ru, Ri)
        else:
            invalid.append((s_list[k], R_list[k], i))
        if (k + 1) % g == 0:
            umbrellas.append((scalar_to_bytes(su), encode_point(Ru), k // g))
            su, Ru = 0, IDENTITY
    return b, CcdC(scalar_to_bytes(sv), encode_point(Rv), umbrellas, invalid)


def sebver_c(Y_bytes: bytes, epochs: list, msgs: list, n2: int, ccd: CcdC, ds: list, mode: str) -> list:
    """POSLO-C.SeBVer (Fig. 3b): 'V' verifies every epoch outside ccd^i against ccd^v (one
    bit); 'U' verifies, per umbrella, its group's epochs outside ccd^i against the umbrella
    (one bit each); 'I' verifies each invalid epoch against its own sigma~_i (one bit each)."""
    bad = {i for _, _, i in ccd.invalid}
    pos = {i: k for k, i in enumerate(epochs)}
    if mode == "V":
        keep = [k for k, i in enumerate(epochs) if i not in bad]
        return [aver_c(Y_bytes, [epochs[k] for k in keep], [msgs[k] for k in keep], n2, ccd.sv, ccd.Rv, ds)]
    if mode == "U":
        g = len(epochs) // len(ccd.umbrellas)
        out = []
        for su, Ru, l in ccd.umbrellas:
            keep = [k for k in range(l * g, (l + 1) * g) if epochs[k] not in bad]
            out.append(aver_c(Y_bytes, [epochs[k] for k in keep], [msgs[k] for k in keep], n2, su, Ru, ds))
        return out
    if mode == "I":
        return [aver_c(Y_bytes, [i], [msgs[pos[i]]], n2, si, [Ri], ds) for si, Ri, i in ccd.invalid]
    raise ValueError("mode must be V, U or I")


# ----------------------------------------------------------------------------------
# POSLO-F (Fig. 4) with the BPV generator (Definition 3)
# ----------------------------------------------------------------------------------

@dataclass
class SecretKeyF:
    y: int
    root: bytes
    D: int
    n2: int
    bpv_r: list
    bpv_R: list        # extended points


def kg_f(y_bytes: bytes, root: bytes, D_: int, n2: int, bpv_r_bytes: bytes):
    """POSLO-F.Kg: Y = yG and the BPV table {r_k, R_k = r_k G}."""
    y = int.from_bytes(y_bytes, "little") % Q
    if y == 0:
        raise ValueError("y must be non-zero")
    v = len(bpv_r_bytes) // 32
    rs = [int.from_bytes(bpv_r_bytes[32 * k:32 * k + 32], "little") % Q for k in range(v)]
    Rs = [scalar_mult(r, G) for r in rs]
    return SecretKeyF(y, root, D_, n2, rs, Rs), encode_point(scalar_mult(y, G))


def bpv_table_encoded(sk: SecretKeyF) -> list:
    return [encode_point(R) for R in sk.bpv_R]


def sig_f(sk: SecretKeyF, t: int, m: bytes, subset):
    """POSLO-F.Sig for entry t: (r_t, R_t) = BPV.Online over `subset`, e_t = H(m || x_t)
    with x_t = PRF_0(x_0[i] || j), s_t = r_t - e_t y.  Returns (s, R, x) as bytes."""
    i, j = divmod(t, sk.n2)
    x0 = SC(sk.root, sk.D, 0, 0, i)
    r = sum(sk.bpv_r[k] for k in subset) % Q
    R = IDENTITY
    for k in subset:
        R = point_add(R, sk.bpv_R[k])
    x = entry_seed(x0, j)
    e = hash_to_scalar(m, x)
    s = (r - e * sk.y) % Q
    return scalar_to_bytes(s), encode_point(R), x


def entry_scalar(ds: list, n2: int, t: int, m: bytes) -> int:
    """e_t of entry t under the disclosed seeds ds."""
    i, j = divmod(t, n2)
    return hash_to_scalar(m, entry_seed(SRet(ds, i), j))


def verify_entry_f(Y, e: int, s_bytes: bytes, R_bytes: bytes) -> bool:
    """Single-entry POSLO-F check (Fig. 4 AVer, |m| = 1): s canonical, R decodable and
    [8](R - eY - sG) = O."""
    s = scalar_from_bytes(s_bytes)
    R = decode_point(R_bytes)
    if s is None or R is None:
        return False
    return cofactored_check(R, e, Y, s)


def aver_f(Y_bytes: bytes, msgs: list, first_index: int, n2: int, s_list: list, R_list: list,
           ds: list) -> bool:
    """POSLO-F.AVer over a batch (Fig. 4: C.AVer steps 2-8 with R~ = sum R_t): all s_t
    canonical, all R_t decodable, and [8](sum R_t - (sum e_t) Y - (sum s_t) G) = O."""
    Y = decode_point(Y_bytes)
    if Y is None:
        raise ValueError("bad public key")
    R = IDENTITY
    s = 0
    e = 0
    for k, m in enumerate(msgs):
        sk = scalar_from_bytes(s_list[k])
        Rk = decode_point(R_list[k])
        if sk is None or Rk is None:
            return False
        R = point_add(R, Rk)
        s = (s + sk) % Q
        e = (e + entry_scalar(ds, n2, first_index + k, m)) % Q
    return cofactored_check(R, e, Y, s)


def distill_f(Y_bytes: bytes, msgs: list, first_index: int, n2: int, s_list: list, R_list: list,
              ds: list):
    """POSLO-F Distill (Sec. 4.3 prose, Fig. 3b semantics at entry granularity): the
    invalid set is exactly the entries that fail their own check; ccd^v aggregates the
    rest.  Returns (sorted global indices, ccd_s bytes, ccd_R bytes)."""
    Y = decode_point(Y_bytes)
    if Y is None:
        raise ValueError("bad public key")
    invalid = []
    s_v, R_v = 0, IDENTITY
    for k, m in enumerate(msgs):
        t = first_index + k
        e = entry_scalar(ds, n2, t, m)
        if verify_entry_f(Y, e, s_list[k], R_list[k]):
            s_v = (s_v + int.from_bytes(s_list[k], "little")) % Q
            R_v = point_add(R_v, decode_point(R_list[k]))
        else:
            invalid.append(t)
    return invalid, scalar_to_bytes(s_v), encode_point(R_v)


def msm(scalars: list, points: list):
    """sum_t k_t P_t by the definition (one scalar multiplication per term)."""
    acc = IDENTITY
    for k, b in zip(scalars, points):
        pt = decode_point(b)
        if pt is None:
            raise ValueError("undecodable point")
        acc = point_add(acc, scalar_mult(k, pt))
    return encode_point(acc)


def verify_multi(devices: list):
    """Many single-signer POSLO-F batches, each by its own definition: device d is accepted
    iff every entry passes its own check; the invalid (device, index) pairs are listed by
    device, then index.  devices[d] = (Y, msgs, first_index, n2, s_list, R_list, ds)."""
    accept, pairs = [], []
    for d, (Y, msgs, first, n2, s_list, R_list, ds) in enumerate(devices):
        inv, _, _ = distill_f(Y, msgs, first, n2, s_list, R_list, ds)
        accept.append(not inv)
        pairs.extend((d, t) for t in inv)
    return accept, pairs
