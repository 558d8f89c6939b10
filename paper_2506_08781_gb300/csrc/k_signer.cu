// Signer-side kernels for synthetic workloads: key generation and POSLO-C/F signing.
#include "common.cuh"

namespace poslo {

__global__ void k_keygen_y(const uint8_t* y, const uint32_t* tableG, uint8_t* Y_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t yv[8], enc[8];
  load_sc_bytes(y, yv);
  ge_encode(base_mult_table(yv, tableG), enc);
  store_words_bytes(Y_out, enc);
}

__global__ void k_keygen_c_epochs(const uint8_t* r, uint32_t n1, uint32_t n2, const uint32_t* tableG,
                                  uint8_t* epoch_R) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n1) return;
  uint32_t rw[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    rw[k] = ((uint32_t)r[4 * k] << 24) | (r[4 * k + 1] << 16) | (r[4 * k + 2] << 8) | r[4 * k + 3];
  sc acc;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc.v[k] = 0;
  for (uint32_t j = 0; j < n2; ++j) acc = sc_add(acc, nonce_c(rw, i, j));
  uint32_t enc[8];
  ge_encode(base_mult_table(acc.v, tableG), enc);
  store_words_bytes(epoch_R + 32 * (size_t)i, enc);
}

__global__ void k_keygen_bpv(const uint8_t* bpv_r, uint32_t v, const uint32_t* tableG, uint8_t* bpv_R) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v) return;
  uint32_t rv[8], enc[8];
  load_sc_bytes(bpv_r + 32 * (size_t)k, rv);
  ge_encode(base_mult_table(rv, tableG), enc);
  store_words_bytes(bpv_R + 32 * (size_t)k, enc);
}

__global__ void k_decode_table(const uint8_t* enc, uint32_t v, uint32_t* out, uint32_t* status) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v) return;
  uint32_t b[8];
  load_sc_bytes(enc + 32 * (size_t)k, b);
  ge P;
  if (!ge_decode(b, P)) atomicOr(status, kErrPoint);
  ge_store(out + 32 * (size_t)k, P);
}

template <int INST>
__global__ void k_sign_f(const SignFArgs a) {
  AesCtx c{};
  if constexpr (INST == kInstAes) {
    __shared__ AesShared sh;
    aes_tables_init(sh);
    c = aes_ctx(&sh);
  }
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n) return;
  const uint64_t gi = a.first_index + t;
  const uint64_t i = gi / a.n2, j = gi - i * a.n2;
  const uint4 xs = a.seeds ? reinterpret_cast<const uint4*>(a.seeds)[i - a.e0] : make_uint4(0, 0, 0, 0);
  const uint32_t x0[4] = {xs.x, xs.y, xs.z, xs.w};
  uint32_t x[4];
  prf_entry_i<INST>(c, x0, (uint32_t)j, x);
  const uint64_t o0 = a.offs[t] - a.base_off, o1 = a.offs[t + 1] - a.base_off;
  uint32_t d[8];
  entry_digest<INST>(c, a.msgs + o0, (uint32_t)(o1 - o0), x, d);
  const sc e = sc_reduce256(d);
  sc r;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.v[k] = 0;
  ge R = ge_identity();
  for (uint32_t kk = 0; kk < a.k; ++kk) {
    const uint32_t idx = a.subsets[t * a.k + kk];
    sc rk;
    load_sc_bytes(a.bpv_r + 32 * (size_t)idx, rk.v);
    r = sc_add(r, rk);
    R = ge_add(R, ge_load(a.bpv_pts + 32 * (size_t)idx));
  }
  sc y;
  load_sc_bytes(a.y, y.v);
  const sc s = sc_sub(r, sc_mul(e, y));
  store_words_bytes(a.s_out + 32 * t, s.v);
  uint32_t enc[8];
  ge_encode(R, enc);
  store_words_bytes(a.R_out + 32 * t, enc);
  if (a.x_out) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a.x_out[16 * t + 4 * k] = (uint8_t)(x[k] >> 24);
      a.x_out[16 * t + 4 * k + 1] = (uint8_t)(x[k] >> 16);
      a.x_out[16 * t + 4 * k + 2] = (uint8_t)(x[k] >> 8);
      a.x_out[16 * t + 4 * k + 3] = (uint8_t)x[k];
    }
  }
}

template <int INST>
__global__ void k_sign_c(const SignCArgs a) {
  AesCtx c{};
  if constexpr (INST == kInstAes) {
    __shared__ AesShared sh;
    aes_tables_init(sh);
    c = aes_ctx(&sh);
  }
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_epochs) return;
  const uint64_t i = a.first_epoch + k;
  const uint4 xs = reinterpret_cast<const uint4*>(a.seeds)[k];
  const uint32_t x0[4] = {xs.x, xs.y, xs.z, xs.w};
  uint32_t rw[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    rw[q] = ((uint32_t)a.r[4 * q] << 24) | (a.r[4 * q + 1] << 16) | (a.r[4 * q + 2] << 8) | a.r[4 * q + 3];
  sc y;
  load_sc_bytes(a.y, y.v);
  sc acc;
#pragma unroll
  for (int q = 0; q < 8; ++q) acc.v[q] = 0;
  for (uint32_t j = 0; j < a.n2; ++j) {
    const uint64_t t = k * a.n2 + j;
    uint32_t x[4];
    prf_entry_i<INST>(c, x0, j, x);
    const uint64_t o0 = a.offs[t] - a.base_off, o1 = a.offs[t + 1] - a.base_off;
    uint32_t d[8];
    entry_digest<INST>(c, a.msgs + o0, (uint32_t)(o1 - o0), x, d);
    const sc e = sc_reduce256(d);
    acc = sc_add(acc, sc_sub(nonce_c(rw, (uint32_t)i, j), sc_mul(e, y)));
  }
  store_words_bytes(a.s_out + 32 * k, acc.v);
}

void launch_sign_f(int inst, unsigned grid, unsigned block, cudaStream_t st, const SignFArgs& a) {
  if (inst == kInstAes) k_sign_f<kInstAes><<<grid, block, 0, st>>>(a);
  else k_sign_f<kInstSha><<<grid, block, 0, st>>>(a);
}

void launch_sign_c(int inst, unsigned grid, unsigned block, cudaStream_t st, const SignCArgs& a) {
  if (inst == kInstAes) k_sign_c<kInstAes><<<grid, block, 0, st>>>(a);
  else k_sign_c<kInstSha><<<grid, block, 0, st>>>(a);
}

}  // namespace poslo
