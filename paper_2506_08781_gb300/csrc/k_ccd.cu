// POSLO-C distillation and selective batch verification (Fig. 3b): per-epoch sums of e,
// grouped sums of scalars and points (ccd^v, the umbrellas ccd^u, SeBVer's V and U sums),
// and a list of independent cofactored checks [8](R_k - e_k Y - s_k G) = O (the per-epoch
// C.AVer of Distill and the checks of SeBVer).
#include "common.cuh"

namespace poslo {

// out[g] = sum of the 32-byte scalars x[g G .. (g+1) G) not flagged in skip, mod q.
// One block per group; each thread keeps 64-bit limb sums, reduced once per group.
__global__ void __launch_bounds__(kCcdThreads) k_scalar_group_sums(const uint8_t* x, uint64_t G, uint64_t n,
                                                                   const uint8_t* skip, uint32_t* out) {
  const uint64_t g = blockIdx.x;
  acc13 a;
  acc_zero(a);
  const uint64_t lo = g * G, hi = min(lo + G, n);
  for (uint64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if (skip && skip[t]) continue;
    uint32_t v[8];
    const uint4* p = reinterpret_cast<const uint4*>(x + 32 * t);
    const uint4 v0 = p[0], v1 = p[1];
    v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w; v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
    acc_add<8>(a, v);
  }
  __shared__ unsigned long long red[kCcdThreads / 32][13];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 13; ++k) {
    unsigned long long v = a.v[k];
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sums[13];
    for (int k = 0; k < 13; ++k) {
      unsigned long long v = 0;
      for (int w = 0; w < kCcdThreads / 32; ++w) v += red[w][k];
      sums[k] = v;
    }
    const sc r = limb_sums_to_scalar(sums);
    for (int k = 0; k < 8; ++k) out[8 * g + k] = r.v[k];
  }
}

// enc[g] = encoding of the sum of the decoded points pts[g G .. (g+1) G) that are neither
// flagged in skip nor undecodable (bad).  One block per group.
__global__ void __launch_bounds__(kCcdThreads) k_point_group_sums(const uint32_t* pts, const uint8_t* bad, uint64_t G,
                                                                  uint64_t n, const uint8_t* skip, uint8_t* enc) {
  const uint64_t g = blockIdx.x;
  ge acc = ge_identity();
  const uint64_t lo = g * G, hi = min(lo + G, n);
  for (uint64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if ((skip && skip[t]) || (bad && bad[t])) continue;
    fe x, y, t2d;
    pts_load(pts + (size_t)kPtsWords * t, x, y, t2d);
    acc = ge_madd(acc, x, y, t2d);
  }
  __shared__ uint32_t sp[kCcdThreads][32];
  ge_store(sp[threadIdx.x], acc);
  __syncthreads();
  for (int h = kCcdThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) ge_store(sp[threadIdx.x], ge_add(ge_load(sp[threadIdx.x]), ge_load(sp[threadIdx.x + h])));
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    uint32_t b[8];
    ge_encode(ge_load(sp[0]), b);
    for (int k = 0; k < 8; ++k) reinterpret_cast<uint32_t*>(enc + 32 * g)[k] = b[k];
  }
}

// ok[k] = s_k canonical, R_k decodable (not bad), and [8](R_k - e_k Y - s_k G) = O, for n
// independent checks; one quad of lanes per check (quad-cooperative table additions), the
// surplus quads repeating the last check without writing.
__global__ void __launch_bounds__(128) k_check_list(const uint32_t* e, const uint8_t* s, const uint32_t* pts,
                                                    const uint8_t* bad, uint32_t n, const uint32_t* tableY,
                                                    const uint32_t* tableG, uint8_t* ok) {
  const uint32_t quad = ((uint32_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const uint32_t k = quad < n ? quad : n - 1;
  uint32_t ek[8], sk[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) ek[i] = e[8 * (size_t)k + i];
  const uint4* sp = reinterpret_cast<const uint4*>(s + 32 * (size_t)k);
  const uint4 s0 = sp[0], s1 = sp[1];
  sk[0] = s0.x; sk[1] = s0.y; sk[2] = s0.z; sk[3] = s0.w; sk[4] = s1.x; sk[5] = s1.y; sk[6] = s1.z; sk[7] = s1.w;
  const bool canon = sc_is_canonical(sk);
  // every lane runs every quad operation (full-mask shuffles)
  ge acc = ge_identity();
  int ce = 0, cs = 0;
  for (int w = 0; w < 64; ++w) {
    acc = ge_add_quad(acc, table_pick(tableY, w, sc_digit4(ek, w, ce)));
    acc = ge_add_quad(acc, table_pick(tableG, w, sc_digit4(sk, w, cs)));
  }
  ge R;
  fe t2d;
  pts_load(pts + (size_t)kPtsWords * k, R.X, R.Y, t2d);
  R.Z = fe_one();
  R.T = fe_mul(R.X, R.Y);
  const bool good = canon && !bad[k] && ge_is_identity(ge_mul_cofactor(ge_sub(R, acc)));
  if ((threadIdx.x & 3) == 0 && quad < n) ok[k] = good ? 1 : 0;
}

// dst[k] = src[idx[k]] for 32-byte records.
__global__ void k_gather32(const uint8_t* src, const uint64_t* idx, uint64_t n, uint8_t* dst) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * n) return;
  const uint64_t k = t >> 1, half = t & 1;
  reinterpret_cast<uint4*>(dst + 32 * k)[half] = reinterpret_cast<const uint4*>(src + 32 * idx[k])[half];
}

// flag[k] = 1 - ok[k] (the invalid epochs of Distill, for the compaction and as skip mask).
__global__ void k_flip(const uint8_t* ok, uint64_t n, uint8_t* flag) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) flag[t] = ok[t] ? 0 : 1;
}

}  // namespace poslo
