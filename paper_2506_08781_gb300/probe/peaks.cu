// Throughput probes for the integer pipes of the GPU this library runs on.  The POSLO path
// has no dense contraction, so its roofline is set by the integer units: the ALU pipe
// (LOP3 / IADD3 / SHF: SHA-256) and the IMAD pipe (mad.lo / mad.hi: 255-bit field
// multiplication).  Each probe runs eight independent dependency chains per thread so that
// issue, not latency, limits it, and reports operations per second.
#include <cuda_runtime.h>
#include <cstdint>

namespace {

constexpr int kChains = 8;

template <int OP>
__global__ void __launch_bounds__(256) k_probe(uint32_t* out, int iters, uint32_t m, uint32_t c) {
  uint32_t a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 0x9e3779b9u + k * 0x85ebca6bu + blockIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (OP == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(m), "r"(c));
      if (OP == 1) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(m), "r"(c));
      if (OP == 2) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(m), "r"(c));
      if (OP == 3) asm volatile("add.u32 %0, %0, %1;\n\tadd.u32 %0, %0, %2;" : "+r"(a[k]) : "r"(m), "r"(c));
      if (OP == 4) asm volatile("shf.r.wrap.b32 %0, %0, %0, %1;" : "+r"(a[k]) : "r"(m));
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x ^= a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

template <int OP>
double run(int sms, uint32_t* buf, int iters, int ops_per_step) {
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t b, e;
  cudaEventCreate(&b);
  cudaEventCreate(&e);
  k_probe<OP><<<blocks, threads>>>(buf, iters / 8, 3u, 7u);   // warm-up
  cudaEventRecord(b);
  k_probe<OP><<<blocks, threads>>>(buf, iters, 3u, 7u);
  cudaEventRecord(e);
  cudaEventSynchronize(e);
  float ms = 0;
  cudaEventElapsedTime(&ms, b, e);
  cudaEventDestroy(b);
  cudaEventDestroy(e);
  const double ops = (double)blocks * threads * iters * kChains * ops_per_step;
  return ops / (ms * 1e-3);
}

}  // namespace

extern "C" int poslo_probe_int_peaks(int device, double out[5]) {
  if (cudaSetDevice(device) != cudaSuccess) return -3;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  uint32_t* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)sms * 8 * 256 * 4) != cudaSuccess) return -2;
  const int iters = 1 << 14;
  out[0] = run<0>(sms, buf, iters, 1);   // mad.lo.u32
  out[1] = run<1>(sms, buf, iters, 1);   // mad.hi.u32
  out[2] = run<2>(sms, buf, iters, 1);   // lop3
  out[3] = run<3>(sms, buf, iters, 2);   // integer add
  out[4] = run<4>(sms, buf, iters, 1);   // funnel shift
  cudaFree(buf);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
