// Throughput probes behind the integer roofline of the mesh (no counterpart in
// the paper): the rate of 32-bit integer multiply-adds, and of the
// carry-chained two-limb x 64-bit multiply-accumulate the mesh runs per
// stencil weight (wmac2_u64), on independent chains that fill every SM.
#include "abf_internal.cuh"

namespace abf {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) probe_imad_kernel(uint32_t* sink, int iters, uint32_t seed) {
  uint32_t a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = seed ^ (threadIdx.x * 2654435761u + k);
  // a[k] <- a[k] a[k+1 mod 8] + c: distinct products of two variables, so no
  // two iterations fold into one multiply-add and no product is shared (a
  // constant multiplier would let the compiler compose the affine steps)
  for (int i = 0; i < iters; ++i) {
    uint32_t b[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) b[k] = a[k] * a[(k + 1) % kProbeChains] + (uint32_t)(2 * k + 1);
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = b[k];
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x ^= a[k];
  if (x == 0x5bd1e995u) sink[blockIdx.x] = x;  // keeps the chains alive
}

__global__ void __launch_bounds__(kProbeThreads) probe_mac_kernel(uint64_t* sink, int iters, uint64_t seed) {
  Wide<2> acc[kProbeChains];
  Wide<2> gv;
  gv.w[0] = seed ^ (threadIdx.x * 0x9E3779B97F4A7C15ull);
  gv.w[1] = ~gv.w[0];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) {
    acc[k].w[0] = seed + k;
    acc[k].w[1] = k;
  }
  uint64_t w = 0x0123456789abcdefull ^ seed;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) wmac2_u64(acc[k], gv, w + (uint64_t)k);
  }
  uint64_t x = 0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x ^= acc[k].w[0] ^ acc[k].w[1];
  if (x == 0x5bd1e9955bd1e995ull) sink[blockIdx.x] = x;
}

}  // namespace abf

extern "C" abf_status abf_probe_alu(int32_t kind, double* ops_per_s) {
  if (!ops_per_s || (kind != 0 && kind != 1)) return ABF_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ABF_ERR_CUDA;
  void* sink = nullptr;
  if (cudaMalloc(&sink, 8 * 4096) != cudaSuccess) return ABF_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8;
  const int iters = kind == 0 ? 1 << 16 : 1 << 12;
  auto launch = [&](int it) {
    if (kind == 0) abf::probe_imad_kernel<<<blocks, abf::kProbeThreads>>>((uint32_t*)sink, it, 12345u);
    else abf::probe_mac_kernel<<<blocks, abf::kProbeThreads>>>((uint64_t*)sink, it, 12345ull);
  };
  launch(iters / 8);  // warm-up
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  abf_status st = ABF_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
    st = ABF_ERR_CUDA;
  else
    *ops_per_s = (double)blocks * abf::kProbeThreads * (double)iters * abf::kProbeChains / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}
