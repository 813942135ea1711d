// ak_probe_fp64_rate: the FP64 instruction rate this GPU sustains, measured, for the
// roofline of the FP64 form (whose stage kernels are bound by the FP64 unit, not by HBM).
// Every thread runs eight independent chains of fused multiply-adds, so that the FP64
// pipe, not the latency of one chain, limits the rate.
#include "ak_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kIters = 4096;

__device__ double g_probe_sink;

__global__ void dfma_chains_kernel(double b, double c) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == -1.0) g_probe_sink = s;  // never true: keeps the chains alive
}

}  // namespace

extern "C" ak_status ak_probe_fp64_rate(void* cuda_stream, double* dfma_per_s) {
  if (!dfma_per_s) {
    ak_set_error("ak_probe_fp64_rate: NULL argument");
    return AK_EINVAL;
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  const unsigned grid = (unsigned)(8 * nsm);  // several CTAs per SM: every SMSP busy
  float best = 1e30f;
  // b, c keep the chains at a fixed point near 1 (no overflow, no subnormals)
  const double b = 0.9999, c = 1e-4;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first one warms up
    e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) {
      dfma_chains_kernel<<<grid, kThreads, 0, s>>>(b, c);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) {
    ak_set_error("ak_probe_fp64_rate: %s", cudaGetErrorString(e));
    return AK_ECUDA;
  }
  *dfma_per_s = (double)grid * kThreads * kChains * kIters / (best * 1e-3);
  return AK_OK;
}
