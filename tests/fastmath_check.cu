// Test helper: evaluates the library's integer-pipe conversions and Newton-refined
// reciprocal / rsqrt / sqrt next to CUDA's IEEE operations on the same inputs.
#include <cuda_runtime.h>

#include "../paper_2409_16053_gb300/csrc/fastmath.cuh"

__global__ void fastmath_kernel(const double* x, int n, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  double* o = out + 9 * (long long)i;
  o[0] = ak::rcp64(v);
  o[1] = 1.0 / v;
  o[2] = ak::rsqrt64(fabs(v));
  o[3] = 1.0 / sqrt(fabs(v));
  o[4] = ak::sqrt64(fabs(v));
  o[5] = sqrt(fabs(v));
  o[6] = (double)ak::f64_to_f32(v);
  o[7] = (double)__double2float_rn(v);
  const float f = __double2float_rn(v);
  o[8] = ak::f32_to_f64(f) - (double)f;  // exact conversion: 0
}

// sqrt(a / b) on the integer pipe and FP32 next to the IEEE expression: out[2i], out[2i+1]
__global__ void ratio_kernel(const double* a, const double* b, int n, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[2 * (long long)i] = ak::sqrt_ratio64(a[i], b[i]);
  out[2 * (long long)i + 1] = sqrt(a[i] / b[i]);
}

extern "C" int ratio_eval(const double* host_a, const double* host_b, int n, double* host_out) {
  double *da = nullptr, *db = nullptr, *dout = nullptr;
  if (cudaMalloc(&da, sizeof(double) * n) != cudaSuccess) return 1;
  if (cudaMalloc(&db, sizeof(double) * n) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, sizeof(double) * 2 * (size_t)n) != cudaSuccess) return 2;
  cudaMemcpy(da, host_a, sizeof(double) * n, cudaMemcpyHostToDevice);
  cudaMemcpy(db, host_b, sizeof(double) * n, cudaMemcpyHostToDevice);
  ratio_kernel<<<(n + 255) / 256, 256>>>(da, db, n, dout);
  cudaError_t e = cudaMemcpy(host_out, dout, sizeof(double) * 2 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 3;
}

// sqrt(g a / b) with g split into two floats, next to the IEEE expression
__global__ void gratio_kernel(const double* a, const double* b, int n, double g, float gh,
                              float gl, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[2 * (long long)i] = ak::sqrt_gratio64(a[i], b[i], g, gh, gl);
  out[2 * (long long)i + 1] = sqrt(g * a[i] / b[i]);
}

extern "C" int gratio_eval(const double* host_a, const double* host_b, int n, double g,
                           double* host_out) {
  const float gh = (float)g, gl = (float)(g - (double)gh);
  double *da = nullptr, *db = nullptr, *dout = nullptr;
  if (cudaMalloc(&da, sizeof(double) * n) != cudaSuccess) return 1;
  if (cudaMalloc(&db, sizeof(double) * n) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, sizeof(double) * 2 * (size_t)n) != cudaSuccess) return 2;
  cudaMemcpy(da, host_a, sizeof(double) * n, cudaMemcpyHostToDevice);
  cudaMemcpy(db, host_b, sizeof(double) * n, cudaMemcpyHostToDevice);
  gratio_kernel<<<(n + 255) / 256, 256>>>(da, db, n, g, gh, gl, dout);
  cudaError_t e = cudaMemcpy(host_out, dout, sizeof(double) * 2 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 3;
}

extern "C" int fastmath_eval(const double* host_x, int n, double* host_out) {
  double *dx = nullptr, *dout = nullptr;
  if (cudaMalloc(&dx, sizeof(double) * n) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, sizeof(double) * 9 * (size_t)n) != cudaSuccess) return 2;
  cudaMemcpy(dx, host_x, sizeof(double) * n, cudaMemcpyHostToDevice);
  fastmath_kernel<<<(n + 255) / 256, 256>>>(dx, n, dout);
  cudaError_t e = cudaMemcpy(host_out, dout, sizeof(double) * 9 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 3;
}
