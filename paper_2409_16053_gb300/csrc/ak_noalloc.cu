// ak_cfl_dt_noalloc: the CFL time step of a register, computed with no device-memory
// allocation at all.  Its scratch is a file-scope static __device__ array, so the
// call works for callers that cannot call cudaMalloc (see include/ak.h).
#include "ak_internal.cuh"

namespace {

constexpr int kThreads = 256;

// Scratch of every call on a device: one partial minimum per MeshBlock, and the
// result in the last slot.  Every GPU that loads the library holds it until exit.
__device__ __align__(256) double g_cfl_scratch[AK_NOALLOC_MAX_BLOCKS + 1];

// Device address of g_cfl_scratch on the current device, looked up on every call: a
// cached address would go stale when the module is loaded again (after cudaDeviceReset,
// or in another context on the same device).  The lookup allocates nothing.
cudaError_t scratch_address(double** out) {
  double* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_cfl_scratch);
  if (e == cudaSuccess) *out = p;
  return e;
}

// One CTA per MeshBlock: minimum over the block's interior of dx_d / (|v_d| + c_s).
__global__ void block_min_kernel(const double* __restrict__ reg, int nx1, int nx2, int nx3,
                                 int ng, int s1, long long front, long long block_stride,
                                 double dx1, double dx2, double dx3, double gamma,
                                 double* partial) {
  __shared__ double red[kThreads / 32];
  const int p2 = nx2 + 2 * ng, p3 = nx3 + 2 * ng;
  const long long var_stride = (long long)s1 * p2 * p3;
  const long long n = (long long)nx1 * nx2 * nx3;
  const double* ub = reg + (long long)blockIdx.x * block_stride + front;
  double m = __longlong_as_double(0x7ff0000000000000ll);
  for (long long c = threadIdx.x; c < n; c += blockDim.x) {
    const int i = (int)(c % nx1);
    const int j = (int)((c / nx1) % nx2);
    const int k = (int)(c / ((long long)nx1 * nx2));
    const long long e = ((long long)(k + ng) * p2 + (j + ng)) * s1 + (i + ng);
    double u[AK_NVAR];
#pragma unroll
    for (int v = 0; v < AK_NVAR; ++v) u[v] = ub[e + v * var_stride];
    double rho = u[0] >= AK_RHO_FLOOR ? u[0] : AK_RHO_FLOOR;
    const double v1 = u[1] / rho, v2 = u[2] / rho, v3 = u[3] / rho;
    double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / rho;
    ug = ug >= AK_UG_FLOOR ? ug : AK_UG_FLOOR;
    const double cs = sqrt(gamma * (gamma - 1.0) * ug / rho);
    double t = dx1 / (fabs(v1) + cs);
    t = fmin(t, dx2 / (fabs(v2) + cs));
    t = fmin(t, dx3 / (fabs(v3) + cs));
    m = fmin(m, t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? red[threadIdx.x]
                                           : __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

// One CTA: result = cfl * min(partial[0 .. nblocks)), stored after the partials.
__global__ void final_min_kernel(double* partial, int nblocks, double cfl) {
  __shared__ double red[1024 / 32];
  double m = __longlong_as_double(0x7ff0000000000000ll);
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) m = fmin(m, partial[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) partial[AK_NOALLOC_MAX_BLOCKS] = cfl * v;
  }
}

}  // namespace

extern "C" ak_status ak_cfl_dt_noalloc(const double* reg, int32_t nblocks, const int32_t nx[3],
                                       int32_t nghost, const double dx[3], double gamma,
                                       double cfl, void* cuda_stream, double* dt_out) {
  if (!reg || !nx || !dx || !dt_out) {
    ak_set_error("ak_cfl_dt_noalloc: NULL argument");
    return AK_EINVAL;
  }
  if (nblocks < 1 || nblocks > AK_NOALLOC_MAX_BLOCKS) {
    ak_set_error("ak_cfl_dt_noalloc: nblocks = %d outside [1, %d] (size of the static scratch)",
                 nblocks, AK_NOALLOC_MAX_BLOCKS);
    return AK_EINVAL;
  }
  if (nghost < 1 || nx[0] < 1 || nx[1] < 1 || nx[2] < 1 || !(dx[0] > 0.0) || !(dx[1] > 0.0) ||
      !(dx[2] > 0.0) || !(gamma > 1.0) || !(cfl > 0.0)) {
    ak_set_error("ak_cfl_dt_noalloc: invalid block size, nghost, dx, gamma or cfl");
    return AK_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    ak_set_error("ak_cfl_dt_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return AK_ECUDA;
  }
  // the register layout of ak_mesh_layout: row pitch, front pad and block stride
  const int s1 = (nx[0] + 2 * nghost + 3) / 4 * 4;
  const long long front = (4 - nghost % 4) % 4;
  const long long var_stride = (long long)s1 * (nx[1] + 2 * nghost) * (nx[2] + 2 * nghost);
  const long long block_stride = ((front + AK_NVAR * var_stride + 31) / 32) * 32;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  block_min_kernel<<<nblocks, kThreads, 0, s>>>(reg, nx[0], nx[1], nx[2], nghost, s1, front,
                                                 block_stride, dx[0], dx[1], dx[2], gamma,
                                                 scratch);
  final_min_kernel<<<1, 1024, 0, s>>>(scratch, nblocks, cfl);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dt_out, scratch + AK_NOALLOC_MAX_BLOCKS, sizeof(double),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ak_set_error("ak_cfl_dt_noalloc: %s", cudaGetErrorString(e));
    return AK_ECUDA;
  }
  return AK_OK;
}
