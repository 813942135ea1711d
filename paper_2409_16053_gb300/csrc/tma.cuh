// Bulk-tensor (TMA) copies and their completion, as inline PTX for sm_103a.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace ak {

// One box of a 5-D tensor map from shared memory to global memory (bulk-group
// completion).  The shared source must be 128-byte aligned and written before the
// issuing thread's fence.proxy.async + barrier.
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, const void* smem, int c0,
                                             int c1, int c2, int c3, int c4) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];"
      :
      : "l"((unsigned long long)map), "r"(s), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until at most N committed bulk groups still read their shared source.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// Wait until at most N committed bulk groups are still in flight (writes done).
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}
// Makes this thread's generic-proxy shared-memory writes visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace ak
