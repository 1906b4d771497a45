// gate_common.cuh -- device helpers shared by the two gate kernels (kernels.cu, fast.cu).
#pragma once
#include "launch.h"

namespace qc {

// Asynchronous 16-byte global -> shared copies (the next item's directory entries).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// Waits until at most N of this thread's most recent copy groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// Section 3.7: the bound of the running gate, from E after the previous gate.  Every
// CTA evaluates the same rule on the same values (only the post kernel writes them).
__device__ __forceinline__ uint32_t gate_bits(const GateLaunch& L) {
  return (uint32_t)level_bits(L.ctl, next_level(L.ctl, L.P.ctl->E, L.P.ctl->level, L.P.ctl->n64));
}

// The chunk index of the k-th active chunk (or pair): the bits of k deposited into the
// free chunk-index bits, run by run.
__device__ __forceinline__ unsigned long long item_chunk(const GateLaunch& L, unsigned long long k) {
  if (L.nruns < 0) return deposit_bits(k, L.free_mask);
  unsigned long long out = 0;
  for (int i = 0; i < L.nruns; ++i) out |= (k << L.run_shift[i]) & L.run_mask[i];
  return out;
}

}  // namespace qc
