// select.cu -- inference of the learned chunk-mode selector (not from the paper).
//
// Before a gate runs, one thread per active chunk reads the chunk's image header from
// the page pool, forms the network's 16 inputs with the gate's features, runs the
// float32 fixed-order inference of device.cuh and writes one decision byte: which of
// the expensive trials (SPLIT, PALETTE) the gate's encoder runs for that chunk.  The
// weights sit in shared memory as float32 (every thread of a warp reads the same
// weight at the same time: a broadcast).  Reads are 32 bytes of directory entry and 16
// bytes of header per chunk, so the kernel takes a small fraction of a gate.
#include "device.cuh"
#include "gate_common.cuh"
#include "launch.h"

namespace qc {

constexpr int kSelThreads = 256;

__global__ void __launch_bounds__(kSelThreads) k_select(const __grid_constant__ GateLaunch L,
                                                        const unsigned short* __restrict__ mlp,
                                                        uint8_t* __restrict__ dec) {
  __shared__ __align__(16) float w[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += kSelThreads) w[i] = __uint_as_float((uint32_t)mlp[i] << 16);
  __syncthreads();
  const Pool& P = L.P;
  const int kc = P.kc;
  // the bound the gate will run at (the same rule on the same values as the gate kernels)
  const uint32_t S = gate_bits(L);
  const unsigned long long n = L.pair ? 2ull * L.items : L.nact;
  for (unsigned long long k = (unsigned long long)blockIdx.x * kSelThreads + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * kSelThreads) {
    const unsigned long long ch = L.pair ? ((item_chunk(L, k >> 1) | L.hi_vals) | ((k & 1ull) ? L.pair_bit : 0ull))
                                         : (item_chunk(L, k) | L.hi_vals);
    const uint32_t* e = dir_entry(P, ch);
    const uint32_t len = e[0], np = e[1];
    uint4 h = make_uint4(0u, 0u, 0u, 0u);
    if (len >= 16u) {
      if (np == 0u) h = *reinterpret_cast<const uint4*>(e + 4);
      else if (e[4] < P.npages) h = *reinterpret_cast<const uint4*>(P.pages + (unsigned long long)e[4] * kPage);
    }
    const uint32_t hdr[4] = {h.x, h.y, h.z, h.w};
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = sel_feature(hdr, len, kc, L.gfeat, S, i);
    dec[k] = (uint8_t)sel_decide(w, x);
  }
}

cudaError_t launch_select(const GateLaunch& L, const unsigned short* mlp, uint8_t* dec, int grid, cudaStream_t st) {
  k_select<<<grid, kSelThreads, 0, st>>>(L, mlp, dec);
  return cudaGetLastError();
}

}  // namespace qc
