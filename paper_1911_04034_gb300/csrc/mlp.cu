// mlp.cu -- training of the learned chunk-mode selector (not from the paper).
//
// The selector (inference in device.cuh) is a 16 -> 32 -> 32 -> 8 network with
// bfloat16 weights.  Training keeps float32 master weights; every step rounds them
// to bfloat16, runs the forward and backward passes over a minibatch with float32
// arithmetic (one thread per sample, gradients summed in shared memory, then across
// blocks), and applies an Adam update.  Loss: softmax cross-entropy of the seven mode
// logits (outputs 0..6) against the mode the exhaustive trial chose, plus the squared
// error of the bit budget (output 7) against the best image's size over the RAW size.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/qcsim.h"
#include "launch.h"

namespace {

constexpr int NIN = 16, NH = 32, NOUT = 8, NMODES = 7, NSIZE = NOUT - NMODES;
constexpr int OW1 = 0, OB1 = 512, OW2 = 544, OB2 = 1568, OW3 = 1600, OB3 = 1856, NP = 1864;
static_assert(NP == qc::kMlpParams, "parameter layout");

__device__ __forceinline__ float bf16_round_dev(float v) {
  uint32_t u = __float_as_uint(v);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  return __uint_as_float(u);
}

// Rounds the float32 masters to bfloat16 (as float, and as 16-bit words).
__global__ void k_mlp_round(const float* __restrict__ w, float* __restrict__ wq, unsigned short* __restrict__ wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NP; i += gridDim.x * blockDim.x) {
    const float q = bf16_round_dev(w[i]);
    wq[i] = q;
    if (wb) wb[i] = (unsigned short)(__float_as_uint(q) >> 16);
  }
}

// Forward + backward for samples idx[0..n); grad (NP floats) and loss are summed.
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ wq, const float* __restrict__ x,
                                                  const int* __restrict__ mode, const float* __restrict__ sizes,
                                                  const int* __restrict__ idx, int n, float inv_b,
                                                  float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float sw[NP];
  __shared__ float sg[NP];
  __shared__ float sl;
  for (int i = threadIdx.x; i < NP; i += blockDim.x) {
    sw[i] = wq[i];
    sg[i] = 0.0f;
  }
  if (threadIdx.x == 0) sl = 0.0f;
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const int smp = idx[t];
    float in[NIN], z1[NH], h1[NH], z2[NH], h2[NH], o[NOUT];
    for (int i = 0; i < NIN; ++i) in[i] = x[smp * NIN + i];
    for (int j = 0; j < NH; ++j) {
      float a = sw[OB1 + j];
      for (int i = 0; i < NIN; ++i) a += sw[OW1 + j * NIN + i] * in[i];
      z1[j] = a;
      h1[j] = a > 0.0f ? a : 0.0f;
    }
    for (int j = 0; j < NH; ++j) {
      float a = sw[OB2 + j];
      for (int i = 0; i < NH; ++i) a += sw[OW2 + j * NH + i] * h1[i];
      z2[j] = a;
      h2[j] = a > 0.0f ? a : 0.0f;
    }
    for (int j = 0; j < NOUT; ++j) {
      float a = sw[OB3 + j];
      for (int i = 0; i < NH; ++i) a += sw[OW3 + j * NH + i] * h2[i];
      o[j] = a;
    }
    // loss and d loss / d outputs (mean over the minibatch: factor inv_b)
    float mx = o[0];
    for (int m = 1; m < NMODES; ++m) mx = fmaxf(mx, o[m]);
    float se = 0.0f;
    for (int m = 0; m < NMODES; ++m) se += expf(o[m] - mx);
    const int y = mode[smp];
    float dout[NOUT];
    float l = -(o[y] - mx - logf(se));
    for (int m = 0; m < NMODES; ++m) dout[m] = (expf(o[m] - mx) / se - (m == y ? 1.0f : 0.0f)) * inv_b;
    for (int k = 0; k < NSIZE; ++k) {
      const float d = o[NMODES + k] - sizes[smp * NSIZE + k];
      l += d * d;
      dout[NMODES + k] = 2.0f * d * inv_b;
    }
    atomicAdd(&sl, l * inv_b);
    // backward
    float dh2[NH];
    for (int i = 0; i < NH; ++i) dh2[i] = 0.0f;
    for (int j = 0; j < NOUT; ++j) {
      atomicAdd(&sg[OB3 + j], dout[j]);
      for (int i = 0; i < NH; ++i) {
        atomicAdd(&sg[OW3 + j * NH + i], dout[j] * h2[i]);
        dh2[i] += sw[OW3 + j * NH + i] * dout[j];
      }
    }
    float dh1[NH];
    for (int i = 0; i < NH; ++i) dh1[i] = 0.0f;
    for (int j = 0; j < NH; ++j) {
      const float dz = z2[j] > 0.0f ? dh2[j] : 0.0f;
      if (dz == 0.0f) continue;
      atomicAdd(&sg[OB2 + j], dz);
      for (int i = 0; i < NH; ++i) {
        atomicAdd(&sg[OW2 + j * NH + i], dz * h1[i]);
        dh1[i] += sw[OW2 + j * NH + i] * dz;
      }
    }
    for (int j = 0; j < NH; ++j) {
      const float dz = z1[j] > 0.0f ? dh1[j] : 0.0f;
      if (dz == 0.0f) continue;
      atomicAdd(&sg[OB1 + j], dz);
      for (int i = 0; i < NIN; ++i) atomicAdd(&sg[OW1 + j * NIN + i], dz * in[i]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NP; i += blockDim.x)
    if (sg[i] != 0.0f) atomicAdd(&grad[i], sg[i]);
  if (threadIdx.x == 0 && loss) atomicAdd(loss, sl);
}

__global__ void k_mlp_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NP; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

sim_status mlp_fail(sim_status s, const char* msg) {
  qc::set_last_error(msg);
  return s;
}

#define MCK(call)                                                           \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) return mlp_fail(SIM_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

// Copies the training set to the device; layout: x (n*16 f32), sizes (n*NSIZE f32),
// mode (n i32), idx (n i32), grad (NP), loss (1), wq (NP), w, m, v (NP each).
struct TrainSet {
  DevBuf buf;
  float *x, *sizes, *grad, *loss, *wq, *w, *m, *v;
  int *mode, *idx;
};

sim_status upload(TrainSet& T, const float* x, const int32_t* mode, const float* sizes, uint64_t n) {
  const size_t fl = (size_t)n * (NIN + NSIZE) + 5 * NP + 1, in = (size_t)n * 2;
  MCK(cudaMalloc(&T.buf.p, fl * 4 + in * 4 + 64));
  float* f = static_cast<float*>(T.buf.p);
  T.x = f;
  T.sizes = T.x + n * NIN;
  T.grad = T.sizes + n * NSIZE;
  T.loss = T.grad + NP;
  T.wq = T.loss + 1;
  T.w = T.wq + NP;
  T.m = T.w + NP;
  T.v = T.m + NP;
  T.mode = reinterpret_cast<int*>(T.v + NP);
  T.idx = T.mode + n;
  MCK(cudaMemcpy(T.x, x, n * NIN * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(T.sizes, sizes, n * NSIZE * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(T.mode, mode, n * 4, cudaMemcpyHostToDevice));
  return SIM_OK;
}

}  // namespace

extern "C" {

sim_status sim_mlp_grad(const float* params, const float* x, const int32_t* mode, const float* sizes, uint64_t n,
                        float* grad_out, float* loss_out) {
  if (!params || !x || !mode || !sizes || !grad_out || n == 0 || n > (1ull << 26))
    return mlp_fail(SIM_ERR_INVALID, "bad arguments");
  for (uint64_t i = 0; i < n; ++i)
    if (mode[i] < 0 || mode[i] >= NMODES) return mlp_fail(SIM_ERR_INVALID, "mode label outside 0..6");
  TrainSet T;
  if (sim_status r = upload(T, x, mode, sizes, n)) return r;
  std::vector<int> idx(n);
  for (uint64_t i = 0; i < n; ++i) idx[i] = (int)i;
  MCK(cudaMemcpy(T.idx, idx.data(), n * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(T.w, params, NP * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemset(T.grad, 0, (NP + 1) * 4));
  k_mlp_round<<<8, 256>>>(T.w, T.wq, nullptr);
  const int blocks = (int)((n + 255) / 256);
  k_mlp_grad<<<blocks, 256>>>(T.wq, T.x, T.mode, T.sizes, T.idx, (int)n, 1.0f / (float)n, T.grad, T.loss);
  MCK(cudaGetLastError());
  MCK(cudaMemcpy(grad_out, T.grad, NP * 4, cudaMemcpyDeviceToHost));
  float l = 0.0f;
  MCK(cudaMemcpy(&l, T.loss, 4, cudaMemcpyDeviceToHost));
  if (loss_out) *loss_out = l;
  return SIM_OK;
}

sim_status sim_mlp_train(const float* x, const int32_t* mode, const float* sizes, uint64_t n, int epochs, int batch,
                         float lr, uint64_t seed, float* params, uint16_t* bf16_out, float* last_loss) {
  if (!x || !mode || !sizes || !params || n == 0 || n > (1ull << 26) || epochs < 1 || batch < 1 || !(lr > 0.0f))
    return mlp_fail(SIM_ERR_INVALID, "bad arguments");
  for (uint64_t i = 0; i < n; ++i)
    if (mode[i] < 0 || mode[i] >= NMODES) return mlp_fail(SIM_ERR_INVALID, "mode label outside 0..6");
  TrainSet T;
  if (sim_status r = upload(T, x, mode, sizes, n)) return r;
  MCK(cudaMemcpy(T.w, params, NP * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemset(T.m, 0, 2 * NP * 4));
  std::vector<int> idx(n);
  for (uint64_t i = 0; i < n; ++i) idx[i] = (int)i;
  uint64_t s = seed;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int step = 0;
  float epoch_loss = 0.0f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (uint64_t i = n - 1; i > 0; --i) {  // Fisher-Yates with splitmix64
      const uint64_t j = splitmix(s) % (i + 1);
      const int t = idx[i];
      idx[i] = idx[j];
      idx[j] = t;
    }
    MCK(cudaMemcpy(T.idx, idx.data(), n * 4, cudaMemcpyHostToDevice));
    MCK(cudaMemset(T.loss, 0, 4));
    for (uint64_t b0 = 0; b0 < n; b0 += (uint64_t)batch) {
      const int nb = (int)((n - b0) < (uint64_t)batch ? (n - b0) : (uint64_t)batch);
      MCK(cudaMemset(T.grad, 0, NP * 4));
      k_mlp_round<<<8, 256>>>(T.w, T.wq, nullptr);
      k_mlp_grad<<<(nb + 255) / 256, 256>>>(T.wq, T.x, T.mode, T.sizes, T.idx + b0, nb, 1.0f / (float)nb, T.grad,
                                            T.loss);
      ++step;
      const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
      k_mlp_adam<<<8, 256>>>(T.w, T.m, T.v, T.grad, lr, b1, b2, eps, bc1, bc2);
    }
    MCK(cudaGetLastError());
    MCK(cudaMemcpy(&epoch_loss, T.loss, 4, cudaMemcpyDeviceToHost));
    epoch_loss *= (float)batch / (float)n;  // loss was summed per minibatch mean
  }
  unsigned short* wb = nullptr;
  MCK(cudaMalloc(&wb, NP * 2));
  k_mlp_round<<<8, 256>>>(T.w, T.wq, wb);
  cudaError_t e = cudaMemcpy(params, T.w, NP * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && bf16_out) e = cudaMemcpy(bf16_out, wb, NP * 2, cudaMemcpyDeviceToHost);
  cudaFree(wb);
  if (e != cudaSuccess) return mlp_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  if (last_loss) *last_loss = epoch_loss;
  return SIM_OK;
}

}  // extern "C"
