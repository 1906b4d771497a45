// noalloc.cu -- sim_codec_encode_noalloc: the device chunk encoder for callers that
// must not allocate device memory.
//
// sim_codec_encode (host-buffer form) stages the caller's chunks and the encoded
// images in a device buffer it obtains with cudaMalloc for every call.  Some callers
// cannot allow that: a process whose device memory is already handed out to another
// allocator (a framework's caching allocator that has reserved the free memory), or
// one that runs under a fixed device-memory budget enforced by the host application
// and cannot risk an allocation failure in the middle of its work.  This entry point
// stages through a fixed, file-scope device array instead, so it never calls
// cudaMalloc, cudaFree or an allocating library routine.
//
// The array lives in every GPU that loads the library, from module load until the
// process exits.  All calls on a device share it, so two calls whose work overlaps
// on that device (different host threads or streams) race on it: callers must
// serialise them.  Each call rewrites the parts it uses (inputs, images, lengths,
// error word), so nothing from an earlier call leaks into its result.  The first
// call on a device looks up the array's device address (under a lock, so concurrent
// first calls from several host threads are safe) and keeps it; a cudaDeviceReset
// unloads the module and invalidates that address, so this entry point must not be
// used on a device after it was reset.
#include <mutex>

#include "../../include/qcsim.h"
#include "launch.h"

namespace {

// 8 MiB: input chunks + their images + lengths + the error word of one call.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device with that
// device current (host code cannot use the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_lock;

sim_status noalloc_fail(sim_status s, const char* msg) {
  qc::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" sim_status sim_codec_encode_noalloc(const double* in, uint64_t n_chunks, int chunk_log2, double eps,
                                               int force_mode, uint8_t* out, uint64_t out_stride, uint32_t* out_len) {
  if (!in || !out || !out_len) return noalloc_fail(SIM_ERR_INVALID, "NULL argument");
  if (chunk_log2 < 0 || chunk_log2 > qc::kMaxKC) return noalloc_fail(SIM_ERR_INVALID, "chunk_log2 outside [0, 11]");
  if (force_mode >= (int)qc::M_NMODES) return noalloc_fail(SIM_ERR_INVALID, "unknown mode");
  const int S = qc::sig_bits_of(eps);  // Eq. sigbits, as every other entry point maps eps
  if (S < 0) return noalloc_fail(SIM_ERR_INVALID, "eps outside {0} U [2^-52, 1)");
  const uint64_t need = 16 + (16ull << chunk_log2) + (1ull << chunk_log2) / 2 + 32;
  if (out_stride < need || (out_stride & 15)) return noalloc_fail(SIM_ERR_INVALID, "out_stride too small or not 16-aligned");
  if (n_chunks == 0) return SIM_OK;
  // Bound the request before forming any product with n_chunks, so that none can wrap:
  // each chunk needs its input, its image slot and its length in the array.
  if (out_stride > kNoAllocScratchBytes ||
      n_chunks > kNoAllocScratchBytes / ((16ull << chunk_log2) + out_stride + 4))
    return noalloc_fail(SIM_ERR_INVALID, "request larger than the 8 MiB scratch");
  // layout inside the static array: [error word | pad to 256][inputs][images][lengths]
  const uint64_t in_bytes = n_chunks * (16ull << chunk_log2);
  const uint64_t img_bytes = n_chunks * out_stride;
  const uint64_t len_bytes = n_chunks * 4;
  const uint64_t off_in = 256, off_img = off_in + ((in_bytes + 255) & ~255ull);
  const uint64_t off_len = off_img + ((img_bytes + 255) & ~255ull);
  if (off_len + len_bytes > kNoAllocScratchBytes) return noalloc_fail(SIM_ERR_INVALID, "request larger than the 8 MiB scratch");

  // set-up, once per device, with that device current: the first call on a device
  // looks up the array's device address
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(SIM_ERR_CUDA, "cudaGetDevice failed or device index too large");
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> guard(g_scratch_lock);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
        return noalloc_fail(SIM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      g_scratch_ptr[dev] = p;
    }
    ptr = g_scratch_ptr[dev];
  }
  unsigned char* base = static_cast<unsigned char*>(ptr);
  unsigned int* derr = reinterpret_cast<unsigned int*>(base);
  double* din = reinterpret_cast<double*>(base + off_in);
  uint8_t* dimg = base + off_img;
  uint32_t* dlen = reinterpret_cast<uint32_t*>(base + off_len);

  cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(unsigned int), 0);  // the error word starts at zero
  if (e == cudaSuccess) e = cudaMemcpyAsync(din, in, in_bytes, cudaMemcpyHostToDevice, 0);
  if (e == cudaSuccess)
    e = qc::launch_codec_encode(din, n_chunks, chunk_log2, (uint32_t)S, force_mode, dimg, out_stride, dlen, derr, 0);
  unsigned int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_len, dlen, len_bytes, cudaMemcpyDeviceToHost, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dimg, img_bytes, cudaMemcpyDeviceToHost, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) return noalloc_fail(SIM_ERR_CUDA, cudaGetErrorString(e));
  if (herr & qc::E_NONFINITE) return noalloc_fail(SIM_ERR_INVALID, "input holds a non-finite value");
  if (herr & qc::E_MODE) return noalloc_fail(SIM_ERR_INVALID, "forced mode does not apply to a chunk");
  return SIM_OK;
}
