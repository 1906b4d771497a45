// launch.h -- host-side launch wrappers of the kernels in kernels.cu (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"

namespace qc {

constexpr int kMaxRuns = 6;

// One gate on the compressed state.
struct GateLaunch {
  Pool P;
  CtlParams ctl;
  GateCoef g;
  unsigned long long items;      // work items (chunk pairs)
  unsigned long long nact;       // active chunks (in-chunk gates pair them up)
  unsigned long long free_mask;  // chunk-index bits enumerated by the item counter
  unsigned long long run_mask[kMaxRuns];  // free_mask as runs of contiguous bits ...
  uint32_t run_shift[kMaxRuns];           // ... each receiving the counter's bits shifted up by run_shift
  int nruns;                              // -1: more runs than kMaxRuns (deposit bit by bit)
  unsigned long long hi_vals;    // control values on chunk-index bits
  unsigned long long pair_bit;   // chunk-index bit of the target (cross-chunk gates), else 0
  uint32_t lo_mask, lo_vals;     // controls inside a chunk
  int target;                    // target bit (in-chunk gates)
  int pair;                      // 1: target >= chunk_log2
  int prof;                      // 1: accumulate per-phase SM cycles
  uint32_t modes;                // chunk modes the encoder may choose (bit m = mode m)
  const uint8_t* sel_dec;        // the selector's decisions, one byte per active chunk (index 2 item + side;
                                 // bit 0 SPLIT trial, bit 1 PALETTE trial), or nullptr: the mode set decides
  uint32_t gfeat;                // gate features for the selector (see SelCtx)
  float* trace;                  // selector training records (device) or nullptr
  unsigned long long* trace_n;
  unsigned long long trace_cap;
  uint8_t* bc;                   // block cache lines (kBcLines of bc_line_bytes) or nullptr
  uint32_t* defer;               // streaming kernel: items left to the general kernel (device list)
  int fast_kind;                 // streaming kernel: 0 cross-chunk pairs, 1 in-chunk target < 2, 2 in-chunk
                                 // target 2..6 (partner in another lane), 3 in-chunk diagonal gate
  int list;                      // general kernel: 1 = run the items the streaming kernel left
  // streaming kernel arithmetic (the same values as the kept-term sums of GateCoef):
  int arith;                     // 0 dense: the four sums with every coefficient, zeros included;
                                 // 1 diagonal (u01 = u10 = 0); 2 anti-diagonal (u00 = u11 = 0);
                                 // 3 real (every imaginary part zero): the real products only;
                                 // 4 every coefficient part +-2^sk, none zero: signed sums, then scaled
  int rop[2];                    // diagonal / anti-diagonal, per output row: 0 complex product, 1 copy
                                 // (the entry is exactly 1), 2 negation (exactly -1)
  double cf[16];                 // dense: row r's coefficients of (ar, ai, br, bi) / (ai, ar, bi, br) at 4r
  double du[4];                  // diagonal: u00, u11; anti-diagonal: u01, u10 (re, im)
  uint32_t sgn;                  // arith 4: bit q set if coefficient cf[q] is negative
  int sk;                        // arith 4: log2 of the coefficients' common magnitude
};

// One gate of one simulator inside a batched launch; its work items are the global
// items [begin, begin + L.items).
struct BatchJob {
  GateLaunch L;
  unsigned long long begin;
};

// Records the message sim_last_error() returns on the calling thread.
void set_last_error(const char* msg);

// Eq. sigbits: significant bits S = 12 - EXP(eps) kept of a binary64 value under the
// pointwise relative bound eps (EXP = the IEEE exponent of eps); 64 for eps = 0 (the
// lossless stage); -1 for a bound outside {0} U [2^-52, 1).
int sig_bits_of(double eps);

int vpt_for(int kc);
size_t gate_smem_bytes(int kc);
size_t codec_smem_bytes(int kc);
int gate_ctas_per_sm(int kc);

cudaError_t launch_gate(const GateLaunch& L, int grid, cudaStream_t st);
// The streaming kernel (chunk_log2 in [7, 11]): the work items it can take whole, the
// rest appended to L.defer for launch_gate with L.list = 1 right after it.
constexpr int kFastMinKC = 7;
int fast_ctas_per_sm(int kc);
int fast_warps();        // warps per CTA of the streaming kernel (a pair of warps per work item)
int fast_pairs();        // work items a CTA of the streaming kernel runs at once
int fast_warp_cache();   // page ids each of its warps may hold
cudaError_t launch_gate_fast(const GateLaunch& L, int grid, cudaStream_t st);
cudaError_t launch_post(const Pool& P, const CtlParams& cp, int grid_ctas, cudaStream_t st);
// The learned selector's decisions for every active chunk of the gate L describes,
// written to dec (one byte per chunk, index 2 item + side) before the gate runs; mlp
// holds the bfloat16 parameters (device, 16-byte aligned).
cudaError_t launch_select(const GateLaunch& L, const unsigned short* mlp, uint8_t* dec, int grid, cudaStream_t st);
cudaError_t launch_gate_batch(const BatchJob* jobs, int njobs, unsigned long long total, int kc, int grid,
                              cudaStream_t st);
cudaError_t launch_post_batch(const BatchJob* jobs, int njobs, int grid_ctas, cudaStream_t st);
cudaError_t launch_pool_init(const Pool& P, unsigned long long nchunks, cudaStream_t st);
cudaError_t launch_init_chunk0(const Pool& P, unsigned long long nchunks, cudaStream_t st);
cudaError_t launch_codec_encode(const double* in, unsigned long long nchunks, int kc, uint32_t S, int force,
                                uint8_t* out, unsigned long long stride, uint32_t* lens, unsigned int* err,
                                cudaStream_t st);
cudaError_t launch_codec_encode(const double* in, unsigned long long nchunks, int kc, uint32_t S, int force,
                                uint32_t modes, uint8_t* out, unsigned long long stride, uint32_t* lens,
                                unsigned int* err, cudaStream_t st);
cudaError_t launch_codec_decode(const uint8_t* in, unsigned long long stride, const uint32_t* lens,
                                unsigned long long nchunks, int kc, double* out, unsigned int* err, cudaStream_t st);
cudaError_t launch_decode_range(const Pool& P, unsigned long long first_amp, unsigned long long count, double* out,
                                cudaStream_t st);
cudaError_t launch_chunk_norms(const Pool& P, unsigned long long cfirst, unsigned long long nchunks, double* out,
                              cudaStream_t st);
cudaError_t launch_chunk_dots(const Pool& P, unsigned long long cfirst, unsigned long long nchunks, const double* ref,
                             double* out, cudaStream_t st);
cudaError_t launch_mode_counts(const Pool& P, unsigned long long nchunks, unsigned long long* counts,
                               unsigned long long* wide, cudaStream_t st);
cudaError_t launch_copy_image(const Pool& P, unsigned long long chunk, uint8_t* out, cudaStream_t st);

cudaError_t launch_sv_init(double* psi, unsigned long long amps, cudaStream_t st);
cudaError_t launch_sv_gate(double* psi, int n, const GateCoef& g, int target, unsigned long long cmask,
                           unsigned long long cvals, uint32_t rows, cudaStream_t st);

// Checkpoint: image lengths, gather of all images, and the rebuild of directory and
// page arena from saved images (pages [0, used) in chunk order).
cudaError_t launch_checkpoint_lengths(const Pool& P, unsigned long long nchunks, uint32_t* len, cudaStream_t st);
cudaError_t launch_checkpoint_gather(const Pool& P, unsigned long long nchunks, const unsigned long long* off,
                                     uint8_t* out, cudaStream_t st);
cudaError_t launch_checkpoint_scatter(const Pool& P, unsigned long long nchunks, const unsigned long long* off,
                                      const unsigned long long* pbase, const uint32_t* len, const uint8_t* in,
                                      unsigned long long used, cudaStream_t st);

}  // namespace qc
