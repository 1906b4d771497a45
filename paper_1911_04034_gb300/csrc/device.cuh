// device.cuh -- device-side building blocks of libqcsim (sm_103a).
//
//  * block-wide scans (warp shuffles)
//  * chunk decoder and encoder working on shared-memory tiles: bit-plane truncation
//    (Section 4.2, Eq. sigbits), XOR leading-zero coding with a 2-bit code
//    (Section 4.2, Solution C) and the ZERO/CONST/PERIOD/STREAM/RAW modes that stand
//    in for the Zstd stage
//  * gate arithmetic on an amplitude pair (Section 3.1, Eq. matrix1 / Eq. matrix2)
//  * the compressed-block pool: 512-byte pages, per-CTA page caches, a global stack
//    of free pages, and a directory entry per chunk
//
// One CTA of kThreads threads owns one work item at a time; every function named
// *_block is called by all threads of the CTA.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qc {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPage = 512;
constexpr int kCacheCap = 128;
constexpr int kMaxKC = 11;

enum : uint32_t {
  M_ZERO = 0, M_CONST = 1, M_PERIOD = 2, M_STREAM = 3, M_RAW = 4, M_SPLIT = 5, M_PALETTE = 6, M_NMODES = 7
};
// Solution C's modes; SPLIT (Solution D, re parts then im parts) and PALETTE (distinct
// values plus k-bit indices) only on request
constexpr uint32_t kDefaultModes = 0x1Fu;
constexpr uint32_t kAllModes = 0x7Fu;  // every mode, SPLIT and PALETTE trials included
constexpr uint32_t kPaletteMax = 256;  // most distinct values a PALETTE image lists
// Index width of a palette of P entries: the smallest k >= 1 with 2^k >= P.
__host__ __device__ __forceinline__ uint32_t palette_bits(uint32_t P) {
  uint32_t k = 1;
  while ((1u << k) < P) ++k;
  return k;
}

enum : uint32_t { E_OK = 0, E_OOM = 1, E_CORRUPT = 2, E_NONFINITE = 4, E_MODE = 8, E_TIMEOUT = 16 };

// ---------------------------------------------------------------- sizes ---- //
__host__ __device__ __forceinline__ uint32_t round16(uint32_t x) { return (x + 15u) & ~15u; }
// Codes: 2 bits per coded value, padded to 16 bytes.
__host__ __device__ __forceinline__ uint32_t code_bytes(uint32_t nv) { return round16((nv + 3u) >> 2); }
// Residual stream: 64-bit words, padded to 16 bytes.
__host__ __device__ __forceinline__ uint32_t resid_bytes(uint32_t bits) { return ((bits + 127u) >> 7) << 4; }
// Largest image the encoder writes for a chunk of 2^kc amplitudes (RAW).
__host__ __device__ __forceinline__ uint32_t max_image_bytes(int kc) { return 16u + (16u << kc); }
// Largest image any mode can produce, a forced STREAM of incompressible values included.
__host__ __device__ __forceinline__ uint32_t max_coded_bytes(int kc) {
  return 16u + code_bytes(2u << kc) + resid_bytes(64u * (2u << kc));
}
__host__ __device__ __forceinline__ uint32_t max_pages(int kc) { return (max_image_bytes(kc) + kPage - 1) / kPage; }
// Directory entry: [bytes u32][npages u32][8 reserved][data: page ids or the image itself]
__host__ __device__ __forceinline__ uint32_t dir_stride(int kc) { return round16(16u + 4u * max_pages(kc)); }
__host__ __device__ __forceinline__ uint32_t inline_cap(int kc) { return dir_stride(kc) - 16u; }

// ------------------------------------------------------------- device state -- //
// Counters and controller state of one simulator, in device memory.
struct DevCtl {
  unsigned long long E;         // sum of image bytes after the last finished gate
  unsigned long long dE;        // change of E during the running gate (two's complement)
  unsigned long long Emax;      // largest E after any gate
  long long top;                // free pages on the global stack
  unsigned long long nfreed;    // pages pushed to the overflow list during the running gate
  unsigned long long gates;     // gates finished
  unsigned long long amp_updates;
  unsigned long long peak_pages;
  long long switch_gate;        // first gate run lossy, -1 if none
  double lb_sum;                // sum of delta_i over lossy gates
  double lb_prod;               // prod (1 - delta_i)
  int level;                    // ladder level of the last gate (0 = lossless)
  int S_last;                   // significant bits of the last gate
  unsigned int err;             // E_* flags
  unsigned int pad;
  unsigned long long bytes_in;  // image bytes the gate kernels read (cumulative)
  unsigned long long bytes_out; // image bytes the gate kernels wrote (cumulative)
  unsigned long long phase_cycles[6];  // SM cycles of CTA thread 0 per phase when profiling
  unsigned long long split_trials;     // chunk encodes that ran the Solution D trial
  unsigned long long trace_n;          // selector training records written
  unsigned long long bc_lookups;       // block-cache lookups (cumulative)
  unsigned long long bc_hits;          // block-cache hits (cumulative)
  unsigned long long bc_gate_lookups;  // ... during the running gate
  unsigned long long bc_gate_hits;
  unsigned int bc_zero_streak;         // gates in a row with lookups and no hit
  unsigned int bc_off;                 // gates the cache still sits out (0 = on)
  unsigned long long ndefer;           // work items of the running gate the streaming kernel left to the general one
  unsigned int fast_all;               // 1: the streaming kernel left every item of the running gate
  unsigned int fast_pad;
  unsigned long long fast_items;       // work items the streaming kernel committed (cumulative)
  unsigned long long fast_deferred;    // work items it left to the general kernel (cumulative)
  unsigned int timeout_site;           // where a bounded wait gave up (E_TIMEOUT): 1 item start, 2 pass, 3 item end
  unsigned int timeout_pad;
  unsigned long long wc_pages;         // free pages the streaming kernel's warps keep in their caches
  unsigned long long palette_trials;   // chunk encodes that ran the PALETTE trial
  long long n64;                       // images whose header says S = 64 (as of the last gate)
  long long dn64;                      // ... its change during the running gate
};

// Controller parameters (host-computed, constant for the handle).
struct CtlParams {
  unsigned long long thresh;    // floor(tau * budget)
  unsigned long long inflight;  // two decompressed blocks (Eq. totalnbBytes, r = 1)
  int nlevels;                  // lossy levels on the ladder (0 = lossless only)
  int ladder;                   // 0 jump, 1 one level per gate, 2 guarded (worst case fits)
  int S[8];                     // significant bits per level (index level-1)
  double delta[8];              // 2^EXP(eps) per level
  unsigned long long nchunks;   // chunks of the state
  unsigned long long touched;   // chunks the running gate rewrites (set per gate)
  unsigned long long maxb[9];   // largest image the encoder can write at level l (0 = lossless)
  int wide_gate;                // the running gate has a nonzero coefficient below 2^-52 (set per gate)
  int pad;
};

// Section 3.7: before a gate, relax the bound if E + inflight > floor(tau * budget).
// Guarded ladder: the smallest level (never below the current one) at which even
// the largest images on every chunk the gate rewrites keep E within floor(tau *
// budget): a gate rewriting every chunk ends with at most the sum of those images,
// otherwise E grows by at most that sum.  A chunk holding a subnormal is coded at 64
// bits at any level (Eq. sigbits cannot truncate it): once the run is lossy, the n64
// images still at 64 bits are assumed to be among the rewritten chunks, and a gate
// that may make subnormals of normal values (a nonzero coefficient below 2^-52)
// counts all of its chunks at 64 bits.
__host__ __device__ __forceinline__ int next_level(const CtlParams& p, unsigned long long E, int level, long long n64) {
  if (p.nlevels == 0 || level >= p.nlevels) return level;
  if (p.ladder == 2) {
    unsigned long long wide = 0;
    if (p.wide_gate) wide = p.touched;
    else if (level > 0) wide = n64 < 0 ? 0ull : ((unsigned long long)n64 < p.touched ? (unsigned long long)n64 : p.touched);
    for (int l = level; l < p.nlevels; ++l) {
      const unsigned long long worst = (p.touched - wide) * p.maxb[l] + wide * p.maxb[0];
      if ((p.touched >= p.nchunks ? worst : E + worst) <= p.thresh) return l;
    }
    return p.nlevels;
  }
  if (E + p.inflight <= p.thresh) return level;
  return p.ladder == 1 ? level + 1 : p.nlevels;
}
// Largest image of a chunk at S significant bits: STREAM with every value fully
// explicit, or RAW if smaller (the encoder never writes more than both).
__host__ __device__ __forceinline__ unsigned long long max_level_image(int kc, int S) {
  const uint32_t N = 2u << kc;
  const unsigned long long stream = 16ull + code_bytes(N) + resid_bytes((uint32_t)S * N);
  const unsigned long long raw = 16ull + 8ull * N;
  return stream < raw ? stream : raw;
}
__host__ __device__ __forceinline__ int level_bits(const CtlParams& p, int level) {
  return level == 0 ? 64 : p.S[level - 1];
}

struct Pool {
  uint8_t* pages;          // npages * kPage bytes
  uint32_t* dir;           // nchunks * dir_stride(kc) bytes
  uint32_t* stack;         // free page ids, [0, top)
  uint32_t* freed;         // overflow list, [0, nfreed)
  uint32_t* cache;         // grid * kCacheCap page ids
  uint32_t* cache_n;       // grid counts
  uint32_t* wcache;        // streaming kernel: page ids each of its warps keeps across launches
  uint32_t* wcache_n;      // ... and their counts (one per warp of its grid)
  DevCtl* ctl;
  unsigned long long npages;
  uint32_t dir_words;      // dir_stride / 4
  int kc;
};

// ------------------------------------------------------- block cache ---- //
// Section 3.4: a line holds the two compressed input blocks of a work item and the two
// output blocks the running gate made of them; another item of the same gate with the
// same inputs takes the outputs instead of decoding, applying and encoding.  Lines are
// valid for one gate (tag = gate serial << 2 | state; states 0 empty, 1 being written,
// 2 ready); a hit is confirmed byte by byte.
constexpr int kBcLines = 256;
constexpr uint32_t kBcHead = 64;
constexpr unsigned int kBcZeroGates = 16;  // gates with lookups and no hit before the cache pauses
constexpr unsigned int kBcPause = 64;      // gates it then sits out before probing again
struct BcLine {
  unsigned long long tag;
  unsigned long long key;
  uint32_t len[4];  // input 0, input 1, output 0, output 1
};
__host__ __device__ __forceinline__ uint64_t bc_line_bytes(uint32_t img_cap) { return kBcHead + 4ull * img_cap; }

// -------------------------------------------------------------- scans ----- //
__device__ __forceinline__ uint32_t warp_incl_add(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}
__device__ __forceinline__ int warp_incl_max(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = max(v, n);
  }
  return v;
}

// Warp totals of the block scans, double-buffered: each scan uses buffer pp and flips
// pp, so two consecutive scans never share a buffer and one barrier per scan is
// enough (the other scan's barrier separates a buffer's readers from its next writer).
struct ScanSmem {
  uint32_t wsum2[2][kWarps];
  uint32_t wsum[2][kWarps];
  uint32_t wor[2][kWarps];
  uint32_t wand[2][kWarps];
  uint32_t wlm[2][kWarps];  // lead-byte scan: bytes set, and their values
  uint32_t wlv[2][kWarps];
  uint32_t wlm2[2][kWarps];  // the second chunk's lead-byte scan (decode_stream32_pair)
  uint32_t wlv2[2][kWarps];
  uint32_t bits_period;
  unsigned long long bc_part[kWarps];  // block cache: per-warp partial hashes
  int bc_flag;                         // block cache: 0 miss, 1 candidate line, 2 line claimed
};

// Exclusive prefix sum over the CTA with one barrier; also ORs `fo` and ANDs `fa`
// over the CTA.  All threads must call it.
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t fo, uint32_t fa, ScanSmem& s, int& pp,
                                               uint32_t* total, uint32_t* all_or, uint32_t* all_and) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_add(v);
  const uint32_t wo = __reduce_or_sync(0xffffffffu, fo);
  const uint32_t wa = __reduce_and_sync(0xffffffffu, fa);
  if (lane == 31) {
    s.wsum[pp][w] = inc;
    s.wor[pp][w] = wo;
    s.wand[pp][w] = wa;
  }
  __syncthreads();
  // lane i < kWarps reads warp i's totals; warp reductions combine them
  const uint32_t x = lane < kWarps ? s.wsum[pp][lane] : 0u;
  const uint32_t xo = lane < kWarps ? s.wor[pp][lane] : 0u;
  const uint32_t xa = lane < kWarps ? s.wand[pp][lane] : 0xffffffffu;
  const uint32_t base = __reduce_add_sync(0xffffffffu, lane < w ? x : 0u);
  pp ^= 1;
  *total = __reduce_add_sync(0xffffffffu, x);
  *all_or = __reduce_or_sync(0xffffffffu, xo);
  *all_and = __reduce_and_sync(0xffffffffu, xa);
  return base + inc - v;
}

// Two exclusive prefix sums at once (same barrier), plus OR/AND flags.
__device__ __forceinline__ void block_scan2(uint32_t v, uint32_t v2, uint32_t fo, uint32_t fa, ScanSmem& s, int& pp,
                                            uint32_t* ex, uint32_t* ex2, uint32_t* total, uint32_t* total2,
                                            uint32_t* all_or, uint32_t* all_and) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_add(v);
  const uint32_t inc2 = warp_incl_add(v2);
  const uint32_t wo = __reduce_or_sync(0xffffffffu, fo);
  const uint32_t wa = __reduce_and_sync(0xffffffffu, fa);
  if (lane == 31) {
    s.wsum[pp][w] = inc;
    s.wsum2[pp][w] = inc2;
    s.wor[pp][w] = wo;
    s.wand[pp][w] = wa;
  }
  __syncthreads();
  const uint32_t x = lane < kWarps ? s.wsum[pp][lane] : 0u, x2 = lane < kWarps ? s.wsum2[pp][lane] : 0u;
  const uint32_t xo = lane < kWarps ? s.wor[pp][lane] : 0u;
  const uint32_t xa = lane < kWarps ? s.wand[pp][lane] : 0xffffffffu;
  const uint32_t base = __reduce_add_sync(0xffffffffu, lane < w ? x : 0u);
  const uint32_t base2 = __reduce_add_sync(0xffffffffu, lane < w ? x2 : 0u);
  pp ^= 1;
  *ex = base + inc - v;
  *ex2 = base2 + inc2 - v2;
  *total = __reduce_add_sync(0xffffffffu, x);
  *total2 = __reduce_add_sync(0xffffffffu, x2);
  *all_or = __reduce_or_sync(0xffffffffu, xo);
  *all_and = __reduce_and_sync(0xffffffffu, xa);
}

// The leading three bytes of a value that a thread's run of coded values leaves for its
// successor: bytes a value writes explicitly replace the running ones, bytes it copies
// keep them.  A run is summarised as (M, V): the bits of the top three bytes (of the
// value's high word) that it sets, and their values.  Composition (earlier, later) =
// (M1 | M2, (V1 & ~M2) | V2) is associative; this is its exclusive scan over the CTA
// (identity (0, 0): the first value's predecessor is 0), one barrier
// (block_lead_scan returns V).
constexpr uint32_t kLeadFull = 0xFFFFFF00u;  // all three leading bytes set: earlier runs no longer matter

// The warp part: inclusive (im, iv) and exclusive (em, ev) composition within the warp.
__device__ __forceinline__ void warp_lead_scan(uint32_t M, uint32_t V, uint32_t& im, uint32_t& iv, uint32_t& em,
                                               uint32_t& ev) {
  const int lane = threadIdx.x & 31;
  im = M;
  iv = V;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    // lanes below d already cover the whole warp prefix; full lanes cannot change
    if (__all_sync(0xffffffffu, im == kLeadFull || lane < d)) break;
    const uint32_t um = __shfl_up_sync(0xffffffffu, im, d), uv = __shfl_up_sync(0xffffffffu, iv, d);
    if (lane >= d) {
      iv = (uv & ~im) | iv;
      im |= um;
    }
  }
  em = __shfl_up_sync(0xffffffffu, im, 1);
  ev = __shfl_up_sync(0xffffffffu, iv, 1);
  if (lane == 0) em = ev = 0u;
}
// Earlier warps' totals, nearest first, until every leading byte is set; then the
// thread's exclusive prefix.
__device__ __forceinline__ uint32_t lead_prefix(const uint32_t* wlm, const uint32_t* wlv, uint32_t em, uint32_t ev) {
  uint32_t pm = 0u, pv = 0u;
  for (int i = (int)(threadIdx.x >> 5) - 1; i >= 0 && pm != kLeadFull; --i) {
    pv |= wlv[i] & ~pm;
    pm |= wlm[i];
  }
  return (pv & ~em) | ev;
}
__device__ __forceinline__ uint32_t block_lead_scan(uint32_t M, uint32_t V, ScanSmem& s, int& pp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t im, iv, em, ev;
  warp_lead_scan(M, V, im, iv, em, ev);
  if (lane == 31) {
    s.wlm[pp][w] = im;
    s.wlv[pp][w] = iv;
  }
  __syncthreads();
  const uint32_t P = lead_prefix(s.wlm[pp], s.wlv[pp], em, ev);
  pp ^= 1;
  return P;
}
// The same scan for two independent runs (two chunks), one barrier.
__device__ __forceinline__ void block_lead_scan2(uint32_t M0, uint32_t V0, uint32_t M1, uint32_t V1, ScanSmem& s,
                                                 int& pp, uint32_t& P0, uint32_t& P1) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t im0, iv0, em0, ev0, im1, iv1, em1, ev1;
  warp_lead_scan(M0, V0, im0, iv0, em0, ev0);
  warp_lead_scan(M1, V1, im1, iv1, em1, ev1);
  if (lane == 31) {
    s.wlm[pp][w] = im0;
    s.wlv[pp][w] = iv0;
    s.wlm2[pp][w] = im1;
    s.wlv2[pp][w] = iv1;
  }
  __syncthreads();
  P0 = lead_prefix(s.wlm[pp], s.wlv[pp], em0, ev0);
  P1 = lead_prefix(s.wlm2[pp], s.wlv2[pp], em1, ev1);
  pp ^= 1;
}

// Block cache key of a work item: a hash of its two staged images (every 16-byte
// unit mixed with its position, summed).  All threads; one barrier.
__device__ __forceinline__ unsigned long long bc_mix(uint4 v, uint32_t pos) {
  unsigned long long z = (((unsigned long long)v.y << 32) | v.x) + 0x9E3779B97F4A7C15ull * (pos + 1u);
  z ^= (((unsigned long long)v.w << 32) | v.z) * 0xD1B54A32D192ED03ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long bc_key(const uint8_t* img0, uint32_t b0, const uint8_t* img1, uint32_t b1,
                                                     ScanSmem& s) {
  const uint32_t u0 = b0 >> 4, u1 = b1 >> 4;
  unsigned long long h = 0ull;
  for (uint32_t u = threadIdx.x; u < u0 + u1; u += kThreads)
    h += bc_mix(u < u0 ? reinterpret_cast<const uint4*>(img0)[u] : reinterpret_cast<const uint4*>(img1)[u - u0],
                u < u0 ? u : 0x80000000u + (u - u0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31u) == 0) s.bc_part[threadIdx.x >> 5] = h;
  __syncthreads();
  unsigned long long k = (unsigned long long)b0 * 0x100000001B3ull + b1;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) k += s.bc_part[i];
  return k;
}

// ---------------------------------------------------------- bit helpers --- //
// Leading identical bytes of v and its predecessor, capped at 3 (the 2-bit code).
__device__ __forceinline__ uint32_t xor_code(uint64_t v, uint64_t prev) {
  uint64_t d = v ^ prev;
  uint32_t L = d ? (uint32_t)(__clzll((long long)d) >> 3) : 8u;
  return L < 3u ? L : 3u;
}
__device__ __forceinline__ uint32_t resid_len(uint32_t c, uint32_t S) {
  int r = (int)S - 8 * (int)c;
  return r > 0 ? (uint32_t)r : 0u;
}
// r bits (1..64) starting at MSB-first bit position `pos` of the word array.
__device__ __forceinline__ uint64_t get_bits(const uint64_t* w, uint32_t pos, uint32_t r) {
  uint32_t wi = pos >> 6, off = pos & 63u;
  uint64_t hi = w[wi] << off;
  if (off + r > 64u) hi |= w[wi + 1] >> (64u - off);
  return hi >> (64u - r);
}
__device__ __forceinline__ uint64_t trunc_mask(uint32_t S) { return S >= 64u ? ~0ull : (~0ull << (64u - S)); }

// The residual stream is a sequence of 64-bit little-endian words read most
// significant bit first; as 32-bit units in stream order, unit q is memory word q ^ 1.
// 64 stream bits starting at bit position o (needs 8 readable bytes past the stream).
__device__ __forceinline__ void stream_window(const uint32_t* m32, uint32_t o, uint32_t& hi, uint32_t& lo) {
  const uint32_t q = o >> 5, sh = o & 31u;
  const uint32_t x0 = m32[q ^ 1u], x1 = m32[(q + 1u) ^ 1u], x2 = m32[(q + 2u) ^ 1u];
  hi = __funnelshift_l(x1, x0, sh);
  lo = __funnelshift_l(x2, x1, sh);
}

// ------------------------------------------------------------ tile layout -- //
// A decoded chunk lives in shared memory as 2^kc amplitudes of 16 bytes with one
// unused 16-byte slot after every 8 amplitudes.  Threads own contiguous runs of
// values (what the prefix scans need); the padding spreads those runs over all
// banks, so every 16-byte access of a warp is conflict-free.
__host__ __device__ __forceinline__ uint32_t tile_amp(uint32_t a) { return a + (a >> 3); }
__host__ __device__ __forceinline__ uint32_t tile_val(uint32_t j) { return 2u * tile_amp(j >> 1) + (j & 1u); }
__host__ __device__ __forceinline__ uint32_t tile_words(int kc) {
  const uint32_t A = 1u << kc;
  return 2u * (A + (A >> 3));
}

// Thread t owns values [t*VPT, t*VPT + VPT) (whole amplitudes when VPT >= 2).
template <int VPT>
__device__ __forceinline__ void load_vals(const uint64_t* tile, uint32_t j0, uint32_t N, uint64_t v[VPT]) {
  if (VPT >= 2) {
    const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(tile);
#pragma unroll
    for (int m = 0; m < VPT / 2; ++m) {
      const uint32_t a = (j0 >> 1) + m;
      if (2u * a < N) {
        const ulonglong2 q = t2[tile_amp(a)];
        v[2 * m] = q.x;
        v[2 * m + 1] = q.y;
      } else {
        v[2 * m] = v[2 * m + 1] = 0ull;
      }
    }
  } else {
    v[0] = j0 < N ? tile[tile_val(j0)] : 0ull;
  }
}
template <int VPT>
__device__ __forceinline__ void store_vals(uint64_t* tile, uint32_t j0, uint32_t N, const uint64_t v[VPT]) {
  if (VPT >= 2) {
    ulonglong2* t2 = reinterpret_cast<ulonglong2*>(tile);
#pragma unroll
    for (int m = 0; m < VPT / 2; ++m) {
      const uint32_t a = (j0 >> 1) + m;
      if (2u * a < N) t2[tile_amp(a)] = make_ulonglong2(v[2 * m], v[2 * m + 1]);
    }
  } else {
    if (j0 < N) tile[tile_val(j0)] = v[0];
  }
}

// ----------------------------------------------------------- decoder ----- //
// Position in the chunk of the k-th coded value: k itself, or for SPLIT (Solution D)
// the real parts of all amplitudes first, then the imaginary parts.
template <bool SPLIT>
__device__ __forceinline__ uint32_t coded_pos(uint32_t k, uint32_t A) {
  return SPLIT ? (k < A ? 2u * k : 2u * (k - A) + 1u) : k;
}

// Bits of the top three bytes of a high word that a value with code c writes
// explicitly (bytes c..2), and those it copies from its predecessor (bytes 0..c-1).
__device__ __forceinline__ uint32_t lead_explicit(uint32_t c) { return 0xFFFFFF00u & (0xFFFFFFFFu >> (8u * c)); }
__device__ __forceinline__ uint32_t lead_copied(uint32_t c) { return ~(0xFFFFFFFFu >> (8u * c)); }

// Decodes the XOR-coded values of a PERIOD / STREAM / SPLIT image.  W32: S <= 32, so
// every value's low word is zero and only high words are read from the stream.
// FULL: all 2^(kc+1) values are coded (STREAM, SPLIT), so with VPT >= 2 every value
// of every thread exists.
template <int VPT, bool SPLIT, bool W32, bool FULL>
__device__ bool decode_xor_block(const uint8_t* payload, uint32_t plen, uint32_t nv, uint32_t S, uint32_t bits,
                                 uint64_t* tile, ScanSmem& s, int& pp) {
  const uint32_t A = nv >> 1;
  const uint32_t* codes32 = reinterpret_cast<const uint32_t*>(payload);
  const uint32_t cb = code_bytes(nv);
  const uint32_t* m32 = reinterpret_cast<const uint32_t*>(payload + cb);
  const uint32_t j0 = threadIdx.x * VPT;
  bool has[VPT];
#pragma unroll
  for (int k = 0; k < VPT; ++k) has[k] = FULL ? (VPT >= 2 || j0 < nv) : (j0 + k < nv);
  // the 2-bit codes of this thread's values share one 32-bit word (VPT divides 16)
  const uint32_t cword = j0 < nv ? codes32[j0 >> 4] : 0u;
  const uint32_t cbase = VPT >= 4 ? cword >> (8u * ((j0 >> 2) & 3u)) : cword;
  uint32_t c[VPT], r[VPT];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const uint32_t j = j0 + k;
    c[k] = 3u;
    r[k] = 0u;
    if (has[k]) {
      c[k] = VPT >= 4 ? (cbase >> (8 * (k >> 2) + 6 - 2 * (k & 3))) & 3u
                      : (cword >> (8u * ((j >> 2) & 3u) + 6u - 2u * (j & 3u))) & 3u;
      r[k] = resid_len(c[k], S);
      sum += r[k];
    }
  }
  uint32_t total, fo, fa;
  uint32_t o = block_scan(sum, 0u, 0u, s, pp, &total, &fo, &fa);
  if (total != bits || cb + resid_bytes(bits) != plen) return false;
  // explicit part of every value (the residual bits placed at [8c, S)) and the run's
  // effect on the leading bytes
  const uint64_t mS = trunc_mask(S);
  const uint32_t mhi = (uint32_t)(mS >> 32), mlo = (uint32_t)mS;
  uint32_t ehi[VPT], elo[VPT];
  uint32_t M = 0u, V = 0u;
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    ehi[k] = elo[k] = 0u;
    if (has[k]) {
      const uint32_t d = 8u * c[k];
      if (W32) {
        const uint32_t q = o >> 5, sh = o & 31u;
        const uint32_t x = __funnelshift_l(m32[(q + 1u) ^ 1u], m32[q ^ 1u], sh);
        ehi[k] = (x >> d) & mhi;
      } else {
        uint32_t hi, lo;
        stream_window(m32, o, hi, lo);
        ehi[k] = (hi >> d) & mhi;
        elo[k] = __funnelshift_r(lo, hi, d) & mlo;
      }
      o += r[k];
      const uint32_t ex = lead_explicit(c[k]);
      V = (V & ~ex) | (ehi[k] & 0xFFFFFF00u);
      M |= ex;
    }
  }
  // leading bytes of the predecessor of value j0, then the copies in order
  uint32_t P = block_lead_scan(M, V, s, pp);
  uint64_t e[VPT];
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    e[k] = 0ull;
    if (has[k]) {
      const uint32_t hi = ehi[k] | (P & lead_copied(c[k]));
      P = hi;
      e[k] = ((uint64_t)hi << 32) | (uint64_t)(W32 ? 0u : elo[k]);
    }
  }
  if (SPLIT) {
#pragma unroll
    for (int k = 0; k < VPT; ++k)
      if (has[k]) tile[tile_val(coded_pos<true>(j0 + k, A))] = e[k];
  } else {
    store_vals<VPT>(tile, j0, nv, e);
  }
  __syncthreads();
  return true;
}

// Decodes the staged image (header + payload in shared memory) into the tile.
// Returns false (tile zero-filled) if the image fails its checks.
template <int VPT>
__device__ bool decode_block(const uint8_t* img, uint32_t img_bytes, int kc, uint64_t* tile, ScanSmem& s, int& pp) {
  // img_bytes <= the caller's staging buffer; images in the pool are at most RAW size,
  // images handed to the codec entry points at most max_coded_bytes(kc)
  const uint32_t N = 2u << kc;
  const uint32_t* h = reinterpret_cast<const uint32_t*>(img);
  const uint32_t mode = h[0] & 0xffu, S = (h[0] >> 8) & 0xffu, lp = (h[0] >> 16) & 0xffu, flags = h[0] >> 24;
  const uint32_t plen = h[1], nv = h[2], bits = h[3];
  const uint8_t* payload = img + 16;
  bool ok = flags == 0 && img_bytes >= 16 && plen + 16u == img_bytes && (plen & 15u) == 0 &&
            img_bytes <= max_coded_bytes(kc) && (mode == M_ZERO || (S >= 13u && S <= 64u));
  if (ok) {
    switch (mode) {
      case M_ZERO: ok = S == 0 && lp == 0 && plen == 0 && nv == 0 && bits == 0; break;
      case M_CONST: ok = lp == 0 && plen == 16 && nv == 2 && bits == 0; break;
      case M_PERIOD: ok = lp >= 1 && (int)lp < kc && nv == (2u << lp); break;
      case M_STREAM: ok = lp == 0 && nv == N; break;
      case M_RAW: ok = lp == 0 && nv == N && bits == 0 && plen == 8u * N; break;
      case M_SPLIT: ok = lp == 0 && nv == N; break;
      case M_PALETTE:  // lp = k, bits = P
        ok = nv == N && bits >= 1u && bits <= kPaletteMax && lp == palette_bits(bits) &&
             plen == round16(8u * bits) + resid_bytes(N * lp);
        break;
      default: ok = false;
    }
  }
  if (ok && mode == M_PALETTE) {
    // the list strictly ascending, every index inside it
    const uint32_t P = bits, k = lp;
    const uint64_t* pal = reinterpret_cast<const uint64_t*>(payload);
    const uint64_t* w = reinterpret_cast<const uint64_t*>(payload + round16(8u * P));
    bool good = true;
    for (uint32_t i = threadIdx.x + 1u; i < P; i += kThreads) good &= pal[i] > pal[i - 1];
    for (uint32_t j = threadIdx.x; j < N; j += kThreads) {
      const uint32_t ix = (uint32_t)get_bits(w, j * k, k);
      good &= ix < P;
      tile[tile_val(j)] = ix < P ? pal[ix] : 0ull;
    }
    if (__syncthreads_and(good)) return true;
    ok = false;
  }
  if (ok && mode == M_SPLIT) {
    if (S <= 32u ? decode_xor_block<VPT, true, true, true>(payload, plen, nv, S, bits, tile, s, pp)
                 : decode_xor_block<VPT, true, false, true>(payload, plen, nv, S, bits, tile, s, pp))
      return true;
    ok = false;
  }
  if (ok && (mode == M_PERIOD || mode == M_STREAM)) {
    if (mode == M_STREAM)
      ok = S <= 32u ? decode_xor_block<VPT, false, true, true>(payload, plen, nv, S, bits, tile, s, pp)
                    : decode_xor_block<VPT, false, false, true>(payload, plen, nv, S, bits, tile, s, pp);
    else
      ok = S <= 32u ? decode_xor_block<VPT, false, true, false>(payload, plen, nv, S, bits, tile, s, pp)
                    : decode_xor_block<VPT, false, false, false>(payload, plen, nv, S, bits, tile, s, pp);
    if (ok && mode == M_PERIOD) {
      ulonglong2* t2 = reinterpret_cast<ulonglong2*>(tile);
      const uint32_t P = nv >> 1;  // period in amplitudes
      for (uint32_t a = P + threadIdx.x; a < (N >> 1); a += kThreads) t2[tile_amp(a)] = t2[tile_amp(a & (P - 1u))];
      __syncthreads();
    }
    if (ok) return true;
  }
  const uint64_t* pw = reinterpret_cast<const uint64_t*>(payload);
  ulonglong2* t2 = reinterpret_cast<ulonglong2*>(tile);
  for (uint32_t a = threadIdx.x; a < (N >> 1); a += kThreads) {
    ulonglong2 q = make_ulonglong2(0ull, 0ull);
    if (ok && mode == M_CONST) q = make_ulonglong2(pw[0], pw[1]);
    else if (ok && mode == M_RAW) q = make_ulonglong2(pw[2 * a], pw[2 * a + 1]);
    t2[tile_amp(a)] = q;
  }
  __syncthreads();
  return ok;
}

// True if a staged image is a STREAM image of width S <= 32 that passes decode_block's
// header checks: the case decode_stream32_pair takes.
__device__ __forceinline__ bool stream32_image(const uint8_t* img, uint32_t img_bytes, int kc) {
  const uint32_t* h = reinterpret_cast<const uint32_t*>(img);
  const uint32_t mode = h[0] & 0xffu, S = (h[0] >> 8) & 0xffu, lp = (h[0] >> 16) & 0xffu, flags = h[0] >> 24;
  return mode == M_STREAM && flags == 0 && lp == 0 && S >= 13u && S <= 32u && img_bytes >= 16u &&
         h[1] + 16u == img_bytes && (h[1] & 15u) == 0 && img_bytes <= max_coded_bytes(kc) && h[2] == (2u << kc);
}

// The 2-bit code of value j0 + k from the 32-bit code word holding values j0 .. j0 + VPT - 1.
template <int VPT>
__device__ __forceinline__ uint32_t code_in_word(uint32_t cword, uint32_t j0, int k) {
  if (VPT >= 4) return (cword >> (8u * ((j0 >> 2) & 3u) + 8 * (k >> 2) + 6 - 2 * (k & 3))) & 3u;
  const uint32_t j = j0 + (uint32_t)k;
  return (cword >> (8u * ((j >> 2) & 3u) + 6u - 2u * (j & 3u))) & 3u;
}

// Decodes the two STREAM images of a work item (both stream32_image) into their tiles
// in one pass: decode_xor_block's steps for each chunk, the two chunks sharing every
// barrier.  Every thread holds VPT values of each chunk (kThreads * VPT = 2^(kc+1)).
// Returns false if either image's residual lengths disagree with its header.
template <int VPT>
__device__ bool decode_stream32_pair(const uint8_t* img0, const uint8_t* img1, uint32_t N, uint64_t* tile0,
                                     uint64_t* tile1, ScanSmem& s, int& pp) {
  const uint32_t* hd0 = reinterpret_cast<const uint32_t*>(img0);
  const uint32_t* hd1 = reinterpret_cast<const uint32_t*>(img1);
  const uint32_t S0 = (hd0[0] >> 8) & 0xffu, S1 = (hd1[0] >> 8) & 0xffu;
  const uint32_t cb = code_bytes(N);
  const uint32_t j0 = threadIdx.x * VPT;
  const uint32_t cw0 = reinterpret_cast<const uint32_t*>(img0 + 16)[j0 >> 4];
  const uint32_t cw1 = reinterpret_cast<const uint32_t*>(img1 + 16)[j0 >> 4];
  uint32_t sum0 = 0u, sum1 = 0u;
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    sum0 += resid_len(code_in_word<VPT>(cw0, j0, k), S0);
    sum1 += resid_len(code_in_word<VPT>(cw1, j0, k), S1);
  }
  uint32_t o0, o1, total0, total1, fo, fa;
  block_scan2(sum0, sum1, 0u, 0u, s, pp, &o0, &o1, &total0, &total1, &fo, &fa);
  if (total0 != hd0[3] || total1 != hd1[3] || cb + resid_bytes(total0) != hd0[1] || cb + resid_bytes(total1) != hd1[1])
    return false;
  // explicit parts (the residual placed at [8c, S) of the high word) and each run's
  // effect on the leading bytes
  const uint32_t* m0 = reinterpret_cast<const uint32_t*>(img0 + 16 + cb);
  const uint32_t* m1 = reinterpret_cast<const uint32_t*>(img1 + 16 + cb);
  const uint32_t mh0 = (uint32_t)(trunc_mask(S0) >> 32), mh1 = (uint32_t)(trunc_mask(S1) >> 32);
  uint32_t e0[VPT], e1[VPT];
  uint32_t M0 = 0u, V0 = 0u, M1 = 0u, V1 = 0u;
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    {
      const uint32_t c = code_in_word<VPT>(cw0, j0, k), q = o0 >> 5, sh = o0 & 31u;
      e0[k] = (__funnelshift_l(m0[(q + 1u) ^ 1u], m0[q ^ 1u], sh) >> (8u * c)) & mh0;
      o0 += resid_len(c, S0);
      const uint32_t ex = lead_explicit(c);
      V0 = (V0 & ~ex) | (e0[k] & 0xFFFFFF00u);
      M0 |= ex;
    }
    {
      const uint32_t c = code_in_word<VPT>(cw1, j0, k), q = o1 >> 5, sh = o1 & 31u;
      e1[k] = (__funnelshift_l(m1[(q + 1u) ^ 1u], m1[q ^ 1u], sh) >> (8u * c)) & mh1;
      o1 += resid_len(c, S1);
      const uint32_t ex = lead_explicit(c);
      V1 = (V1 & ~ex) | (e1[k] & 0xFFFFFF00u);
      M1 |= ex;
    }
  }
  uint32_t P0, P1;
  block_lead_scan2(M0, V0, M1, V1, s, pp, P0, P1);
  uint64_t v[VPT];
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    P0 = e0[k] | (P0 & lead_copied(code_in_word<VPT>(cw0, j0, k)));
    v[k] = (uint64_t)P0 << 32;
  }
  store_vals<VPT>(tile0, j0, N, v);
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    P1 = e1[k] | (P1 & lead_copied(code_in_word<VPT>(cw1, j0, k)));
    v[k] = (uint64_t)P1 << 32;
  }
  store_vals<VPT>(tile1, j0, N, v);
  __syncthreads();
  return true;
}

// ------------------------------------------------------- learned selector -- //
// Not from the paper.  For every chunk a gate is about to rewrite, a 16 -> 32 -> 32 -> 8
// network with bfloat16 weights predicts the best chunk mode (outputs 0..6: logits of
// ZERO, CONST, PERIOD, STREAM, RAW, SPLIT, PALETTE) and a bit budget (output 7: the best
// image's size over the RAW size) from the chunk's current image header and the gate
// alone.  Needing no decoded value, the decisions of a whole gate come from one small
// kernel that runs before the gate.  The SPLIT (Solution D) and PALETTE trials run
// only for chunks whose decision grants them; the cheap modes are always computed, and
// the codec keeps the error bound whatever the network says.
//
// Inference is float32 with a fixed order: each unit sums its products over its
// inputs in index order, one rounding per product and per sum (no fused
// multiply-add), then adds its bias; ReLU maps non-positive sums to +0.  A trial runs
// iff its mode's logit plus 2 reaches the largest of the seven logits; both run when
// the budget is below half the chunk's current size fraction (input 7), a predicted
// collapse of the image that the logits may miss.  Both rules lean towards a trial: a
// missed one costs memory, a needless one only time.
constexpr int kMlpParams = 1864;  // W1[32][16] b1[32] W2[32][32] b2[32] W3[8][32] b3[8]
constexpr int kTraceFloats = 20;  // features[16], best mode, best size / RAW size, 0, 0
constexpr uint32_t kSelSplit = 1u, kSelPalette = 2u;  // decision bits

// Gate features of the selector (bits): 0 the matrix is real, 1 diagonal, 2
// anti-diagonal, 3 the target lies inside the chunk.
struct SelCtx {
  uint32_t gfeat;
  uint32_t S_gate;                 // significant bits the controller chose for this gate
  uint32_t prev_hdr[4];            // header of the chunk's current (pre-gate) image
  uint32_t prev_len;               // and its length
  float* trace;                    // training records (device) or nullptr
  unsigned long long* trace_n;
  unsigned long long trace_cap;
  unsigned long long* split_trials;    // counts chunk encodes that ran the SPLIT trial
  unsigned long long* palette_trials;  // ... and the PALETTE trial
};

// The chunk modes a decision grants: Solution C's set plus the trials.
__host__ __device__ __forceinline__ uint32_t sel_modes(uint32_t dec) {
  return kDefaultModes | ((dec & kSelSplit) ? (1u << M_SPLIT) : 0u) | ((dec & kSelPalette) ? (1u << M_PALETTE) : 0u);
}

// Input i of the network for a chunk whose current image has header hdr and length
// len (kc = chunk_log2): one-hot of the image mode (0..6), its size over the RAW size
// (7), its S / 64 (8), header word 3 / (64 N) (9: residual bits, or the palette size),
// header byte 2 / 16 (10: log2 period, or the palette index width), the gate features
// (11..14), the gate's S / 64 (15).
__device__ __forceinline__ float sel_feature(const uint32_t hdr[4], uint32_t len, int kc, uint32_t gfeat,
                                             uint32_t S_gate, int i) {
  const uint32_t mode = hdr[0] & 0xffu, S = (hdr[0] >> 8) & 0xffu, b2 = (hdr[0] >> 16) & 0xffu;
  if (i < 7) return mode == (uint32_t)i ? 1.0f : 0.0f;
  if (i == 7) return __fdiv_rn(__uint2float_rn(len), __uint2float_rn(16u + (16u << kc)));
  if (i == 8) return __fdiv_rn(__uint2float_rn(S), 64.0f);
  if (i == 9) return __fdiv_rn(__uint2float_rn(hdr[3]), __uint2float_rn(64u * (2u << kc)));
  if (i == 10) return __fdiv_rn(__uint2float_rn(b2), 16.0f);
  if (i < 15) return ((gfeat >> (i - 11)) & 1u) ? 1.0f : 0.0f;
  return __fdiv_rn(__uint2float_rn(S_gate), 64.0f);
}

// One unit: the float32 sum over NIN inputs in input order, then the bias.
template <int NIN>
__device__ __forceinline__ float sel_unit(const float* w, const float* in, float bias) {
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < NIN; ++i) acc = __fadd_rn(acc, __fmul_rn(w[i], in[i]));
  return __fadd_rn(acc, bias);
}

// The decision bits for one chunk (one thread; w: the parameters as float32, in
// shared memory; x: the 16 inputs).
__device__ __forceinline__ uint32_t sel_decide(const float* w, const float x[16]) {
  float h1[32], h2[32], o[8];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float z = sel_unit<16>(w + 16 * j, x, w[512 + j]);
    h1[j] = z > 0.0f ? z : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float z = sel_unit<32>(w + 544 + 32 * j, h1, w[1568 + j]);
    h2[j] = z > 0.0f ? z : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) o[j] = sel_unit<32>(w + 1600 + 32 * j, h2, w[1856 + j]);
  float mx = o[0];
#pragma unroll
  for (int m = 1; m < 7; ++m)
    if (o[m] > mx) mx = o[m];
  const bool shrink = o[7] < __fmul_rn(x[7], 0.5f);
  uint32_t d = 0;
  if (__fadd_rn(o[5], 2.0f) >= mx || shrink) d |= kSelSplit;
  if (__fadd_rn(o[6], 2.0f) >= mx || shrink) d |= kSelPalette;
  return d;
}

// ----------------------------------------------------------- encoder ----- //
// The 2-bit codes of values [j0, j0 + VPT) placed in their 32-bit code word (four
// codes per byte, the first in the top bits); values >= nv get no code.
template <int VPT>
__device__ __forceinline__ uint32_t code_word(const uint32_t c[VPT], uint32_t j0, uint32_t nv) {
  uint32_t cw = 0;
  if constexpr (VPT >= 4) {  // j0 is a multiple of 4: the layout within the thread's bytes is fixed
#pragma unroll
    for (int k = 0; k < VPT; ++k)
      if (j0 + k < nv) cw |= c[k] << (8 * (k >> 2) + 6 - 2 * (k & 3));
    return cw << (8u * ((j0 >> 2) & 3u));
  } else {
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const uint32_t j = j0 + k;
      if (j < nv) cw |= c[k] << (8u * ((j >> 2) & 3u) + 6u - 2u * (j & 3u));
    }
    return cw;
  }
}

// Writes the 2-bit codes and the residual stream of coded values [j0, j0 + VPT) of this
// thread (values >= nv are not coded) into an image whose payload was cleared; o0 is
// the stream offset of value j0.
template <int VPT>
__device__ __forceinline__ void pack_xor(uint8_t* img, uint32_t nv, uint32_t j0, uint32_t o0, const uint64_t t[VPT],
                                         const uint32_t c[VPT], const uint32_t r[VPT]) {
  // codes: one 32-bit word per 16 values
  uint32_t* codes32 = reinterpret_cast<uint32_t*>(img + 16);
  const uint32_t cw = code_word<VPT>(c, j0, nv);
  uint32_t oend = o0;
#pragma unroll
  for (int k = 0; k < VPT; ++k)
    if (j0 + k < nv) oend += r[k];
  if (j0 < nv && cw) atomicOr(&codes32[j0 >> 4], cw);
  // residual bits: this thread owns stream bits [o0, oend); interior 32-bit units are
  // written once with plain stores, the two end units (shared with the neighbours)
  // with atomicOr into the cleared payload
  if (oend > o0) {
    uint32_t* m32 = reinterpret_cast<uint32_t*>(img + 16 + code_bytes(nv));
    const uint32_t qf = o0 >> 5, ql = (oend - 1u) >> 5;
    uint32_t qb = qf, w0 = 0, w1 = 0, w2 = 0, o = o0;
#define QC_FLUSH(q, v)                                        \
do {                                                        \
  if ((q) <= ql && (v) != 0u) {                             \
    if ((q) == qf || (q) == ql) atomicOr(&m32[(q) ^ 1u], (v)); \
    else m32[(q) ^ 1u] = (v);                               \
  }                                                         \
} while (0)
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      if (j0 + k < nv && r[k]) {
        const uint32_t q = o >> 5, sh = o & 31u;
        while (qb < q) {
          QC_FLUSH(qb, w0);
          w0 = w1;
          w1 = w2;
          w2 = 0;
          ++qb;
        }
        const uint32_t d = 8u * c[k];
        const uint32_t thi = (uint32_t)(t[k] >> 32), tlo = (uint32_t)t[k];
        const uint32_t xhi = __funnelshift_l(tlo, thi, d), xlo = tlo << d;
        w0 |= xhi >> sh;
        w1 |= __funnelshift_r(xlo, xhi, sh);
        w2 |= __funnelshift_r(0u, xlo, sh);
        o += r[k];
      }
    }
    QC_FLUSH(qb, w0);
    QC_FLUSH(qb + 1u, w1);
    QC_FLUSH(qb + 2u, w2);
#undef QC_FLUSH
  }
}


// pack_xor for S <= 32: every residual is at most 32 bits of the value's high word h.
// The thread fills 32-bit stream units in order in a register; a completed unit is
// stored (the first one with atomicOr: the previous thread may own its leading bits),
// the unfinished last one is ORed in (the next thread owns its trailing bits).
template <int VPT>
__device__ __forceinline__ void pack_xor32(uint8_t* img, uint32_t nv, uint32_t j0, uint32_t o0, const uint32_t h[VPT],
                                           const uint32_t c[VPT], const uint32_t r[VPT]) {
  uint32_t* codes32 = reinterpret_cast<uint32_t*>(img + 16);
  const uint32_t cw = code_word<VPT>(c, j0, nv);
  if (j0 < nv && cw) atomicOr(&codes32[j0 >> 4], cw);
  uint32_t* m32 = reinterpret_cast<uint32_t*>(img + 16 + code_bytes(nv));
  uint32_t q = o0 >> 5, fill = o0 & 31u, cur = 0u;
  bool first = true;
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    if (j0 + k < nv) {
      const uint32_t f = h[k] << (8u * c[k]);  // the residual in the top r bits, zeros below
      cur |= f >> fill;
      const uint32_t nf = fill + r[k];
      if (nf >= 32u) {
        if (first) atomicOr(&m32[q ^ 1u], cur);
        else m32[q ^ 1u] = cur;
        first = false;
        ++q;
        cur = __funnelshift_r(0u, f, fill);  // the residual's bits past the unit
        fill = nf - 32u;
      } else {
        fill = nf;
      }
    }
  }
  if (fill > 0u && cur) atomicOr(&m32[q ^ 1u], cur);
}

// PALETTE trial over a tile of N values (already truncated), using the payload area
// `area` (at least 8 N bytes, nothing in it live) as scratch: the values are copied
// there and sorted ascending (bitonic network), the distinct ones compacted to the
// front.  Returns their number P if P <= kPaletteMax (the list stays at area[0, 8P)),
// else 0.  All threads; barriers.
template <int VPT>
__device__ __forceinline__ uint32_t palette_block(const uint64_t* tile, uint32_t N, uint8_t* area, ScanSmem& s,
                                                  int& pp) {
  uint64_t* a = reinterpret_cast<uint64_t*>(area);
  for (uint32_t j = threadIdx.x; j < N; j += kThreads) a[j] = tile[tile_val(j)];
  __syncthreads();
  for (uint32_t k = 2; k <= N; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < N; i += kThreads) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const uint64_t x = a[i], y = a[l];
          if ((x > y) == ((i & k) == 0u)) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  // distinct values: first of each run of equal ones; rank by a block scan
  // thread t holds values [t VPT, t VPT + VPT) of the sorted list (VPT = N / kThreads,
  // or 1 with fewer values than threads)
  uint64_t v[VPT];
  uint32_t first = 0u, cnt = 0u;
  const uint32_t j0 = threadIdx.x * VPT;
#pragma unroll
  for (uint32_t q = 0; q < VPT; ++q) {
    v[q] = 0ull;
    if (j0 + q < N) {
      v[q] = a[j0 + q];
      if (j0 + q == 0u || v[q] != a[j0 + q - 1u]) {
        first |= 1u << q;
        ++cnt;
      }
    }
  }
  uint32_t total, fo, fa;
  uint32_t r = block_scan(cnt, 0u, 0u, s, pp, &total, &fo, &fa);
  if (total > kPaletteMax) {
    __syncthreads();
    return 0u;
  }
#pragma unroll
  for (uint32_t q = 0; q < VPT; ++q)
    if ((first >> q) & 1u) a[r++] = v[q];
  __syncthreads();
  return total;
}

// Writes the k-bit indices of a tile's N values into a PALETTE payload whose list of P
// values is at pay[0, 8P) (the index stream follows at round16(8 P), MSB first in 64-bit
// little-endian words, cleared here first).  All threads; one barrier.
template <int VPT>
__device__ __forceinline__ void palette_pack(const uint64_t* tile, uint32_t N, uint8_t* pay, uint32_t P) {
  const uint64_t* pal = reinterpret_cast<const uint64_t*>(pay);
  const uint32_t k = palette_bits(P);
  uint32_t* m32 = reinterpret_cast<uint32_t*>(pay + round16(8u * P));
  const uint32_t words = resid_bytes(N * k) / 4u;
  for (uint32_t u = threadIdx.x; u < words; u += kThreads) m32[u] = 0u;
  if (threadIdx.x == 0 && (P & 1u)) reinterpret_cast<uint64_t*>(pay)[P] = 0ull;  // the list's padding
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < N; j += kThreads) {
    const uint64_t x = tile[tile_val(j)];
    uint32_t lo = 0, hi = P - 1u;  // the value is in the list
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (pal[mid] < x) lo = mid + 1u;
      else hi = mid;
    }
    // k bits at stream position j k: one or two 32-bit units (unit q is word q ^ 1)
    const uint32_t pos = j * k, q = pos >> 5, off = pos & 31u;
    const uint32_t f = lo << (32u - k);  // the index in the top k bits
    atomicOr(&m32[q ^ 1u], f >> off);
    if (off + k > 32u) atomicOr(&m32[(q + 1u) ^ 1u], f << (32u - off));
  }
  __syncthreads();
}

// Leading identical bytes of two high words (values whose low words are zero), capped at 3.
__device__ __forceinline__ uint32_t xor_code32(uint32_t v, uint32_t prev) {
  return min((uint32_t)__clz((int)(v ^ prev)) >> 3, 3u);
}

// Steps 2-6 of encode_block once the chunk's width S is known.  W32 (S <= 32): the
// truncated values' low words are zero, so codes, the Solution D trial and packing
// work on high words only.
template <int VPT, bool W32>
__device__ __forceinline__ uint32_t encode_core(uint64_t* tile, int kc, uint32_t S, int force_mode, uint32_t modes,
                                                uint8_t* img, uint32_t img_cap, ScanSmem& s, int& pp,
                                                unsigned int* err, const SelCtx* sel, uint64_t t[VPT]) {
  const uint32_t N = 2u << kc, A = 1u << kc;
  const uint32_t j0 = threadIdx.x * VPT;
  const bool act = VPT >= 2 || j0 < N;  // every value of a run with VPT >= 2 exists
  const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(tile);
  const uint64_t mask = trunc_mask(S);
  // 2. truncate (and store -0 as +0)
  bool nz = false;
  uint32_t h[VPT];  // W32: high words of the truncated values
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    if constexpr (W32) {
      uint32_t v = (uint32_t)(t[k] >> 32) & (uint32_t)(mask >> 32);
      if (v == 0x80000000u || !act) v = 0u;
      h[k] = v;
      t[k] = (uint64_t)v << 32;
      nz |= v != 0u;
    } else {
      uint64_t v = t[k] & mask;
      if (v == 0x8000000000000000ull) v = 0;
      t[k] = act ? v : 0ull;
      nz |= t[k] != 0ull;
    }
  }
  store_vals<VPT>(tile, j0, N, t);
  __syncthreads();
  // 3. codes and residual lengths (predecessor of value 0 is 0); CONST and top-level
  //    PERIOD tests on this thread's values
  uint32_t c[VPT], r[VPT], sum = 0;
  uint64_t prev = (j0 > 0 && j0 <= N) ? tile[tile_val(j0 - 1)] : 0ull;
  const uint64_t a0x = tile[tile_val(0)], a0y = tile[tile_val(1)];
  const uint32_t Ptop = kc >= 2 ? (1u << (kc - 1)) : 0u;
  bool cst = true, gtop = true;
  if constexpr (W32) {
    uint32_t ph = (uint32_t)(prev >> 32);
    const uint32_t a0xh = (uint32_t)(a0x >> 32), a0yh = (uint32_t)(a0y >> 32);
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      c[k] = 3u;
      r[k] = 0u;
      if (act) {
        c[k] = xor_code32(h[k], ph);
        r[k] = resid_len(c[k], S);
        sum += r[k];
        ph = h[k];
        cst &= h[k] == (((j0 + k) & 1u) ? a0yh : a0xh);
      }
    }
    if (act && ((j0 >> 1) & Ptop))
      gtop = h[0] == reinterpret_cast<const uint32_t*>(tile)[2u * tile_val(j0 ^ (2u * Ptop)) + 1u];
  } else {
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      c[k] = 3u;
      r[k] = 0u;
      if (act) {
        c[k] = xor_code(t[k], prev);
        r[k] = resid_len(c[k], S);
        sum += r[k];
        prev = t[k];
        cst &= t[k] == (((j0 + k) & 1u) ? a0y : a0x);
      }
    }
    if (act && ((j0 >> 1) & Ptop)) gtop = t[0] == tile[tile_val(j0 ^ (2u * Ptop))];
  }
  // Solution D order (SPLIT): only its residual length is needed unless it wins
  const bool want_split = force_mode == (int)M_SPLIT || (force_mode < 0 && ((modes >> M_SPLIT) & 1u));
  uint32_t sum2 = 0;
  if (want_split) {
    uint64_t pv = j0 > 0 && j0 <= N ? tile[tile_val(coded_pos<true>(j0 - 1, A))] : 0ull;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      if (act) {
        const uint64_t v = tile[tile_val(coded_pos<true>(j0 + k, A))];
        if constexpr (W32) sum2 += resid_len(xor_code32((uint32_t)(v >> 32), (uint32_t)(pv >> 32)), S);
        else sum2 += resid_len(xor_code(v, pv), S);
        pv = v;
      }
    }
  }
  uint32_t total, f_or, f_and, o0, o2 = 0, total2 = 0;
  if (want_split)
    block_scan2(sum, sum2, nz ? 1u : 0u, (cst ? 1u : 0u) | (gtop ? 2u : 0u), s, pp, &o0, &o2, &total, &total2, &f_or,
                &f_and);
  else
    o0 = block_scan(sum, nz ? 1u : 0u, (cst ? 1u : 0u) | (gtop ? 2u : 0u), s, pp, &total, &f_or, &f_and);
  const bool allzero = (f_or & 1u) == 0u;
  const bool allconst = (f_and & 1u) != 0u;
  // PALETTE trial: the chunk's values sorted in the (still unused) payload area, the
  // distinct ones kept in place ascending; the area is cleared again for the packers
  uint32_t npal = 0;
  const bool want_pal = force_mode == (int)M_PALETTE || (force_mode < 0 && ((modes >> M_PALETTE) & 1u));
  if (want_pal) npal = palette_block<VPT>(tile, N, img + 16, s, pp);
  // 4. smallest power-of-two period P (amplitudes), 2 <= P < 2^kc: the chunk is
  //    P-periodic iff flipping any amplitude-index bit >= log2 P leaves it unchanged.
  //    The scan's flag compared one value per thread with its partner half a chunk
  //    away (a necessary condition); the loop checks every candidate in full.
  int period = -1;
  if (kc >= 2 && (f_and & 2u) && (!allconst || force_mode == (int)M_PERIOD)) {
    int p = kc - 1;
    for (; p >= 1; --p) {
      const uint32_t P = 1u << p;
      bool ok = true;
      for (uint32_t i = threadIdx.x; i < A; i += kThreads) {
        if (i & P) {
          const ulonglong2 q = t2[tile_amp(i)], w = t2[tile_amp(i ^ P)];
          ok &= (q.x == w.x) && (q.y == w.y);
        }
      }
      if (!__syncthreads_and(ok)) break;
    }
    period = p + 1 < kc ? p + 1 : -1;
  }
  // residual bits of the first 2P values (rare: only periodic chunks)
  uint32_t bits_p = 0;
  if (period > 0) {
    if (threadIdx.x == 0) s.bits_period = 0;
    __syncthreads();
    const uint32_t nvp = 2u << period;
    uint32_t o = o0;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      if (j0 + k == nvp) s.bits_period = o;
      o += r[k];
    }
    __syncthreads();
    bits_p = s.bits_period;
    __syncthreads();
  }
  // 5. sizes and the choice (every thread computes the same)
  uint32_t size[M_NMODES];
  size[M_ZERO] = allzero ? 16u : 0u;
  size[M_CONST] = allconst ? 32u : 0u;
  size[M_PERIOD] = period > 0 ? 16u + code_bytes(2u << period) + resid_bytes(bits_p) : 0u;
  size[M_STREAM] = 16u + code_bytes(N) + resid_bytes(total);
  size[M_RAW] = 16u + 8u * N;
  size[M_SPLIT] = want_split ? 16u + code_bytes(N) + resid_bytes(total2) : 0u;
  size[M_PALETTE] = npal ? 16u + round16(8u * npal) + resid_bytes(N * palette_bits(npal)) : 0u;
  uint32_t mode = 0, best = 0;
  if (force_mode >= 0) {
    if (force_mode >= (int)M_NMODES || size[force_mode] == 0 || size[force_mode] > img_cap) {
      if (threadIdx.x == 0) atomicOr(err, (unsigned)E_MODE);
      return 0;
    }
    mode = (uint32_t)force_mode;
    best = size[mode];
  } else {
    best = 0xffffffffu;
#pragma unroll
    for (uint32_t m = 0; m < M_NMODES; ++m)
      if (((modes >> m) & 1u) && size[m] != 0 && size[m] < best) { best = size[m]; mode = m; }
    if (best > img_cap) {  // cannot happen: RAW always fits a buffer of max_image_bytes
      if (threadIdx.x == 0) atomicOr(err, (unsigned)E_MODE);
      return 0;
    }
  }
  // 6. write the image
  uint32_t nv = 0, rbits = 0;
  if (mode == M_CONST) nv = 2;
  if (mode == M_PERIOD) { nv = 2u << period; rbits = bits_p; }
  if (mode == M_STREAM) { nv = N; rbits = total; }
  if (mode == M_RAW) nv = N;
  if (mode == M_SPLIT) { nv = N; rbits = total2; }
  if (mode == M_PALETTE) { nv = N; rbits = npal; }
  if (sel && threadIdx.x == 0 && force_mode < 0) {
    if (want_split && sel->split_trials) atomicAdd(sel->split_trials, 1ull);
    if (want_pal && sel->palette_trials) atomicAdd(sel->palette_trials, 1ull);
  }
  // training record: the chunk's pre-gate inputs, the mode the mode set chose and its
  // size over the RAW size
  if (sel && sel->trace && threadIdx.x == 0 && force_mode < 0) {
    const unsigned long long k = atomicAdd(sel->trace_n, 1ull);
    if (k < sel->trace_cap) {
      float* rec = sel->trace + k * kTraceFloats;
      for (int i = 0; i < 16; ++i) rec[i] = sel_feature(sel->prev_hdr, sel->prev_len, kc, sel->gfeat, sel->S_gate, i);
      rec[16] = (float)mode;
      rec[17] = __fdiv_rn(__uint2float_rn(best), __uint2float_rn(16u + 8u * N));
      rec[18] = 0.0f;
      rec[19] = 0.0f;
    }
  }
  if (threadIdx.x == 0) {
    uint32_t* h = reinterpret_cast<uint32_t*>(img);
    const uint32_t b2 = mode == M_PERIOD ? (uint32_t)period : (mode == M_PALETTE ? palette_bits(npal) : 0u);
    h[0] = mode | ((mode == M_ZERO ? 0u : S) << 8) | (b2 << 16);
    h[1] = best - 16u;
    h[2] = nv;
    h[3] = rbits;
  }
  uint64_t* pay64 = reinterpret_cast<uint64_t*>(img + 16);
  if (mode == M_PALETTE) {
    // the list is in place; each value's index by binary search, packed k bits each
    palette_pack<VPT>(tile, N, img + 16, npal);
  } else if (want_pal) {
    // another mode won: the sort scratch goes, the packers need a cleared payload
    const uint32_t span = min(img_cap, max_coded_bytes(kc)) - 16u;
    uint4* z = reinterpret_cast<uint4*>(img + 16);
    for (uint32_t u = threadIdx.x; u < span / 16u; u += kThreads) z[u] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
  }
  if (mode == M_PALETTE) {
    // written above
  } else if (mode == M_CONST) {
    if (threadIdx.x == 0) {
      pay64[0] = a0x;
      pay64[1] = a0y;
    }
  } else if (mode == M_RAW) {
    ulonglong2* p2 = reinterpret_cast<ulonglong2*>(pay64);
    for (uint32_t a = threadIdx.x; a < A; a += kThreads) p2[a] = t2[tile_amp(a)];
  } else if (mode == M_SPLIT) {
    // recompute the Solution D codes (the scan kept only their total)
    uint64_t pv = j0 > 0 && j0 <= N ? tile[tile_val(coded_pos<true>(j0 - 1, A))] : 0ull;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      if (act) {
        t[k] = tile[tile_val(coded_pos<true>(j0 + k, A))];
        if constexpr (W32) {
          h[k] = (uint32_t)(t[k] >> 32);
          c[k] = xor_code32(h[k], (uint32_t)(pv >> 32));
        } else {
          c[k] = xor_code(t[k], pv);
        }
        r[k] = resid_len(c[k], S);
        pv = t[k];
      } else {
        t[k] = 0ull;
        h[k] = 0u;
        c[k] = 3u;
        r[k] = 0u;
      }
    }
    if constexpr (W32) pack_xor32<VPT>(img, nv, j0, o2, h, c, r);
    else pack_xor<VPT>(img, nv, j0, o2, t, c, r);
  } else if (mode == M_PERIOD || mode == M_STREAM) {
    if constexpr (W32) pack_xor32<VPT>(img, nv, j0, o0, h, c, r);
    else pack_xor<VPT>(img, nv, j0, o0, t, c, r);
  }
  __syncthreads();
  return best;
}

// Encodes the tile (raw bit patterns; overwritten with the truncated values) into
// img (img_cap bytes, nothing else in it is live).  S_req = 12 - EXP(eps) or 64.
// force_mode < 0: smallest image (never larger than RAW).  Returns the image length,
// or 0 with *err set (non-finite value, or a forced mode that does not apply or does
// not fit in img_cap).
template <int VPT>
__device__ uint32_t encode_block(uint64_t* tile, int kc, uint32_t S_req, int force_mode, uint32_t modes, uint8_t* img,
                                 uint32_t img_cap, ScanSmem& s, int& pp, unsigned int* err,
                                 const SelCtx* sel = nullptr) {
  const uint32_t N = 2u << kc;
  const uint32_t j0 = threadIdx.x * VPT;
  // 0. clear the payload area the packers OR into (the buffer is free here)
  {
    const uint32_t span = min(img_cap, max_coded_bytes(kc)) - 16u;
    uint4* z = reinterpret_cast<uint4*>(img + 16);
    for (uint32_t u = threadIdx.x; u < span / 16u; u += kThreads) z[u] = make_uint4(0u, 0u, 0u, 0u);
  }
  // 1. chunk-wide width: a nonzero subnormal forces 64 bits; non-finite is an error
  //    (with VPT >= 2 every thread's run of values lies inside the chunk)
  const bool act = VPT >= 2 || j0 < N;
  uint64_t t[VPT];
  load_vals<VPT>(tile, j0, N, t);
  bool sub = false, nonfin = false;
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    if (act) {
      const uint32_t hi = (uint32_t)(t[k] >> 32) & 0x7fffffffu;
      nonfin |= hi >= 0x7ff00000u;
      sub |= hi < 0x00100000u && (hi | (uint32_t)t[k]) != 0u;
    }
  }
  bool anysub = false;
  if (__syncthreads_or(nonfin || sub)) {  // rare: settle which of the two it was
    if (__syncthreads_or(nonfin)) {
      if (threadIdx.x == 0) atomicOr(err, (unsigned)E_NONFINITE);
      return 0;
    }
    anysub = true;
  }
  const uint32_t S = anysub ? 64u : S_req;
  if (S <= 32u) return encode_core<VPT, true>(tile, kc, S, force_mode, modes, img, img_cap, s, pp, err, sel, t);
  return encode_core<VPT, false>(tile, kc, S, force_mode, modes, img, img_cap, s, pp, err, sel, t);
}

// Step 3 of encode_core (W32) for one chunk of a pair: the codes of this thread's
// values packed two bits each (value k at bits 2k), their residual bits, and the CONST
// and top-level PERIOD tests.  All values of the thread exist (kThreads * VPT = N).
template <int VPT>
__device__ __forceinline__ void codes32_pair_part(const uint64_t* tile, uint32_t j0, const uint32_t h[VPT], uint32_t S,
                                                  uint32_t Ptop, uint32_t& cc, uint32_t& sum, bool& cst, bool& gtop) {
  const uint32_t* t32 = reinterpret_cast<const uint32_t*>(tile);
  uint32_t ph = j0 > 0 ? t32[2u * tile_val(j0 - 1u) + 1u] : 0u;
  const uint32_t a0xh = t32[2u * tile_val(0) + 1u], a0yh = t32[2u * tile_val(1) + 1u];
  cc = 0u;
  sum = 0u;
  cst = true;
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const uint32_t c = xor_code32(h[k], ph);
    cc |= c << (2 * k);
    sum += resid_len(c, S);
    ph = h[k];
    cst &= h[k] == (((j0 + k) & 1u) ? a0yh : a0xh);
  }
  gtop = true;
  if ((j0 >> 1) & Ptop) gtop = h[0] == t32[2u * tile_val(j0 ^ (2u * Ptop)) + 1u];
}

// Steps 4-6 of encode_core (W32, smallest image, no Solution D trial) for one chunk of
// a pair, once the shared scan has given its stream offset o0, its residual total and
// its chunk-wide flags.  Returns the image length, or 0 with *err set.
template <int VPT>
__device__ __forceinline__ uint32_t finish32_pair_part(const uint64_t* tile, int kc, uint32_t S, uint32_t modes,
                                                       uint8_t* img, uint32_t img_cap, ScanSmem& s, unsigned int* err,
                                                       const uint32_t h[VPT], uint32_t cc, uint32_t o0, uint32_t total,
                                                       bool allzero, bool allconst, bool gtop) {
  const uint32_t N = 2u << kc, A = 1u << kc;
  const uint32_t j0 = threadIdx.x * VPT;
  const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(tile);
  // 4. smallest power-of-two period (as in encode_core)
  int period = -1;
  if (kc >= 2 && gtop && !allconst) {
    int p = kc - 1;
    for (; p >= 1; --p) {
      const uint32_t P = 1u << p;
      bool ok = true;
      for (uint32_t i = threadIdx.x; i < A; i += kThreads) {
        if (i & P) {
          const ulonglong2 q = t2[tile_amp(i)], w = t2[tile_amp(i ^ P)];
          ok &= (q.x == w.x) && (q.y == w.y);
        }
      }
      if (!__syncthreads_and(ok)) break;
    }
    period = p + 1 < kc ? p + 1 : -1;
  }
  uint32_t bits_p = 0;
  if (period > 0) {
    if (threadIdx.x == 0) s.bits_period = 0;
    __syncthreads();
    const uint32_t nvp = 2u << period;
    uint32_t o = o0;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      if (j0 + k == nvp) s.bits_period = o;
      o += resid_len((cc >> (2 * k)) & 3u, S);
    }
    __syncthreads();
    bits_p = s.bits_period;
    __syncthreads();
  }
  // 5. sizes and the choice
  uint32_t size[M_NMODES];
  size[M_ZERO] = allzero ? 16u : 0u;
  size[M_CONST] = allconst ? 32u : 0u;
  size[M_PERIOD] = period > 0 ? 16u + code_bytes(2u << period) + resid_bytes(bits_p) : 0u;
  size[M_STREAM] = 16u + code_bytes(N) + resid_bytes(total);
  size[M_RAW] = 16u + 8u * N;
  size[M_SPLIT] = 0u;
  uint32_t mode = 0, best = 0xffffffffu;
#pragma unroll
  for (uint32_t m = 0; m < M_NMODES; ++m)
    if (((modes >> m) & 1u) && size[m] != 0 && size[m] < best) {
      best = size[m];
      mode = m;
    }
  if (best > img_cap) {  // cannot happen: RAW always fits a buffer of max_image_bytes
    if (threadIdx.x == 0) atomicOr(err, (unsigned)E_MODE);
    return 0;
  }
  // 6. the image
  uint32_t nv = 0, rbits = 0;
  if (mode == M_CONST) nv = 2;
  if (mode == M_PERIOD) { nv = 2u << period; rbits = bits_p; }
  if (mode == M_STREAM) { nv = N; rbits = total; }
  if (mode == M_RAW) nv = N;
  if (threadIdx.x == 0) {
    uint32_t* hd = reinterpret_cast<uint32_t*>(img);
    hd[0] = mode | ((mode == M_ZERO ? 0u : S) << 8) | ((mode == M_PERIOD ? (uint32_t)period : 0u) << 16);
    hd[1] = best - 16u;
    hd[2] = nv;
    hd[3] = rbits;
  }
  uint64_t* pay64 = reinterpret_cast<uint64_t*>(img + 16);
  if (mode == M_CONST) {
    if (threadIdx.x == 0) {
      pay64[0] = tile[tile_val(0)];
      pay64[1] = tile[tile_val(1)];
    }
  } else if (mode == M_RAW) {
    ulonglong2* p2 = reinterpret_cast<ulonglong2*>(pay64);
    for (uint32_t a = threadIdx.x; a < A; a += kThreads) p2[a] = t2[tile_amp(a)];
  } else if (mode == M_PERIOD || mode == M_STREAM) {
    uint32_t c[VPT], r[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      c[k] = (cc >> (2 * k)) & 3u;
      r[k] = resid_len(c[k], S);
    }
    pack_xor32<VPT>(img, nv, j0, o0, h, c, r);
  }
  return best;
}

// Encodes both tiles of a work item in one pass: encode_core's steps for each chunk,
// the two chunks sharing every barrier.  Taken for the common case only: width
// S <= 32, the smallest image among modes without SPLIT, no selector network, and every
// thread holding VPT values of each chunk (kThreads * VPT = 2^(kc+1)).  Returns false,
// with both tiles untouched, if either chunk holds a subnormal or non-finite value (the
// caller then runs encode_block on each); otherwise true with the image lengths in
// n0 / n1 (0 with *err set on error).
template <int VPT>
__device__ bool encode_pair32(uint64_t* tile0, uint64_t* tile1, int kc, uint32_t S, uint32_t modes, uint8_t* img0,
                              uint8_t* img1, uint32_t img_cap, ScanSmem& s, int& pp, unsigned int* err, uint32_t& n0,
                              uint32_t& n1) {
  const uint32_t N = 2u << kc;
  const uint32_t j0 = threadIdx.x * VPT;
  // 0. clear both payload areas the packers OR into
  {
    const uint32_t span = (min(img_cap, max_coded_bytes(kc)) - 16u) / 16u;
    uint4* z0 = reinterpret_cast<uint4*>(img0 + 16);
    uint4* z1 = reinterpret_cast<uint4*>(img1 + 16);
    for (uint32_t u = threadIdx.x; u < 2u * span; u += kThreads) {
      if (u < span) z0[u] = make_uint4(0u, 0u, 0u, 0u);
      else z1[u - span] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  // 1. truncated high words (-0 stored as +0); a subnormal or non-finite value anywhere
  //    sends both chunks to the general path
  const uint32_t mh = (uint32_t)(trunc_mask(S) >> 32);
  uint32_t h0[VPT], h1[VPT];
  bool bad = false, nz0 = false, nz1 = false;
  {
    uint64_t t[VPT];
    load_vals<VPT>(tile0, j0, N, t);
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const uint32_t hi = (uint32_t)(t[k] >> 32), ahi = hi & 0x7fffffffu;
      bad |= ahi >= 0x7ff00000u || (ahi < 0x00100000u && (ahi | (uint32_t)t[k]) != 0u);
      const uint32_t v = hi & mh;
      h0[k] = v == 0x80000000u ? 0u : v;
      nz0 |= h0[k] != 0u;
    }
    load_vals<VPT>(tile1, j0, N, t);
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const uint32_t hi = (uint32_t)(t[k] >> 32), ahi = hi & 0x7fffffffu;
      bad |= ahi >= 0x7ff00000u || (ahi < 0x00100000u && (ahi | (uint32_t)t[k]) != 0u);
      const uint32_t v = hi & mh;
      h1[k] = v == 0x80000000u ? 0u : v;
      nz1 |= h1[k] != 0u;
    }
  }
  if (__syncthreads_or(bad)) return false;
  // 2. the truncated values back into the tiles
  {
    uint64_t t[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) t[k] = (uint64_t)h0[k] << 32;
    store_vals<VPT>(tile0, j0, N, t);
#pragma unroll
    for (int k = 0; k < VPT; ++k) t[k] = (uint64_t)h1[k] << 32;
    store_vals<VPT>(tile1, j0, N, t);
  }
  __syncthreads();
  // 3. codes, residual lengths and flags of both chunks; one scan for both
  const uint32_t Ptop = kc >= 2 ? (1u << (kc - 1)) : 0u;
  uint32_t cc0, cc1, sum0, sum1;
  bool cst0, cst1, gt0, gt1;
  codes32_pair_part<VPT>(tile0, j0, h0, S, Ptop, cc0, sum0, cst0, gt0);
  codes32_pair_part<VPT>(tile1, j0, h1, S, Ptop, cc1, sum1, cst1, gt1);
  uint32_t o0, o1, total0, total1, f_or, f_and;
  block_scan2(sum0, sum1, (nz0 ? 1u : 0u) | (nz1 ? 2u : 0u),
              (cst0 ? 1u : 0u) | (gt0 ? 2u : 0u) | (cst1 ? 4u : 0u) | (gt1 ? 8u : 0u), s, pp, &o0, &o1, &total0,
              &total1, &f_or, &f_and);
  // 4-6. period, choice and image of each chunk
  n0 = finish32_pair_part<VPT>(tile0, kc, S, modes, img0, img_cap, s, err, h0, cc0, o0, total0, (f_or & 1u) == 0u,
                               (f_and & 1u) != 0u, (f_and & 2u) != 0u);
  n1 = finish32_pair_part<VPT>(tile1, kc, S, modes, img1, img_cap, s, err, h1, cc1, o1, total1, (f_or & 2u) == 0u,
                               (f_and & 4u) != 0u, (f_and & 8u) != 0u);
  __syncthreads();
  return true;
}

// -------------------------------------------------------- gate arithmetic -- //
// Each output component is a sum of four products with (ar, ai, br, bi):
//   a'r = u00r ar - u00i ai + u01r br - u01i bi      a'i = u00r ai + u00i ar + u01r bi + u01i br
//   b'r = u10r ar - u10i ai + u11r br - u11i bi      b'i = u10r ai + u10i ar + u11r bi + u11i br
// taken in the order written.  A term whose coefficient is exactly zero is left out;
// the first kept term is one rounded product and every later term one fused
// multiply-add; with no term the result is +0.  The host lists the kept terms of
// each row (coefficient and operand) and marks a first coefficient of +1 / -1, whose
// product is an exact copy / sign flip and needs no FP64 instruction.
struct GateCoef {
  double c[16];      // row r: c[4r .. 4r + cnt[r]) in execution order
  uint8_t op[16];    // operand of each term: 0 ar, 1 ai, 2 br, 3 bi
  uint8_t cnt[4];    // kept terms per row
  uint8_t first[4];  // first term: 0 product, 1 copy, 2 sign flip
  uint8_t dense;     // all 16 terms kept: rows in the order written, no operand lookup
};

__device__ __forceinline__ double pick4(const double x[4], uint32_t i) {
  return i == 0 ? x[0] : (i == 1 ? x[1] : (i == 2 ? x[2] : x[3]));
}
__device__ __forceinline__ double flip_sign(double v) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
}

__device__ __forceinline__ double row_eval(const GateCoef& g, int r, const double x[4]) {
  const uint32_t n = g.cnt[r];
  if (n == 0) return 0.0;
  const double v0 = pick4(x, g.op[4 * r]);
  double acc;
  if (g.first[r] == 0) acc = __dmul_rn(g.c[4 * r], v0);
  else acc = g.first[r] == 1 ? v0 : flip_sign(v0);
  if (n > 1) acc = __fma_rn(g.c[4 * r + 1], pick4(x, g.op[4 * r + 1]), acc);
  if (n > 2) acc = __fma_rn(g.c[4 * r + 2], pick4(x, g.op[4 * r + 2]), acc);
  if (n > 3) acc = __fma_rn(g.c[4 * r + 3], pick4(x, g.op[4 * r + 3]), acc);
  return acc;
}

__device__ __forceinline__ void apply_pair(const GateCoef& g, double2& a, double2& b) {
  if (g.dense) {  // the same sums with the operands fixed (a first coefficient of +-1 multiplies exactly)
    const double* c = g.c;
    const double ar = a.x, ai = a.y, br = b.x, bi = b.y;
    a.x = __fma_rn(c[3], bi, __fma_rn(c[2], br, __fma_rn(c[1], ai, __dmul_rn(c[0], ar))));
    a.y = __fma_rn(c[7], br, __fma_rn(c[6], bi, __fma_rn(c[5], ar, __dmul_rn(c[4], ai))));
    b.x = __fma_rn(c[11], bi, __fma_rn(c[10], br, __fma_rn(c[9], ai, __dmul_rn(c[8], ar))));
    b.y = __fma_rn(c[15], br, __fma_rn(c[14], bi, __fma_rn(c[13], ar, __dmul_rn(c[12], ai))));
    return;
  }
  const double x[4] = {a.x, a.y, b.x, b.y};
  a.x = row_eval(g, 0, x);
  a.y = row_eval(g, 1, x);
  b.x = row_eval(g, 2, x);
  b.y = row_eval(g, 3, x);
}

// The first row pair (a'r, a'i) or the second (b'r, b'i) of apply_pair alone, with the
// same sums in the same order (for a thread that owns only one amplitude of the pair).
__device__ __forceinline__ double2 apply_rows01(const GateCoef& g, const double2 a, const double2 b) {
  if (g.dense) {
    const double* c = g.c;
    return make_double2(__fma_rn(c[3], b.y, __fma_rn(c[2], b.x, __fma_rn(c[1], a.y, __dmul_rn(c[0], a.x)))),
                        __fma_rn(c[7], b.x, __fma_rn(c[6], b.y, __fma_rn(c[5], a.x, __dmul_rn(c[4], a.y)))));
  }
  const double x[4] = {a.x, a.y, b.x, b.y};
  return make_double2(row_eval(g, 0, x), row_eval(g, 1, x));
}
__device__ __forceinline__ double2 apply_rows23(const GateCoef& g, const double2 a, const double2 b) {
  if (g.dense) {
    const double* c = g.c;
    return make_double2(__fma_rn(c[11], b.y, __fma_rn(c[10], b.x, __fma_rn(c[9], a.y, __dmul_rn(c[8], a.x)))),
                        __fma_rn(c[15], b.x, __fma_rn(c[14], b.y, __fma_rn(c[13], a.x, __dmul_rn(c[12], a.y)))));
  }
  const double x[4] = {a.x, a.y, b.x, b.y};
  return make_double2(row_eval(g, 2, x), row_eval(g, 3, x));
}

// Image of a chunk whose amplitudes all equal (v0, v1): what encode_block writes
// for a constant tile (the subnormal rule, truncation, -0 -> +0, then ZERO if both
// values are +0, else CONST).  h receives 8 words (16-byte header + 16-byte payload
// as u32); returns the image length, 0 for a non-finite value.
__device__ __forceinline__ uint32_t const_image(uint64_t v0, uint64_t v1, uint32_t S_req, uint32_t h[8]) {
  const uint32_t e0 = (uint32_t)(v0 >> 52) & 0x7ffu, e1 = (uint32_t)(v1 >> 52) & 0x7ffu;
  if (e0 == 0x7ffu || e1 == 0x7ffu) return 0;
  const bool sub = (e0 == 0u && (v0 << 12) != 0ull) || (e1 == 0u && (v1 << 12) != 0ull);
  const uint32_t S = sub ? 64u : S_req;
  const uint64_t m = trunc_mask(S);
  uint64_t t0 = v0 & m, t1 = v1 & m;
  if (t0 == 0x8000000000000000ull) t0 = 0;
  if (t1 == 0x8000000000000000ull) t1 = 0;
  for (int k = 0; k < 8; ++k) h[k] = 0u;
  if (t0 == 0ull && t1 == 0ull) return 16u;
  h[0] = M_CONST | (S << 8);
  h[1] = 16u;
  h[2] = 2u;
  h[3] = 0u;
  h[4] = (uint32_t)t0;
  h[5] = (uint32_t)(t0 >> 32);
  h[6] = (uint32_t)t1;
  h[7] = (uint32_t)(t1 >> 32);
  return 32u;
}

// --------------------------------------------------------------- pool ---- //
__device__ __forceinline__ uint32_t* dir_entry(const Pool& P, unsigned long long chunk) {
  return P.dir + chunk * (unsigned long long)P.dir_words;
}

// Stages chunk's image into smem (all threads).  Returns the image length.
__device__ __forceinline__ uint32_t load_image_block(const Pool& P, unsigned long long chunk, uint8_t* smem_img,
                                                     uint32_t* smem_pages, uint32_t cap) {
  const uint32_t* e = dir_entry(P, chunk);
  const uint32_t bytes = e[0], np = e[1];
  if (bytes > cap) return bytes;  // caller reports corruption
  uint4* dst = reinterpret_cast<uint4*>(smem_img);
  const uint32_t units = bytes >> 4;
  if (np == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(e + 4);
    for (uint32_t u = threadIdx.x; u < units; u += kThreads) dst[u] = src[u];
  } else {
    for (uint32_t q = threadIdx.x; q < np; q += kThreads) smem_pages[q] = e[4 + q];
    __syncthreads();
    constexpr uint32_t upp = kPage / 16;
    for (uint32_t u = threadIdx.x; u < units; u += kThreads) {
      const uint32_t pid = smem_pages[u / upp];
      const uint4* src = reinterpret_cast<const uint4*>(P.pages + (unsigned long long)pid * kPage);
      dst[u] = __ldcs(src + (u % upp));
    }
  }
  __syncthreads();
  return bytes;
}

// A CTA's page cache: ids of pages its work items freed, reused first by its later
// items, held in shared memory during a launch (the post kernel returns the rest).
struct CtaCache {
  uint32_t* ids;  // shared memory, kCacheCap entries
  uint32_t* n;    // shared memory
};

// Warp 0: returns the old pages of the two staged chunks (p0[0..np0), p1[0..np1)) to the
// CTA cache; what does not fit goes to the global freed list, merged into the stack
// after the gate.
__device__ __forceinline__ void free_pages_warp(const Pool& P, const CtaCache& cc, const uint32_t* p0, uint32_t np0,
                                                const uint32_t* p1, uint32_t np1) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = *cc.n, tot = np0 + np1, room = (uint32_t)kCacheCap - n;
  unsigned long long base = 0;
  if (tot > room) {
    if (lane == 0)
      base = atomicAdd(reinterpret_cast<unsigned long long*>(&P.ctl->nfreed), (unsigned long long)(tot - room));
    base = __shfl_sync(0xffffffffu, base, 0);
  }
  for (uint32_t q = lane; q < tot; q += 32u) {
    const uint32_t id = q < np0 ? p0[q] : p1[q - np0];
    if (q < room) {
      cc.ids[n + q] = id;
    } else {
      const unsigned long long at = base + (q - room);
      if (at < P.npages) P.freed[at] = id;  // the list holds every page at most once
      else atomicOr(&P.ctl->err, (unsigned)E_CORRUPT);
    }
  }
  __syncwarp();
  if (lane == 0) *cc.n = n + min(tot, room);
  __syncwarp();
}

// Warp 0: takes np0 + np1 pages (the cache's most recent first, then the global stack)
// into out0 / out1.  False: the pool is dry.
__device__ __forceinline__ bool alloc_pages_warp(const Pool& P, const CtaCache& cc, uint32_t* out0, uint32_t np0,
                                                 uint32_t* out1, uint32_t np1) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = *cc.n, tot = np0 + np1, take = min(tot, n), need = tot - take;
  long long old = 0;
  if (need) {
    if (lane == 0)
      old = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&P.ctl->top), (unsigned long long)(-(long long)need));
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old - (long long)need < 0) {  // dry: give the reservation back (top never stays below 0)
      if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&P.ctl->top), (unsigned long long)need);
      return false;
    }
  }
  for (uint32_t q = lane; q < tot; q += 32u) {
    const uint32_t id = q < take ? cc.ids[n - 1u - q] : P.stack[old - 1 - (long long)(q - take)];
    if (q < np0) out0[q] = id;
    else out1[q - np0] = id;
  }
  __syncwarp();
  if (lane == 0) *cc.n = n - take;
  __syncwarp();
  return true;
}

// Writes the image in smem to the chunk (inline in the directory when it fits,
// else to freshly allocated pages) and updates the directory entry.  All threads.
// smem_pages must hold the page ids (thread 0 allocated them).
__device__ __forceinline__ void store_image_block(const Pool& P, unsigned long long chunk, const uint8_t* smem_img,
                                                  uint32_t bytes, const uint32_t* smem_pages, uint32_t np) {
  uint32_t* e = dir_entry(P, chunk);
  const uint4* src = reinterpret_cast<const uint4*>(smem_img);
  const uint32_t units = bytes >> 4;
  if (np == 0) {
    uint4* dst = reinterpret_cast<uint4*>(e + 4);
    for (uint32_t u = threadIdx.x; u < units; u += kThreads) dst[u] = src[u];
  } else {
    constexpr uint32_t upp = kPage / 16;
    for (uint32_t u = threadIdx.x; u < units; u += kThreads) {
      uint4* dst = reinterpret_cast<uint4*>(P.pages + (unsigned long long)smem_pages[u / upp] * kPage);
      __stcs(dst + (u % upp), src[u]);
    }
    for (uint32_t q = threadIdx.x; q < np; q += kThreads) e[4 + q] = smem_pages[q];
  }
  if (threadIdx.x == 0) {
    e[0] = bytes;
    e[1] = np;
  }
}

__host__ __device__ __forceinline__ uint32_t pages_for(uint32_t bytes, int kc) {
  return bytes <= inline_cap(kc) ? 0u : (bytes + kPage - 1) / kPage;
}

// Scatter the bits of j into the positions that are set in `free_mask` (low first).
__device__ __forceinline__ unsigned long long deposit_bits(unsigned long long j, unsigned long long free_mask) {
  unsigned long long out = 0;
  while (free_mask) {
    const unsigned long long low = free_mask & (~free_mask + 1ull);
    if (j & 1ull) out |= low;
    j >>= 1;
    free_mask ^= low;
  }
  return out;
}

}  // namespace qc
