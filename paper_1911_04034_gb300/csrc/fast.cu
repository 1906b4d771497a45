// fast.cu -- the streaming form of the fused gate kernel (sm_103a).
//
// The general kernel (k_gate) gives a work item of two chunks to a whole CTA: decode
// into shared-memory tiles, apply, encode, each step a CTA-wide pass with barriers.
// For the case that dominates a lossy run -- both input chunks coded as STREAM at a
// width S <= 32 and the output again a STREAM image at the gate's S <= 32 -- this
// kernel gives a work item to a pair of warps instead, one chunk each; a warp walks its
// chunk in passes of 256 values (8 per lane) and keeps every value in registers from
// the decoder through the gate arithmetic to the encoder (a cross-chunk gate swaps the
// partner values of each pass with the other warp through shared memory):
//
//   per pass: codes -> residual lengths -> warp scan of the offsets ->
//             explicit parts from the staged input window -> warp scan of the
//             leading bytes (Section 4.2, Solution C decoding) -> the 2x2 unitary on
//             the amplitude pairs (Section 3.1, Eq. matrix1/matrix2) -> truncation to
//             S bits (Eq. sigbits) -> XOR leading-byte codes -> warp scan of the output
//             offsets -> packing into the output window -> finished 16-byte blocks out
//             to freshly allocated pages.
//
// Scans are warp shuffles and every carry between passes (stream offsets, the
// predecessor's leading bytes, the encoder's predecessor) stays in registers, so the
// kernel has no CTA-wide barrier; the warps of an SM overlap their FP64 arithmetic
// with each other's integer codec work.  Input windows are double-buffered with
// cp.async (the next pass's window is in flight while the current one is decoded).
//
// Anything else goes to the general kernel unchanged: an item whose input images are
// not STREAM at S <= 32, whose output chunk would not be a STREAM image (all-zero,
// constant, possibly periodic -- Section 4.2's period rule needs the whole chunk; a
// chunk whose sampled values all equal their partners half a chunk away is left to
// the general kernel, which runs the full test -- or holding a subnormal or non-finite
// value), or one whose chunk the learned selector granted a SPLIT / PALETTE trial, is
// appended to a device list before any of its state changes, and k_gate runs the list
// right after this kernel.  Both kernels write the bytes the oracle writes.
#include "gate_common.cuh"

namespace qc {

constexpr int kFastWarps = 8;   // four pairs: the two warps of a pair share a work item, one chunk each
constexpr int kFastPairs = kFastWarps / 2;
constexpr int kFastThreads = 32 * kFastWarps;
#ifndef QC_FAST_MIN_CTAS
#define QC_FAST_MIN_CTAS 3
#endif
constexpr uint32_t kFastWin = 1056;   // bytes of a pass window: 1024 bytes of stream at most, plus alignment and read slack
constexpr uint32_t kWinBlocks = kFastWin / 16;
constexpr uint32_t kWarpCache = 64;   // page ids a warp keeps between its items

__host__ __device__ __forceinline__ uint32_t fast_pg_words(int kc) { return (max_pages(kc) + 3u) & ~3u; }
// Per warp (one chunk): two input windows, one output window, the input and the output
// page ids, the values it shows its partner warp (two passes), its page cache, one
// sample per lane of each pass of the chunk's first half.
__host__ __device__ __forceinline__ uint32_t fast_warp_bytes(int kc) {
  return 3u * kFastWin + 8u * fast_pg_words(kc) + 2u * 1024u + 4u * kWarpCache + 16u + (1u << (kc - 1));
}
// Largest STREAM image of a chunk at S <= 32 bits.
__host__ __device__ __forceinline__ uint32_t fast_max_image(int kc) {
  return 16u + code_bytes(2u << kc) + resid_bytes(32u * (2u << kc));
}

// A warp's own page cache in shared memory: ids[0, *n).
struct WarpPages {
  uint32_t* ids;
  uint32_t* n;
};

// All lanes: at least `want` (<= 32) ids in the cache, refilled 32 at a time from the
// global stack.  False (E_OOM set, the stack top restored) if the stack is dry.
__device__ __forceinline__ bool wp_reserve(const Pool& P, const WarpPages& wp, uint32_t want) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = *wp.n;
  if (n >= want) return true;
  long long old = 0;
  if (lane == 0)
    old = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&P.ctl->top), (unsigned long long)(-32ll));
  old = __shfl_sync(0xffffffffu, old, 0);
  if (old - 32 < 0) {  // the stack is dry: give the reservation back (top never stays below 0)
    if (lane == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&P.ctl->top), 32ull);
      atomicOr(&P.ctl->err, (unsigned)E_OOM);
    }
    return false;
  }
  wp.ids[n + lane] = P.stack[old - 1 - (long long)lane];
  __syncwarp();
  if (lane == 0) *wp.n = n + 32u;
  __syncwarp();
  return true;
}

// All lanes: pushes ids[0, cnt) into the cache; what does not fit goes to the global
// freed list (merged into the stack after the gate).
__device__ __forceinline__ void wp_free(const Pool& P, const WarpPages& wp, const uint32_t* ids, uint32_t cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = *wp.n, room = kWarpCache - n;
  unsigned long long base = 0;
  if (cnt > room) {
    if (lane == 0) base = atomicAdd(&P.ctl->nfreed, (unsigned long long)(cnt - room));
    base = __shfl_sync(0xffffffffu, base, 0);
  }
  for (uint32_t q = lane; q < cnt; q += 32u) {
    const uint32_t id = ids[q];
    if (q < room) {
      wp.ids[n + q] = id;
    } else {
      const unsigned long long at = base + (q - room);
      if (at < P.npages) P.freed[at] = id;  // the list holds every page at most once
      else atomicOr(&P.ctl->err, (unsigned)E_CORRUPT);
    }
  }
  __syncwarp();
  if (lane == 0) *wp.n = n + min(cnt, room);
  __syncwarp();
}

// All lanes: the output page list grows to `need` pages.
__device__ __forceinline__ bool wp_grow(const Pool& P, const WarpPages& wp, uint32_t* opg, uint32_t& onp,
                                        uint32_t need) {
  while (onp < need) {
    const uint32_t k = min(need - onp, 32u);
    if (!wp_reserve(P, wp, k)) return false;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t n = *wp.n;
    if (lane < k) opg[onp + lane] = wp.ids[n - 1u - lane];
    __syncwarp();
    if (lane == 0) *wp.n = n - k;
    __syncwarp();
    onp += k;
  }
  return true;
}

// Bit position (within a lane's 16-bit code field) of the 2-bit code of the lane's
// value k: four codes per byte, the first in the top bits, bytes in memory order.
__host__ __device__ constexpr uint32_t code_shift(int k) { return 8u * (uint32_t)(k >> 2) + 6u - 2u * (uint32_t)(k & 3); }
// 8 * (code of value k) from the lane's code field.
template <int k>
__device__ __forceinline__ uint32_t code8(uint32_t cw) {
  constexpr uint32_t s = code_shift(k);
  if constexpr (s >= 3) return (cw >> (s - 3)) & 0x18u;
  else return (cw << (3 - s)) & 0x18u;
}
__device__ __forceinline__ uint32_t code8_at(uint32_t cw, int k) {
  switch (k) {
    case 0: return code8<0>(cw);
    case 1: return code8<1>(cw);
    case 2: return code8<2>(cw);
    case 3: return code8<3>(cw);
    case 4: return code8<4>(cw);
    case 5: return code8<5>(cw);
    case 6: return code8<6>(cw);
    default: return code8<7>(cw);
  }
}
__device__ __forceinline__ uint32_t rlen(uint32_t S, uint32_t c8) { return S > c8 ? S - c8 : 0u; }

// Sum of the residual lengths max(S - 8c, 0) of the 8 codes of a lane's 16-bit field.
__device__ __forceinline__ uint32_t rsum8(uint32_t cw, uint32_t S) {
  const uint32_t lo = cw & 0x5555u, hi = (cw >> 1) & 0x5555u;
  const uint32_t n1 = __popc(lo & ~hi), n2 = __popc(hi & ~lo), n3 = __popc(lo & hi);
  return (8u - n1 - n2 - n3) * S + n1 * rlen(S, 8u) + n2 * rlen(S, 16u) + n3 * rlen(S, 24u);
}

// Exclusive warp scan (plus the warp total, to all lanes).
__device__ __forceinline__ uint32_t warp_excl(uint32_t v, uint32_t& total) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= (uint32_t)d) inc += u;
  }
  total = __shfl_sync(0xffffffffu, inc, 31);
  return inc - v;
}

// The leading-byte run of a lane, packed: bits 8..31 the bytes its values set, bits 0..1
// the smallest code among them (3: none set).  Composition (earlier A, later B): B's
// explicit bytes replace A's; the smallest code is the smaller of the two.
__device__ __forceinline__ uint32_t lead_compose(uint32_t A, uint32_t B) {
  const uint32_t mb = B & 3u;
  const uint32_t ex = 0xFFFFFF00u & (0xFFFFFFFFu >> (8u * mb));
  return (A & ~ex & 0xFFFFFF00u) | (B & 0xFFFFFF00u) | min(A & 3u, mb);
}
// Exclusive warp scan of lead runs after `carry` (the top bytes of the value before the
// warp's first): returns the top bytes of the lane's predecessor; `after` receives (on
// all lanes) the top bytes of the warp's last value.
__device__ __forceinline__ uint32_t lead_scan_warp(uint32_t W, uint32_t carry, uint32_t& after) {
  const uint32_t lane = threadIdx.x & 31u;
  if (__all_sync(0xffffffffu, (W & 3u) == 0u)) {
    // every lane has a value with code 0 (all three leading bytes explicit): a lane's
    // predecessor's leading bytes are the previous lane's run alone
    uint32_t exc = __shfl_up_sync(0xffffffffu, W, 1);
    if (lane == 0) exc = carry;
    after = __shfl_sync(0xffffffffu, W, 31) & 0xFFFFFF00u;
    return exc & 0xFFFFFF00u;
  }
  uint32_t inc = W;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= (uint32_t)d) inc = lead_compose(u, inc);
  }
  uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) exc = 3u;  // empty run
  const uint32_t last = __shfl_sync(0xffffffffu, inc, 31);
  const uint32_t cw = (carry & 0xFFFFFF00u) | 3u;
  after = lead_compose(cw, last) & 0xFFFFFF00u;
  return lead_compose(cw, exc) & 0xFFFFFF00u;
}

// Stages stream blocks [wb, wb + kWinBlocks) of the input image (only those inside its
// nbs stream blocks) into a window with cp.async.  16-byte block k of the stream is
// image byte 16 + cb + 16k.
__device__ __forceinline__ void fast_issue_window(const Pool& P, const uint32_t* ipg, uint32_t* win, uint32_t cb,
                                                  uint32_t wb, uint32_t nbs) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (uint32_t k = lane; k < kWinBlocks; k += 32u) {
    const uint32_t blk = wb + k;
    if (blk < nbs) {
      const uint32_t b = 16u + cb + 16u * blk;
      cp_async16(win + 4u * k, P.pages + (unsigned long long)ipg[b >> 9] * kPage + (b & (kPage - 1u)));
    }
  }
}

__device__ __forceinline__ double hi_as_double(uint32_t h) { return __longlong_as_double((long long)((uint64_t)h << 32)); }

// The truncated high word of a result (S <= 32: the low word is always cut); a signed
// zero becomes +0.  `spec` is set for a subnormal or non-finite result: a chunk holding
// one is coded at 64 bits or is an error, which the general kernel handles.
__device__ __forceinline__ uint32_t fast_trunc(double v, uint32_t mh, bool& spec) {
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const uint32_t hi = (uint32_t)(u >> 32), ahi = hi & 0x7fffffffu;
  const bool zero = (ahi | (uint32_t)u) == 0u;
  spec |= (ahi - 0x00100000u) >= 0x7fe00000u && !zero;
  return zero ? 0u : (hi & mh);
}

// The explicit parts of a lane's 8 values from the input window (stream unit q at
// win[(q ^ 1) - w4]), starting at stream bit o; e[k] receives bits [8c, S) of value k's
// high word; returns the lane's lead run (see lead_compose).
__device__ __forceinline__ uint32_t fast_extract(const uint32_t* win, uint32_t w4, uint32_t o, uint32_t cw,
                                                 uint32_t S, uint32_t mh, uint32_t e[8]) {
  uint32_t W = 3u;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t c8 = code8_at(cw, k);
    const uint32_t q = o >> 5;
    const uint32_t x = __funnelshift_l(win[((q + 1u) ^ 1u) - w4], win[(q ^ 1u) - w4], o);
    e[k] = (x >> c8) & mh;
    o += rlen(S, c8);
    const uint32_t ex = 0xFFFFFF00u & (0xFFFFFFFFu >> c8);
    W = (W & ~ex & 0xFFFFFF00u) | (e[k] & ex) | min(W & 3u, c8 >> 3);
  }
  return W;
}

// Rebuilds the high words from the explicit parts: value k takes its copied leading
// bytes from its predecessor (P: the top bytes of the lane's predecessor).
__device__ __forceinline__ void fast_rebuild(uint32_t e[8], uint32_t cw, uint32_t P) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    P = e[k] | (P & ~(0xFFFFFFFFu >> code8_at(cw, k)));
    e[k] = P;
  }
}

// Codes of a lane's 8 truncated values (predecessor of the first: pr), as the lane's
// 16-bit code field; `sum` receives their residual-length sum.
__device__ __forceinline__ uint32_t fast_codes(const uint32_t t[8], uint32_t pr, uint32_t S, uint32_t& sum) {
  uint32_t cw = 0u, s = 0u;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t x = t[k] ^ (k ? t[k - 1] : pr);
    const uint32_t c8 = min((uint32_t)__clz((int)x), 24u) & 0x18u;
    s += rlen(S, c8);
    cw |= (c8 >> 3) << code_shift(k);
  }
  sum = s;
  return cw;
}

// Packs the residuals of a lane's 8 values (high words t, codes in the lane's code
// field cw) at stream bit o of a cleared window whose block 0 is stream block w4 / 4
// (stream unit q is win[(q ^ 1) - w4]).  The first unit the lane touches and its last,
// unfinished one may be shared with the neighbouring lanes: atomicOr; units in
// between are stored.
__device__ __forceinline__ void fast_pack(uint32_t* win, uint32_t w4, uint32_t o, const uint32_t t[8], uint32_t cw,
                                          uint32_t S) {
  uint32_t q = o >> 5, fill = o & 31u, cur = 0u;
  bool first = true;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t c8 = code8_at(cw, k);
    const uint32_t r = rlen(S, c8);
    const uint32_t f = t[k] << c8;  // the residual in the top r bits, zeros below
    cur |= f >> fill;
    const uint32_t nf = fill + r;
    if (nf >= 32u) {
      if (first) atomicOr(&win[(q ^ 1u) - w4], cur);
      else win[(q ^ 1u) - w4] = cur;
      first = false;
      ++q;
      cur = __funnelshift_r(0u, f, fill);
      fill = nf - 32u;
    } else {
      fill = nf;
    }
  }
  if (fill > 0u && cur) atomicOr(&win[(q ^ 1u) - w4], cur);
}

// The two warps of a pair meet through a sequence number per warp in shared memory:
// each raises its own to `phase` (after its earlier shared-memory writes) and waits
// until the partner's has reached it.  The wait is bounded: after kSpinLimit polls it
// sets E_TIMEOUT (and the site) and returns false, so no protocol error can hang the
// kernel.
constexpr uint32_t kSpinLimit = 1u << 22;
__device__ __forceinline__ bool pair_sync(volatile uint32_t* seq, uint32_t side, uint32_t phase, DevCtl* ctl,
                                          uint32_t site) {
  __syncwarp();
  bool ok = true;
  if ((threadIdx.x & 31u) == 0) {
    __threadfence_block();
    seq[side] = phase;
    uint32_t it = 0;
    while ((int)(seq[side ^ 1u] - phase) < 0) {
      if (++it > kSpinLimit) {
        ok = false;
        atomicOr(&ctl->err, (unsigned)E_TIMEOUT);
        atomicExch(&ctl->timeout_site, site);
        break;
      }
    }
    __threadfence_block();
  }
  ok = __shfl_sync(0xffffffffu, ok ? 1u : 0u, 0) != 0u;
  __syncwarp();  // orders lane 0's acquire before the other lanes' reads
  return ok;
}

// The two warps of a pair agree on a flag word: each publishes its own, then both read
// both.  Slots alternate, so a slot is rewritten only after the partner has passed the
// next meeting, i.e. after it read the slot.  A failed wait reads as an error (bit 1).
__device__ __forceinline__ uint32_t pair_agree(uint32_t* slots, volatile uint32_t* seq, uint32_t& phase,
                                               uint32_t side, uint32_t mine, DevCtl* ctl, uint32_t site) {
  volatile uint32_t* s = slots + 2u * (phase & 1u);
  if ((threadIdx.x & 31u) == 0) s[side] = mine;
  ++phase;
  if (!pair_sync(seq, side, phase, ctl, site)) return 2u;
  return s[side ^ 1u];
}

// One output amplitude of a dense-class gate: row pair (r, r + 1) of Eq. matrix1 /
// matrix2 over every coefficient (cf: that row pair's eight, from GateLaunch.cf), in
// the order of the kept-term sums; zero coefficients add exact zeros.
__device__ __forceinline__ double2 dense_rows(const double* cf, double2 a, double2 b) {
  return make_double2(__fma_rn(cf[3], b.y, __fma_rn(cf[2], b.x, __fma_rn(cf[1], a.y, __dmul_rn(cf[0], a.x)))),
                      __fma_rn(cf[7], b.x, __fma_rn(cf[6], b.y, __fma_rn(cf[5], a.x, __dmul_rn(cf[4], a.y)))));
}

// The same output for a real matrix (every imaginary coefficient zero): the chains
// above with their zero terms left out -- each dropped term adds an exact zero -- so
// the products of the real parts alone, in the same order (cf[0] = cf[4] = the row's
// first real coefficient, cf[2] = cf[6] its second).
__device__ __forceinline__ double2 real_rows(const double* cf, double2 a, double2 b) {
  return make_double2(__fma_rn(cf[2], b.x, __dmul_rn(cf[0], a.x)), __fma_rn(cf[2], b.y, __dmul_rn(cf[0], a.y)));
}

// The same output for a gate whose coefficient parts are all +-2^k, none zero (sqrt(X),
// sqrt(Y)): every product of the chains above is exact, so each chain equals 2^k times
// the chain of the signed inputs in the same order (scaling by a power of two commutes
// with rounding while no partial sum leaves the normal range): three additions per
// output part, then the scale added to the exponent field.  The inputs are checked
// once per pass (an item holding a value below 2^-959 goes to the general kernel), and
// then no partial sum leaves the normal range: inputs of at least 2^-959 truncated to at
// most 20 mantissa bits are multiples of 2^-979, so a nonzero sum is at least that, and
// 2^k <= 1.  Only an overflow to infinity is left to catch.  Bit q of L.sgn is the sign
// of coefficient cf[q].
__device__ __forceinline__ void signed_rows(const GateLaunch& L, uint32_t r, uint32_t ar, uint32_t ai, uint32_t br,
                                            uint32_t bi, uint32_t mh, uint32_t& outr, uint32_t& outi, bool& spec) {
  const uint32_t sg = L.sgn >> (8u * r);
  auto t = [&](int q, uint32_t h) { return hi_as_double(h ^ ((sg >> q) << 31)); };
  const double re = __dadd_rn(__dadd_rn(__dadd_rn(t(0, ar), t(1, ai)), t(2, br)), t(3, bi));
  const double im = __dadd_rn(__dadd_rn(__dadd_rn(t(4, ai), t(5, ar)), t(6, bi)), t(7, br));
  auto scaled = [&](double y) -> uint32_t {
    const uint64_t u = (uint64_t)__double_as_longlong(y);
    const uint32_t hi = (uint32_t)(u >> 32);
    if ((hi & 0x7fffffffu) == 0u && (uint32_t)u == 0u) return 0u;
    spec |= (hi & 0x7ff00000u) == 0x7ff00000u;
    return (hi + ((uint32_t)L.sk << 20)) & mh;
  };
  outr = scaled(re);
  outi = scaled(im);
}

// Row r of a diagonal (x = the amplitude itself) or anti-diagonal (x = its partner)
// gate on x, given as high words: a complex product in the order of the kept-term sums,
// or an exact copy / negation done on the high words (no FP64); results truncated.
__device__ __forceinline__ void row_op(const GateLaunch& L, uint32_t r, uint32_t xr, uint32_t xi, uint32_t mh,
                                       uint32_t& outr, uint32_t& outi, bool& spec) {
  const int op = L.rop[r];
  if (op == 0) {
    const double ur = L.du[2u * r], ui = L.du[2u * r + 1u];
    const double x = hi_as_double(xr), y = hi_as_double(xi);
    outr = fast_trunc(__fma_rn(-ui, y, __dmul_rn(ur, x)), mh, spec);
    outi = fast_trunc(__fma_rn(ui, x, __dmul_rn(ur, y)), mh, spec);
  } else if (op == 1) {
    outr = xr & mh;
    outi = xi & mh;
  } else {
    outr = xr ? ((xr ^ 0x80000000u) & mh) : 0u;
    outi = xi ? ((xi ^ 0x80000000u) & mh) : 0u;
  }
}

// A pair of amplitudes (slots k0 < k1) held by the same lane: both outputs.
template <int ARITH>
__device__ __forceinline__ void fast_pair_in_lane(const GateLaunch& L, uint32_t ibase, int k0, int k1, uint32_t v[8],
                                                  uint32_t mh, bool& spec) {
  const uint32_t ar = v[2 * k0], ai = v[2 * k0 + 1], br = v[2 * k1], bi = v[2 * k1 + 1];
  uint32_t o[4] = {ar & mh, ai & mh, br & mh, bi & mh};
  if (((ibase + (uint32_t)k0) & L.lo_mask) == L.lo_vals) {
    if constexpr (ARITH == 4) {
      signed_rows(L, 0u, ar, ai, br, bi, mh, o[0], o[1], spec);
      signed_rows(L, 1u, ar, ai, br, bi, mh, o[2], o[3], spec);
    } else if constexpr (ARITH == 0 || ARITH == 3) {
      const double2 a = make_double2(hi_as_double(ar), hi_as_double(ai)), b = make_double2(hi_as_double(br), hi_as_double(bi));
      const double2 x = ARITH == 0 ? dense_rows(L.cf, a, b) : real_rows(L.cf, a, b);
      const double2 y = ARITH == 0 ? dense_rows(L.cf + 8, a, b) : real_rows(L.cf + 8, a, b);
      o[0] = fast_trunc(x.x, mh, spec);
      o[1] = fast_trunc(x.y, mh, spec);
      o[2] = fast_trunc(y.x, mh, spec);
      o[3] = fast_trunc(y.y, mh, spec);
    } else {  // anti-diagonal: a' from b, b' from a
      row_op(L, 0u, br, bi, mh, o[0], o[1], spec);
      row_op(L, 1u, ar, ai, mh, o[2], o[3], spec);
    }
  }
  v[2 * k0] = o[0];
  v[2 * k0 + 1] = o[1];
  v[2 * k1] = o[2];
  v[2 * k1 + 1] = o[3];
}

// Shared-memory buffers of one warp (its chunk of the pair's item).
struct FastWarp {
  uint32_t* iwin0;
  uint32_t* iwin1;
  uint32_t* owin;
  uint32_t* ipg;
  uint32_t* opg;
  uint32_t* xch;  // [2][256]: the pass's decoded high words, for the partner warp
  uint32_t* half;  // [passes / 2][32]: one sample per lane of each first-half pass
};

__device__ __forceinline__ FastWarp fast_warp(uint8_t* base, int kc) {
  FastWarp f;
  f.iwin0 = reinterpret_cast<uint32_t*>(base);
  f.iwin1 = f.iwin0 + kFastWin / 4u;
  f.owin = f.iwin1 + kFastWin / 4u;
  f.ipg = f.owin + kFastWin / 4u;
  f.opg = f.ipg + fast_pg_words(kc);
  f.xch = f.opg + fast_pg_words(kc);
  f.half = f.xch + 512u + kWarpCache + 4u;
  return f;
}

// One work item: this warp's chunk (side 0 or 1 of the pair).  Returns 0 when both
// chunks were committed, 1 when the pair left the item to the general kernel (nothing
// of the state changed), 2 when the pair stops (a device error is set).
// Per-phase SM cycles of a warp when profiling (lane 0 counts): 0 staging (directory
// entries, headers, the partners' agreement, waits for input windows), 1 decoding, 2 the
// gate (with the exchange between the partners), 3 encoding, 4 committing (finished
// blocks, header, codes, directory entry, pages).
struct FastPhases {
  long long* t;  // shared memory: the five sums, then the last clock
  bool on;
  __device__ __forceinline__ void mark(int k) {
    if (on) {
      const long long now = clock64();
      t[k] += now - t[5];
      t[5] = now;
    }
  }
};

template <int KIND, int ARITH>
__device__ __forceinline__ int fast_item(const GateLaunch& L, unsigned long long item, uint32_t S, const FastWarp& fw,
                                         const uint32_t* xpeer, const WarpPages& wp, uint32_t side,
                                         volatile uint32_t* seq, uint32_t* slots, uint32_t& phase, long long& dE,
                                         unsigned long long& rd, unsigned long long& wr, FastPhases& ph) {
  const Pool& P = L.P;
  const int kc = P.kc;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t N = 2u << kc, cb = N >> 2, NP = N >> 8;
  // this warp's chunk; an in-chunk gate with an odd number of chunks has a last item of one
  const bool whole = L.pair || 2ull * item + 1ull < L.nact;
  unsigned long long ch = 0;
  if (whole) ch = L.pair ? ((item_chunk(L, item) | L.hi_vals) | (side ? L.pair_bit : 0ull))
                         : (item_chunk(L, 2ull * item + side) | L.hi_vals);
  // directory entry and header: a STREAM image at S <= 32, granted no selector trial
  uint32_t ib = 0, inp = 0, Sin = 0, bits_in = 0;
  bool ok = whole && (!L.sel_dec || L.sel_dec[2ull * item + side] == 0u);
  if (ok) {
    const uint32_t* e = dir_entry(P, ch);
    const uint2 h = *reinterpret_cast<const uint2*>(e);
    ib = h.x;
    inp = h.y;
    ok = inp >= 1u && ib >= 16u + cb && ib <= fast_max_image(kc) && (ib & 15u) == 0u && inp == (ib + kPage - 1u) / kPage;
    if (ok) {
      bool good = true;
      for (uint32_t k = lane; k < inp; k += 32u) {
        const uint32_t pid = e[4 + k];
        fw.ipg[k] = pid;
        good &= pid < P.npages;
      }
      ok = __all_sync(0xffffffffu, good);
      __syncwarp();
    }
    if (ok) {
      const uint4 hd = *reinterpret_cast<const uint4*>(P.pages + (unsigned long long)fw.ipg[0] * kPage);
      const uint32_t mode = hd.x & 0xffu, lp = (hd.x >> 16) & 0xffu, fl = hd.x >> 24;
      Sin = (hd.x >> 8) & 0xffu;
      bits_in = hd.w;
      ok = mode == M_STREAM && fl == 0u && lp == 0u && Sin >= 13u && Sin <= 32u && hd.y + 16u == ib && hd.z == N &&
           cb + resid_bytes(hd.w) == hd.y;
    }
  }
  unsigned int err = 0;
  if (lane == 0) err = *(volatile unsigned int*)&P.ctl->err;
  err = __shfl_sync(0xffffffffu, err, 0);
  {
    const uint32_t mine = (ok ? 1u : 0u) | (err ? 2u : 0u);
    const uint32_t other = pair_agree(slots, seq, phase, side, mine, P.ctl, 1u);
    if ((mine | other) & 2u) return 2;
    if (!((mine & other) & 1u)) return 1;
  }
  if constexpr (KIND == 0 && ARITH == 1) {
    // A diagonal row that is an exact copy (T's and CZ's first row) leaves this chunk's
    // values as they are; already coded at the gate's S, they would be re-encoded to the
    // same bytes (truncation is idempotent, and the smallest-image choice sees the same
    // values), so the image stays and the warp only joins the pair's final agreement
    // (there are no meetings in between for a diagonal gate).
    if (L.rop[side] == 1 && Sin == S) {
      const uint32_t other = pair_agree(slots, seq, phase, side, 1u, P.ctl, 3u);
      if (other & 2u) return 2;
      return (other & 1u) ? 0 : 1;
    }
  }
  const uint32_t nbs = (ib - 16u - cb) >> 4;
  // the code word of this lane's values in pass p (image byte 16 + 64 p + 4 (lane / 2))
  auto code_word_at = [&](uint32_t p) -> uint32_t {
    const uint32_t b = 16u + 64u * p + 4u * (lane >> 1);
    return *reinterpret_cast<const uint32_t*>(P.pages + (unsigned long long)fw.ipg[b >> 9] * kPage + (b & (kPage - 1u)));
  };
  uint32_t cw_next = code_word_at(0u);
  // the first pass's window; output window cleared; the output pages of header and codes
  fast_issue_window(P, fw.ipg, fw.iwin0, cb, 0u, nbs);
  cp_async_commit();
  for (uint32_t k = lane; k < kWinBlocks; k += 32u) reinterpret_cast<uint4*>(fw.owin)[k] = make_uint4(0u, 0u, 0u, 0u);
  uint32_t onp = 0u;
  bool oom = !wp_grow(P, wp, fw.opg, onp, (16u + cb + kPage - 1u) / kPage);
  __syncwarp();
  ph.mark(0);
  const uint32_t mh = (uint32_t)(trunc_mask(S) >> 32), mhin = (uint32_t)(trunc_mask(Sin) >> 32);
  uint32_t ioff = 0u, ooff = 0u, lead = 0u, prv = 0u, refr = 0u, refi = 0u, nzor = 0u;
  bool spec = false, cst = true, halves = true, lost = false;
  for (uint32_t p = 0; p < NP; ++p) {
    uint32_t* const win = (p & 1u) ? fw.iwin1 : fw.iwin0;
    uint32_t* const wnext = (p & 1u) ? fw.iwin0 : fw.iwin1;
    // residual lengths of this lane's 8 values, their offsets in the pass
    const uint32_t cw = (cw_next >> (16u * (lane & 1u))) & 0xffffu;
    if (p + 1u < NP) cw_next = code_word_at(p + 1u);  // in flight while this pass runs
    uint32_t tot;
    const uint32_t ps = ioff;
    const uint32_t o = ps + warp_excl(rsum8(cw, Sin), tot);
    ioff += tot;
    // the next pass's window is in flight while this pass runs
    if (p + 1u < NP) fast_issue_window(P, fw.ipg, wnext, cb, ioff >> 7, nbs);
    cp_async_commit();
    ph.mark(1);
    cp_async_wait_group<1>();
    __syncwarp();
    ph.mark(0);
    // explicit parts, leading bytes from the predecessors
    uint32_t v[8];
    {
      const uint32_t W = fast_extract(win, 4u * (ps >> 7), o, cw, Sin, mhin, v);
      uint32_t after;
      const uint32_t Pl = lead_scan_warp(W, lead, after);
      lead = after;
      fast_rebuild(v, cw, Pl);
    }
    if constexpr (ARITH == 4) {
      // signed_rows needs every input at least 2^-959 (or zero): each warp checks its own
      // values, and the pair's agreement defers the item if either chunk has one below
#pragma unroll
      for (int k = 0; k < 8; ++k) spec |= ((v[k] & 0x7fffffffu) - 1u) < ((64u << 20) - 1u);  // nonzero, exponent < 64
    }
    ph.mark(1);
    // the gate on every amplitude pair whose in-chunk control bits match; results
    // truncated to S bits in place
    const uint32_t ibase = 128u * p + 4u * lane;  // the lane's first amplitude in the chunk
    uint32_t w[8];                                // the partner amplitudes' high words (kinds 0 and 2)
    if constexpr (KIND == 0 && ARITH != 1) {
      // the partner warp holds the other amplitude of every pair, at the same position
      // (a diagonal gate needs only the amplitude itself)
      uint32_t* xs = fw.xch + 256u * (p & 1u);
      reinterpret_cast<uint4*>(xs)[2u * lane] = make_uint4(v[0], v[1], v[2], v[3]);
      reinterpret_cast<uint4*>(xs)[2u * lane + 1u] = make_uint4(v[4], v[5], v[6], v[7]);
      ++phase;
      if (!lost) lost = !pair_sync(seq, side, phase, P.ctl, 2u);
      const uint32_t* xo = xpeer + 256u * (p & 1u);
      const uint4 w0 = reinterpret_cast<const uint4*>(xo)[2u * lane], w1 = reinterpret_cast<const uint4*>(xo)[2u * lane + 1u];
      w[0] = w0.x; w[1] = w0.y; w[2] = w0.z; w[3] = w0.w; w[4] = w1.x; w[5] = w1.y; w[6] = w1.z; w[7] = w1.w;
    } else if constexpr (KIND == 2) {
      // partner amplitude i ^ 2^t (2 <= t <= 6): the same slot of lane ^ 2^(t-2)
#pragma unroll
      for (int k = 0; k < 8; ++k) w[k] = __shfl_xor_sync(0xffffffffu, v[k], 1u << (L.target - 2));
    }
    if constexpr (KIND == 1) {
      // partner in the lane: amplitudes k and k ^ 2^t, t = 0 or 1
      if (L.target == 0) {
        fast_pair_in_lane<ARITH>(L, ibase, 0, 1, v, mh, spec);
        fast_pair_in_lane<ARITH>(L, ibase, 2, 3, v, mh, spec);
      } else {
        fast_pair_in_lane<ARITH>(L, ibase, 0, 2, v, mh, spec);
        fast_pair_in_lane<ARITH>(L, ibase, 1, 3, v, mh, spec);
      }
    } else {
      // which row pair this lane's amplitudes take: the pair's second amplitude (b) takes
      // rows 2-3 (kind 0: the second warp; kind 2: lanes with bit t - 2 set; kind 3 per
      // amplitude, bit t)
      const uint32_t lane_row = KIND == 0 ? side : (KIND == 2 ? ((lane >> (L.target - 2)) & 1u) : 0u);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t i = ibase + (uint32_t)k;
        const uint32_t row = KIND == 3 ? ((i >> L.target) & 1u) : lane_row;
        const uint32_t i0 = i & ~(1u << (KIND == 0 ? 31u : (uint32_t)L.target));
        uint32_t outr = v[2 * k] & mh, outi = v[2 * k + 1] & mh;  // unchanged amplitude, truncated
        if ((i0 & L.lo_mask) == L.lo_vals) {
          if constexpr (ARITH == 4) {
            const uint32_t ar = row ? w[2 * k] : v[2 * k], ai = row ? w[2 * k + 1] : v[2 * k + 1];
            const uint32_t br = row ? v[2 * k] : w[2 * k], bi = row ? v[2 * k + 1] : w[2 * k + 1];
            signed_rows(L, row, ar, ai, br, bi, mh, outr, outi, spec);
          } else if constexpr (ARITH == 0 || ARITH == 3) {
            // a = the pair's first amplitude, b = its second
            const uint32_t ar = row ? w[2 * k] : v[2 * k], ai = row ? w[2 * k + 1] : v[2 * k + 1];
            const uint32_t br = row ? v[2 * k] : w[2 * k], bi = row ? v[2 * k + 1] : w[2 * k + 1];
            const double2 a = make_double2(hi_as_double(ar), hi_as_double(ai));
            const double2 b = make_double2(hi_as_double(br), hi_as_double(bi));
            const double2 out = ARITH == 0 ? dense_rows(L.cf + 8u * row, a, b) : real_rows(L.cf + 8u * row, a, b);
            outr = fast_trunc(out.x, mh, spec);
            outi = fast_trunc(out.y, mh, spec);
          } else if constexpr (ARITH == 1) {
            row_op(L, row, v[2 * k], v[2 * k + 1], mh, outr, outi, spec);
          } else {
            row_op(L, row, w[2 * k], w[2 * k + 1], mh, outr, outi, spec);
          }
        }
        v[2 * k] = outr;
        v[2 * k + 1] = outi;
      }
    }
    ph.mark(2);
    // encoder: constant-chunk and period filters, codes, output offsets
    if (p == 0u) {
      refr = __shfl_sync(0xffffffffu, v[0], 0);
      refi = __shfl_sync(0xffffffffu, v[1], 0);
    }
    uint32_t pr = __shfl_up_sync(0xffffffffu, v[7], 1);
    if (lane == 0) pr = prv;
    prv = __shfl_sync(0xffffffffu, v[7], 31);
    {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        nzor |= v[k];
        cst &= v[k] == ((k & 1) ? refi : refr);
      }
      // period filter: a chunk with a period below its length equals itself shifted by
      // half a chunk; two values per lane are compared with their partners
      if (NP == 1u) {  // both halves in this pass: lanes 0-15 and 16-31 (every lane shuffles)
        const uint32_t a = __shfl_xor_sync(0xffffffffu, v[0], 16);
        const uint32_t b = __shfl_xor_sync(0xffffffffu, v[5], 16);
        halves &= (a == v[0]) & (b == v[5]);
      } else if (p < NP / 2u) {
        fw.half[32u * p + lane] = v[0] ^ __funnelshift_l(v[5], v[5], 13);
      } else {
        halves &= fw.half[32u * (p - NP / 2u) + lane] == (v[0] ^ __funnelshift_l(v[5], v[5], 13));
      }
    }
    uint32_t osum, otot;
    const uint32_t ocw = fast_codes(v, pr, S, osum);
    const uint32_t ob = ooff >> 7;
    fast_pack(fw.owin, 4u * ob, ooff + warp_excl(osum, otot), v, ocw, S);
    // codes: two lanes fill one 32-bit word
    const uint32_t pairw = ocw | (__shfl_down_sync(0xffffffffu, ocw, 1) << 16);
    if ((lane & 1u) == 0u && !oom) {  // image byte 16 + 64 p + 2 lane
      const uint32_t b = 16u + 64u * p + 2u * lane;
      *reinterpret_cast<uint32_t*>(P.pages + (unsigned long long)fw.opg[b >> 9] * kPage + (b & (kPage - 1u))) = pairw;
    }
    ooff += otot;
    __syncwarp();
    ph.mark(3);
    // finished blocks to the pages (the last pass also its unfinished one, zero-padded)
    const bool last = p + 1u == NP;
    const uint32_t endb = last ? (ooff + 127u) >> 7 : ooff >> 7;
    const uint32_t nb = endb - ob;
    if (!oom) oom = !wp_grow(P, wp, fw.opg, onp, (16u + cb + 16u * endb + kPage - 1u) / kPage);
    const uint4* w4 = reinterpret_cast<const uint4*>(fw.owin);
    if (!oom)
      for (uint32_t k = lane; k < nb; k += 32u) {
        const uint32_t b = 16u + cb + 16u * (ob + k);
        reinterpret_cast<uint4*>(P.pages + (unsigned long long)fw.opg[b >> 9] * kPage + (b & (kPage - 1u)))[0] = w4[k];
      }
    if (!last) {
      uint4 carry = make_uint4(0u, 0u, 0u, 0u);
      if (lane == 0) carry = w4[nb];
      __syncwarp();
      // the unfinished block becomes block 0 of the next pass's window
      uint4* z = reinterpret_cast<uint4*>(fw.owin);
      for (uint32_t k = lane; k <= nb; k += 32u) z[k] = k == 0u ? carry : make_uint4(0u, 0u, 0u, 0u);
      __syncwarp();
    }
    ph.mark(4);
  }
  // every input bit consumed exactly (else the image is corrupt); this chunk a STREAM
  // image unless it is constant or possibly periodic, or holds special values
  const bool corrupt = ioff != bits_in;
  // (every lane takes every vote: a warp-wide primitive must never sit behind a branch)
  const bool any_spec = __any_sync(0xffffffffu, spec), all_cst = __all_sync(0xffffffffu, cst);
  const bool any_nz = __any_sync(0xffffffffu, nzor != 0u), all_halves = __all_sync(0xffffffffu, halves);
  const bool keep = !any_spec && !all_cst && any_nz && !all_halves;
  if (corrupt && lane == 0) atomicOr(&P.ctl->err, (unsigned)E_CORRUPT);
  const uint32_t mine = (keep ? 1u : 0u) | ((corrupt || oom || lost) ? 2u : 0u);
  const uint32_t other = lost ? 2u : pair_agree(slots, seq, phase, side, mine, P.ctl, 3u);
  if (((mine | other) & 2u) || !((mine & other) & 1u)) {
    wp_free(P, wp, fw.opg, onp);
    cp_async_wait_all();
    __syncwarp();
    return ((mine | other) & 2u) ? 2 : 1;
  }
  // the header, then the directory entry; the old pages freed
  const uint32_t plen = cb + resid_bytes(ooff), bytes = 16u + plen;
  if (lane == 0)
    reinterpret_cast<uint4*>(P.pages + (unsigned long long)fw.opg[0] * kPage)[0] = make_uint4(M_STREAM | (S << 8), plen, N, ooff);
  uint32_t* e = dir_entry(P, ch);
  for (uint32_t k = lane; k < onp; k += 32u) e[4 + k] = fw.opg[k];
  if (lane == 0) {
    e[0] = bytes;
    e[1] = onp;
    dE += (long long)bytes - (long long)ib;
    rd += ib;
    wr += bytes;
  }
  wp_free(P, wp, fw.ipg, inp);
  ph.mark(4);
  return 0;
}

template <int KIND, int ARITH>
__global__ void __launch_bounds__(kFastThreads, QC_FAST_MIN_CTAS) k_gate_fast(const __grid_constant__ GateLaunch L) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_slots[kFastPairs][4];
  __shared__ uint32_t s_seq[kFastPairs][2];
  const int kc = L.P.kc;
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const uint32_t pr = wid >> 1, side = wid & 1u;
  if (threadIdx.x < 2u * kFastPairs) s_seq[threadIdx.x >> 1][threadIdx.x & 1u] = 0u;
  __syncthreads();  // the only CTA-wide barrier: every sequence number starts at 0
  DevCtl* ctl = L.P.ctl;
  const uint32_t S = gate_bits(L);
  if (S > 32u) {  // lossless or wide values: the general kernel takes the whole gate
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->fast_all = 1u;
    return;
  }
  uint8_t* wb = smem + (size_t)wid * fast_warp_bytes(kc);
  const FastWarp fw = fast_warp(wb, kc);
  const uint32_t* xpeer = fast_warp(smem + (size_t)(wid ^ 1u) * fast_warp_bytes(kc), kc).xch;
  // the warp's page cache, kept in global memory between launches
  WarpPages wp;
  wp.ids = fw.xch + 512u;
  wp.n = wp.ids + kWarpCache;
  const size_t gw = (size_t)blockIdx.x * kFastWarps + wid;
  const uint32_t n_start = L.P.wcache_n[gw];
  {
    const uint32_t n = n_start;
    for (uint32_t q = lane; q < n; q += 32u) wp.ids[q] = L.P.wcache[gw * kWarpCache + q];
    if (lane == 0) *wp.n = n;
    __syncwarp();
  }
  uint32_t phase = 0;
  __shared__ long long s_ph[kFastWarps][6];
  FastPhases ph;
  ph.t = s_ph[wid];
  ph.on = L.prof && lane == 0;
  if (ph.on) {
    for (int k = 0; k < 5; ++k) ph.t[k] = 0;
    ph.t[5] = clock64();
  }
  long long dE = 0;
  unsigned long long rd = 0, wr = 0, done = 0, deferred = 0;
  const unsigned long long pairs = (unsigned long long)gridDim.x * kFastPairs;
  for (unsigned long long item = (unsigned long long)blockIdx.x * kFastPairs + pr; item < L.items; item += pairs) {
    const int r = fast_item<KIND, ARITH>(L, item, S, fw, xpeer, wp, side, s_seq[pr], s_slots[pr], phase, dE, rd, wr, ph);
    if (r == 2) break;
    if (r == 1) {
      if (side == 0 && lane == 0) {
        const unsigned long long k = atomicAdd(&ctl->ndefer, 1ull);
        L.defer[k] = (uint32_t)item;
        ++deferred;
      }
    } else if (side == 0) {
      ++done;
    }
  }
  cp_async_wait_all();
  __syncwarp();
  // the warp's cached pages stay with it for the next launch
  {
    const uint32_t n = *wp.n;
    for (uint32_t q = lane; q < n; q += 32u) L.P.wcache[gw * kWarpCache + q] = wp.ids[q];
    if (lane == 0) {
      L.P.wcache_n[gw] = n;
      if (n != n_start) atomicAdd(&ctl->wc_pages, (unsigned long long)((long long)n - (long long)n_start));
    }
  }
  if (lane == 0) {
    if (dE) atomicAdd(&ctl->dE, (unsigned long long)dE);
    if (rd) atomicAdd(&ctl->bytes_in, rd);
    if (wr) atomicAdd(&ctl->bytes_out, wr);
    if (done) atomicAdd(&ctl->fast_items, done);
    if (deferred) atomicAdd(&ctl->fast_deferred, deferred);
    if (ph.on)
      for (int k = 0; k < 5; ++k)
        if (ph.t[k]) atomicAdd(&ctl->phase_cycles[k], (unsigned long long)ph.t[k]);
  }
}

// ------------------------------------------------------------- launchers -- //
template <typename K>
static cudaError_t prep_fast(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

size_t fast_smem_bytes(int kc) { return (size_t)kFastWarps * fast_warp_bytes(kc); }
int fast_warps() { return kFastWarps; }
int fast_pairs() { return kFastPairs; }
int fast_warp_cache() { return (int)kWarpCache; }

int fast_ctas_per_sm(int kc) {
  int n = 0;
  const size_t smem = fast_smem_bytes(kc);
  prep_fast(k_gate_fast<0, 0>, smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gate_fast<0, 0>, kFastThreads, smem) != cudaSuccess || n < 1)
    n = 1;
  return n;
}

template <int KIND, int ARITH>
static cudaError_t launch_fast_as(const GateLaunch& L, int grid, size_t smem, cudaStream_t st) {
  const cudaError_t e = prep_fast(k_gate_fast<KIND, ARITH>, smem);
  if (e != cudaSuccess) return e;
  k_gate_fast<KIND, ARITH><<<grid, kFastThreads, smem, st>>>(L);
  return cudaGetLastError();
}

// Kinds and arithmetic forms that occur: cross-chunk pairs of any gate class, in-chunk
// partners of dense, real, power-of-two or anti-diagonal gates, in-chunk diagonal gates.
cudaError_t launch_gate_fast(const GateLaunch& L, int grid, cudaStream_t st) {
  const size_t smem = fast_smem_bytes(L.P.kc);
  switch (L.fast_kind * 8 + L.arith) {
    case 0: return launch_fast_as<0, 0>(L, grid, smem, st);
    case 1: return launch_fast_as<0, 1>(L, grid, smem, st);
    case 2: return launch_fast_as<0, 2>(L, grid, smem, st);
    case 3: return launch_fast_as<0, 3>(L, grid, smem, st);
    case 4: return launch_fast_as<0, 4>(L, grid, smem, st);
    case 8: return launch_fast_as<1, 0>(L, grid, smem, st);
    case 10: return launch_fast_as<1, 2>(L, grid, smem, st);
    case 11: return launch_fast_as<1, 3>(L, grid, smem, st);
    case 12: return launch_fast_as<1, 4>(L, grid, smem, st);
    case 16: return launch_fast_as<2, 0>(L, grid, smem, st);
    case 18: return launch_fast_as<2, 2>(L, grid, smem, st);
    case 19: return launch_fast_as<2, 3>(L, grid, smem, st);
    case 20: return launch_fast_as<2, 4>(L, grid, smem, st);
    case 25: return launch_fast_as<3, 1>(L, grid, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qc
