/*
 * qc_oracle.c -- CPU oracle for compressed full-state quantum circuit simulation
 * (Wu et al., "Full-State Quantum Circuit Simulation by Using Data Compression", SC'19).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this file: it is used by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline leg of bench.py.  It shares no code, header, table or helper with the
 * CUDA library; the only thing both sides see is the seeded circuit description.
 *
 * Plain, slow, sequential fp64 C.  Compiled with -ffp-contract=off so that every
 * product and every fma below is exactly the operation written.
 *
 * Contents
 *   1. Bit-plane truncation (Section 4.2, Solution C, Eq. sigbits; interval of Section 3.7)
 *   2. XOR leading-zero coding with a 2-bit code (Section 4.2, Solution C, step 1)
 *   3. Chunk image format: modes ZERO/CONST/PERIOD/STREAM/RAW standing in for the
 *      Zstd stage (Section 3.7 lossless stage, Section 4.2 Solution C step 3)
 *   4. Gate application on amplitude pairs (Section 3.1, Eq. matrix1 and Eq. matrix2)
 *   5. Uncompressed state vector simulator (Section 2.1, Eq. 2nrep / Eq. psi)
 *   6. Compressed simulator: decode -> apply -> encode per work item, with the
 *      per-timestep error-bound controller (Section 3.1, Eq. totalnbBytes; Section 3.7)
 *   7. Fidelity (Section 3.8, Eq. idealsim) and its lower bounds
 *   8. Measurement sampling
 *
 * Every function returns ORC_OK (0) or a negative ORC_ERR_* code.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_CORRUPT (-4)
#define ORC_ERR_STATE (-6)

#define ORC_MODE_ZERO 0
#define ORC_MODE_CONST 1
#define ORC_MODE_PERIOD 2
#define ORC_MODE_STREAM 3
#define ORC_MODE_RAW 4
#define ORC_MODE_SPLIT 5
#define ORC_MODE_PALETTE 6
#define ORC_NMODES 7
#define ORC_DEFAULT_MODES 0x1F /* Solution C: ZERO..RAW; SPLIT (Solution D) and PALETTE on request */
#define ORC_PALETTE_MAX 256    /* most distinct values a PALETTE image lists */

/* Planted-mistake switch used only by the mutation tests: each nonzero value
 * introduces one plausible bug so the tests can show that some pin catches it. */
static int g_mutant = 0;
void orc_set_mutant(int m) { g_mutant = m; }

/* ------------------------------------------------------------------------- */
/* 1. Bit-plane truncation                                                    */
/* ------------------------------------------------------------------------- */

/* EXP(eps): the exponent of eps in its IEEE-754 binary64 representation
 * (Section 4.2, Eq. sigbits; the paper's example is EXP(0.01) = -7). */
int orc_exp_of(double eps) {
  uint64_t b;
  memcpy(&b, &eps, 8);
  int field = (int)((b >> 52) & 0x7ff);
  return field - 1023;
}

/* Sig_Bit_Count = Bit_Count(Sign&Exp) - EXP(eps), with 12 sign+exponent bits for
 * binary64 (Eq. sigbits).  eps == 0 selects the lossless stage: all 64 bits.
 * Valid lossy bounds are normal doubles in [2^-52, 1); others are rejected. */
int orc_sig_bits(double eps) {
  if (eps == 0.0) return 64;
  if (!(eps > 0.0) || !(eps < 1.0)) return ORC_ERR_INVALID;
  int e = orc_exp_of(eps);
  if (e < -52) return ORC_ERR_INVALID;
  int s = 12 - e;
  if (g_mutant == 1) s = 12 - e - 1; /* mutant: one bit too few (the worked example's count) */
  return s > 64 ? 64 : s;
}

/* Keep the S leading bits (sign, exponent, S-12 mantissa bits) and zero the rest:
 * truncation toward zero, so |t| <= |x| and |x - t| < 2^(12-S) |x| for a normal x,
 * which is the interval (|D(1-delta)|, |D|] of Section 3.7.  A negative zero is
 * stored as +0 (equal value; the paper is silent on signed zeros). */
uint64_t orc_truncate(uint64_t bits, int S) {
  uint64_t t = bits;
  if (S < 64) {
    int drop = 64 - S;
    if (g_mutant == 2) drop = drop + 1; /* mutant: drops one kept bit */
    t = bits & ~((((uint64_t)1) << drop) - 1);
  }
  if (t == 0x8000000000000000ull) t = 0;
  return t;
}

/* ------------------------------------------------------------------------- */
/* 2. XOR leading-zero coding (Solution C step 1)                             */
/* ------------------------------------------------------------------------- */

/* Number of identical leading bytes of a and its predecessor p (0..8). */
static int leading_equal_bytes(uint64_t a, uint64_t p) {
  uint64_t d = a ^ p;
  int n = 0;
  for (int k = 7; k >= 0; --k) {
    if (((d >> (8 * k)) & 0xff) != 0) break;
    n++;
  }
  return n;
}

/* The 2-bit code: c = min(identical leading bytes, 3). */
static int xor_code(uint64_t v, uint64_t prev) {
  int L = leading_equal_bytes(v, prev);
  if (g_mutant == 3) return L < 2 ? L : 2; /* mutant: caps the code at 2 */
  return L < 3 ? L : 3;
}

/* Residual length: the significant bits that the leading bytes did not cover. */
static int residual_len(int c, int S) {
  int r = S - 8 * c;
  return r > 0 ? r : 0;
}

/* Bit writer over 64-bit words, most significant bit first. */
typedef struct { uint64_t* w; size_t nwords; uint64_t pos; } bitw;

static void bw_put(bitw* b, uint64_t val, int r) {
  if (r == 0) return;
  size_t wi = (size_t)(b->pos >> 6);
  int off = (int)(b->pos & 63);
  if (off + r <= 64) {
    b->w[wi] |= val << (64 - off - r);
  } else {
    b->w[wi] |= val >> (off + r - 64);
    b->w[wi + 1] |= val << (128 - off - r);
  }
  b->pos += (uint64_t)r;
}

static uint64_t bw_get(const uint64_t* w, uint64_t pos, int r) {
  if (r == 0) return 0;
  size_t wi = (size_t)(pos >> 6);
  int off = (int)(pos & 63);
  uint64_t hi = w[wi] << off; /* first bit now at bit 63 */
  if (off + r > 64) hi |= w[wi + 1] >> (64 - off);
  return hi >> (64 - r);
}

/* ------------------------------------------------------------------------- */
/* 3. Chunk image                                                             */
/* ------------------------------------------------------------------------- */
/*
 * A chunk holds 2^kc amplitudes = N = 2^(kc+1) binary64 values in the order
 * re0, im0, re1, im1, ...  Its image is a 16-byte header then a payload whose
 * length is a multiple of 16 bytes.
 *   header: [0] mode  [1] S (0 for ZERO)  [2] log2 period P in amplitudes (PERIOD)
 *           [3] flags = 0   [4..7] payload bytes   [8..11] coded values
 *           [12..15] residual bits   (all little-endian)
 *   ZERO   : every truncated value is +0; no payload.
 *   CONST  : every amplitude equals amplitude 0; payload = its two values (16 B).
 *   PERIOD : smallest power of two P, 2 <= P < 2^kc, with amp[i] == amp[i-P] for all
 *            i >= P; payload = XOR coding of the first 2P values.
 *   STREAM : XOR coding of all N values.
 *   RAW    : the N truncated values verbatim.
 *   SPLIT  : Solution D (Section 4.2): the real parts of all amplitudes, then the
 *            imaginary parts, XOR-coded like STREAM (enabled by a mode mask).
 *   PALETTE: the lossless stage's dictionary part (the role Section 3.7 gives Zstd on
 *            few-valued states): the P <= 256 distinct truncated values, ascending as
 *            unsigned 64-bit integers, 8 bytes each, padded to 16 bytes; then every value's
 *            index in that list in k = max(1, ceil(log2 P)) bits, MSB first in 64-bit
 *            little-endian words like the residual stream, padded to 16 bytes.  Header
 *            byte 2 = k, coded values = N, bytes 12..15 = P (enabled by a mode mask).
 * XOR coding layout: the 2-bit codes, four per byte with the first code in the top
 * two bits, padded to 16 bytes; then the residual bit stream in 64-bit
 * little-endian words, first bit = bit 63 of word 0, padded to 16 bytes.
 * The smallest image wins; ties go to the lower mode number.
 */

static size_t pad16(size_t x) { return (x + 15) & ~(size_t)15; }
static size_t codes_area(size_t nv) { return pad16((nv + 3) / 4); }
static size_t resid_area(uint64_t bits) { return (size_t)((bits + 127) / 128) * 16; }

static void put_u32(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
static uint32_t get_u32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static void put_u64(uint8_t* p, uint64_t v) {
  for (int k = 0; k < 8; ++k) p[k] = (uint8_t)(v >> (8 * k));
}
static uint64_t get_u64(const uint8_t* p) {
  uint64_t v = 0;
  for (int k = 0; k < 8; ++k) v |= (uint64_t)p[k] << (8 * k);
  return v;
}

/* Total residual bits of the XOR coding of t[0..nv). */
static uint64_t xor_bits(const uint64_t* t, size_t nv, int S) {
  uint64_t bits = 0, prev = 0;
  for (size_t j = 0; j < nv; ++j) {
    bits += (uint64_t)residual_len(xor_code(t[j], prev), S);
    prev = t[j];
  }
  return bits;
}

/* Writes codes + residual stream of t[0..nv) into payload p (zeroed by caller). */
static void xor_write(const uint64_t* t, size_t nv, int S, uint8_t* p, uint64_t bits) {
  size_t ca = codes_area(nv);
  size_t nwords = resid_area(bits) / 8;
  uint64_t* w = (uint64_t*)calloc(nwords + 1, 8);
  bitw b = {w, nwords, 0};
  uint64_t prev = 0;
  for (size_t j = 0; j < nv; ++j) {
    int c = xor_code(t[j], prev);
    int r = residual_len(c, S);
    p[j >> 2] |= (uint8_t)(c << (6 - 2 * (int)(j & 3)));
    if (r > 0) bw_put(&b, (t[j] << (8 * c)) >> (64 - r), r);
    prev = t[j];
  }
  for (size_t k = 0; k < nwords; ++k) put_u64(p + ca + 8 * k, w[k]);
  free(w);
}

/* Reads nv values; checks that the residual bits add up. */
static int xor_read(const uint8_t* p, size_t plen, size_t nv, int S, uint64_t bits, uint64_t* out) {
  size_t ca = codes_area(nv);
  size_t ra = resid_area(bits);
  if (ca + ra != plen) return ORC_ERR_CORRUPT;
  size_t nwords = ra / 8;
  uint64_t* w = (uint64_t*)calloc(nwords + 1, 8);
  for (size_t k = 0; k < nwords; ++k) w[k] = get_u64(p + ca + 8 * k);
  uint64_t pos = 0, prev = 0;
  int rc = ORC_OK;
  for (size_t j = 0; j < nv; ++j) {
    int c = (p[j >> 2] >> (6 - 2 * (int)(j & 3))) & 3;
    int r = residual_len(c, S);
    if (pos + (uint64_t)r > bits) { rc = ORC_ERR_CORRUPT; break; }
    uint64_t e = bw_get(w, pos, r);
    pos += (uint64_t)r;
    uint64_t explicit_bits = r ? ((e << (64 - r)) >> (8 * c)) : 0;
    uint64_t top = c ? (~(uint64_t)0) << (64 - 8 * c) : 0;
    uint64_t v = (prev & top) | explicit_bits;
    out[j] = v;
    prev = v;
  }
  if (rc == ORC_OK && pos != bits) rc = ORC_ERR_CORRUPT;
  free(w);
  return rc;
}

/* Chunk-wide significant bit count: a nonzero subnormal anywhere forces 64 bits
 * (truncating a subnormal would not keep the relative bound).  Non-finite -> error. */
int orc_chunk_sig_bits(const uint64_t* v, size_t nv, int S) {
  int s = S;
  for (size_t j = 0; j < nv; ++j) {
    uint64_t e = (v[j] >> 52) & 0x7ff;
    if (e == 0x7ff) return ORC_ERR_INVALID;
    if (e == 0 && (v[j] & 0x000fffffffffffffull) != 0) s = 64;
  }
  return s;
}

/* Smallest power-of-two period p = log2 P in [1, kc) (amplitudes), or -1. */
static int find_period(const uint64_t* t, int kc) {
  size_t A = (size_t)1 << kc;
  for (int p = 1; p < kc; ++p) {
    size_t P = (size_t)1 << p;
    int ok = 1;
    for (size_t i = P; i < A && ok; ++i)
      if (t[2 * i] != t[2 * (i - P)] || t[2 * i + 1] != t[2 * (i - P) + 1]) ok = 0;
    if (ok) return p;
  }
  return -1;
}

/* Solution D order: u[k] = re of amplitude k for k < 2^kc, then the imaginary parts. */
static void split_order(const uint64_t* t, int kc, uint64_t* u) {
  size_t A = (size_t)1 << kc;
  for (size_t k = 0; k < A; ++k) {
    u[k] = t[2 * k];
    u[A + k] = t[2 * k + 1];
  }
}

static int cmp_u64(const void* a, const void* b) {
  const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* The distinct values of t[0..N), ascending, into pal (room for ORC_PALETTE_MAX);
 * returns how many there are, or ORC_PALETTE_MAX + 1 if there are more. */
static int palette_of(const uint64_t* t, size_t N, uint64_t* pal) {
  uint64_t* s = (uint64_t*)malloc(N * 8);
  memcpy(s, t, N * 8);
  qsort(s, N, 8, cmp_u64);
  int P = 0;
  for (size_t j = 0; j < N; ++j) {
    if (j > 0 && s[j] == s[j - 1]) continue;
    if (P == ORC_PALETTE_MAX) { free(s); return ORC_PALETTE_MAX + 1; }
    pal[P++] = s[j];
  }
  free(s);
  return P;
}

/* Index width of a palette of P entries: the smallest k >= 1 with 2^k >= P. */
static int palette_bits(int P) {
  int k = 1;
  while ((1 << k) < P) ++k;
  return k;
}

/* Position of v in pal[0..P) (v is in it). */
static int palette_index(const uint64_t* pal, int P, uint64_t v) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (pal[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

/* Size in bytes of the image in mode m, or 0 if m does not apply. */
static size_t mode_size(int m, const uint64_t* t, int kc, int S, int period) {
  size_t N = (size_t)2 << kc;
  switch (m) {
    case ORC_MODE_ZERO:
      for (size_t j = 0; j < N; ++j) if (t[j] != 0) return 0;
      return 16;
    case ORC_MODE_CONST:
      for (size_t j = 2; j < N; j += 2) if (t[j] != t[0] || t[j + 1] != t[1]) return 0;
      return 32;
    case ORC_MODE_PERIOD: {
      if (period < 0) return 0;
      size_t nv = (size_t)2 << period;
      return 16 + codes_area(nv) + resid_area(xor_bits(t, nv, S));
    }
    case ORC_MODE_STREAM:
      return 16 + codes_area(N) + resid_area(xor_bits(t, N, S));
    case ORC_MODE_RAW:
      return 16 + 8 * N;
    case ORC_MODE_SPLIT: {
      uint64_t* u = (uint64_t*)malloc(N * 8);
      split_order(t, kc, u);
      size_t sz = 16 + codes_area(N) + resid_area(xor_bits(u, N, S));
      free(u);
      return sz;
    }
    case ORC_MODE_PALETTE: {
      uint64_t pal[ORC_PALETTE_MAX];
      int P = palette_of(t, N, pal);
      if (P > ORC_PALETTE_MAX) return 0;
      return 16 + pad16(8 * (size_t)P) + resid_area((uint64_t)N * (uint64_t)palette_bits(P));
    }
  }
  return 0;
}

/* Size of the image the encoder would write for each mode (0 = not applicable).
 * Inputs are the raw bit patterns of the N values. */
int orc_mode_sizes(const uint64_t* x, int kc, int S_req, uint64_t* sizes_out) {
  size_t N = (size_t)2 << kc;
  int S = orc_chunk_sig_bits(x, N, S_req);
  if (S < 0) return S;
  uint64_t* t = (uint64_t*)malloc(N * 8);
  for (size_t j = 0; j < N; ++j) t[j] = orc_truncate(x[j], S);
  int period = find_period(t, kc);
  for (int m = 0; m < ORC_NMODES; ++m) sizes_out[m] = mode_size(m, t, kc, S, period);  /* 7 entries */
  free(t);
  return ORC_OK;
}

/* Encode one chunk (raw bit patterns x[0..N)) with requested bits S_req.
 * force_mode >= 0 selects that mode; otherwise the smallest image among the modes
 * whose bit is set in mode_mask (ties: lower mode number).  Returns the image length
 * or an error. */
long orc_encode_chunk_mask(const uint64_t* x, int kc, int S_req, int force_mode, unsigned mode_mask, uint8_t* out,
                           size_t cap) {
  if (kc < 0 || kc > 20) return ORC_ERR_INVALID;
  if (S_req < 13 || S_req > 64) return ORC_ERR_INVALID;
  size_t N = (size_t)2 << kc;
  int S = orc_chunk_sig_bits(x, N, S_req);
  if (S < 0) return S;
  uint64_t* t = (uint64_t*)malloc(N * 8);
  for (size_t j = 0; j < N; ++j) t[j] = orc_truncate(x[j], S);
  int period = find_period(t, kc);
  size_t best = 0;
  int mode = -1;
  if (force_mode >= 0) {
    if (force_mode >= ORC_NMODES) { free(t); return ORC_ERR_INVALID; }
    best = mode_size(force_mode, t, kc, S, period);
    mode = force_mode;
    if (best == 0) { free(t); return ORC_ERR_INVALID; }
  } else {
    for (int m = 0; m < ORC_NMODES; ++m) {
      if (!((mode_mask >> m) & 1u)) continue;
      size_t sz = mode_size(m, t, kc, S, period);
      if (sz != 0 && (mode < 0 || sz < best)) { best = sz; mode = m; }
    }
    if (mode < 0) { free(t); return ORC_ERR_INVALID; }
  }
  if (best > cap) { free(t); return ORC_ERR_INVALID; }
  memset(out, 0, best);
  uint8_t* p = out + 16;
  uint32_t nv = 0;
  uint64_t bits = 0;
  out[0] = (uint8_t)mode;
  out[1] = (uint8_t)(mode == ORC_MODE_ZERO ? 0 : S);
  out[2] = (uint8_t)(mode == ORC_MODE_PERIOD ? period : 0);
  out[3] = 0;
  switch (mode) {
    case ORC_MODE_ZERO: break;
    case ORC_MODE_CONST:
      nv = 2;
      put_u64(p, t[0]);
      put_u64(p + 8, t[1]);
      break;
    case ORC_MODE_PERIOD:
    case ORC_MODE_STREAM:
      nv = (uint32_t)(mode == ORC_MODE_PERIOD ? ((size_t)2 << period) : N);
      bits = xor_bits(t, nv, S);
      xor_write(t, nv, S, p, bits);
      break;
    case ORC_MODE_RAW:
      nv = (uint32_t)N;
      for (size_t j = 0; j < N; ++j) put_u64(p + 8 * j, t[j]);
      break;
    case ORC_MODE_SPLIT: {
      uint64_t* u = (uint64_t*)malloc(N * 8);
      split_order(t, kc, u);
      nv = (uint32_t)N;
      bits = xor_bits(u, N, S);
      xor_write(u, N, S, p, bits);
      free(u);
      break;
    }
    case ORC_MODE_PALETTE: {
      uint64_t pal[ORC_PALETTE_MAX];
      const int P = palette_of(t, N, pal), k = palette_bits(P);
      const size_t pa = pad16(8 * (size_t)P), nwords = resid_area((uint64_t)N * (uint64_t)k) / 8;
      for (int i = 0; i < P; ++i) put_u64(p + 8 * i, pal[i]);
      uint64_t* w = (uint64_t*)calloc(nwords + 1, 8);
      bitw b = {w, nwords, 0};
      for (size_t j = 0; j < N; ++j) bw_put(&b, (uint64_t)palette_index(pal, P, t[j]), k);
      for (size_t q = 0; q < nwords; ++q) put_u64(p + pa + 8 * q, w[q]);
      free(w);
      out[2] = (uint8_t)k;
      nv = (uint32_t)N;
      bits = (uint64_t)P;  /* bytes 12..15 hold the palette size */
      break;
    }
  }
  put_u32(out + 4, (uint32_t)(best - 16));
  put_u32(out + 8, nv);
  put_u32(out + 12, (uint32_t)bits);
  free(t);
  return (long)best;
}

long orc_encode_chunk(const uint64_t* x, int kc, int S_req, int force_mode, uint8_t* out, size_t cap) {
  return orc_encode_chunk_mask(x, kc, S_req, force_mode, ORC_DEFAULT_MODES, out, cap);
}

/* Decode an image into N raw bit patterns. */
int orc_decode_chunk(const uint8_t* img, size_t len, int kc, uint64_t* out) {
  if (len < 16 || kc < 0 || kc > 20) return ORC_ERR_CORRUPT;
  size_t N = (size_t)2 << kc;
  int mode = img[0], S = img[1], lp = img[2];
  uint32_t plen = get_u32(img + 4), nv = get_u32(img + 8), bits = get_u32(img + 12);
  if (img[3] != 0 || (size_t)plen + 16 != len || (plen & 15) != 0) return ORC_ERR_CORRUPT;
  if (mode != ORC_MODE_ZERO && (S < 13 || S > 64)) return ORC_ERR_CORRUPT;
  const uint8_t* p = img + 16;
  switch (mode) {
    case ORC_MODE_ZERO:
      if (S != 0 || lp != 0 || plen != 0 || nv != 0 || bits != 0) return ORC_ERR_CORRUPT;
      memset(out, 0, N * 8);
      return ORC_OK;
    case ORC_MODE_CONST:
      if (lp != 0 || plen != 16 || nv != 2 || bits != 0) return ORC_ERR_CORRUPT;
      for (size_t j = 0; j < N; j += 2) { out[j] = get_u64(p); out[j + 1] = get_u64(p + 8); }
      return ORC_OK;
    case ORC_MODE_PERIOD: {
      if (lp < 1 || lp >= kc || nv != ((uint32_t)2 << lp)) return ORC_ERR_CORRUPT;
      int rc = xor_read(p, plen, nv, S, bits, out);
      if (rc) return rc;
      for (size_t j = nv; j < N; ++j) out[j] = out[j - nv];
      return ORC_OK;
    }
    case ORC_MODE_STREAM:
      if (lp != 0 || nv != N) return ORC_ERR_CORRUPT;
      return xor_read(p, plen, nv, S, bits, out);
    case ORC_MODE_RAW:
      if (lp != 0 || nv != N || bits != 0 || plen != 8 * N) return ORC_ERR_CORRUPT;
      for (size_t j = 0; j < N; ++j) out[j] = get_u64(p + 8 * j);
      return ORC_OK;
    case ORC_MODE_PALETTE: {
      /* lp = k, bits = P; the list strictly ascending, every index inside it */
      const uint32_t P = bits;
      if (nv != N || P < 1 || P > ORC_PALETTE_MAX || lp != palette_bits((int)P)) return ORC_ERR_CORRUPT;
      const size_t pa = pad16(8 * (size_t)P), ia = resid_area((uint64_t)N * (uint64_t)lp);
      if (pa + ia != plen) return ORC_ERR_CORRUPT;
      uint64_t pal[ORC_PALETTE_MAX];
      for (uint32_t i = 0; i < P; ++i) {
        pal[i] = get_u64(p + 8 * i);
        if (i > 0 && pal[i] <= pal[i - 1]) return ORC_ERR_CORRUPT;
      }
      uint64_t* w = (uint64_t*)calloc(ia / 8 + 1, 8);
      for (size_t q = 0; q < ia / 8; ++q) w[q] = get_u64(p + pa + 8 * q);
      int rc = ORC_OK;
      for (size_t j = 0; j < N; ++j) {
        const uint64_t ix = bw_get(w, (uint64_t)j * (uint64_t)lp, lp);
        if (ix >= P) { rc = ORC_ERR_CORRUPT; break; }
        out[j] = pal[ix];
      }
      free(w);
      return rc;
    }
    case ORC_MODE_SPLIT: {
      if (lp != 0 || nv != N) return ORC_ERR_CORRUPT;
      uint64_t* u = (uint64_t*)malloc(N * 8);
      int rc = xor_read(p, plen, nv, S, bits, u);
      size_t A = N / 2;
      if (!rc)
        for (size_t k = 0; k < A; ++k) {
          out[2 * k] = u[k];
          out[2 * k + 1] = u[A + k];
        }
      free(u);
      return rc;
    }
  }
  return ORC_ERR_CORRUPT;
}

/* ------------------------------------------------------------------------- */
/* 4. Gate application (Eq. matrix1, Eq. matrix2)                             */
/* ------------------------------------------------------------------------- */

typedef struct {
  int32_t target;
  int32_t kind; /* caller's hint; the oracle ignores it */
  uint64_t ctrl_mask;
  uint64_t ctrl_vals;
  double u[8]; /* u00r u00i u01r u01i u10r u10i u11r u11i */
} orc_gate;

/* One real component of a complex 2x2 row times (a, b): the sum of four products,
 * taken in the order written; a product whose coefficient is exactly zero is left
 * out, the first kept product is rounded once and each later one is added with a
 * single fused multiply-add.  With no product kept the result is +0. */
static double row_sum(double c1, double x1, double c2, double x2, double c3, double x3, double c4, double x4) {
  double cs[4] = {c1, c2, c3, c4}, xs[4] = {x1, x2, x3, x4};
  double acc = 0.0;
  int have = 0;
  for (int k = 0; k < 4; ++k) {
    if (cs[k] == 0.0) continue;
    if (!have) { acc = cs[k] * xs[k]; have = 1; }
    else acc = fma(cs[k], xs[k], acc);
  }
  return acc;
}

/* (a, b) <- U (a, b) for one amplitude pair: a has bit t = 0, b has bit t = 1. */
static void apply_pair(const double* u, double* a, double* b) {
  double ar = a[0], ai = a[1], br = b[0], bi = b[1];
  double u00r = u[0], u00i = u[1], u01r = u[2], u01i = u[3];
  double u10r = u[4], u10i = u[5], u11r = u[6], u11i = u[7];
  if (g_mutant == 4) { double s = u01r; u01r = u10r; u10r = s; s = u01i; u01i = u10i; u10i = s; } /* mutant: U transposed */
  if (g_mutant == 5) u01i = -u01i; /* mutant: wrong sign */
  a[0] = row_sum(u00r, ar, -u00i, ai, u01r, br, -u01i, bi);
  a[1] = row_sum(u00r, ai, u00i, ar, u01r, bi, u01i, br);
  b[0] = row_sum(u10r, ar, -u10i, ai, u11r, br, -u11i, bi);
  b[1] = row_sum(u10r, ai, u10i, ar, u11r, bi, u11i, br);
  if (g_mutant == 6) b[1] = row_sum(u10r, ai, u10i, ar, u11r, bi, 0.0, br); /* mutant: dropped term */
}

/* Gate checks: target in range, controls inside the register and not on the
 * target, control values inside the mask, finite entries, and U^H U = I within 1e-12. */
int orc_gate_check(const orc_gate* g, int n) {
  if (g->target < 0 || g->target >= n) return ORC_ERR_INVALID;
  uint64_t all = (n >= 64) ? ~(uint64_t)0 : ((((uint64_t)1) << n) - 1);
  if (g->ctrl_mask & ~all) return ORC_ERR_INVALID;
  if ((g->ctrl_mask >> g->target) & 1) return ORC_ERR_INVALID;
  if (g->ctrl_vals & ~g->ctrl_mask) return ORC_ERR_INVALID;
  for (int k = 0; k < 8; ++k) if (!isfinite(g->u[k])) return ORC_ERR_INVALID;
  /* columns of U: c0 = (u00, u10), c1 = (u01, u11) */
  double c0r[2] = {g->u[0], g->u[4]}, c0i[2] = {g->u[1], g->u[5]};
  double c1r[2] = {g->u[2], g->u[6]}, c1i[2] = {g->u[3], g->u[7]};
  double n0 = 0, n1 = 0, dr = 0, di = 0;
  for (int k = 0; k < 2; ++k) {
    n0 += c0r[k] * c0r[k] + c0i[k] * c0i[k];
    n1 += c1r[k] * c1r[k] + c1i[k] * c1i[k];
    dr += c0r[k] * c1r[k] + c0i[k] * c1i[k]; /* <c0|c1> */
    di += c0r[k] * c1i[k] - c0i[k] * c1r[k];
  }
  if (fabs(n0 - 1.0) > 1e-12 || fabs(n1 - 1.0) > 1e-12 || fabs(dr) > 1e-12 || fabs(di) > 1e-12) return ORC_ERR_INVALID;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* 5. Uncompressed state vector (interleaved re, im; index bit k = qubit k)   */
/* ------------------------------------------------------------------------- */

void orc_sv_init(double* psi, int n) {
  size_t A = (size_t)1 << n;
  memset(psi, 0, 2 * A * sizeof(double));
  psi[0] = 1.0;
}

int orc_sv_apply(double* psi, int n, const orc_gate* g) {
  int rc = orc_gate_check(g, n);
  if (rc) return rc;
  size_t A = (size_t)1 << n, tb = (size_t)1 << g->target;
  for (size_t i = 0; i < A; ++i) {
    if (i & tb) continue;
    if ((i & g->ctrl_mask) != g->ctrl_vals) continue;
    apply_pair(g->u, psi + 2 * i, psi + 2 * (i | tb));
  }
  return ORC_OK;
}

int orc_sv_run(double* psi, int n, const orc_gate* gates, size_t ng) {
  for (size_t k = 0; k < ng; ++k) {
    int rc = orc_sv_apply(psi, n, gates + k);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* Sum of |a_i|^2 in index order (Eq. psi), each term fma(re, re, im*im). */
double orc_sv_norm2(const double* psi, int n) {
  size_t A = (size_t)1 << n;
  double s = 0.0;
  for (size_t i = 0; i < A; ++i) s += fma(psi[2 * i], psi[2 * i], psi[2 * i + 1] * psi[2 * i + 1]);
  return s;
}

/* <x|y> = sum conj(x_i) y_i in index order. */
void orc_sv_inner(const double* x, const double* y, int n, double* out2) {
  size_t A = (size_t)1 << n;
  double re = 0.0, im = 0.0;
  for (size_t i = 0; i < A; ++i) {
    double xr = x[2 * i], xi = x[2 * i + 1], yr = y[2 * i], yi = y[2 * i + 1];
    re += xr * yr + xi * yi;
    im += xr * yi - xi * yr;
  }
  out2[0] = re;
  out2[1] = im;
}

/* ------------------------------------------------------------------------- */
/* 8. Measurement (one shot, splitmix64 draw)                                 */
/* ------------------------------------------------------------------------- */

/* splitmix64 (Steele, Lea, Flood 2014): one output for one 64-bit state. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* u = (splitmix64(seed) >> 11) 2^-53; outcome = smallest i whose running sum of
 * |a|^2 reaches u * total.  prob = |a_outcome|^2 / total. */
int orc_sv_measure(const double* psi, int n, uint64_t seed, uint64_t* outcome, double* prob) {
  size_t A = (size_t)1 << n;
  double total = orc_sv_norm2(psi, n);
  double u = (double)(orc_splitmix64(seed) >> 11) * (1.0 / 9007199254740992.0);
  double target = u * total, run = 0.0;
  size_t pick = A - 1;
  for (size_t i = 0; i < A; ++i) {
    double p = fma(psi[2 * i], psi[2 * i], psi[2 * i + 1] * psi[2 * i + 1]);
    run += p;
    if (run >= target && p > 0.0) { pick = i; break; }
  }
  *outcome = pick;
  *prob = fma(psi[2 * pick], psi[2 * pick], psi[2 * pick + 1] * psi[2 * pick + 1]) / total;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* 9. Learned selector (not from the paper): which trial encodes to run       */
/* ------------------------------------------------------------------------- */
/* 16 -> 32 (ReLU) -> 32 (ReLU) -> 8, parameters W1[32][16] b1[32] W2[32][32] b2[32]
 * W3[8][32] b3[8] (bfloat16 values held as float).  float32, every unit summing its
 * products over its inputs in index order, one rounding per product and per sum. */
#define ORC_MLP_NPARAMS 1864

static float mlp_unit(const float* w, const float* x, int n, float b) {
  float acc = 0.0f;
  for (int i = 0; i < n; ++i) {
    float prod = w[i] * x[i];
    acc = acc + prod;
  }
  return acc + b;
}

void orc_mlp_forward(const float* prm, const float* x, float* out) {
  const float *W1 = prm, *b1 = W1 + 512, *W2 = b1 + 32, *b2 = W2 + 1024, *W3 = b2 + 32, *b3 = W3 + 256;
  float h1[32], h2[32];
  for (int j = 0; j < 32; ++j) {
    float z = mlp_unit(W1 + 16 * j, x, 16, b1[j]);
    h1[j] = z > 0.0f ? z : 0.0f;
  }
  for (int j = 0; j < 32; ++j) {
    float z = mlp_unit(W2 + 32 * j, h1, 32, b2[j]);
    h2[j] = z > 0.0f ? z : 0.0f;
  }
  for (int j = 0; j < 8; ++j) out[j] = mlp_unit(W3 + 32 * j, h2, 32, b3[j]);
}

/* Outputs 0..6: logits of the chunk modes ZERO, CONST, PERIOD, STREAM, RAW, SPLIT,
 * PALETTE; output 7: the bit budget, the predicted size of the chunk's best image as a
 * fraction of the RAW size.  Decision: the SPLIT (bit 0) and PALETTE (bit 1) trials
 * each run iff that mode's logit plus a margin of 2 reaches the largest of the seven
 * logits, and both run when the budget is below half the chunk's current size fraction
 * (input 7) -- a predicted collapse of the image the mode logits may miss; float32
 * sums and comparisons.  Every rule leans towards a trial: a missed trial costs memory,
 * a needless one only time.  The cheap modes are always computed; the codec keeps the
 * bound. */
int orc_mlp_trials(const float* prm, const float* x) {
  float out[8];
  orc_mlp_forward(prm, x, out);
  float mx = out[0];
  for (int m = 1; m < 7; ++m)
    if (out[m] > mx) mx = out[m];
  const int shrink = out[7] < x[7] * 0.5f;
  int t = 0;
  if (out[5] + 2.0f >= mx || shrink) t |= 1;
  if (out[6] + 2.0f >= mx || shrink) t |= 2;
  return t;
}

/* The selector's 16 inputs for a chunk about to be rewritten by gate g, from its current
 * image (img, len bytes) and the gate alone (no decoded value), so that the decisions
 * of a whole gate can be taken before it runs: one-hot of the image mode (7), its
 * size / RAW size, its S / 64, header word 3 / (64 N) (residual bits; the palette size
 * for PALETTE), header byte 2 / 16 (log2 period, palette index width), whether the gate
 * matrix is real, diagonal, anti-diagonal, whether the target lies inside the chunk, and
 * the gate's S / 64. */
void orc_mlp_features(const uint8_t* img, size_t len, int kc, const orc_gate* g, int S_gate, float* x) {
  uint32_t w3 = (uint32_t)img[12] | ((uint32_t)img[13] << 8) | ((uint32_t)img[14] << 16) | ((uint32_t)img[15] << 24);
  const double* u = g->u;
  for (int m = 0; m < 16; ++m) x[m] = 0.0f;
  if (img[0] < 7) x[img[0]] = 1.0f;
  x[7] = (float)len / (float)(16 + (16 << kc));
  x[8] = (float)img[1] / 64.0f;
  x[9] = (float)w3 / (float)(64 * (2 << kc));
  x[10] = (float)img[2] / 16.0f;
  x[11] = (u[1] == 0 && u[3] == 0 && u[5] == 0 && u[7] == 0) ? 1.0f : 0.0f;
  x[12] = (u[2] == 0 && u[3] == 0 && u[4] == 0 && u[5] == 0) ? 1.0f : 0.0f;
  x[13] = (u[0] == 0 && u[1] == 0 && u[6] == 0 && u[7] == 0) ? 1.0f : 0.0f;
  x[14] = g->target < kc ? 1.0f : 0.0f;
  x[15] = (float)S_gate / 64.0f;
}

/* The mode set a chunk is encoded with under the selector: Solution C's modes plus
 * the trials it grants. */
static unsigned mlp_mask(const float* prm, const uint8_t* img, size_t len, int kc, const orc_gate* g, int S_gate) {
  float x[16];
  orc_mlp_features(img, len, kc, g, S_gate, x);
  const int t = orc_mlp_trials(prm, x);
  return ORC_DEFAULT_MODES | ((t & 1) ? (1u << ORC_MODE_SPLIT) : 0u) | ((t & 2) ? (1u << ORC_MODE_PALETTE) : 0u);
}

/* ------------------------------------------------------------------------- */
/* 6. Compressed simulator                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
  uint64_t gates, encoded_bytes, max_encoded_bytes, raw_bytes, inflight_bytes, chunks_by_mode[8];
  double min_ratio, eps_current, fid_lb_sum, fid_lb_prod;
  int64_t eps_switch_gate;
  int32_t S_current, level;
  int32_t guard_fit; /* guarded ladder: 1 if the last gate's level was chosen because its worst case fits */
  int32_t pad;
  uint64_t wide_images; /* images whose header says S = 64 */
} orc_stats;

typedef struct {
  int n, b, kc, ladder, S_cur, level, nlevels;
  unsigned modes;
  int use_mlp;                    /* 1: SPLIT / PALETTE tried only where the selector says so */
  float mlp[ORC_MLP_NPARAMS];
  double levels[8];
  double eps_max, tau;
  uint64_t budget, thresh, inflight, nchunks, E, Emax, gates;
  int64_t switch_gate;
  double lb_sum, lb_prod;
  int guard_fit;
  uint64_t n64; /* images whose header says S = 64 */
  uint8_t** img;
  uint32_t* len;
  int poisoned;
} orc_csim;

void orc_csim_destroy(orc_csim* s);

static int csim_store(orc_csim* s, uint64_t c, const uint64_t* vals, unsigned mask) {
  size_t cap = 16 + 8 * ((size_t)2 << s->kc);
  uint8_t* buf = (uint8_t*)malloc(cap);
  long L = orc_encode_chunk_mask(vals, s->kc, s->S_cur, -1, mask, buf, cap);
  if (L < 0) { free(buf); return (int)L; }
  uint8_t* fit = (uint8_t*)realloc(buf, (size_t)L);
  if (fit) buf = fit;
  if (s->img[c]) {
    s->E -= s->len[c];
    s->n64 -= s->img[c][1] == 64;
    free(s->img[c]);
  }
  s->img[c] = buf;
  s->len[c] = (uint32_t)L;
  s->n64 += buf[1] == 64;
  s->E += (uint64_t)L;
  return ORC_OK;
}

/* ladder: 0 = jump from lossless straight to eps_max, 1 = the paper's ladder
 * 1e-5, 1e-4, ... one level per gate up to eps_max (Section 3.7).
 * Blocks hold 2^block_log2 amplitudes (Section 3.1); each block is coded as
 * 2^(block_log2 - chunk_log2) independent chunks. */
orc_csim* orc_csim_create(int n, int block_log2, int chunk_log2, double eps_max, uint64_t budget, double tau,
                          int ladder) {
  if (n < 1 || n > 40 || block_log2 < 0 || chunk_log2 < 0) return NULL;
  if (eps_max != 0.0 && orc_sig_bits(eps_max) < 0) return NULL;
  orc_csim* s = (orc_csim*)calloc(1, sizeof(orc_csim));
  s->n = n;
  s->b = block_log2 < n ? block_log2 : n;
  s->kc = chunk_log2 < s->b ? chunk_log2 : s->b;
  s->eps_max = eps_max;
  s->tau = tau;
  s->budget = budget;
  s->thresh = (uint64_t)floor(tau * (double)budget);
  /* Eq. totalnbBytes with r = 1: two decompressed blocks are in flight. */
  s->inflight = (uint64_t)2 << (s->b + 4);
  s->ladder = ladder;
  s->modes = ORC_DEFAULT_MODES;
  s->S_cur = 64;
  s->switch_gate = -1;
  s->lb_sum = 0.0;
  s->lb_prod = 1.0;
  static const double paper_levels[5] = {1e-5, 1e-4, 1e-3, 1e-2, 1e-1};
  s->nlevels = 0;
  if (eps_max > 0.0) {
    if (ladder >= 1)
      for (int k = 0; k < 5; ++k) if (paper_levels[k] < eps_max) s->levels[s->nlevels++] = paper_levels[k];
    s->levels[s->nlevels++] = eps_max;
  }
  s->nchunks = (uint64_t)1 << (n - s->kc);
  s->img = (uint8_t**)calloc(s->nchunks, sizeof(uint8_t*));
  s->len = (uint32_t*)calloc(s->nchunks, sizeof(uint32_t));
  size_t N = (size_t)2 << s->kc;
  uint64_t* vals = (uint64_t*)calloc(N, 8);
  for (uint64_t c = 0; c < s->nchunks; ++c) {
    memset(vals, 0, N * 8);
    if (c == 0) { double one = 1.0; memcpy(&vals[0], &one, 8); }
    if (csim_store(s, c, vals, ORC_DEFAULT_MODES)) { free(vals); orc_csim_destroy(s); return NULL; }
  }
  free(vals);
  s->Emax = s->E;
  return s;
}

void orc_csim_destroy(orc_csim* s) {
  if (!s) return;
  for (uint64_t c = 0; c < s->nchunks; ++c) free(s->img[c]);
  free(s->img);
  free(s->len);
  free(s);
}

/* Error-bound controller, evaluated before each gate (Section 3.7): the memory the
 * gate needs is nbBytes = E + W (Eq. totalnbBytes, r = 1), with E the current sum of
 * image bytes and W two decompressed blocks.  If nbBytes exceeds floor(tau * budget)
 * the bound is relaxed: the jump ladder goes from lossless to eps_max at once, the
 * paper's ladder steps one level per gate.  The bound never tightens. */
/* The largest image a chunk can take at S significant bits: every value coded with
 * the full S bits (2-bit code each), or the verbatim values if that is smaller. */
static uint64_t max_level_image(int kc, int S) {
  uint64_t N = (uint64_t)2 << kc;
  uint64_t codes = ((N + 3) / 4 + 15) / 16 * 16;
  uint64_t resid = (S * N + 127) / 128 * 16;
  uint64_t stream = 16 + codes + resid, raw = 16 + 8 * N;
  return stream < raw ? stream : raw;
}

/* Section 3.7, before gate g (touched = chunks the gate rewrites).  Ladders 0 and 1:
 * relax when E + two decompressed blocks (Eq. totalnbBytes) exceed floor(tau budget).
 * Ladder 2 reads the rule for a device that rewrites all of a gate's chunks at once:
 * take the smallest level, never below the current one, whose worst case still fits
 * -- the gate ends with at most the sum of the largest images of the chunks it
 * rewrites if it rewrites every chunk, else with at most E plus that sum.  A chunk
 * holding a subnormal is coded at 64 bits at any level (Eq. sigbits cannot truncate
 * it), so its largest image is the 64-bit one: once the run is lossy, every image
 * still at 64 bits is assumed to be among the rewritten chunks; and a gate with a
 * nonzero coefficient below 2^-52 in magnitude may make subnormals of normal values,
 * so all of its chunks count at 64 bits. */
static void controller(orc_csim* s, uint64_t touched, int wide_gate) {
  if (s->nlevels == 0 || (s->ladder != 2 && s->level >= s->nlevels)) return;
  int lvl = s->level;
  if (s->ladder == 2) {
    uint64_t wide = 0;
    if (wide_gate) wide = touched;
    else if (s->level > 0) wide = s->n64 < touched ? s->n64 : touched;
    const uint64_t full = max_level_image(s->kc, 64);
    lvl = s->nlevels;
    s->guard_fit = 0;
    for (int l = s->level; l <= s->nlevels; ++l) {
      uint64_t worst = (touched - wide) * max_level_image(s->kc, l == 0 ? 64 : orc_sig_bits(s->levels[l - 1])) +
                       wide * full;
      if ((touched >= s->nchunks ? worst : s->E + worst) <= s->thresh) {
        lvl = l;
        s->guard_fit = 1;
        break;
      }
    }
  } else {
    if (s->E + s->inflight <= s->thresh) return;
    lvl = s->ladder == 1 ? s->level + 1 : s->nlevels;
  }
  if (lvl == s->level) return;
  s->level = lvl;
  s->S_cur = orc_sig_bits(s->levels[s->level - 1]);
  if (s->switch_gate < 0) s->switch_gate = (int64_t)s->gates;
}

/* A coefficient that can turn a normal value into a subnormal: nonzero, below 2^-52. */
static int gate_is_wide(const orc_gate* g) {
  for (int k = 0; k < 8; ++k)
    if (g->u[k] != 0.0 && fabs(g->u[k]) < 0x1p-52) return 1;
  return 0;
}

int orc_csim_apply(orc_csim* s, const orc_gate* g) {
  if (s->poisoned) return ORC_ERR_STATE;
  int rc = orc_gate_check(g, s->n);
  if (rc) return rc;
  int kc = s->kc, t = g->target;
  size_t A = (size_t)1 << kc, N = 2 * A;
  uint64_t hi_mask = g->ctrl_mask >> kc, hi_vals = g->ctrl_vals >> kc;
  controller(s, s->nchunks >> __builtin_popcountll(hi_mask & (s->nchunks - 1)), gate_is_wide(g));
  uint64_t lo_mask = g->ctrl_mask & (A - 1), lo_vals = g->ctrl_vals & (A - 1);
  uint64_t* x0 = (uint64_t*)malloc(N * 8);
  uint64_t* x1 = (uint64_t*)malloc(N * 8);
  unsigned m0 = s->modes, m1 = s->modes;
  for (uint64_t q = 0; q < s->nchunks && rc == ORC_OK; ++q) {
    if ((q & hi_mask) != hi_vals) continue;
    if (t < kc) {
      rc = orc_decode_chunk(s->img[q], s->len[q], kc, x0);
      if (rc) break;
      double* d = (double*)x0;
      for (size_t i = 0; i < A; ++i) {
        if ((i >> t) & 1) continue;
        if ((i & lo_mask) != lo_vals) continue;
        apply_pair(g->u, d + 2 * i, d + 2 * (i | ((size_t)1 << t)));
      }
      if (s->use_mlp) m0 = mlp_mask(s->mlp, s->img[q], s->len[q], kc, g, s->S_cur);
      rc = csim_store(s, q, x0, m0);
    } else {
      uint64_t qb = (uint64_t)1 << (t - kc);
      if (q & qb) continue;
      uint64_t q1 = q | qb;
      rc = orc_decode_chunk(s->img[q], s->len[q], kc, x0);
      if (!rc) rc = orc_decode_chunk(s->img[q1], s->len[q1], kc, x1);
      if (rc) break;
      double *d0 = (double*)x0, *d1 = (double*)x1;
      for (size_t i = 0; i < A; ++i) {
        if ((i & lo_mask) != lo_vals) continue;
        apply_pair(g->u, d0 + 2 * i, d1 + 2 * i);
      }
      if (s->use_mlp) {
        m0 = mlp_mask(s->mlp, s->img[q], s->len[q], kc, g, s->S_cur);
        m1 = mlp_mask(s->mlp, s->img[q1], s->len[q1], kc, g, s->S_cur);
      }
      rc = csim_store(s, q, x0, m0);
      if (!rc) rc = csim_store(s, q1, x1, m1);
    }
  }
  free(x0);
  free(x1);
  if (rc) { s->poisoned = 1; return rc; }
  if (s->S_cur < 64) {
    double delta = ldexp(1.0, 12 - s->S_cur); /* 2^EXP(eps): the bound each value keeps */
    s->lb_sum += delta;
    s->lb_prod *= (1.0 - delta);
  }
  s->gates += 1;
  if (s->E > s->Emax) s->Emax = s->E;
  return ORC_OK;
}

int orc_csim_run(orc_csim* s, const orc_gate* gates, size_t ng) {
  for (size_t k = 0; k < ng; ++k) {
    int rc = orc_csim_apply(s, gates + k);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* Decodes the whole state into interleaved doubles. */
int orc_csim_amplitudes(const orc_csim* s, double* out) {
  size_t N = (size_t)2 << s->kc;
  for (uint64_t c = 0; c < s->nchunks; ++c) {
    int rc = orc_decode_chunk(s->img[c], s->len[c], s->kc, (uint64_t*)(out + c * N));
    if (rc) return rc;
  }
  return ORC_OK;
}

/* Copies chunk c's image; *len receives its length. */
int orc_csim_image(const orc_csim* s, uint64_t c, uint8_t* out, size_t cap, uint64_t* len) {
  if (c >= s->nchunks) return ORC_ERR_INVALID;
  *len = s->len[c];
  if (s->len[c] > cap) return ORC_ERR_INVALID;
  memcpy(out, s->img[c], s->len[c]);
  return ORC_OK;
}

/* Replaces chunk c's image (used to start the oracle from a stored state). */
int orc_csim_set_image(orc_csim* s, uint64_t c, const uint8_t* img, size_t len) {
  if (c >= s->nchunks) return ORC_ERR_INVALID;
  size_t N = (size_t)2 << s->kc;
  uint64_t* tmp = (uint64_t*)malloc(N * 8);
  int rc = orc_decode_chunk(img, len, s->kc, tmp);
  free(tmp);
  if (rc) return rc;
  uint8_t* b = (uint8_t*)malloc(len);
  memcpy(b, img, len);
  s->E -= s->len[c];
  free(s->img[c]);
  s->img[c] = b;
  s->len[c] = (uint32_t)len;
  s->E += len;
  return ORC_OK;
}

void orc_csim_stats(const orc_csim* s, orc_stats* st) {
  memset(st, 0, sizeof(*st));
  st->gates = s->gates;
  st->encoded_bytes = s->E;
  st->max_encoded_bytes = s->Emax;
  st->raw_bytes = (uint64_t)16 << s->n;
  st->inflight_bytes = s->inflight;
  for (uint64_t c = 0; c < s->nchunks; ++c) st->chunks_by_mode[s->img[c][0] & 7] += 1;
  st->min_ratio = (double)st->raw_bytes / (double)s->Emax;
  st->eps_current = s->level ? s->levels[s->level - 1] : 0.0;
  st->fid_lb_sum = 1.0 - s->lb_sum;
  st->fid_lb_prod = s->lb_prod;
  st->eps_switch_gate = s->switch_gate;
  st->S_current = s->S_cur;
  st->level = s->level;
  st->guard_fit = s->guard_fit;
  st->wide_images = s->n64;
}

uint64_t orc_csim_nchunks(const orc_csim* s) { return s->nchunks; }

/* Selector for later gates: use_mlp = 0 keeps the mode set; 1 tries Solution D for a
 * chunk only when the network (params, ORC_MLP_NPARAMS floats) says so. */
int orc_csim_set_mlp(orc_csim* s, int use_mlp, const float* params) {
  s->use_mlp = use_mlp;
  if (use_mlp) memcpy(s->mlp, params, sizeof(s->mlp));
  return ORC_OK;
}

/* Mode set the encoder chooses from for later gates (bit m = mode m). */
int orc_csim_set_modes(orc_csim* s, unsigned mask) {
  if ((mask & 0x1Fu) != 0x1Fu || (mask >> ORC_NMODES)) return ORC_ERR_INVALID;
  s->modes = mask;
  return ORC_OK;
}
int orc_csim_chunk_log2(const orc_csim* s) { return s->kc; }
int orc_csim_block_log2(const orc_csim* s) { return s->b; }
