// api.cu -- host side of the libqcsim C ABI (see include/qcsim.h).
//
// Gate classification (Section 3.3 segments): with chunks of 2^kc amplitudes, a
// target below kc pairs amplitudes inside one chunk; a target at or above kc pairs
// chunk q with chunk q | 2^(t-kc) (the paper's "different blocks" segment; one GPU
// has no remote-rank segment).  A control on a chunk-index bit removes whole chunks
// from the work (the paper's block-level skip); controls below kc are tested per
// amplitude pair inside the kernel.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qcsim.h"
#include "launch.h"

using qc::CtlParams;
using qc::DevCtl;
using qc::GateCoef;
using qc::GateLaunch;
using qc::Pool;

namespace {

thread_local std::string g_last_error;

sim_status fail(sim_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

sim_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(SIM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(SIM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

}  // namespace

// Eq. sigbits: S = 12 - EXP(eps) for binary64 (EXP = the IEEE exponent of eps);
// eps = 0 is the lossless stage (64 bits).  -1 for a bound outside {0} U [2^-52, 1).
int qc::sig_bits_of(double eps) {
  if (eps == 0.0) return 64;
  if (!(eps > 0.0) || !(eps < 1.0)) return -1;
  int e2 = 0;
  (void)std::frexp(eps, &e2);  // eps = f 2^e2, f in [0.5, 1): IEEE exponent e2 - 1
  const int ex = e2 - 1;
  if (ex < -52) return -1;
  const int S = 12 - ex;
  return S > 64 ? 64 : S;
}

namespace {

using qc::sig_bits_of;

bool gate_ok(const sim_gate* g, int n, std::string* why) {
  if (g->target < 0 || g->target >= n) { *why = "target outside the register"; return false; }
  const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
  if (g->ctrl_mask & ~all) { *why = "control outside the register"; return false; }
  if ((g->ctrl_mask >> g->target) & 1ull) { *why = "control on the target"; return false; }
  if (g->ctrl_vals & ~g->ctrl_mask) { *why = "control value outside the control mask"; return false; }
  for (int k = 0; k < 8; ++k)
    if (!std::isfinite(g->u[k])) { *why = "non-finite matrix entry"; return false; }
  // U^H U = I: unit columns, orthogonal to each other
  const double* u = g->u;
  const double n0 = u[0] * u[0] + u[1] * u[1] + u[4] * u[4] + u[5] * u[5];
  const double n1 = u[2] * u[2] + u[3] * u[3] + u[6] * u[6] + u[7] * u[7];
  const double dr = u[0] * u[2] + u[1] * u[3] + u[4] * u[6] + u[5] * u[7];
  const double di = u[0] * u[3] - u[1] * u[2] + u[4] * u[7] - u[5] * u[6];
  if (std::fabs(n0 - 1.0) > 1e-12 || std::fabs(n1 - 1.0) > 1e-12 || std::fabs(dr) > 1e-12 || std::fabs(di) > 1e-12) {
    *why = "matrix is not unitary within 1e-12";
    return false;
  }
  return true;
}

GateCoef coef_of(const sim_gate* g) {
  const double* u = g->u;
  // four rows (a'r, a'i, b'r, b'i), four terms each: coefficient and operand
  // (0 ar, 1 ai, 2 br, 3 bi) in the order of the sums of Eq. matrix1
  const double cf[4][4] = {{u[0], -u[1], u[2], -u[3]},
                           {u[0], u[1], u[2], u[3]},
                           {u[4], -u[5], u[6], -u[7]},
                           {u[4], u[5], u[6], u[7]}};
  const uint8_t ops[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {0, 1, 2, 3}, {1, 0, 3, 2}};
  GateCoef c;
  std::memset(&c, 0, sizeof(c));
  for (int r = 0; r < 4; ++r) {
    int k = 0;
    for (int t = 0; t < 4; ++t) {
      if (cf[r][t] == 0.0) continue;  // an exactly-zero coefficient drops its term
      c.c[4 * r + k] = cf[r][t];
      c.op[4 * r + k] = ops[r][t];
      ++k;
    }
    c.cnt[r] = (uint8_t)k;
    c.first[r] = 0;
    if (k > 0 && c.c[4 * r] == 1.0) c.first[r] = 1;
    if (k > 0 && c.c[4 * r] == -1.0) c.first[r] = 2;
  }
  c.dense = (c.cnt[0] == 4 && c.cnt[1] == 4 && c.cnt[2] == 4 && c.cnt[3] == 4) ? 1 : 0;
  return c;
}

int popcount64(uint64_t x) { return __builtin_popcountll(x); }

int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

void qc::set_last_error(const char* msg) { g_last_error = msg; }

struct sim {
  int n = 0, b = 0, kc = 0, ladder = 0;
  double eps_max = 0.0, tau = 0.9;
  uint64_t budget = 0, nchunks = 0, npages = 0;
  cudaStream_t st = 0;
  Pool P{};
  CtlParams cp{};
  DevCtl* d_ctl = nullptr;
  unsigned long long* d_counts = nullptr;
  int grid = 1;
  sim_status poisoned = SIM_OK;
  uint64_t amp_updates = 0;
  uint64_t device_bytes = 0;
  uint8_t* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  double level_eps[8] = {0};
  // gate-kernel timing
  bool timing = false;
  bool phases = false;
  uint32_t modes = qc::kDefaultModes;
  int selector = 0;                  // 0 mode set, 2 selector network
  unsigned short* d_mlp = nullptr;   // bfloat16 parameters of the selector network
  uint8_t* d_dec = nullptr;          // its decisions for the running gate (one byte per chunk)
  float* d_trace = nullptr;          // selector training records
  uint8_t* d_bc = nullptr;           // block cache lines (Section 3.4) or nullptr
  uint32_t* d_defer = nullptr;       // items the streaming kernel leaves to the general one
  int fast_grid = 0;                 // CTAs of the streaming kernel (0: chunk size outside its range)
  bool fast = true;                  // gates try the streaming kernel first
  uint64_t kernel_launches = 0;      // gate, streaming and post kernels enqueued
  uint64_t trace_cap = 0;
  // the graph of the last sim_batch_apply call this handle led, kept for replay
  cudaGraphExec_t bexec = nullptr;
  qc::BatchJob* bjobs = nullptr;     // its job list (device)
  std::vector<uint8_t> bkey;         // what its launches depend on
  std::vector<uint64_t> bupd;        // the amplitude updates it makes, per handle
  uint64_t uid = 0;                  // creation number (never reused)
  uint64_t cfg_gen = 0;              // bumped by every setting that can change a gate's launch
  cudaStream_t bstream = nullptr;    // private capture / replay stream
  cudaEvent_t bready = nullptr;
  uint64_t graph_replays = 0;
  void drop_graph() {
    if (bexec) cudaGraphExecDestroy(bexec);
    cudaFree(bjobs);
    bexec = nullptr;
    bjobs = nullptr;
    bkey.clear();
    bupd.clear();
  }
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  size_t ev_next = 0;
  unsigned long long* d_tlog = nullptr;  // per timed launch: cumulative image bytes read, written after it
  size_t tlog_cap = 0;
  unsigned long long t_bytes_in0 = 0, t_bytes_out0 = 0;

  ~sim() {
    drop_graph();
    if (bready) cudaEventDestroy(bready);
    if (bstream) cudaStreamDestroy(bstream);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    cudaFree(d_tlog);
    cudaFree(d_defer);
    cudaFree(d_mlp);
    cudaFree(d_dec);
    cudaFree(d_trace);
    cudaFree(d_bc);
    cudaFree(P.pages);
    cudaFree(P.dir);
    cudaFree(P.stack);
    cudaFree(P.freed);
    cudaFree(P.cache);
    cudaFree(P.cache_n);
    cudaFree(P.wcache);
    cudaFree(P.wcache_n);
    cudaFree(d_ctl);
    cudaFree(d_counts);
    cudaFree(d_scratch);
  }

  sim_status scratch(size_t bytes) {
    if (bytes <= scratch_bytes) return SIM_OK;
    cudaFree(d_scratch);
    d_scratch = nullptr;
    scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&d_scratch, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
    scratch_bytes = bytes;
    return SIM_OK;
  }

  // Device error word -> status; poisons the handle on a device-side failure.
  sim_status check_device() {
    unsigned int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, &d_ctl->err, sizeof(err), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      poisoned = SIM_ERR_CUDA;
      return cuda_fail(e, "device");
    }
    if (err == 0) return SIM_OK;
    if (err & qc::E_OOM) {
      poisoned = SIM_ERR_OOM;
      return fail(SIM_ERR_OOM, "the page pool ran out of pages (budget too small for the state)");
    }
    if (err & qc::E_TIMEOUT) {
      unsigned int site = 0;
      cudaMemcpy(&site, &d_ctl->timeout_site, sizeof(site), cudaMemcpyDeviceToHost);
      poisoned = SIM_ERR_TIMEOUT;
      return fail(SIM_ERR_TIMEOUT, "a bounded wait in the streaming gate kernel gave up (site %u)", site);
    }
    poisoned = SIM_ERR_CORRUPT;
    return fail(SIM_ERR_CORRUPT, "a chunk image failed its checks or held a non-finite value (flags 0x%x)", err);
  }

  sim_status guard() const {
    if (poisoned != SIM_OK) return fail(SIM_ERR_STATE, "handle is poisoned by an earlier failure");
    return SIM_OK;
  }
};

struct sim_sv {
  int n = 0;
  double* psi = nullptr;
  cudaStream_t st = 0;
  ~sim_sv() { cudaFree(psi); }
};

extern "C" {

const char* sim_last_error(void) { return g_last_error.c_str(); }

sim_status sim_create_ex(int n_qubits, int block_log2, int chunk_log2, double err_bound, uint64_t budget, double tau,
                         int ladder, uint64_t pool_bytes, sim_t** out) {
  if (!out) return fail(SIM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > 40) return fail(SIM_ERR_INVALID, "n_qubits must be in [1, 40]");
  if (block_log2 < 0) return fail(SIM_ERR_INVALID, "block_log2 must be >= 0");
  if (chunk_log2 < 0 || chunk_log2 > qc::kMaxKC) return fail(SIM_ERR_INVALID, "chunk_log2 must be in [0, 11]");
  if (sig_bits_of(err_bound) < 0) return fail(SIM_ERR_INVALID, "err_bound must be 0 or in [2^-52, 1)");
  if (budget == 0) return fail(SIM_ERR_INVALID, "budget must be > 0");
  if (!(tau > 0.0 && tau <= 1.0)) return fail(SIM_ERR_INVALID, "tau must be in (0, 1]");
  if (ladder < 0 || ladder > 2) return fail(SIM_ERR_INVALID, "ladder must be 0, 1 or 2");

  sim* s = new sim();
  s->n = n_qubits;
  s->b = block_log2 < n_qubits ? block_log2 : n_qubits;
  s->kc = chunk_log2 < s->b ? chunk_log2 : s->b;
  s->eps_max = err_bound;
  s->tau = tau;
  s->budget = budget;
  s->ladder = ladder;
  s->nchunks = 1ull << (s->n - s->kc);
  static std::atomic<uint64_t> creations{0};
  s->uid = ++creations;

  // controller parameters (Section 3.7, Eq. totalnbBytes with r = 1)
  CtlParams& cp = s->cp;
  cp.thresh = (unsigned long long)std::floor(tau * (double)budget);
  cp.inflight = 2ull << (s->b + 4);
  cp.ladder = ladder;
  cp.nlevels = 0;
  if (err_bound > 0.0) {
    static const double paper[5] = {1e-5, 1e-4, 1e-3, 1e-2, 1e-1};
    if (ladder >= 1)
      for (double e : paper)
        if (e < err_bound) s->level_eps[cp.nlevels++] = e;
    s->level_eps[cp.nlevels++] = err_bound;
  }
  for (int k = 0; k < cp.nlevels; ++k) {
    cp.S[k] = sig_bits_of(s->level_eps[k]);
    cp.delta[k] = std::ldexp(1.0, 12 - cp.S[k]);
  }
  cp.nchunks = s->nchunks;
  cp.touched = s->nchunks;
  for (int l = 0; l <= cp.nlevels; ++l) cp.maxb[l] = qc::max_level_image(s->kc, l == 0 ? 64 : cp.S[l - 1]);

  // page arena: the budget, 1/8 more for page rounding, and the pages that the
  // per-CTA caches may hold while a gate runs
  s->grid = device_sms() * qc::gate_ctas_per_sm(s->kc);
  s->fast_grid = s->kc >= qc::kFastMinKC ? device_sms() * qc::fast_ctas_per_sm(s->kc) : 0;
  // pages the per-CTA caches of the general kernel, and the per-warp caches and items in
  // flight of the streaming kernel, may hold while a gate runs
  const uint64_t slack_pages = (uint64_t)s->grid * (qc::kCacheCap + 2 * qc::max_pages(s->kc)) +
                               (uint64_t)s->fast_grid * qc::fast_warps() * (qc::fast_warp_cache() + 2 * qc::max_pages(s->kc));
  if (pool_bytes) {
    s->npages = (pool_bytes + qc::kPage - 1) / qc::kPage;
  } else {
    const uint64_t bp = (budget + qc::kPage - 1) / qc::kPage;
    s->npages = bp + bp / 8 + slack_pages;
  }
  if (s->npages >= (1ull << 32)) {
    delete s;
    return fail(SIM_ERR_INVALID, "budget too large for 32-bit page ids");
  }
  if (s->fast_grid) {
    // no more CTAs of the streaming kernel than the largest gate has items for, and,
    // in a pool sized by the caller, no more than let its warps' free-page caches (each
    // up to its capacity plus one refill, and one chunk's output pages) hold a quarter
    // of the pool; none if not even one CTA fits
    const uint64_t need = ((s->nchunks + 1) / 2 + qc::fast_pairs() - 1) / qc::fast_pairs();
    uint64_t cap = need;
    if (pool_bytes) {
      const uint64_t per_cta = (uint64_t)qc::fast_warps() * (qc::fast_warp_cache() + 32 + qc::max_pages(s->kc));
      const uint64_t fit = s->npages / 4 / per_cta;
      cap = fit < cap ? fit : cap;
    }
    s->fast_grid = (uint64_t)s->fast_grid < cap ? s->fast_grid : (int)cap;
  }
  Pool& P = s->P;
  P.kc = s->kc;
  P.npages = s->npages;
  P.dir_words = qc::dir_stride(s->kc) / 4;
  struct A {
    void** p;
    size_t bytes;
    const char* what;
  } allocs[] = {
      {(void**)&P.pages, (size_t)s->npages * qc::kPage, "page arena"},
      {(void**)&P.dir, (size_t)s->nchunks * qc::dir_stride(s->kc), "directory"},
      {(void**)&P.stack, (size_t)s->npages * 4, "free-page stack"},
      {(void**)&P.freed, (size_t)s->npages * 4, "freed list"},
      {(void**)&P.cache, (size_t)s->grid * qc::kCacheCap * 4, "page caches"},
      {(void**)&P.cache_n, (size_t)s->grid * 4, "page cache counts"},
      {(void**)&P.wcache, (size_t)(s->fast_grid ? s->fast_grid : 1) * qc::fast_warps() * qc::fast_warp_cache() * 4,
       "streaming-kernel page caches"},
      {(void**)&P.wcache_n, (size_t)(s->fast_grid ? s->fast_grid : 1) * qc::fast_warps() * 4,
       "streaming-kernel page cache counts"},
      {(void**)&s->d_ctl, sizeof(DevCtl), "counters"},
      {(void**)&s->d_counts, 8 * sizeof(unsigned long long), "mode counts"},
      {(void**)&s->d_defer, (size_t)(s->nchunks / 2 + 1) * sizeof(uint32_t), "deferred-item list"},
  };
  for (auto& a : allocs) {
    cudaError_t e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      delete s;
      return cuda_fail(e, a.what);
    }
    s->device_bytes += a.bytes;
  }
  P.ctl = s->d_ctl;
  DevCtl h{};
  h.top = (long long)s->npages;
  h.switch_gate = -1;
  h.lb_prod = 1.0;
  h.S_last = 64;
  cudaError_t e = cudaMemcpy(s->d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(P.cache_n, 0, (size_t)s->grid * 4);
  if (e == cudaSuccess) e = cudaMemset(P.wcache_n, 0, (size_t)(s->fast_grid ? s->fast_grid : 1) * qc::fast_warps() * 4);
  if (e == cudaSuccess) e = qc::launch_pool_init(P, s->nchunks, 0);
  if (e == cudaSuccess) e = qc::launch_init_chunk0(P, s->nchunks, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "initialisation");
  }
  sim_status rc = s->check_device();
  if (rc != SIM_OK) {
    delete s;
    return rc;
  }
  *out = s;
  return SIM_OK;
}

sim_status sim_create(int n_qubits, int block_log2, double err_bound, sim_t** out) {
  if (n_qubits < 1 || n_qubits > 40 || block_log2 < 0) return fail(SIM_ERR_INVALID, "bad n_qubits or block_log2");
  size_t freeb = 0, totalb = 0;
  if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) return fail(SIM_ERR_CUDA, "cudaMemGetInfo failed");
  const int b = block_log2 < n_qubits ? block_log2 : n_qubits;
  const int kc = b < 10 ? b : 10;
  const uint64_t nchunks = 1ull << (n_qubits - kc);
  const uint64_t raw = 16ull << n_qubits;
  const double overhead = (double)nchunks * qc::dir_stride(kc) + 64.0 * 1024 * 1024;
  double avail = 0.9 * (double)freeb - overhead;
  avail /= (1.0 + 8.0 / qc::kPage);  // stack and freed list: 8 bytes per page
  if (avail < 1e6) return fail(SIM_ERR_OOM, "not enough free device memory");
  uint64_t budget = (uint64_t)avail;
  const uint64_t cap = raw + 16ull * nchunks + 4096;  // RAW images never need more
  if (budget > cap) budget = cap;
  return sim_create_ex(n_qubits, block_log2, kc, err_bound, budget, 0.9, 0, 0, out);
}

sim_status sim_destroy(sim_t* s) {
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  cudaStreamSynchronize(s->st);
  delete s;
  return SIM_OK;
}

sim_status sim_reset(sim_t* s) {
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  if (sim_status r = s->guard()) return r;
  DevCtl h{};
  h.top = (long long)s->npages;
  h.switch_gate = -1;
  h.lb_prod = 1.0;
  h.S_last = 64;
  const size_t nwc = (size_t)(s->fast_grid ? s->fast_grid : 1) * qc::fast_warps();
  cudaError_t e = cudaMemcpyAsync(s->d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->P.cache_n, 0, (size_t)s->grid * 4, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->P.wcache_n, 0, nwc * 4, s->st);
  if (e == cudaSuccess && s->d_bc)  // lines are tagged by gate serial, which starts over
    e = cudaMemsetAsync(s->d_bc, 0, (size_t)qc::kBcLines * qc::bc_line_bytes(qc::round16(qc::max_image_bytes(s->kc))),
                        s->st);
  if (e == cudaSuccess) e = qc::launch_pool_init(s->P, s->nchunks, s->st);
  if (e == cudaSuccess) e = qc::launch_init_chunk0(s->P, s->nchunks, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);  // h is read from the host stack
  if (e != cudaSuccess) return cuda_fail(e, "reset");
  s->amp_updates = 0;
  s->kernel_launches = 0;
  return s->check_device();
}

sim_status sim_set_stream(sim_t* s, void* stream) {
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  s->st = reinterpret_cast<cudaStream_t>(stream);
  return SIM_OK;
}

// Work description of one gate (Section 3.3 segments, see the top of this file).
static GateLaunch make_launch(sim* s, const sim_gate* g) {
  const int kc = s->kc, t = g->target;
  const uint64_t A = 1ull << kc;
  GateLaunch L{};
  L.P = s->P;
  L.ctl = s->cp;
  L.g = coef_of(g);
  const uint64_t chunk_bits = (s->nchunks - 1ull);
  const uint64_t hi_mask = (g->ctrl_mask >> kc) & chunk_bits;
  L.hi_vals = (g->ctrl_vals >> kc) & chunk_bits;
  L.lo_mask = (uint32_t)(g->ctrl_mask & (A - 1ull));
  L.lo_vals = (uint32_t)(g->ctrl_vals & (A - 1ull));
  L.target = t;
  L.prof = s->phases ? 1 : 0;
  L.modes = s->modes;
  L.sel_dec = s->selector == 2 ? s->d_dec : nullptr;
  {
    const double* u = g->u;
    const bool real = u[1] == 0 && u[3] == 0 && u[5] == 0 && u[7] == 0;
    const bool diag = u[2] == 0 && u[3] == 0 && u[4] == 0 && u[5] == 0;
    const bool perm = u[0] == 0 && u[1] == 0 && u[6] == 0 && u[7] == 0;
    L.gfeat = (real ? 1u : 0u) | (diag ? 2u : 0u) | (perm ? 4u : 0u) | (t < kc ? 8u : 0u);
    // a coefficient that can turn a normal value into a subnormal (see next_level)
    L.ctl.wide_gate = 0;
    for (int k = 0; k < 8; ++k)
      if (u[k] != 0.0 && std::fabs(u[k]) < 0x1p-52) L.ctl.wide_gate = 1;
  }
  L.bc = s->d_trace ? nullptr : s->d_bc;
  L.trace = s->d_trace;
  L.trace_n = s->d_trace ? &s->d_ctl->trace_n : nullptr;
  L.trace_cap = s->trace_cap;
  if (t >= kc) {
    L.pair = 1;
    L.pair_bit = 1ull << (t - kc);
    L.free_mask = chunk_bits & ~hi_mask & ~L.pair_bit;
    L.items = 1ull << popcount64(L.free_mask);
    L.nact = 2ull * L.items;
  } else {
    L.pair = 0;
    L.pair_bit = 0;
    L.free_mask = chunk_bits & ~hi_mask;
    L.nact = 1ull << popcount64(L.free_mask);
    L.items = (L.nact + 1ull) / 2ull;
  }
  L.ctl.touched = L.nact;  // the guarded ladder bounds the gate by the chunks it rewrites
  // free_mask as runs: run i at bit p receives counter bits [q, q + len) shifted by p - q
  L.nruns = 0;
  int q = 0;
  for (int p = 0; p < 64 && L.nruns >= 0;) {
    if (!((L.free_mask >> p) & 1ull)) {
      ++p;
      continue;
    }
    int len = 0;
    while (p + len < 64 && ((L.free_mask >> (p + len)) & 1ull)) ++len;
    if (L.nruns == qc::kMaxRuns) {
      L.nruns = -1;
      break;
    }
    L.run_mask[L.nruns] = (len == 64 ? ~0ull : ((1ull << len) - 1ull)) << p;
    L.run_shift[L.nruns] = (uint32_t)(p - q);
    ++L.nruns;
    q += len;
    p += len;
  }
  return L;
}

// True if the streaming kernel can take the gate's items (see kernels.cu): chunk sizes
// 2^7..2^11, Solution C's mode set (under the selector network: the items none of
// whose chunks was granted a trial), no block cache or training records, and a partner
// amplitude within a warp's pass unless the gate is diagonal.  Sets L.fast_kind.
static bool fast_applies(const sim* s, const sim_gate* g, GateLaunch& L) {
  if (!s->fast || s->fast_grid == 0 || L.bc || L.trace) return false;
  if (!L.sel_dec && L.modes != qc::kDefaultModes) return false;
  const double* u = g->u;
  const bool diag = u[2] == 0.0 && u[3] == 0.0 && u[4] == 0.0 && u[5] == 0.0;
  const bool anti = u[0] == 0.0 && u[1] == 0.0 && u[6] == 0.0 && u[7] == 0.0;
  if (L.pair) L.fast_kind = 0;
  else if (diag) L.fast_kind = 3;
  else if (L.target < 2) L.fast_kind = 1;
  else if (L.target < 7) L.fast_kind = 2;
  else return false;
  // Eq. matrix1 / matrix2 with the coefficient order of GateCoef: a term with a zero
  // coefficient contributes an exact zero, so summing every term gives the kept-term
  // sums' value (a zero result may differ in sign, and the encoder stores +0 for both)
  const double cf[16] = {u[0], -u[1], u[2], -u[3], u[0], u[1], u[2], u[3],
                         u[4], -u[5], u[6], -u[7], u[4], u[5], u[6], u[7]};
  for (int k = 0; k < 16; ++k) L.cf[k] = cf[k];
  const bool real = u[1] == 0.0 && u[3] == 0.0 && u[5] == 0.0 && u[7] == 0.0;
  L.arith = diag ? 1 : (anti ? 2 : (real ? 3 : 0));
  if (L.arith == 0) {
    // every coefficient part of the same magnitude 2^k, none zero: exact products
    const double c = std::fabs(cf[0]);
    bool pow2 = c > 0.0;
    for (int k = 1; k < 16 && pow2; ++k) pow2 = std::fabs(cf[k]) == c;
    int e = 0;
    if (pow2 && std::frexp(c, &e) == 0.5 && e - 1 >= -64 && e - 1 <= 0) {
      L.arith = 4;
      L.sk = e - 1;
      L.sgn = 0;
      for (int k = 0; k < 16; ++k)
        if (cf[k] < 0.0) L.sgn |= 1u << k;
    }
  }
  if (L.arith == 1 || L.arith == 2) {
    // the one nonzero entry of each row: a' = d0 x, b' = d1 y (x, y = a, b or b, a)
    const double d[4] = {diag ? u[0] : u[2], diag ? u[1] : u[3], diag ? u[6] : u[4], diag ? u[7] : u[5]};
    for (int r = 0; r < 2; ++r) {
      L.du[2 * r] = d[2 * r];
      L.du[2 * r + 1] = d[2 * r + 1];
      L.rop[r] = d[2 * r + 1] != 0.0 ? 0 : (d[2 * r] == 1.0 ? 1 : (d[2 * r] == -1.0 ? 2 : 0));
    }
  }
  return true;
}

static sim_status enqueue_gate(sim* s, const sim_gate* g) {
  GateLaunch L = make_launch(s, g);
  const int grid = (uint64_t)s->grid < L.items ? s->grid : (int)L.items;
  const bool fast = fast_applies(s, g, L);
  L.defer = s->d_defer;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (s->timing) {
    while (s->ev_pool.size() < s->ev_next + 2) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e), "event create");
      s->ev_pool.push_back(e);
    }
    e0 = s->ev_pool[s->ev_next++];
    e1 = s->ev_pool[s->ev_next++];
    CK(cudaEventRecord(e0, s->st), "event record");
  }
  if (L.sel_dec) {
    // the selector's decisions for every chunk the gate rewrites, before either gate kernel
    const unsigned long long n = L.pair ? 2ull * L.items : L.nact;
    const unsigned long long want = (n + 255ull) / 256ull;
    const int sg = (unsigned long long)s->grid < want ? s->grid : (int)want;
    CK(qc::launch_select(L, s->d_mlp, s->d_dec, sg, s->st), "selector kernel launch");
    s->kernel_launches += 1;
  }
  if (fast) {
    // the streaming kernel first; the general kernel then runs the items it left
    const unsigned long long want = (L.items + qc::fast_pairs() - 1) / qc::fast_pairs();
    const int fg = (unsigned long long)s->fast_grid < want ? s->fast_grid : (int)want;
    CK(qc::launch_gate_fast(L, fg, s->st), "streaming gate kernel launch");
    L.list = 1;
    s->kernel_launches += 1;
  }
  CK(qc::launch_gate(L, grid, s->st), "gate kernel launch");
  s->kernel_launches += 2;  // with the post kernel below
  if (s->timing) {
    CK(cudaEventRecord(e1, s->st), "event record");
    s->ev_pending.emplace_back(e0, e1);
  }
  CK(qc::launch_post(s->P, L.ctl, s->grid, s->st), "post kernel launch");
  if (s->timing) {
    // the traffic counters after this gate, for the per-launch figures of sim_timing_launches
    const size_t k = s->ev_pending.size() - 1;
    if (k >= s->tlog_cap) {
      const size_t cap = s->tlog_cap ? 2 * s->tlog_cap : 4096;
      unsigned long long* p = nullptr;
      CK(cudaMallocAsync(&p, cap * 2 * sizeof(unsigned long long), s->st), "timing log");
      if (s->tlog_cap)
        CK(cudaMemcpyAsync(p, s->d_tlog, s->tlog_cap * 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                           s->st), "timing log copy");
      if (s->d_tlog) CK(cudaFreeAsync(s->d_tlog, s->st), "timing log");
      s->d_tlog = p;
      s->tlog_cap = cap;
    }
    CK(cudaMemcpyAsync(s->d_tlog + 2 * k, &s->d_ctl->bytes_in, 2 * sizeof(unsigned long long),
                       cudaMemcpyDeviceToDevice, s->st), "timing log");
  }
  s->amp_updates += L.nact << s->kc;
  return SIM_OK;
}

sim_status sim_apply_gate(sim_t* s, const sim_gate* g) {
  if (!s || !g) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  std::string why;
  if (!gate_ok(g, s->n, &why)) return fail(SIM_ERR_INVALID, "invalid gate: %s", why.c_str());
  return enqueue_gate(s, g);
}

sim_status sim_apply_circuit(sim_t* s, const sim_gate* gates, size_t n_gates) {
  if (!s || (!gates && n_gates)) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  std::string why;
  for (size_t k = 0; k < n_gates; ++k)
    if (!gate_ok(gates + k, s->n, &why)) return fail(SIM_ERR_INVALID, "invalid gate %zu: %s", k, why.c_str());
  for (size_t k = 0; k < n_gates; ++k)
    if (sim_status r = enqueue_gate(s, gates + k)) return r;
  return s->check_device();
}

sim_status sim_sync(sim_t* s) {
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  if (sim_status r = s->guard()) return r;
  return s->check_device();
}

static sim_status read_traffic(sim* s, unsigned long long* in, unsigned long long* out) {
  unsigned long long v[2];
  CK(cudaMemcpyAsync(v, &s->d_ctl->bytes_in, sizeof(v), cudaMemcpyDeviceToHost, s->st), "copy counters");
  CK(cudaStreamSynchronize(s->st), "sync");
  *in = v[0];
  *out = v[1];
  return SIM_OK;
}

sim_status sim_set_timing(sim_t* s, int on) {
  if (s) ++s->cfg_gen;  // a kept batch graph no longer matches
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  CK(cudaStreamSynchronize(s->st), "sync");
  s->timing = on != 0;
  s->phases = on >= 2;
  if (s->timing && !s->d_tlog) {  // room for the per-launch log of 8192 gates before it has to grow
    CK(cudaMalloc(&s->d_tlog, 8192 * 2 * sizeof(unsigned long long)), "timing log");
    s->tlog_cap = 8192;
  }
  s->ev_pending.clear();
  s->ev_next = 0;
  return read_traffic(s, &s->t_bytes_in0, &s->t_bytes_out0);
}

sim_status sim_timing_launches(sim_t* s, uint64_t cap, float* ms, uint64_t* bytes_read, uint64_t* bytes_written,
                               uint64_t* n) {
  if (!s || !n || (cap && (!ms || !bytes_read || !bytes_written))) return fail(SIM_ERR_INVALID, "NULL argument");
  CK(cudaStreamSynchronize(s->st), "sync");
  const size_t k = s->ev_pending.size();
  *n = k;
  if (k == 0 || cap == 0) return SIM_OK;
  std::vector<unsigned long long> log(2 * k);
  CK(cudaMemcpy(log.data(), s->d_tlog, 2 * k * sizeof(unsigned long long), cudaMemcpyDeviceToHost), "timing log");
  unsigned long long in0 = s->t_bytes_in0, out0 = s->t_bytes_out0;
  for (size_t i = 0; i < k && i < cap; ++i) {
    float m = 0.f;
    CK(cudaEventElapsedTime(&m, s->ev_pending[i].first, s->ev_pending[i].second), "event elapsed");
    ms[i] = m;
    bytes_read[i] = log[2 * i] - in0;
    bytes_written[i] = log[2 * i + 1] - out0;
    in0 = log[2 * i];
    out0 = log[2 * i + 1];
  }
  return SIM_OK;
}

sim_status sim_timing(sim_t* s, double* ms, uint64_t* launches, uint64_t* bytes_read, uint64_t* bytes_written) {
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  CK(cudaStreamSynchronize(s->st), "sync");
  double tot = 0.0;
  for (auto& pr : s->ev_pending) {
    float m = 0.f;
    CK(cudaEventElapsedTime(&m, pr.first, pr.second), "event elapsed");
    tot += m;
  }
  if (ms) *ms = tot;
  if (launches) *launches = s->ev_pending.size();
  unsigned long long in = 0, out = 0;
  if (sim_status r = read_traffic(s, &in, &out)) return r;
  if (bytes_read) *bytes_read = in - s->t_bytes_in0;
  if (bytes_written) *bytes_written = out - s->t_bytes_out0;
  s->t_bytes_in0 = in;
  s->t_bytes_out0 = out;
  s->ev_pending.clear();
  s->ev_next = 0;
  return SIM_OK;
}

sim_status sim_set_budget(sim_t* s, uint64_t bytes) {
  if (s) ++s->cfg_gen;  // a kept batch graph no longer matches
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  if (bytes == 0) return fail(SIM_ERR_INVALID, "budget must be > 0");
  if (sim_status r = s->guard()) return r;
  CK(cudaStreamSynchronize(s->st), "sync");
  s->budget = bytes;
  s->cp.thresh = (unsigned long long)std::floor(s->tau * (double)bytes);
  return SIM_OK;
}

sim_status sim_set_option(sim_t* s, const char* key, int64_t value) {
  if (s) ++s->cfg_gen;  // a kept batch graph no longer matches
  if (!s || !key) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  const std::string k(key);
  if (k == "modes") return sim_set_modes(s, (uint32_t)value);
  if (k == "selector") {
    if (value != 0 && value != 1) return fail(SIM_ERR_INVALID, "selector 2 needs its parameters: sim_set_selector");
    return sim_set_selector(s, (int)value, nullptr);
  }
  if (k == "block_cache") return sim_set_block_cache(s, value != 0);
  if (k == "timing") return sim_set_timing(s, (int)value);
  if (k == "fast_path") {
    if (value != 0 && value != 1) return fail(SIM_ERR_INVALID, "fast_path must be 0 or 1");
    s->fast = value != 0;
    return SIM_OK;
  }
  if (k == "tau_ppm") {
    if (value <= 0 || value > 1000000) return fail(SIM_ERR_INVALID, "tau_ppm must be in (0, 1000000]");
    CK(cudaStreamSynchronize(s->st), "sync");
    s->tau = (double)value * 1e-6;
    s->cp.thresh = (unsigned long long)std::floor(s->tau * (double)s->budget);
    return SIM_OK;
  }
  if (k == "ladder") {
    if (value < 0 || value > 2) return fail(SIM_ERR_INVALID, "ladder must be 0, 1 or 2");
    DevCtl h{};
    CK(cudaMemcpyAsync(&h, s->d_ctl, sizeof(h), cudaMemcpyDeviceToHost, s->st), "copy counters");
    CK(cudaStreamSynchronize(s->st), "sync");
    if (h.gates != 0) return fail(SIM_ERR_INVALID, "the ladder can only change before the first gate");
    CtlParams& cp = s->cp;
    cp.ladder = (int)value;
    s->ladder = (int)value;
    cp.nlevels = 0;
    if (s->eps_max > 0.0) {
      static const double paper[5] = {1e-5, 1e-4, 1e-3, 1e-2, 1e-1};
      if (value >= 1)
        for (double e : paper)
          if (e < s->eps_max) s->level_eps[cp.nlevels++] = e;
      s->level_eps[cp.nlevels++] = s->eps_max;
    }
    for (int l = 0; l < cp.nlevels; ++l) {
      cp.S[l] = sig_bits_of(s->level_eps[l]);
      cp.delta[l] = std::ldexp(1.0, 12 - cp.S[l]);
    }
    for (int l = 0; l <= cp.nlevels; ++l) cp.maxb[l] = qc::max_level_image(s->kc, l == 0 ? 64 : cp.S[l - 1]);
    return SIM_OK;
  }
  if (k == "chunk_log2" || k == "block_log2")
    return fail(SIM_ERR_INVALID, "%s is fixed when the handle is created (sim_create_ex)", key);
  return fail(SIM_ERR_INVALID, "unknown option '%s'", key);
}

sim_status sim_set_block_cache(sim_t* s, int on) {
  if (s) ++s->cfg_gen;  // a kept batch graph no longer matches
  if (!s) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  CK(cudaStreamSynchronize(s->st), "sync");
  if (!on) {
    cudaFree(s->d_bc);
    s->d_bc = nullptr;
    return SIM_OK;
  }
  if (s->d_bc) return SIM_OK;
  const size_t bytes = (size_t)qc::kBcLines * qc::bc_line_bytes(qc::round16(qc::max_image_bytes(s->kc)));
  CK(cudaMalloc(&s->d_bc, bytes), "block cache");
  CK(cudaMemset(s->d_bc, 0, bytes), "block cache");  // every line empty, tag 0
  // a fresh cache starts switched on
  DevCtl h{};
  CK(cudaMemcpy(&h, s->d_ctl, sizeof(h), cudaMemcpyDeviceToHost), "copy counters");
  h.bc_off = 0;
  h.bc_zero_streak = 0;
  CK(cudaMemcpy(s->d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice), "copy counters");
  return SIM_OK;
}

sim_status sim_set_modes(sim_t* s, uint32_t modes) {
  if (s) ++s->cfg_gen;  // a kept batch graph no longer matches
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  if ((modes & qc::kDefaultModes) != qc::kDefaultModes || (modes >> qc::M_NMODES))
    return fail(SIM_ERR_INVALID, "the mode set must contain ZERO..RAW (0x1F) and only known modes");
  s->modes = modes;
  return SIM_OK;
}

sim_status sim_set_selector(sim_t* s, int selector, const uint16_t* bf16_params) {
  if (s) ++s->cfg_gen;  // a kept batch graph no longer matches
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  if (selector < 0 || selector > 2) return fail(SIM_ERR_INVALID, "selector must be 0, 1 or 2");
  if (selector == 2) {
    if (!bf16_params) return fail(SIM_ERR_INVALID, "the selector network needs its parameters");
    if (!s->d_mlp) CK(cudaMalloc(&s->d_mlp, qc::kMlpParams * 2), "selector parameters");
    if (!s->d_dec) CK(cudaMalloc(&s->d_dec, s->nchunks + 16), "selector decisions");
    CK(cudaMemcpy(s->d_mlp, bf16_params, qc::kMlpParams * 2, cudaMemcpyHostToDevice), "selector parameters");
  }
  s->modes = selector == 1 ? qc::kAllModes : qc::kDefaultModes;
  s->selector = selector == 2 ? 2 : 0;
  return SIM_OK;
}

sim_status sim_trace(sim_t* s, uint64_t capacity) {
  if (s) ++s->cfg_gen;  // a kept batch graph no longer matches
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  CK(cudaStreamSynchronize(s->st), "sync");
  cudaFree(s->d_trace);
  s->d_trace = nullptr;
  s->trace_cap = 0;
  CK(cudaMemset(&s->d_ctl->trace_n, 0, sizeof(unsigned long long)), "trace counter");
  if (capacity == 0) return SIM_OK;
  CK(cudaMalloc(&s->d_trace, capacity * qc::kTraceFloats * sizeof(float)), "trace buffer");
  s->trace_cap = capacity;
  return SIM_OK;
}

sim_status sim_trace_read(sim_t* s, float* out, uint64_t cap_records, uint64_t* n_records) {
  if (!s || !out || !n_records) return fail(SIM_ERR_INVALID, "NULL argument");
  unsigned long long n = 0;
  CK(cudaMemcpyAsync(&n, &s->d_ctl->trace_n, sizeof(n), cudaMemcpyDeviceToHost, s->st), "trace counter");
  CK(cudaStreamSynchronize(s->st), "sync");
  if (n > s->trace_cap) n = s->trace_cap;
  if (n > cap_records) n = cap_records;
  if (n) CK(cudaMemcpy(out, s->d_trace, n * qc::kTraceFloats * sizeof(float), cudaMemcpyDeviceToHost), "trace copy");
  *n_records = n;
  return SIM_OK;
}

sim_status sim_layout(sim_t* s, uint64_t* n_chunks, int* chunk_log2, int* block_log2) {
  if (!s) return fail(SIM_ERR_INVALID, "NULL handle");
  if (n_chunks) *n_chunks = s->nchunks;
  if (chunk_log2) *chunk_log2 = s->kc;
  if (block_log2) *block_log2 = s->b;
  return SIM_OK;
}

sim_status sim_amplitudes(sim_t* s, uint64_t first, uint64_t count, double* out, int out_on_device) {
  if (!s || (!out && count)) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  const uint64_t total = 1ull << s->n;
  if (first > total || count > total - first) return fail(SIM_ERR_INVALID, "amplitude range outside the state");
  if (count == 0) return SIM_OK;
  if (out_on_device) {
    CK(qc::launch_decode_range(s->P, first, count, out, s->st), "decode launch");
    return s->check_device();
  }
  const uint64_t slice = 1ull << 22;  // amplitudes per staging pass (64 MiB)
  if (sim_status r = s->scratch((size_t)slice * 16)) return r;
  for (uint64_t off = 0; off < count; off += slice) {
    const uint64_t m = count - off < slice ? count - off : slice;
    CK(qc::launch_decode_range(s->P, first + off, m, reinterpret_cast<double*>(s->d_scratch), s->st), "decode");
    CK(cudaMemcpyAsync(out + 2 * off, s->d_scratch, m * 16, cudaMemcpyDeviceToHost, s->st), "copy out");
    CK(cudaStreamSynchronize(s->st), "sync");
  }
  return s->check_device();
}

static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

sim_status sim_measure(sim_t* s, uint64_t seed, uint64_t* outcome, double* prob) {
  if (!s || !outcome || !prob) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  const uint64_t nc = s->nchunks;
  if (sim_status r = s->scratch((size_t)nc * 8)) return r;
  CK(qc::launch_chunk_norms(s->P, 0, nc, reinterpret_cast<double*>(s->d_scratch), s->st), "norm launch");
  std::vector<double> pc(nc);
  CK(cudaMemcpyAsync(pc.data(), s->d_scratch, nc * 8, cudaMemcpyDeviceToHost, s->st), "copy norms");
  if (sim_status r = s->check_device()) return r;
  double total = 0.0;
  for (double v : pc) total += v;
  const double u = (double)(splitmix64(seed) >> 11) * (1.0 / 9007199254740992.0);
  const double target = u * total;
  double run = 0.0;
  uint64_t c = 0;
  for (; c < nc; ++c) {
    if (run + pc[c] >= target && pc[c] > 0.0) break;
    run += pc[c];
  }
  if (c == nc) {  // rounding put the target past the end: take the last nonzero chunk
    c = nc - 1;
    while (c > 0 && pc[c] == 0.0) --c;
    run = 0.0;
    for (uint64_t k = 0; k < c; ++k) run += pc[k];
  }
  const uint64_t A = 1ull << s->kc;
  std::vector<double> amp(2 * A);
  if (sim_status r = sim_amplitudes(s, c * A, A, amp.data(), 0)) return r;
  uint64_t pick = A;
  uint64_t last_nz = 0;
  for (uint64_t i = 0; i < A; ++i) {
    const double p = std::fma(amp[2 * i], amp[2 * i], amp[2 * i + 1] * amp[2 * i + 1]);
    if (p > 0.0) last_nz = i;
    run += p;
    if (run >= target && p > 0.0) { pick = i; break; }
  }
  if (pick == A) { pick = last_nz; }
  const double p = std::fma(amp[2 * pick], amp[2 * pick], amp[2 * pick + 1] * amp[2 * pick + 1]);
  *outcome = c * A + pick;
  *prob = total > 0.0 ? p / total : 0.0;
  return SIM_OK;
}

sim_status sim_fidelity(sim_t* s, const double* ref, int ref_on_device, double* F, double* re_im, double* norm2) {
  if (!s || !ref || !F) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  const uint64_t nc = s->nchunks, A = 1ull << s->kc;
  const uint64_t per = ref_on_device ? nc : ((1ull << 22) / A > 0 ? (1ull << 22) / A : 1ull);  // chunks per pass
  const size_t ref_bytes = ref_on_device ? 0 : (size_t)per * A * 16;
  if (sim_status r = s->scratch(ref_bytes + (size_t)per * 24)) return r;
  double* d_out = reinterpret_cast<double*>(s->d_scratch + ref_bytes);
  std::vector<double> parts(3 * per);
  double re = 0.0, im = 0.0, nn = 0.0;
  for (uint64_t c0 = 0; c0 < nc; c0 += per) {
    const uint64_t m = nc - c0 < per ? nc - c0 : per;
    const double* dref = ref + 2 * c0 * A;
    if (!ref_on_device) {
      CK(cudaMemcpyAsync(s->d_scratch, ref + 2 * c0 * A, m * A * 16, cudaMemcpyHostToDevice, s->st), "copy ref");
      dref = reinterpret_cast<const double*>(s->d_scratch);
    }
    CK(qc::launch_chunk_dots(s->P, c0, m, dref, d_out, s->st), "dot launch");
    CK(cudaMemcpyAsync(parts.data(), d_out, m * 24, cudaMemcpyDeviceToHost, s->st), "copy parts");
    if (sim_status r = s->check_device()) return r;
    for (uint64_t k = 0; k < m; ++k) {
      re += parts[3 * k];
      im += parts[3 * k + 1];
      nn += parts[3 * k + 2];
    }
  }
  *F = std::sqrt(re * re + im * im);
  if (re_im) { re_im[0] = re; re_im[1] = im; }
  if (norm2) *norm2 = nn;
  return SIM_OK;
}

sim_status sim_stats(sim_t* s, sim_stats_t* o) {
  if (!s || !o) return fail(SIM_ERR_INVALID, "NULL argument");
  DevCtl h{};
  unsigned long long counts[8] = {0};
  CK(cudaMemsetAsync(s->d_counts, 0, sizeof(counts), s->st), "memset");
  CK(qc::launch_mode_counts(s->P, s->nchunks, s->d_counts, nullptr, s->st), "mode count launch");
  CK(cudaMemcpyAsync(&h, s->d_ctl, sizeof(h), cudaMemcpyDeviceToHost, s->st), "copy counters");
  CK(cudaMemcpyAsync(counts, s->d_counts, sizeof(counts), cudaMemcpyDeviceToHost, s->st), "copy counts");
  CK(cudaStreamSynchronize(s->st), "sync");
  std::memset(o, 0, sizeof(*o));
  o->gates = h.gates;
  o->encoded_bytes = h.E;
  o->max_encoded_bytes = h.Emax;
  o->raw_bytes = 16ull << s->n;
  o->inflight_bytes = s->cp.inflight;
  for (int k = 0; k < 8; ++k) o->chunks_by_mode[k] = counts[k];
  o->pool_bytes = s->npages * qc::kPage;
  o->pages_in_use_bytes = (s->npages - (uint64_t)h.top - h.wc_pages) * qc::kPage;  // pages holding images
  o->peak_pages_bytes = h.peak_pages * qc::kPage;
  o->device_bytes = s->device_bytes + s->scratch_bytes;
  o->amp_updates = s->amp_updates;
  o->ratio = h.E ? (double)o->raw_bytes / (double)h.E : 0.0;
  o->min_ratio = h.Emax ? (double)o->raw_bytes / (double)h.Emax : 0.0;
  o->eps_current = h.level ? s->level_eps[h.level - 1] : 0.0;
  o->fidelity_lb_sum = 1.0 - h.lb_sum;
  o->fidelity_lb_prod = h.lb_prod;
  o->eps_switch_gate = h.switch_gate;
  o->sig_bits_current = h.S_last;
  o->level = h.level;
  o->chunk_log2 = s->kc;
  o->block_log2 = s->b;
  for (int k = 0; k < 6; ++k) o->phase_cycles[k] = h.phase_cycles[k];
  o->split_trials = h.split_trials;
  o->cache_lookups = h.bc_lookups;
  o->cache_hits = h.bc_hits;
  o->fast_items = h.fast_items;
  o->fast_deferred = h.fast_deferred;
  o->kernel_launches = s->kernel_launches;
  o->palette_trials = h.palette_trials;
  o->graph_replays = s->graph_replays;
  o->ladder = s->ladder;
  o->modes = s->modes;
  o->wide_images = h.n64 < 0 ? 0 : (uint64_t)h.n64;
  if (h.err) return s->check_device();
  return SIM_OK;
}

sim_status sim_chunk_image(sim_t* s, uint64_t c, uint8_t* out, size_t cap, size_t* len) {
  if (!s || !out || !len) return fail(SIM_ERR_INVALID, "NULL argument");
  if (c >= s->nchunks) return fail(SIM_ERR_INVALID, "chunk index outside the state");
  uint32_t head[2];
  const size_t stride = qc::dir_stride(s->kc);
  CK(cudaMemcpyAsync(head, reinterpret_cast<uint8_t*>(s->P.dir) + c * stride, 8, cudaMemcpyDeviceToHost, s->st),
     "copy dir");
  CK(cudaStreamSynchronize(s->st), "sync");
  *len = head[0];
  if (head[0] > cap) return fail(SIM_ERR_INVALID, "buffer too small for the image (%u bytes)", head[0]);
  if (sim_status r = s->scratch(qc::max_image_bytes(s->kc) + 16)) return r;
  CK(qc::launch_copy_image(s->P, c, s->d_scratch, s->st), "copy image launch");
  CK(cudaMemcpyAsync(out, s->d_scratch, head[0], cudaMemcpyDeviceToHost, s->st), "copy image");
  CK(cudaStreamSynchronize(s->st), "sync");
  return SIM_OK;
}

// ------------------------------------------------------------ batch ------ //
sim_status sim_batch_apply(sim_t* const* sims, int count, const sim_gate* const* circuits, const size_t* n_gates,
                           int use_graph) {
  if (!sims || !circuits || !n_gates || count < 1) return fail(SIM_ERR_INVALID, "bad batch arguments");
  const int kc = sims[0] ? sims[0]->kc : -1;
  size_t steps = 0;
  std::string why;
  for (int k = 0; k < count; ++k) {
    sim* s = sims[k];
    if (!s) return fail(SIM_ERR_INVALID, "NULL handle in the batch");
    if (s->kc != kc) return fail(SIM_ERR_INVALID, "all handles of a batch must share chunk_log2");
    if (sim_status r = s->guard()) return r;
    for (int j = 0; j < k; ++j)
      if (sims[j] == s) return fail(SIM_ERR_INVALID, "a handle appears twice in the batch");
    if (n_gates[k] && !circuits[k]) return fail(SIM_ERR_INVALID, "NULL circuit in the batch");
    for (size_t i = 0; i < n_gates[k]; ++i)
      if (!gate_ok(circuits[k] + i, s->n, &why)) return fail(SIM_ERR_INVALID, "circuit %d gate %zu: %s", k, i, why.c_str());
    if (n_gates[k] > steps) steps = n_gates[k];
  }
  if (steps == 0) return SIM_OK;
  cudaStream_t st = sims[0]->st;
  sim* lead = sims[0];
  // What the launch sequence depends on: the handles (by creation number, so that a
  // new handle at a freed address never matches) with the generation of their
  // settings, and the gates.  A call with the same key makes the same launches, so the
  // graph the lead handle kept can be replayed as it stands.
  std::vector<uint8_t> key;
  if (use_graph) {
    auto put = [&key](const void* p, size_t n) {
      const uint8_t* b = static_cast<const uint8_t*>(p);
      key.insert(key.end(), b, b + n);
    };
    put(&count, sizeof count);
    for (int k = 0; k < count; ++k) {
      put(&sims[k]->uid, sizeof(uint64_t));
      put(&sims[k]->cfg_gen, sizeof(uint64_t));
      put(&n_gates[k], sizeof(size_t));
    }
    for (int k = 0; k < count; ++k) put(circuits[k], n_gates[k] * sizeof(sim_gate));
  }
  cudaError_t e = cudaSuccess;
  std::vector<uint64_t> upd(count, 0);  // amplitude updates each circuit makes
  if (use_graph && lead->bexec && key == lead->bkey) {
    // the job list is still on the device, unchanged: launch the instantiated graph
    upd = lead->bupd;
    e = cudaEventRecord(lead->bready, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(lead->bstream, lead->bready, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(lead->bexec, lead->bstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lead->bstream);
    if (e == cudaSuccess) ++lead->graph_replays;
  } else {
    if (use_graph) lead->drop_graph();
    // step t holds gate t of every circuit that has one; its jobs' items are numbered
    // consecutively
    std::vector<qc::BatchJob> jobs;
    std::vector<sim*> job_sim;  // the handle of each job
    std::vector<size_t> off(steps + 1, 0);
    std::vector<unsigned long long> total(steps, 0);
    int grid = sims[0]->grid;
    for (int k = 1; k < count; ++k) grid = sims[k]->grid < grid ? sims[k]->grid : grid;
    for (size_t t = 0; t < steps; ++t) {
      off[t] = jobs.size();
      unsigned long long begin = 0;
      for (int k = 0; k < count; ++k) {
        if (t >= n_gates[k]) continue;
        qc::BatchJob j;
        j.L = make_launch(sims[k], circuits[k] + t);
        j.begin = begin;
        begin += j.L.items;
        upd[k] += j.L.nact << sims[k]->kc;
        jobs.push_back(j);
        job_sim.push_back(sims[k]);
      }
      total[t] = begin;
    }
    off[steps] = jobs.size();
    qc::BatchJob* d_jobs = nullptr;
    CK(cudaMalloc(&d_jobs, jobs.size() * sizeof(qc::BatchJob)), "batch job list");
    e = cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(qc::BatchJob), cudaMemcpyHostToDevice, st);
    // A graph is captured on a private stream (the legacy default stream cannot be
    // captured), ordered after the work already queued on the handles' stream.
    cudaStream_t cs = st;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && use_graph) {
      if (!lead->bstream) e = cudaStreamCreateWithFlags(&lead->bstream, cudaStreamNonBlocking);
      if (e == cudaSuccess && !lead->bready) e = cudaEventCreateWithFlags(&lead->bready, cudaEventDisableTiming);
      if (e == cudaSuccess) cs = lead->bstream;
      if (e == cudaSuccess) e = cudaEventRecord(lead->bready, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, lead->bready, 0);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    }
    for (size_t t = 0; t < steps && e == cudaSuccess; ++t) {
      const int n = (int)(off[t + 1] - off[t]);
      const int g = (unsigned long long)grid < total[t] ? grid : (int)total[t];
      // the selector's decisions of every handle that runs the network, before the step
      for (size_t j = off[t]; j < off[t + 1] && e == cudaSuccess; ++j) {
        const GateLaunch& L = jobs[j].L;
        if (!L.sel_dec) continue;
        const unsigned long long na = L.pair ? 2ull * L.items : L.nact;
        const int sg = (unsigned long long)grid < (na + 255ull) / 256ull ? grid : (int)((na + 255ull) / 256ull);
        e = qc::launch_select(L, job_sim[j]->d_mlp, const_cast<uint8_t*>(L.sel_dec), sg, cs);
      }
      if (e == cudaSuccess) e = qc::launch_gate_batch(d_jobs + off[t], n, total[t], kc, g, cs);
      if (e == cudaSuccess) e = qc::launch_post_batch(d_jobs + off[t], n, grid, cs);
    }
    if (use_graph && cs != st) {
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (e == cudaSuccess) e = cudaGraphLaunch(exec, cs);
      if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess && exec) {
      // kept for the next call with the same key (the job list stays with it)
      lead->bexec = exec;
      lead->bjobs = d_jobs;
      lead->bkey.swap(key);
      lead->bupd = upd;
    } else {
      if (exec) cudaGraphExecDestroy(exec);
      cudaFree(d_jobs);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    for (int k = 0; k < count; ++k) sims[k]->poisoned = SIM_ERR_CUDA;
    return cuda_fail(e, "batched launch");
  }
  for (int k = 0; k < count; ++k) sims[k]->amp_updates += upd[k];
  sim_status worst = SIM_OK;
  for (int k = 0; k < count; ++k) {
    sim_status r = sims[k]->check_device();
    if (r != SIM_OK && worst == SIM_OK) worst = r;
  }
  return worst;
}

sim_status sim_batch_run(int n_circ, const int* n_qubits, const sim_gate* const* circ, const size_t* n_gates,
                         double err_bound, sim_stats_t* out) {
  if (n_circ < 1 || !n_qubits || !circ || !n_gates || !out) return fail(SIM_ERR_INVALID, "bad batch arguments");
  int nmin = 64, big = 0;
  for (int k = 0; k < n_circ; ++k) {
    if (n_qubits[k] < 1 || n_qubits[k] > 40) return fail(SIM_ERR_INVALID, "n_qubits must be in [1, 40]");
    if (n_qubits[k] < nmin) nmin = n_qubits[k];
    if (n_qubits[k] > n_qubits[big] || (n_qubits[k] == n_qubits[big] && n_gates[k] > n_gates[big])) big = k;
  }
  // one setting for the whole batch, autotuned on the largest circuit when it is long
  // enough: block size 2^10..2^16, chunk (tile) size 2^8..2^10, bound ladder, mode set
  sim_tune_point cfg{};
  cfg.block_log2 = 20;
  cfg.chunk_log2 = nmin < 10 ? nmin : 10;
  cfg.ladder = 0;
  cfg.modes = qc::kDefaultModes;
  if (n_gates[big] >= 4 && nmin >= 8) {
    const int32_t bs[7] = {16, 10, 11, 12, 13, 14, 15}, ls[3] = {0, 1, 2};
    const uint32_t ms[2] = {qc::kDefaultModes, qc::kDefaultModes | (1u << qc::M_PALETTE)};
    int32_t cs[3];
    int nc = 0;
    for (int c = 10; c >= 8 && nc < 3; --c)
      if (c <= nmin) cs[nc++] = c;
    if (sim_status r = sim_autotune(n_qubits[big], err_bound, circ[big], n_gates[big], bs, 7, cs, nc, ls, 3, ms, 2, &cfg,
                                    nullptr, 0, nullptr))
      return r;
  }
  std::vector<sim_t*> sims(n_circ, nullptr);
  sim_status r = SIM_OK;
  for (int k = 0; k < n_circ && r == SIM_OK; ++k) {
    const uint64_t raw = 16ull << n_qubits[k];
    r = sim_create_ex(n_qubits[k], cfg.block_log2, cfg.chunk_log2, err_bound, raw / 4 ? raw / 4 : 1, 0.9, cfg.ladder,
                      raw + raw / 8 + (8ull << 20), &sims[k]);
    if (r == SIM_OK) r = sim_set_modes(sims[k], cfg.modes);
  }
  if (r == SIM_OK) r = sim_batch_apply(sims.data(), n_circ, circ, n_gates, 1);
  for (int k = 0; k < n_circ && r == SIM_OK; ++k) r = sim_stats(sims[k], &out[k]);
  for (sim_t* s : sims)
    if (s) sim_destroy(s);
  return r;
}

// One autotuner measurement: a handle with the point's settings (budget raw/4, pool
// raw + 1/8 + 64 MiB) runs the first half of the probe untimed, then the second half
// with gate-kernel timing; fills rate, ratio (raw over the peak encoded bytes) and the
// fidelity bound.
static sim_status tune_eval(int n_qubits, double err_bound, const sim_gate* probe, size_t n_probe, sim_tune_point& p) {
  const uint64_t raw = 16ull << n_qubits;
  sim_t* s = nullptr;
  sim_status r = sim_create_ex(n_qubits, p.block_log2, p.chunk_log2, err_bound, raw / 4 ? raw / 4 : 1, 0.9, p.ladder,
                               raw + raw / 8 + (64ull << 20), &s);
  if (r != SIM_OK) return r;
  r = sim_set_modes(s, p.modes);
  const size_t half = n_probe / 2;
  if (r == SIM_OK) r = sim_apply_circuit(s, probe, half);
  if (r == SIM_OK) r = sim_set_timing(s, 1);
  const uint64_t before = s->amp_updates;
  if (r == SIM_OK) r = sim_apply_circuit(s, probe + half, n_probe - half);
  double ms = 0.0;
  if (r == SIM_OK) r = sim_timing(s, &ms, nullptr, nullptr, nullptr);
  sim_stats_t st{};
  if (r == SIM_OK) r = sim_stats(s, &st);
  p.rate = (r == SIM_OK && ms > 0.0) ? (double)(s->amp_updates - before) / (ms * 1e-3) : 0.0;
  p.ratio = st.min_ratio;
  p.fidelity_lb_sum = st.fidelity_lb_sum;
  sim_destroy(s);
  return r;
}

sim_status sim_autotune_chunk(int n_qubits, int block_log2, double err_bound, const sim_gate* probe, size_t n_probe,
                              const int* candidates, int n_candidates, int* best, double* rates) {
  if (!probe || !candidates || !best || n_candidates < 1 || n_probe < 2)
    return fail(SIM_ERR_INVALID, "bad autotune arguments");
  double best_rate = -1.0;
  *best = candidates[0];
  for (int i = 0; i < n_candidates; ++i) {
    sim_tune_point p{};
    p.block_log2 = block_log2;
    p.chunk_log2 = candidates[i];
    p.ladder = 0;
    p.modes = qc::kDefaultModes;
    if (sim_status r = tune_eval(n_qubits, err_bound, probe, n_probe, p)) return r;
    if (rates) rates[i] = p.rate;
    if (p.rate > best_rate) {
      best_rate = p.rate;
      *best = candidates[i];
    }
  }
  return SIM_OK;
}

sim_status sim_autotune(int n_qubits, double err_bound, const sim_gate* probe, size_t n_probe,
                        const int32_t* block_log2s, int n_b, const int32_t* chunk_log2s, int n_c, const int32_t* ladders,
                        int n_l, const uint32_t* mode_sets, int n_m, sim_tune_point* best, sim_tune_point* tried,
                        size_t cap_tried, size_t* n_tried) {
  if (!probe || n_probe < 2 || !block_log2s || !chunk_log2s || !ladders || !mode_sets || n_b < 1 || n_c < 1 ||
      n_l < 1 || n_m < 1 || !best || n_qubits < 1 || n_qubits > 40)
    return fail(SIM_ERR_INVALID, "bad autotune arguments");
  std::string why;
  for (size_t i = 0; i < n_probe; ++i)
    if (!gate_ok(probe + i, n_qubits, &why)) return fail(SIM_ERR_INVALID, "probe gate %zu: %s", i, why.c_str());
  for (int i = 0; i < n_b; ++i)
    if (block_log2s[i] < 0) return fail(SIM_ERR_INVALID, "block_log2 must be >= 0");
  for (int i = 0; i < n_c; ++i)
    if (chunk_log2s[i] < 0 || chunk_log2s[i] > 11) return fail(SIM_ERR_INVALID, "chunk_log2 must be in [0, 11]");
  for (int i = 0; i < n_l; ++i)
    if (ladders[i] < 0 || ladders[i] > 2) return fail(SIM_ERR_INVALID, "ladder must be 0, 1 or 2");
  for (int i = 0; i < n_m; ++i)
    if ((mode_sets[i] & qc::kDefaultModes) != qc::kDefaultModes || (mode_sets[i] >> qc::M_NMODES))
      return fail(SIM_ERR_INVALID, "a mode set must contain 0x1F and only known modes");
  // the settings as the handle applies them: blocks clamp to n, chunks to the block
  auto canon = [n_qubits](sim_tune_point p) {
    p.block_log2 = p.block_log2 < n_qubits ? p.block_log2 : n_qubits;
    p.chunk_log2 = p.chunk_log2 < p.block_log2 ? p.chunk_log2 : p.block_log2;
    return p;
  };
  std::vector<sim_tune_point> seen;
  auto eval = [&](sim_tune_point p, sim_tune_point& out) -> sim_status {
    p = canon(p);
    for (const sim_tune_point& q : seen)
      if (q.block_log2 == p.block_log2 && q.chunk_log2 == p.chunk_log2 && q.ladder == p.ladder && q.modes == p.modes) {
        out = q;
        return SIM_OK;
      }
    if (sim_status r = tune_eval(n_qubits, err_bound, probe, n_probe, p)) return r;
    seen.push_back(p);
    out = p;
    return SIM_OK;
  };
  // coordinate descent from the first value of every axis: the tile (chunk) size, the
  // block size, the bound ladder, the mode set; repeated until a sweep changes nothing
  sim_tune_point cur{};
  cur.block_log2 = block_log2s[0];
  cur.chunk_log2 = chunk_log2s[0];
  cur.ladder = ladders[0];
  cur.modes = mode_sets[0];
  if (sim_status r = eval(cur, cur)) return r;
  for (int sweep = 0; sweep < 3; ++sweep) {
    const sim_tune_point start = cur;
    for (int axis = 0; axis < 4; ++axis) {
      const int n = axis == 0 ? n_c : axis == 1 ? n_b : axis == 2 ? n_l : n_m;
      sim_tune_point pick = cur;
      for (int i = 0; i < n; ++i) {
        sim_tune_point p = cur;
        if (axis == 0) p.chunk_log2 = chunk_log2s[i];
        if (axis == 1) p.block_log2 = block_log2s[i];
        if (axis == 2) p.ladder = ladders[i];
        if (axis == 3) p.modes = mode_sets[i];
        sim_tune_point got{};
        if (sim_status r = eval(p, got)) return r;
        if (got.rate > pick.rate) pick = got;
      }
      cur = pick;
    }
    if (cur.block_log2 == start.block_log2 && cur.chunk_log2 == start.chunk_log2 && cur.ladder == start.ladder &&
        cur.modes == start.modes)
      break;
  }
  *best = cur;
  if (n_tried) *n_tried = seen.size();
  for (size_t i = 0; tried && i < seen.size() && i < cap_tried; ++i) tried[i] = seen[i];
  return SIM_OK;
}

// ----------------------------------------------------------- checkpoint -- //
namespace {

struct CkHeader {
  char magic[8];  // "QCSIMCK1"
  uint32_t version, n, b, kc;
  double eps_max;
  uint64_t budget;
  double tau;
  int32_t ladder;
  uint32_t modes;
  int32_t level, S_last;
  uint64_t E, Emax, gates;
  int64_t switch_gate;
  double lb_sum, lb_prod;
  uint64_t amp_updates, peak_pages, nchunks, image_bytes;
};
static_assert(sizeof(CkHeader) <= 256, "checkpoint header must fit 256 bytes");
constexpr uint64_t kCkHead = 256;
const char kCkMagic[8] = {'Q', 'C', 'S', 'I', 'M', 'C', 'K', '1'};

// Image lengths of every chunk on the host, and their exclusive prefix sums.
sim_status ck_lengths(sim* s, std::vector<uint32_t>& len, std::vector<unsigned long long>& off, uint64_t& total) {
  uint32_t* d_len = nullptr;
  CK(cudaMalloc(&d_len, s->nchunks * 4), "checkpoint lengths");
  cudaError_t e = qc::launch_checkpoint_lengths(s->P, s->nchunks, d_len, s->st);
  len.resize(s->nchunks);
  if (e == cudaSuccess) e = cudaMemcpyAsync(len.data(), d_len, s->nchunks * 4, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(d_len);
  if (e != cudaSuccess) return cuda_fail(e, "checkpoint lengths");
  off.resize(s->nchunks);
  total = 0;
  for (uint64_t c = 0; c < s->nchunks; ++c) {
    off[c] = total;
    total += len[c];
  }
  return SIM_OK;
}

}  // namespace

sim_status sim_checkpoint_size(sim_t* s, uint64_t* bytes) {
  if (!s || !bytes) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  std::vector<uint32_t> len;
  std::vector<unsigned long long> off;
  uint64_t total = 0;
  if (sim_status r = ck_lengths(s, len, off, total)) return r;
  *bytes = kCkHead + 4 * s->nchunks + total;
  return SIM_OK;
}

sim_status sim_checkpoint_save(sim_t* s, void* out, uint64_t cap, int out_on_device) {
  if (!s || !out) return fail(SIM_ERR_INVALID, "NULL argument");
  if (sim_status r = s->guard()) return r;
  std::vector<uint32_t> len;
  std::vector<unsigned long long> off;
  uint64_t total = 0;
  if (sim_status r = ck_lengths(s, len, off, total)) return r;
  const uint64_t need = kCkHead + 4 * s->nchunks + total;
  if (cap < need) return fail(SIM_ERR_INVALID, "checkpoint buffer too small (see sim_checkpoint_size)");
  DevCtl h{};
  CK(cudaMemcpyAsync(&h, s->d_ctl, sizeof(h), cudaMemcpyDeviceToHost, s->st), "copy counters");
  CK(cudaStreamSynchronize(s->st), "sync");
  if (h.err) return s->check_device();
  uint8_t head[kCkHead] = {0};
  CkHeader k{};
  std::memcpy(k.magic, kCkMagic, 8);
  k.version = 1;
  k.n = (uint32_t)s->n;
  k.b = (uint32_t)s->b;
  k.kc = (uint32_t)s->kc;
  k.eps_max = s->eps_max;
  k.budget = s->budget;
  k.tau = s->tau;
  k.ladder = s->ladder;
  k.modes = s->modes;
  k.level = h.level;
  k.S_last = h.S_last;
  k.E = h.E;
  k.Emax = h.Emax;
  k.gates = h.gates;
  k.switch_gate = h.switch_gate;
  k.lb_sum = h.lb_sum;
  k.lb_prod = h.lb_prod;
  k.amp_updates = s->amp_updates;
  k.peak_pages = h.peak_pages;
  k.nchunks = s->nchunks;
  k.image_bytes = total;
  std::memcpy(head, &k, sizeof(k));
  // images: gathered on the device, straight into the caller's buffer when it is there
  unsigned long long* d_off = nullptr;
  uint8_t* d_img = nullptr;
  CK(cudaMalloc(&d_off, s->nchunks * 8), "checkpoint offsets");
  uint8_t* base = reinterpret_cast<uint8_t*>(out);
  cudaError_t e = cudaMemcpyAsync(d_off, off.data(), s->nchunks * 8, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess && !out_on_device && total) e = cudaMalloc(&d_img, total);
  uint8_t* dst = out_on_device ? base + kCkHead + 4 * s->nchunks : d_img;
  if (e == cudaSuccess && total) e = qc::launch_checkpoint_gather(s->P, s->nchunks, d_off, dst, s->st);
  const cudaMemcpyKind k_to = out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  if (e == cudaSuccess) e = cudaMemcpyAsync(base, head, kCkHead, k_to, s->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kCkHead, len.data(), 4 * s->nchunks, k_to, s->st);
  if (e == cudaSuccess && !out_on_device && total)
    e = cudaMemcpyAsync(base + kCkHead + 4 * s->nchunks, d_img, total, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(d_off);
  cudaFree(d_img);
  if (e != cudaSuccess) return cuda_fail(e, "checkpoint save");
  return SIM_OK;
}

sim_status sim_checkpoint_load(sim_t* s, const void* in, uint64_t in_len, int in_on_device) {
  if (s) ++s->cfg_gen;  // a kept batch graph no longer matches
  if (!s || !in) return fail(SIM_ERR_INVALID, "NULL argument");
  if (in_len < kCkHead) return fail(SIM_ERR_INVALID, "checkpoint shorter than its header");
  const uint8_t* base = reinterpret_cast<const uint8_t*>(in);
  const cudaMemcpyKind k_from = in_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  uint8_t head[kCkHead];
  CK(cudaMemcpy(head, base, kCkHead, k_from), "checkpoint header");
  CkHeader k{};
  std::memcpy(&k, head, sizeof(k));
  if (std::memcmp(k.magic, kCkMagic, 8) != 0 || k.version != 1) return fail(SIM_ERR_INVALID, "not a checkpoint");
  if (k.n != (uint32_t)s->n || k.b != (uint32_t)s->b || k.kc != (uint32_t)s->kc || k.nchunks != s->nchunks ||
      k.eps_max != s->eps_max || k.ladder != s->ladder || k.budget != s->budget || k.tau != s->tau)
    return fail(SIM_ERR_INVALID, "checkpoint taken with other qubits, block/chunk sizes or controller settings");
  if (k.level < 0 || k.level > s->cp.nlevels || (k.modes & qc::kDefaultModes) != qc::kDefaultModes ||
      (k.modes >> qc::M_NMODES))
    return fail(SIM_ERR_INVALID, "checkpoint controller state out of range");
  if (in_len < kCkHead + 4 * s->nchunks + k.image_bytes) return fail(SIM_ERR_INVALID, "checkpoint truncated");
  std::vector<uint32_t> len(s->nchunks);
  CK(cudaMemcpy(len.data(), base + kCkHead, 4 * s->nchunks, k_from), "checkpoint lengths");
  std::vector<unsigned long long> off(s->nchunks), pbase(s->nchunks);
  uint64_t total = 0, used = 0;
  const uint32_t cap = qc::round16(qc::max_image_bytes(s->kc));
  for (uint64_t c = 0; c < s->nchunks; ++c) {
    if (len[c] < 16 || len[c] > cap || (len[c] & 15u)) return fail(SIM_ERR_INVALID, "checkpoint image length out of range");
    off[c] = total;
    pbase[c] = used;
    total += len[c];
    used += qc::pages_for(len[c], s->kc);
  }
  if (total != k.image_bytes || total != k.E) return fail(SIM_ERR_INVALID, "checkpoint image bytes disagree");
  if (used > s->npages) return fail(SIM_ERR_OOM, "checkpoint needs more pages than the arena holds");
  unsigned long long *d_off = nullptr, *d_pb = nullptr;
  uint32_t* d_len = nullptr;
  uint8_t* d_img = nullptr;
  cudaError_t e = cudaMalloc(&d_off, s->nchunks * 8);
  if (e == cudaSuccess) e = cudaMalloc(&d_pb, s->nchunks * 8);
  if (e == cudaSuccess) e = cudaMalloc(&d_len, s->nchunks * 4);
  if (e == cudaSuccess && !in_on_device && total) e = cudaMalloc(&d_img, total);
  const uint8_t* src = in_on_device ? base + kCkHead + 4 * s->nchunks : d_img;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), s->nchunks * 8, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_pb, pbase.data(), s->nchunks * 8, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, len.data(), s->nchunks * 4, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess && !in_on_device && total)
    e = cudaMemcpyAsync(d_img, base + kCkHead + 4 * s->nchunks, total, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = qc::launch_checkpoint_scatter(s->P, s->nchunks, d_off, d_pb, d_len, src, used, s->st);
  // controller and pool counters as they were, the page caches empty
  DevCtl h{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, s->d_ctl, sizeof(h), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e == cudaSuccess) {
    h.E = k.E;
    h.dE = 0;
    h.Emax = k.Emax;
    h.top = (long long)(s->npages - used);
    h.nfreed = 0;
    h.gates = k.gates;
    h.peak_pages = k.peak_pages > used ? k.peak_pages : used;
    h.switch_gate = k.switch_gate;
    h.lb_sum = k.lb_sum;
    h.lb_prod = k.lb_prod;
    h.level = k.level;
    h.S_last = k.S_last;
    h.err = 0;
    h.n64 = 0;  // counted from the loaded images below
    h.dn64 = 0;
    e = cudaMemcpyAsync(s->d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s->st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_counts, 0, 8 * sizeof(unsigned long long), s->st);
  if (e == cudaSuccess)
    e = qc::launch_mode_counts(s->P, s->nchunks, s->d_counts,
                               reinterpret_cast<unsigned long long*>(&s->d_ctl->n64), s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->P.cache_n, 0, (size_t)s->grid * sizeof(uint32_t), s->st);
  if (e == cudaSuccess)  // the streaming kernel's warp caches held pages of the replaced arena
    e = cudaMemsetAsync(s->P.wcache_n, 0, (size_t)(s->fast_grid ? s->fast_grid : 1) * qc::fast_warps() * 4, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(d_off);
  cudaFree(d_pb);
  cudaFree(d_len);
  cudaFree(d_img);
  if (e != cudaSuccess) return cuda_fail(e, "checkpoint load");
  s->amp_updates = k.amp_updates;
  s->modes = k.modes;
  s->poisoned = SIM_OK;
  return SIM_OK;
}

// ------------------------------------------------------------ codec ------ //
sim_status sim_codec_encode(const double* in, uint64_t n_chunks, int chunk_log2, double eps, int force_mode,
                            uint8_t* out, uint64_t out_stride, uint32_t* out_len, int on_device) {
  return sim_codec_encode_ex(in, n_chunks, chunk_log2, eps, force_mode, qc::kDefaultModes, out, out_stride, out_len,
                             on_device);
}

sim_status sim_codec_encode_ex(const double* in, uint64_t n_chunks, int chunk_log2, double eps, int force_mode,
                               uint32_t modes, uint8_t* out, uint64_t out_stride, uint32_t* out_len, int on_device) {
  if ((modes & qc::kDefaultModes) != qc::kDefaultModes || (modes >> qc::M_NMODES))
    return fail(SIM_ERR_INVALID, "the mode set must contain ZERO..RAW (0x1F) and only known modes");
  if (!in || !out || !out_len) return fail(SIM_ERR_INVALID, "NULL argument");
  if (chunk_log2 < 0 || chunk_log2 > qc::kMaxKC) return fail(SIM_ERR_INVALID, "chunk_log2 must be in [0, 11]");
  const int S = sig_bits_of(eps);
  if (S < 0) return fail(SIM_ERR_INVALID, "eps must be 0 or in [2^-52, 1)");
  if (force_mode >= (int)qc::M_NMODES) return fail(SIM_ERR_INVALID, "unknown mode");
  const uint64_t need = 16 + (16ull << chunk_log2) + (1ull << chunk_log2) / 2 + 32;
  if (out_stride < need || (out_stride & 15)) return fail(SIM_ERR_INVALID, "out_stride too small or not a multiple of 16");
  if (n_chunks == 0) return SIM_OK;
  // every size below is a product with n_chunks: bound it first so that none wraps
  if (out_stride > (1ull << 40) || n_chunks > (1ull << 62) / (out_stride + (16ull << chunk_log2) + 4))
    return fail(SIM_ERR_INVALID, "n_chunks or out_stride too large");
  const size_t in_bytes = (size_t)n_chunks * (16ull << chunk_log2);
  const double* din = in;
  uint8_t* dout = out;
  uint32_t* dlen = out_len;
  unsigned int* derr = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = sizeof(unsigned int) + (on_device ? 0 : in_bytes + n_chunks * out_stride + n_chunks * 4 + 64);
  CK(cudaMalloc(&tmp, tmp_bytes), "codec buffers");
  derr = reinterpret_cast<unsigned int*>(tmp);
  if (!on_device) {
    uint8_t* base = reinterpret_cast<uint8_t*>(tmp) + 16;
    din = reinterpret_cast<double*>(base);
    dout = base + ((in_bytes + 15) & ~15ull);
    dlen = reinterpret_cast<uint32_t*>(dout + n_chunks * out_stride);
    cudaMemcpy((void*)din, in, in_bytes, cudaMemcpyHostToDevice);
  }
  cudaMemset(derr, 0, sizeof(unsigned int));
  cudaError_t e = qc::launch_codec_encode(din, n_chunks, chunk_log2, (uint32_t)S, force_mode, modes, dout, out_stride,
                                          dlen, derr, 0);
  unsigned int herr = 0;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && !on_device) {
    e = cudaMemcpy(out, dout, n_chunks * out_stride, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_len, dlen, n_chunks * 4, cudaMemcpyDeviceToHost);
  }
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "codec encode");
  if (herr & qc::E_NONFINITE) return fail(SIM_ERR_INVALID, "input holds a non-finite value");
  if (herr & qc::E_MODE) return fail(SIM_ERR_INVALID, "forced mode does not apply to a chunk");
  return SIM_OK;
}

sim_status sim_codec_decode(const uint8_t* in, uint64_t in_stride, const uint32_t* in_len, uint64_t n_chunks,
                            int chunk_log2, double* out, int on_device) {
  if (!in || !in_len || !out) return fail(SIM_ERR_INVALID, "NULL argument");
  if (chunk_log2 < 0 || chunk_log2 > qc::kMaxKC) return fail(SIM_ERR_INVALID, "chunk_log2 must be in [0, 11]");
  if (in_stride & 15) return fail(SIM_ERR_INVALID, "in_stride must be a multiple of 16");
  if (n_chunks == 0) return SIM_OK;
  // every size below is a product with n_chunks: bound it first so that none wraps
  if (in_stride > (1ull << 40) || n_chunks > (1ull << 62) / (in_stride + (16ull << chunk_log2) + 4))
    return fail(SIM_ERR_INVALID, "n_chunks or in_stride too large");
  const size_t out_bytes = (size_t)n_chunks * (16ull << chunk_log2);
  const uint8_t* din = in;
  const uint32_t* dlen = in_len;
  double* dout = out;
  void* tmp = nullptr;
  const size_t tmp_bytes = 16 + (on_device ? 0 : n_chunks * in_stride + n_chunks * 4 + 16 + out_bytes);
  CK(cudaMalloc(&tmp, tmp_bytes), "codec buffers");
  unsigned int* derr = reinterpret_cast<unsigned int*>(tmp);
  if (!on_device) {
    uint8_t* base = reinterpret_cast<uint8_t*>(tmp) + 16;
    din = base;
    uint32_t* l = reinterpret_cast<uint32_t*>(base + n_chunks * in_stride);
    dlen = l;
    dout = reinterpret_cast<double*>(base + ((n_chunks * in_stride + n_chunks * 4 + 15) & ~15ull));
    cudaMemcpy((void*)din, in, n_chunks * in_stride, cudaMemcpyHostToDevice);
    cudaMemcpy(l, in_len, n_chunks * 4, cudaMemcpyHostToDevice);
  }
  cudaMemset(derr, 0, sizeof(unsigned int));
  cudaError_t e = qc::launch_codec_decode(din, in_stride, dlen, n_chunks, chunk_log2, dout, derr, 0);
  unsigned int herr = 0;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && !on_device) e = cudaMemcpy(out, dout, out_bytes, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "codec decode");
  if (herr) return fail(SIM_ERR_CORRUPT, "an image failed its checks");
  return SIM_OK;
}

// ------------------------------------------------- uncompressed path ----- //
sim_status sim_sv_create(int n_qubits, sim_sv_t** out) {
  if (!out) return fail(SIM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > 34) return fail(SIM_ERR_INVALID, "n_qubits must be in [1, 34]");
  sim_sv* v = new sim_sv();
  v->n = n_qubits;
  cudaError_t e = cudaMalloc(&v->psi, (size_t)16 << n_qubits);
  if (e != cudaSuccess) {
    delete v;
    return cuda_fail(e, "state vector allocation");
  }
  e = qc::launch_sv_init(v->psi, 1ull << n_qubits, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete v;
    return cuda_fail(e, "state vector init");
  }
  *out = v;
  return SIM_OK;
}

sim_status sim_sv_destroy(sim_sv_t* v) {
  if (!v) return fail(SIM_ERR_INVALID, "NULL handle");
  cudaStreamSynchronize(v->st);
  delete v;
  return SIM_OK;
}

sim_status sim_sv_set_stream(sim_sv_t* v, void* stream) {
  if (!v) return fail(SIM_ERR_INVALID, "NULL handle");
  v->st = reinterpret_cast<cudaStream_t>(stream);
  return SIM_OK;
}

sim_status sim_sv_apply_circuit(sim_sv_t* v, const sim_gate* gates, size_t n_gates) {
  if (!v || (!gates && n_gates)) return fail(SIM_ERR_INVALID, "NULL argument");
  std::string why;
  for (size_t k = 0; k < n_gates; ++k)
    if (!gate_ok(gates + k, v->n, &why)) return fail(SIM_ERR_INVALID, "invalid gate %zu: %s", k, why.c_str());
  for (size_t k = 0; k < n_gates; ++k) {
    // which amplitudes of a pair the gate reads and writes (see k_sv_gate)
    const double* u = gates[k].u;
    const bool z01 = u[2] == 0.0 && u[3] == 0.0, z10 = u[4] == 0.0 && u[5] == 0.0;
    const bool wa = !(u[0] == 1.0 && u[1] == 0.0 && z01), wb = !(u[6] == 1.0 && u[7] == 0.0 && z10);
    const uint32_t rows = (wa ? 1u : 0u) | (wb ? 2u : 0u) | ((wa || (wb && !z10)) ? 4u : 0u) |
                          ((wb || (wa && !z01)) ? 8u : 0u);
    CK(qc::launch_sv_gate(v->psi, v->n, coef_of(gates + k), gates[k].target, gates[k].ctrl_mask, gates[k].ctrl_vals,
                          rows, v->st),
       "state vector gate");
  }
  CK(cudaStreamSynchronize(v->st), "sync");
  return SIM_OK;
}

sim_status sim_sv_amplitudes(sim_sv_t* v, uint64_t first, uint64_t count, double* out, int out_on_device) {
  if (!v || (!out && count)) return fail(SIM_ERR_INVALID, "NULL argument");
  const uint64_t total = 1ull << v->n;
  if (first > total || count > total - first) return fail(SIM_ERR_INVALID, "amplitude range outside the state");
  CK(cudaMemcpyAsync(out, v->psi + 2 * first, count * 16, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     v->st),
     "copy");
  CK(cudaStreamSynchronize(v->st), "sync");
  return SIM_OK;
}

sim_status sim_sv_data(sim_sv_t* v, double** dev_ptr) {
  if (!v || !dev_ptr) return fail(SIM_ERR_INVALID, "NULL argument");
  *dev_ptr = v->psi;
  return SIM_OK;
}

}  // extern "C"
