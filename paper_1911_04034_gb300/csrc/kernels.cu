// kernels.cu -- CUDA kernels of libqcsim (sm_103a).
//
// k_gate   the fused persistent kernel of the hot path: for each work item (two
//          chunks) it stages the compressed images in shared memory, decodes them,
//          applies the gate to every amplitude pair (Section 3.1, Eq. matrix1/2) and
//          re-encodes them with the hybrid codec (Section 4.2, Solution C) under the
//          bound chosen by the controller (Section 3.7), then commits the new images
//          to the page pool.  Decoded amplitudes never leave shared memory.
// k_post   after each gate: returns freed pages to the stack, adds the gate's byte
//          change to E, and records the controller's level and fidelity bounds.
// others   initialisation, codec entry points, readout and the uncompressed path.
#include "launch.h"
#include "gate_common.cuh"

// Resident CTAs per SM that the fused kernel's register budget is sized for (the grid
// follows the occupancy the build achieves).
#ifndef QC_GATE_MIN_CTAS
#define QC_GATE_MIN_CTAS 3
#endif

namespace qc {

int vpt_for(int kc) {
  const int N = 2 << kc;
  return N <= kThreads ? 1 : N / kThreads;
}
__host__ __device__ __forceinline__ uint32_t imgcap(int kc) { return round16(max_image_bytes(kc)); }
// staging buffer of the codec entry points: any forced image fits
__host__ __device__ __forceinline__ uint32_t codedcap(int kc) { return round16(max_coded_bytes(kc)); }
__host__ __device__ __forceinline__ uint32_t pagelist_words(int kc) { return (max_pages(kc) + 3u) & ~3u; }

// Each image buffer keeps 16 spare bytes: the decoder's bit window reads up to 8 bytes
// past the end of a residual stream.
__host__ __device__ __forceinline__ uint32_t imgbuf(int kc) { return imgcap(kc) + 16u; }
size_t gate_smem_bytes(int kc) {
  return 2 * size_t(tile_words(kc)) * 8 + 2 * size_t(imgbuf(kc)) + 4 * size_t(dir_stride(kc)) +
         round16(sizeof(ScanSmem));
}
size_t codec_smem_bytes(int kc) {
  return size_t(tile_words(kc)) * 8 + size_t(codedcap(kc)) + 4 * size_t(pagelist_words(kc)) + round16(sizeof(ScanSmem));
}

// ------------------------------------------------------------- the gate -- //
// Shared-memory layout of the fused kernel and the per-CTA state it carries between
// work items (page cache, byte counters, scan-buffer parity).
struct GateSmem {
  uint64_t *tile0, *tile1;
  uint8_t *img0, *img1;
  uint32_t* ent[2][2];    // two sets of copies of the two directory entries (header, page
                          // ids or image): the current item's and the next item's
  ScanSmem* s;
  long long* ph;          // per-phase cycles, [6] = last clock (profiling)
  int* oom;
  uint32_t* np;
};
// Per-CTA counters that only thread 0 updates (kept in shared memory so that they
// hold no registers during the codec phases).
struct CtaAcc {
  long long dE;
  long long dn64;          // change in the number of images at S = 64
  unsigned long long rd, wr;
  unsigned long long key;  // block-cache key of the running item
};
struct GateCta {
  CtaCache cc;
  CtaAcc* acc;
  unsigned int err;        // thread 0: the error word as read during the previous item
  int pp;
  int cur;                        // directory-entry buffer set of the current item
  unsigned long long next_item;   // item whose entries were prefetched into set cur ^ 1
};

// Bulk asynchronous shared -> global copy (one page of a new image); the issuing thread
// later waits until the source has been read before the buffer is reused.
__device__ __forceinline__ void bulk_store(void* gmem, const void* smem, uint32_t bytes) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem), "r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// Makes this thread's earlier shared-memory writes visible to bulk copies.
__device__ __forceinline__ void fence_to_bulk() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Writes the two new images of a work item: pages by bulk copies (a lane of warp 0 per
// page), inline images and the directory entries by plain stores (warp 1).  All threads
// call it; the images in shared memory must stay untouched until bulk_wait_read.
__device__ __forceinline__ void commit_images(const Pool& P, unsigned long long c0, const uint8_t* img0, uint32_t n0,
                                              const uint32_t* pg0, uint32_t np0, bool has1, unsigned long long c1,
                                              const uint8_t* img1, uint32_t n1, const uint32_t* pg1, uint32_t np1) {
  if (threadIdx.x < 32u) {
    const uint32_t tot = np0 + (has1 ? np1 : 0u);
    bool issued = false;
    for (uint32_t k = threadIdx.x; k < tot; k += 32u) {
      const bool second = k >= np0;
      const uint32_t q = second ? k - np0 : k, bytes = second ? n1 : n0;
      const uint32_t len = min((uint32_t)kPage, bytes - q * kPage);
      if (!issued) fence_to_bulk();
      bulk_store(P.pages + (unsigned long long)(second ? pg1[q] : pg0[q]) * kPage,
                 (second ? img1 : img0) + q * kPage, len);
      issued = true;
    }
    if (issued) bulk_commit();
  } else if (threadIdx.x < 64u) {
    const uint32_t lane = threadIdx.x - 32u;
    for (int w = 0; w < (has1 ? 2 : 1); ++w) {
      uint32_t* e = dir_entry(P, w ? c1 : c0);
      const uint32_t bytes = w ? n1 : n0, np = w ? np1 : np0;
      const uint32_t* pg = w ? pg1 : pg0;
      if (np == 0u) {
        const uint4* src = reinterpret_cast<const uint4*>(w ? img1 : img0);
        for (uint32_t u = lane; u < bytes / 16u; u += 32u) reinterpret_cast<uint4*>(e + 4)[u] = src[u];
      } else {
        for (uint32_t q = lane; q < np; q += 32u) e[4 + q] = pg[q];
      }
      if (lane == 0) {
        e[0] = bytes;
        e[1] = np;
      }
    }
  }
}

// Pulls one page of a later item's image into L2 (no data returned to the SM).
__device__ __forceinline__ void prefetch_l2_page(const void* gmem) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"((uint32_t)kPage) : "memory");
}

__device__ __forceinline__ GateSmem gate_smem(uint8_t* smem, int kc, uint32_t dir_words, long long* ph, int* oom,
                                               uint32_t* np) {
  GateSmem m;
  m.tile0 = reinterpret_cast<uint64_t*>(smem);
  m.tile1 = m.tile0 + tile_words(kc);
  m.img0 = reinterpret_cast<uint8_t*>(m.tile1 + tile_words(kc));
  m.img1 = m.img0 + imgbuf(kc);
  m.ent[0][0] = reinterpret_cast<uint32_t*>(m.img1 + imgbuf(kc));
  m.ent[0][1] = m.ent[0][0] + dir_words;
  m.ent[1][0] = m.ent[0][1] + dir_words;
  m.ent[1][1] = m.ent[1][0] + dir_words;
  m.s = reinterpret_cast<ScanSmem*>(m.ent[1][1] + dir_words);
  m.ph = ph;
  m.oom = oom;
  m.np = np;
  return m;
}

// Warp 0 loads this CTA's page cache of the simulator into shared memory (empty
// unless this CTA already worked for it in the same launch).
__device__ __forceinline__ void cta_begin(const Pool& P, GateCta& st, bool prof, long long* ph) {
  if (threadIdx.x < 32u) {
    const uint32_t n = P.cache_n[blockIdx.x];
    for (uint32_t q = threadIdx.x; q < n; q += 32u) st.cc.ids[q] = P.cache[(size_t)blockIdx.x * kCacheCap + q];
    if (threadIdx.x == 0) *st.cc.n = n;
    __syncwarp();
  }
  if (threadIdx.x == 0) {
    st.acc->dE = 0;
    st.acc->dn64 = 0;
    st.acc->rd = st.acc->wr = 0;
  }
  // the error word as the launch finds it: after a device error even a CTA's first item
  // stops before it touches the pool
  st.err = threadIdx.x == 0 ? *(volatile unsigned int*)&P.ctl->err : 0u;
  st.pp = 0;
  st.cur = 0;
  st.next_item = ~0ull;
  if (prof && threadIdx.x == 0) {
    for (int k = 0; k < 6; ++k) ph[k] = 0;
    ph[6] = clock64();
  }
}

// Warp 0: hands the CTA's page cache and counters back to the simulator.
__device__ __forceinline__ void cta_end(const GateLaunch& L, GateCta& st, const long long* ph) {
  if (threadIdx.x >= 32u) return;
  const uint32_t n = *st.cc.n;
  for (uint32_t q = threadIdx.x; q < n; q += 32u) L.P.cache[(size_t)blockIdx.x * kCacheCap + q] = st.cc.ids[q];
  if (threadIdx.x != 0) return;
  DevCtl* ctl = L.P.ctl;
  if (L.prof)
    for (int k = 0; k < 6; ++k)
      if (ph[k]) atomicAdd(&ctl->phase_cycles[k], (unsigned long long)ph[k]);
  L.P.cache_n[blockIdx.x] = n;
  if (st.acc->dE) atomicAdd(&ctl->dE, (unsigned long long)st.acc->dE);
  if (st.acc->dn64) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->dn64), (unsigned long long)st.acc->dn64);
  if (st.acc->rd) atomicAdd(&ctl->bytes_in, st.acc->rd);
  if (st.acc->wr) atomicAdd(&ctl->bytes_out, st.acc->wr);
}

// One work item (two chunks) of a gate: stage, decode, apply, encode, commit.
// Returns false if the simulator's error word is set (nothing more to do for it).
// PREF: nx is the CTA's next item of the same gate (~0 if none); its directory
// entries are fetched asynchronously during this item and its pages pulled into L2.
template <int VPT, bool PREF>
__device__ __forceinline__ bool gate_item(const GateLaunch& L, unsigned long long item, unsigned long long nx,
                                          uint32_t S, unsigned long long serial, bool bc_on, const GateSmem& m,
                                          GateCta& st) {
  const int kc = L.P.kc;
  const uint32_t A = 1u << kc;
  const uint32_t cap = imgcap(kc);
  const Pool& P = L.P;
  DevCtl* ctl = P.ctl;
  const uint32_t dw4 = P.dir_words / 4u;  // 16-byte units of a directory entry
#define QC_PHASE(k)                     \
  if (L.prof && threadIdx.x == 0) {     \
    const long long now_ = clock64();   \
    m.ph[k] += now_ - m.ph[6];          \
    m.ph[6] = now_;                     \
  }
  // one barrier that also broadcasts thread 0's view of the error word (and publishes
  // the entries prefetched during the previous item); the previous item's bulk page
  // stores must have read the image buffers before they are refilled
  bulk_wait_read();
  if (PREF) cp_async_wait_all();
  if (__syncthreads_or(threadIdx.x == 0 && st.err != 0u)) return false;
  const bool have_entries = PREF && st.next_item == item;
  if (PREF && st.next_item != ~0ull) st.cur ^= 1;
  st.next_item = ~0ull;
  uint32_t* const ent0 = m.ent[st.cur][0];
  uint32_t* const ent1 = m.ent[st.cur][1];
  // the item's chunks (recomputed at commit rather than kept through the codec)
  auto chunks_of = [&](unsigned long long& x0, unsigned long long& x1) {
    if (L.pair) {
      x0 = item_chunk(L, item) | L.hi_vals;
      x1 = x0 | L.pair_bit;
    } else {
      x0 = item_chunk(L, 2ull * item) | L.hi_vals;
      x1 = 2ull * item + 1 < L.nact ? (item_chunk(L, 2ull * item + 1) | L.hi_vals) : 0ull;
    }
  };
  unsigned long long c0, c1;
  chunks_of(c0, c1);
  const bool has1 = L.pair || 2ull * item + 1 < L.nact;
  // stage 1: both directory entries (warp 0 and warp 1), unless prefetched
  if (!have_entries) {
    if (threadIdx.x < 32u) {
      const uint4* src = reinterpret_cast<const uint4*>(dir_entry(P, c0));
      for (uint32_t i = threadIdx.x; i < dw4; i += 32u) reinterpret_cast<uint4*>(ent0)[i] = src[i];
    } else if (threadIdx.x < 64u && has1) {
      const uint4* src = reinterpret_cast<const uint4*>(dir_entry(P, c1));
      for (uint32_t i = threadIdx.x - 32u; i < dw4; i += 32u) reinterpret_cast<uint4*>(ent1)[i] = src[i];
    }
    __syncthreads();
  }
  // the next item's entries (asynchronously, into the other set); no other CTA writes
  // them, and this item touches only its own chunks
  unsigned long long nc0 = 0, nc1 = 0;
  bool nhas1 = false;
  if (PREF && nx != ~0ull) {
    if (L.pair) {
      nc0 = item_chunk(L, nx) | L.hi_vals;
      nc1 = nc0 | L.pair_bit;
      nhas1 = true;
    } else {
      nc0 = item_chunk(L, 2ull * nx) | L.hi_vals;
      nhas1 = 2ull * nx + 1 < L.nact;
      nc1 = nhas1 ? (item_chunk(L, 2ull * nx + 1) | L.hi_vals) : 0ull;
    }
    if (threadIdx.x < 32u) {
      const uint4* src = reinterpret_cast<const uint4*>(dir_entry(P, nc0));
      for (uint32_t i = threadIdx.x; i < dw4; i += 32u) cp_async16(reinterpret_cast<uint4*>(m.ent[st.cur ^ 1][0]) + i, src + i);
    } else if (threadIdx.x < 64u && nhas1) {
      const uint4* src = reinterpret_cast<const uint4*>(dir_entry(P, nc1));
      for (uint32_t i = threadIdx.x - 32u; i < dw4; i += 32u)
        cp_async16(reinterpret_cast<uint4*>(m.ent[st.cur ^ 1][1]) + i, src + i);
    }
    cp_async_commit();
    st.next_item = nx;
  }
  const uint32_t np0 = ent0[1], np1 = has1 ? ent1[1] : 0u;
  const uint32_t b0 = ent0[0], b1 = has1 ? ent1[0] : 0u;
  if (b0 > cap || b1 > cap || np0 > max_pages(kc) || np1 > max_pages(kc) || (np0 == 0u && b0 > inline_cap(kc)) ||
      (np1 == 0u && b1 > inline_cap(kc)) || (b0 & 15u) || (b1 & 15u)) {
    if (threadIdx.x == 0) atomicOr(&ctl->err, (unsigned)E_CORRUPT);
    return false;
  }
  // An all-zero chunk maps to an all-zero chunk under any gate (signed zeros are
  // stored as +0), and its image does not depend on the bound: skip it.
  const bool z0 = np0 == 0 && b0 == 16u && ent0[4] == 0u;
  const bool z1 = !has1 || (np1 == 0 && b1 == 16u && ent1[4] == 0u);
  if (threadIdx.x == 0) st.acc->rd += b0 + b1;
  if (z0 && z1) {
    QC_PHASE(5);
    return true;
  }
  // Two constant chunks (ZERO or CONST images, held inline) under a cross-chunk gate
  // with no in-chunk controls: every pair sees the same inputs, so one pair gives
  // both output chunks, which are constant again.
  if (L.pair && L.lo_mask == 0u && inline_cap(kc) >= 32u && np0 == 0u && np1 == 0u &&
      (z0 || (ent0[4] & 0xffu) == M_CONST) && (z1 || (ent1[4] & 0xffu) == M_CONST)) {
    if (threadIdx.x == 0) {
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (!z0) a = make_double2(__longlong_as_double(((const long long*)(ent0 + 8))[0]),
                                __longlong_as_double(((const long long*)(ent0 + 8))[1]));
      if (!z1) b = make_double2(__longlong_as_double(((const long long*)(ent1 + 8))[0]),
                                __longlong_as_double(((const long long*)(ent1 + 8))[1]));
      apply_pair(L.g, a, b);
      uint32_t h0[8], h1[8];
      const uint32_t n0 = const_image((uint64_t)__double_as_longlong(a.x), (uint64_t)__double_as_longlong(a.y), S, h0);
      const uint32_t n1 = const_image((uint64_t)__double_as_longlong(b.x), (uint64_t)__double_as_longlong(b.y), S, h1);
      if (n0 == 0u || n1 == 0u) {
        atomicOr(&ctl->err, (unsigned)E_NONFINITE);
      } else {
        uint32_t* w0 = dir_entry(P, c0);
        uint32_t* w1 = dir_entry(P, c1);
        for (int k = 0; k < 8; ++k) {
          w0[4 + k] = h0[k];
          w1[4 + k] = h1[k];
        }
        w0[0] = n0;
        w1[0] = n1;
        st.acc->dE += (long long)n0 + (long long)n1 - (long long)b0 - (long long)b1;
        auto wide = [](uint32_t h) { return ((h >> 8) & 0xffu) == 64u ? 1ll : 0ll; };
        st.acc->dn64 += wide(h0[0]) + wide(h1[0]) - (z0 ? 0ll : wide(ent0[4])) - (z1 ? 0ll : wide(ent1[4]));
        st.acc->wr += n0 + n1;
      }
    }
    QC_PHASE(5);
    return true;
  }
  // stage 2: both images in one pass (inline ones from the entry copies); page data is
  // copied asynchronously, so every copy of the thread is in flight at once
  {
    const uint32_t u0 = b0 >> 4, u1 = b1 >> 4;
    constexpr uint32_t upp = kPage / 16;
    for (uint32_t u = threadIdx.x; u < u0 + u1; u += kThreads) {
      const bool second = u >= u0;
      const uint32_t uu = second ? u - u0 : u;
      const uint32_t* ent = second ? ent1 : ent0;
      uint4* dst = reinterpret_cast<uint4*>(second ? m.img1 : m.img0) + uu;
      if ((second ? np1 : np0) == 0u) *dst = reinterpret_cast<const uint4*>(ent + 4)[uu];
      else cp_async16(dst, reinterpret_cast<const uint4*>(P.pages + (unsigned long long)ent[4 + uu / upp] * kPage) + (uu % upp));
    }
    cp_async_commit();
    cp_async_wait_all();
  }
  __syncthreads();
  if (threadIdx.x < 32u) free_pages_warp(P, st.cc, ent0 + 4, np0, ent1 + 4, has1 ? np1 : 0u);
  QC_PHASE(0);
  // the input images coded at 64 bits (thread 0), for the controller's count
  const long long old64 = threadIdx.x == 0 ? (long long)(m.img0[1] == 64u) + (long long)(has1 && m.img1[1] == 64u) : 0ll;
  // the next item's pages into L2: warp 0 for its first chunk, warp 1 for its second
  // (each warp waits only for the entry copies it issued itself)
  auto prefetch_next = [&]() {
    if (PREF && st.next_item != ~0ull && threadIdx.x < 64u && (threadIdx.x < 32u || nhas1)) {
      cp_async_wait_all();
      __syncwarp();
      const uint32_t* e = m.ent[st.cur ^ 1][threadIdx.x >> 5];
      const uint32_t q = min(e[1], max_pages(kc));
      for (uint32_t k = threadIdx.x & 31u; k < q; k += 32u) {
        const uint32_t pid = e[4 + k];
        if (pid < P.npages) prefetch_l2_page(P.pages + (unsigned long long)pid * kPage);
      }
    }
  };
  // Section 3.4: an earlier item of this gate with the same two input blocks left its
  // outputs in the block cache (confirmed byte by byte); otherwise claim the line
  bool bc_hit = false, bc_claim = false;
  uint32_t n0 = 0, n1 = 1;
  if (L.bc && bc_on && has1) {
    const unsigned long long key = bc_key(m.img0, b0, m.img1, b1, *m.s);
    if (threadIdx.x == 0) st.acc->key = key;
    BcLine* line = reinterpret_cast<BcLine*>(L.bc + (key % (unsigned long long)kBcLines) * bc_line_bytes(cap));
    uint8_t* ldat = reinterpret_cast<uint8_t*>(line) + kBcHead;
    if (threadIdx.x == 0) {
      const unsigned long long t = atomicAdd(&line->tag, 0ull);
      int flag = 0;
      if (t == ((serial << 2) | 2ull)) {
        __threadfence();
        if (__ldcg(&line->key) == key && __ldcg(&line->len[0]) == b0 && __ldcg(&line->len[1]) == b1) flag = 1;
      } else if ((t >> 2) != serial && atomicCAS(&line->tag, t, (serial << 2) | 1ull) == t) {
        flag = 2;
      }
      m.s->bc_flag = flag;
      atomicAdd(&ctl->bc_gate_lookups, 1ull);
    }
    __syncthreads();
    const int flag = m.s->bc_flag;
    const uint4* lin = reinterpret_cast<const uint4*>(ldat);
    if (flag == 1) {
      const uint32_t u0 = b0 >> 4, u1 = b1 >> 4, c16 = cap >> 4;
      bool eq = true;
      for (uint32_t u = threadIdx.x; u < u0 + u1; u += kThreads) {
        const uint4 a = u < u0 ? reinterpret_cast<const uint4*>(m.img0)[u] : reinterpret_cast<const uint4*>(m.img1)[u - u0];
        const uint4 b = __ldcg(lin + (u < u0 ? u : c16 + (u - u0)));
        eq &= a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
      }
      if (__syncthreads_and(eq)) {
        n0 = __ldcg(&line->len[2]);
        n1 = __ldcg(&line->len[3]);
        const uint32_t v0 = n0 >> 4, v1 = n1 >> 4;
        for (uint32_t u = threadIdx.x; u < v0 + v1; u += kThreads) {
          if (u < v0) reinterpret_cast<uint4*>(m.img0)[u] = __ldcg(lin + 2u * c16 + u);
          else reinterpret_cast<uint4*>(m.img1)[u - v0] = __ldcg(lin + 3u * c16 + (u - v0));
        }
        __syncthreads();
        bc_hit = true;
        if (threadIdx.x == 0) atomicAdd(&ctl->bc_gate_hits, 1ull);
      }
    } else if (flag == 2) {
      const uint32_t u0 = b0 >> 4, u1 = b1 >> 4, c16 = cap >> 4;
      uint4* lout = reinterpret_cast<uint4*>(ldat);
      for (uint32_t u = threadIdx.x; u < u0 + u1; u += kThreads) {
        if (u < u0) lout[u] = reinterpret_cast<const uint4*>(m.img0)[u];
        else lout[c16 + (u - u0)] = reinterpret_cast<const uint4*>(m.img1)[u - u0];
      }
      bc_claim = true;
    }
  }
  if (bc_hit) {
    prefetch_next();
  } else {
  // two STREAM images of 32-bit width (the common case once the run is lossy) decode
  // together, sharing barriers; anything else chunk by chunk
  const bool paired = has1 && kThreads * VPT == 2u * A;
  bool ok0, ok1;
  if (paired && stream32_image(m.img0, b0, kc) && stream32_image(m.img1, b1, kc)) {
    ok0 = ok1 = decode_stream32_pair<VPT>(m.img0, m.img1, 2u * A, m.tile0, m.tile1, *m.s, st.pp);
  } else {
    ok0 = decode_block<VPT>(m.img0, b0, kc, m.tile0, *m.s, st.pp);
    ok1 = has1 ? decode_block<VPT>(m.img1, b1, kc, m.tile1, *m.s, st.pp) : true;
  }
  prefetch_next();
  QC_PHASE(1);
  if (!ok0 || !ok1) {
    if (threadIdx.x == 0) atomicOr(&ctl->err, (unsigned)E_CORRUPT);
    return false;
  }
  // apply the gate to every amplitude pair whose in-chunk control bits match
  double2* t0 = reinterpret_cast<double2*>(m.tile0);
  double2* t1 = reinterpret_cast<double2*>(m.tile1);
  if (L.pair) {
    for (uint32_t i = threadIdx.x; i < A; i += kThreads) {
      if ((i & L.lo_mask) != L.lo_vals) continue;
      const uint32_t pi = tile_amp(i);
      double2 a = t0[pi], b = t1[pi];
      apply_pair(L.g, a, b);
      t0[pi] = a;
      t1[pi] = b;
    }
  } else {
    const uint32_t tb = 1u << L.target, lowm = tb - 1u;
    const uint32_t tot = has1 ? A : A / 2u;  // pairs over both tiles
    for (uint32_t q = threadIdx.x; q < tot; q += kThreads) {
      const uint32_t p = q & (A / 2u - 1u);
      double2* tt = (q < A / 2u) ? t0 : t1;
      const uint32_t i0 = ((p & ~lowm) << 1) | (p & lowm);
      if ((i0 & L.lo_mask) != L.lo_vals) continue;
      const uint32_t p0 = tile_amp(i0), p1 = tile_amp(i0 | tb);
      double2 a = tt[p0], b = tt[p1];
      apply_pair(L.g, a, b);
      tt[p0] = a;
      tt[p1] = b;
    }
  }
  __syncthreads();
  QC_PHASE(2);
  // chunk modes: the mode set, or Solution C's set plus the trials the selector granted
  uint32_t md0 = L.modes, md1 = L.modes;
  if (L.sel_dec) {
    md0 = sel_modes(L.sel_dec[2ull * item]);
    md1 = has1 ? sel_modes(L.sel_dec[2ull * item + 1ull]) : kDefaultModes;
  }
  SelCtx sel;
  sel.gfeat = L.gfeat;
  sel.S_gate = S;
  sel.trace = L.trace;
  sel.trace_n = L.trace_n;
  sel.trace_cap = L.trace_cap;
  sel.split_trials = &ctl->split_trials;
  sel.palette_trials = &ctl->palette_trials;
  {
    const uint4 h = reinterpret_cast<const uint4*>(m.img0)[0];  // the pre-gate image header (still staged)
    sel.prev_hdr[0] = h.x; sel.prev_hdr[1] = h.y; sel.prev_hdr[2] = h.z; sel.prev_hdr[3] = h.w;
    sel.prev_len = b0;
  }
  // both chunks in one pass when neither needs a SPLIT or PALETTE trial, a training
  // record or 64-bit widths; otherwise (or if a chunk holds a subnormal) chunk by chunk
  const bool enc_paired = paired && S <= 32u && !L.trace && ((md0 | md1) >> M_SPLIT) == 0u &&
                          encode_pair32<VPT>(m.tile0, m.tile1, kc, S, md0, m.img0, m.img1, cap, *m.s, st.pp,
                                             &ctl->err, n0, n1);
  if (!enc_paired) {
    n0 = encode_block<VPT>(m.tile0, kc, S, -1, md0, m.img0, cap, *m.s, st.pp, &ctl->err, &sel);
    if (has1) {
      const uint4 h = reinterpret_cast<const uint4*>(m.img1)[0];
      sel.prev_hdr[0] = h.x; sel.prev_hdr[1] = h.y; sel.prev_hdr[2] = h.z; sel.prev_hdr[3] = h.w;
      sel.prev_len = b1;
      n1 = encode_block<VPT>(m.tile1, kc, S, -1, md1, m.img1, cap, *m.s, st.pp, &ctl->err, &sel);
    }
  }
  QC_PHASE(3);
  // the error word for the next item's check (the load completes while this one ends)
  if (threadIdx.x == 0) st.err = *(volatile unsigned int*)&ctl->err;
  // a claimed cache line receives the outputs and is published for the rest of the gate
  if (bc_claim && n0 != 0u && n1 != 0u) {
    const unsigned long long key = st.acc->key;
    BcLine* line = reinterpret_cast<BcLine*>(L.bc + (key % (unsigned long long)kBcLines) * bc_line_bytes(cap));
    uint8_t* ldat = reinterpret_cast<uint8_t*>(line) + kBcHead;
    const uint32_t v0 = n0 >> 4, v1 = n1 >> 4, c16 = cap >> 4;
    uint4* lout = reinterpret_cast<uint4*>(ldat);
    for (uint32_t u = threadIdx.x; u < v0 + v1; u += kThreads) {
      if (u < v0) lout[2u * c16 + u] = reinterpret_cast<const uint4*>(m.img0)[u];
      else lout[3u * c16 + (u - v0)] = reinterpret_cast<const uint4*>(m.img1)[u - v0];
    }
    if (threadIdx.x == 0) {
      line->key = key;
      line->len[0] = b0;
      line->len[1] = b1;
      line->len[2] = n0;
      line->len[3] = n1;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(&line->tag, (serial << 2) | 2ull);
  }
  }
  if (n0 == 0u || n1 == 0u) return false;
  fence_to_bulk();  // every thread's image writes, before the barrier below, for the bulk page stores
  if (threadIdx.x < 32u) {
    const uint32_t q0 = pages_for(n0, kc), q1 = has1 ? pages_for(n1, kc) : 0u;
    const bool ok = alloc_pages_warp(P, st.cc, ent0 + 4, q0, ent1 + 4, q1);
    if (threadIdx.x == 0) {
      m.np[0] = q0;
      m.np[1] = q1;
      if (!ok) atomicOr(&ctl->err, (unsigned)E_OOM);
      m.oom[0] = !ok;
    }
  }
  __syncthreads();
  if (m.oom[0]) return false;
  {
    unsigned long long x0, x1;
    chunks_of(x0, x1);
    commit_images(P, x0, m.img0, n0, ent0 + 4, m.np[0], has1, x1, m.img1, n1, ent1 + 4, m.np[1]);
  }
  if (threadIdx.x == 0) {
    const uint32_t i0 = ent0[0], i1 = has1 ? ent1[0] : 0u;  // the old image lengths (entry copies)
    st.acc->dE += (long long)n0 - (long long)i0 + (has1 ? (long long)n1 - (long long)i1 : 0ll);
    st.acc->dn64 += (long long)(m.img0[1] == 64u) + (long long)(has1 && m.img1[1] == 64u) - old64;
    st.acc->wr += n0 + (has1 ? n1 : 0u);
  }
  __syncthreads();
  QC_PHASE(4);

  return true;
#undef QC_PHASE
}

template <int VPT>
__global__ void __launch_bounds__(kThreads, VPT >= 16 ? 1 : QC_GATE_MIN_CTAS) k_gate(const __grid_constant__ GateLaunch L) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ long long s_ph[7];
  __shared__ int s_oom;
  __shared__ uint32_t s_np[2];
  __shared__ uint32_t s_cache[kCacheCap];
  __shared__ uint32_t s_cache_n;
  __shared__ CtaAcc s_acc;
  const GateSmem m = gate_smem(smem, L.P.kc, L.P.dir_words, s_ph, &s_oom, s_np);
  GateCta st;
  st.cc.ids = s_cache;
  st.cc.n = &s_cache_n;
  st.acc = &s_acc;
  cta_begin(L.P, st, L.prof, s_ph);
  const uint32_t S = gate_bits(L);
  const unsigned long long serial = L.P.ctl->gates + 1ull;
  const bool bc_on = L.bc != nullptr && L.P.ctl->bc_off == 0u;
  // all items of the gate, or (list) those the streaming kernel left to this one
  const bool listed = L.list && !L.P.ctl->fast_all;
  const unsigned long long count = listed ? L.P.ctl->ndefer : L.items;
  for (unsigned long long k = blockIdx.x; k < count; k += gridDim.x) {
    const unsigned long long nk = k + gridDim.x;
    const unsigned long long item = listed ? (unsigned long long)L.defer[k] : k;
    const unsigned long long nx = nk < count ? (listed ? (unsigned long long)L.defer[nk] : nk) : ~0ull;
    if (!gate_item<VPT, true>(L, item, nx, S, serial, bc_on, m, st)) break;
  }
  cp_async_wait_all();  // no copy may still target shared memory at exit
  bulk_wait_all();      // nor read from it
  cta_end(L, st, s_ph);
}

// Many simulators in one launch: job j is one gate of one simulator, and its work
// items are the global items [begin_j, begin_{j+1}).  All simulators share chunk_log2.
template <int VPT>
__global__ void __launch_bounds__(kThreads, VPT >= 16 ? 1 : QC_GATE_MIN_CTAS)
    k_gate_batch(const BatchJob* __restrict__ jobs, int njobs, unsigned long long total) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ long long s_ph[7];
  __shared__ int s_oom;
  __shared__ uint32_t s_np[2];
  __shared__ uint32_t s_cache[kCacheCap];
  __shared__ uint32_t s_cache_n;
  __shared__ CtaAcc s_acc;
  const GateSmem m = gate_smem(smem, jobs[0].L.P.kc, jobs[0].L.P.dir_words, s_ph, &s_oom, s_np);
  GateCta st;
  st.cc.ids = s_cache;
  st.cc.n = &s_cache_n;
  st.acc = &s_acc;
  int cur = -1;
  uint32_t S = 64;
  unsigned long long serial = 0;
  bool bc_on = false;
  for (unsigned long long g = blockIdx.x; g < total; g += gridDim.x) {
    int lo = 0, hi = njobs - 1;  // last job whose first item is <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].begin <= g) lo = mid;
      else hi = mid - 1;
    }
    if (lo != cur) {
      if (cur >= 0) cta_end(jobs[cur].L, st, s_ph);
      cur = lo;
      __syncthreads();  // the previous job's items are done with the shared parameters
      cta_begin(jobs[cur].L.P, st, jobs[cur].L.prof, s_ph);
      S = gate_bits(jobs[cur].L);
      serial = jobs[cur].L.P.ctl->gates + 1ull;
      bc_on = jobs[cur].L.bc != nullptr && jobs[cur].L.P.ctl->bc_off == 0u;
    }
    gate_item<VPT, false>(jobs[cur].L, g - jobs[cur].begin, ~0ull, S, serial, bc_on, m, st);
  }
  bulk_wait_all();  // no bulk page store may still read shared memory at exit
  if (cur >= 0) cta_end(jobs[cur].L, st, s_ph);
}

// After a gate: free pages back to the stack, then the controller bookkeeping.
// Called by one block of 1024 threads.
__device__ __forceinline__ void post_body(const Pool& P, const CtlParams& cp, int grid_ctas) {
  DevCtl* ctl = P.ctl;
  __shared__ unsigned long long s_top;
  __shared__ int s_skip;
  if (threadIdx.x == 0) {
    // after a device error (the pool ran dry, a corrupt image ...) the handle is
    // finished: no bookkeeping, and never a stack index from a top below 0
    const long long top = *(volatile long long*)&ctl->top;
    s_skip = *(volatile unsigned int*)&ctl->err != 0u || top < 0;
    s_top = s_skip ? 0ull : (unsigned long long)top;
  }
  __syncthreads();
  if (s_skip) return;
  // every warp takes its slots of the stack with one atomic (loop bounds rounded to whole
  // warps, so all lanes vote)
  const uint32_t lane = threadIdx.x & 31u, below = (1u << lane) - 1u;
  const unsigned long long slots = (unsigned long long)grid_ctas * kCacheCap;
  for (unsigned long long q = threadIdx.x; q < ((slots + 31ull) & ~31ull); q += blockDim.x) {
    const bool has = q < slots && (q % kCacheCap) < P.cache_n[q / kCacheCap];
    const uint32_t m = __ballot_sync(0xffffffffu, has);
    unsigned long long base = 0;
    if (lane == 0 && m) base = atomicAdd(&s_top, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (has) {
      const unsigned long long at = base + __popc(m & below);
      if (at < P.npages) P.stack[at] = P.cache[q];
      else atomicOr(&ctl->err, (unsigned)E_CORRUPT);
    }
  }
  const unsigned long long nf = ctl->nfreed;
  for (unsigned long long i = threadIdx.x; i < ((nf + 31ull) & ~31ull); i += blockDim.x) {
    const bool has = i < nf;
    const uint32_t m = __ballot_sync(0xffffffffu, has);
    unsigned long long base = 0;
    if (lane == 0 && m) base = atomicAdd(&s_top, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (has) {
      const unsigned long long at = base + __popc(m & below);
      if (at < P.npages) P.stack[at] = P.freed[i];
      else atomicOr(&ctl->err, (unsigned)E_CORRUPT);
    }
  }
  __syncthreads();
  for (unsigned long long b = threadIdx.x; b < (unsigned long long)grid_ctas; b += blockDim.x) P.cache_n[b] = 0;
  if (threadIdx.x == 0) {
    ctl->top = (long long)s_top;
    ctl->nfreed = 0;
    ctl->ndefer = 0;
    ctl->fast_all = 0u;
    const int lvl = next_level(cp, ctl->E, ctl->level, ctl->n64);
    const int S = level_bits(cp, lvl);
    if (lvl > 0 && ctl->switch_gate < 0) ctl->switch_gate = (long long)ctl->gates;
    if (S < 64) {
      ctl->lb_sum += cp.delta[lvl - 1];
      ctl->lb_prod *= (1.0 - cp.delta[lvl - 1]);
    }
    ctl->level = lvl;
    ctl->S_last = S;
    ctl->E += ctl->dE;
    ctl->dE = 0;
    ctl->n64 += ctl->dn64;
    ctl->dn64 = 0;
    if (ctl->E > ctl->Emax) ctl->Emax = ctl->E;
    ctl->gates += 1;
    // block cache: pause it after kBcZeroGates gates in a row with lookups and no hit
    // (Section 3.4 switches it off when the hit rate stays zero), probe again later
    const unsigned long long lk = ctl->bc_gate_lookups, hit = ctl->bc_gate_hits;
    ctl->bc_lookups += lk;
    ctl->bc_hits += hit;
    ctl->bc_gate_lookups = ctl->bc_gate_hits = 0;
    if (ctl->bc_off) {
      ctl->bc_off -= 1u;
    } else if (lk) {
      ctl->bc_zero_streak = hit ? 0u : ctl->bc_zero_streak + 1u;
      if (ctl->bc_zero_streak >= kBcZeroGates) {
        ctl->bc_off = kBcPause;
        ctl->bc_zero_streak = 0u;
      }
    }
    const unsigned long long in_use = P.npages - s_top - ctl->wc_pages;  // pages holding images
    if (in_use > ctl->peak_pages) ctl->peak_pages = in_use;
  }
}

__global__ void __launch_bounds__(1024) k_post(const Pool P, const CtlParams cp, int grid_ctas) {
  post_body(P, cp, grid_ctas);
}

// One block per job of a batched launch.
__global__ void __launch_bounds__(1024) k_post_batch(const BatchJob* __restrict__ jobs, int grid_ctas) {
  const BatchJob& j = jobs[blockIdx.x];
  post_body(j.L.P, j.L.ctl, grid_ctas);
}

// ------------------------------------------------------------ initialise -- //
__global__ void k_pool_init(const Pool P, unsigned long long nchunks) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < P.npages; i += stride)
    P.stack[i] = (uint32_t)i;
  // every chunk starts as a ZERO image held inline: header only, all fields 0
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < nchunks; c += stride) {
    uint32_t* e = dir_entry(P, c);
    e[0] = 16u;
    e[1] = 0u;
    e[2] = e[3] = 0u;
    e[4] = e[5] = e[6] = e[7] = 0u;
  }
}

// Chunk 0 holds amplitude 1 at index 0 (the state |0...0>), encoded losslessly.
template <int VPT>
__global__ void __launch_bounds__(kThreads) k_init_chunk0(const Pool P, unsigned long long nchunks) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int kc = P.kc;
  const uint32_t N = 2u << kc, cap = codedcap(kc);
  uint64_t* tile = reinterpret_cast<uint64_t*>(smem);
  uint8_t* img = reinterpret_cast<uint8_t*>(tile + tile_words(kc));
  uint32_t* pages = reinterpret_cast<uint32_t*>(img + cap);
  ScanSmem& s = *reinterpret_cast<ScanSmem*>(pages + pagelist_words(kc));
  __shared__ uint32_t s_np;
  __shared__ int s_ok;
  for (uint32_t j = threadIdx.x; j < N; j += kThreads) tile[tile_val(j)] = j == 0 ? 0x3FF0000000000000ull : 0ull;
  __syncthreads();
  int pp = 0;
  const uint32_t n0 = encode_block<VPT>(tile, kc, 64u, -1, kDefaultModes, img, imgcap(kc), s, pp, &P.ctl->err);
  __shared__ uint32_t s_cache_n;
  if (threadIdx.x < 32u) {
    const uint32_t q0 = pages_for(n0, kc);
    if (threadIdx.x == 0) s_cache_n = 0u;
    __syncwarp();
    CtaCache cc;
    cc.ids = nullptr;  // empty cache: every page comes from the stack
    cc.n = &s_cache_n;
    const bool ok = n0 != 0u && alloc_pages_warp(P, cc, pages, q0, nullptr, 0u);
    if (threadIdx.x == 0) {
      s_np = q0;
      s_ok = ok;
      if (!ok) atomicOr(&P.ctl->err, (unsigned)E_OOM);
    }
  }
  __syncthreads();
  if (!s_ok) return;
  store_image_block(P, 0ull, img, n0, pages, s_np);
  if (threadIdx.x == 0) {
    P.ctl->E = 16ull * (nchunks - 1ull) + n0;
    P.ctl->Emax = P.ctl->E;
    P.ctl->n64 = ((reinterpret_cast<const uint32_t*>(img)[0] >> 8) & 0xffu) == 64u ? 1 : 0;
    P.ctl->peak_pages = P.npages - (unsigned long long)P.ctl->top;
  }
}

// -------------------------------------------------------- codec entries -- //
template <int VPT>
__global__ void __launch_bounds__(kThreads)
    k_codec_encode(const double* in, unsigned long long nchunks, int kc, uint32_t S, int force, uint32_t modes,
                   uint8_t* out, unsigned long long stride, uint32_t* lens, unsigned int* err) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t N = 2u << kc, cap = codedcap(kc);
  uint64_t* tile = reinterpret_cast<uint64_t*>(smem);
  uint8_t* img = reinterpret_cast<uint8_t*>(tile + tile_words(kc));
  uint32_t* pages = reinterpret_cast<uint32_t*>(img + cap);
  ScanSmem& s = *reinterpret_cast<ScanSmem*>(pages + pagelist_words(kc));
  int pp = 0;
  for (unsigned long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(in) + c * N;
    for (uint32_t j = threadIdx.x; j < N; j += kThreads) tile[tile_val(j)] = src[j];
    __syncthreads();
    const uint32_t n = encode_block<VPT>(tile, kc, S, force, modes, img, cap, s, pp, err);
    uint4* dst = reinterpret_cast<uint4*>(out + c * stride);
    const uint4* sv = reinterpret_cast<const uint4*>(img);
    for (uint32_t u = threadIdx.x; u < n / 16u; u += kThreads) dst[u] = sv[u];
    if (threadIdx.x == 0) lens[c] = n;
    __syncthreads();
  }
}

template <int VPT>
__global__ void __launch_bounds__(kThreads)
    k_codec_decode(const uint8_t* in, unsigned long long stride, const uint32_t* lens, unsigned long long nchunks,
                   int kc, double* out, unsigned int* err) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t N = 2u << kc, cap = codedcap(kc);
  uint64_t* tile = reinterpret_cast<uint64_t*>(smem);
  uint8_t* img = reinterpret_cast<uint8_t*>(tile + tile_words(kc));
  uint32_t* pages = reinterpret_cast<uint32_t*>(img + cap);
  ScanSmem& s = *reinterpret_cast<ScanSmem*>(pages + pagelist_words(kc));
  int pp = 0;
  for (unsigned long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint32_t len = lens[c];
    const bool fits = len <= cap && (len & 15u) == 0u && len >= 16u;
    if (fits) {
      const uint4* src = reinterpret_cast<const uint4*>(in + c * stride);
      uint4* d = reinterpret_cast<uint4*>(img);
      for (uint32_t u = threadIdx.x; u < len / 16u; u += kThreads) d[u] = src[u];
    } else if (threadIdx.x == 0) {
      reinterpret_cast<uint32_t*>(img)[0] = 0xffu;  // fails the header checks
    }
    __syncthreads();
    const bool ok = decode_block<VPT>(img, fits ? len : 16u, kc, tile, s, pp);
    if (!ok && threadIdx.x == 0) atomicOr(err, (unsigned)E_CORRUPT);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(out) + c * N;
    for (uint32_t j = threadIdx.x; j < N; j += kThreads) dst[j] = tile[tile_val(j)];
    __syncthreads();
  }
}

// --------------------------------------------------------------- readout -- //
// Decodes the chunks overlapping [first_amp, first_amp + count) into out.
template <int VPT>
__global__ void __launch_bounds__(kThreads)
    k_decode_range(const Pool P, unsigned long long first_amp, unsigned long long count, double* out) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int kc = P.kc;
  const uint32_t A = 1u << kc, cap = imgcap(kc);
  uint64_t* tile = reinterpret_cast<uint64_t*>(smem);
  uint8_t* img = reinterpret_cast<uint8_t*>(tile + tile_words(kc));
  uint32_t* pages = reinterpret_cast<uint32_t*>(img + cap);
  ScanSmem& s = *reinterpret_cast<ScanSmem*>(pages + pagelist_words(kc));
  int pp = 0;
  const unsigned long long cfirst = first_amp >> kc, clast = (first_amp + count - 1ull) >> kc;
  for (unsigned long long c = cfirst + blockIdx.x; c <= clast; c += gridDim.x) {
    const uint32_t* e = dir_entry(P, c);
    const uint32_t b = e[0];
    if (b > cap || e[1] > max_pages(kc)) {
      if (threadIdx.x == 0) atomicOr(&P.ctl->err, (unsigned)E_CORRUPT);
      return;
    }
    load_image_block(P, c, img, pages, cap);
    if (!decode_block<VPT>(img, b, kc, tile, s, pp) && threadIdx.x == 0) atomicOr(&P.ctl->err, (unsigned)E_CORRUPT);
    const unsigned long long base = c << kc;
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(out);
    for (uint32_t i = threadIdx.x; i < A; i += kThreads) {
      const unsigned long long a = base + i;
      if (a >= first_amp && a < first_amp + count) {
        dst[2 * (a - first_amp)] = tile[tile_val(2 * i)];
        dst[2 * (a - first_amp) + 1] = tile[tile_val(2 * i + 1)];
      }
    }
    __syncthreads();
  }
}

// Per chunk: sum over its amplitudes of fma(re, re, im*im) (measurement), or the
// partial inner product with a reference state and the norm (fidelity).
template <int VPT, bool DOT>
__global__ void __launch_bounds__(kThreads)
    k_chunk_reduce(const Pool P, unsigned long long cfirst, unsigned long long nchunks, const double* ref, double* out) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int kc = P.kc;
  const uint32_t A = 1u << kc, cap = imgcap(kc);
  uint64_t* tile = reinterpret_cast<uint64_t*>(smem);
  uint8_t* img = reinterpret_cast<uint8_t*>(tile + tile_words(kc));
  uint32_t* pages = reinterpret_cast<uint32_t*>(img + cap);
  ScanSmem& s = *reinterpret_cast<ScanSmem*>(pages + pagelist_words(kc));
  int pp = 0;
  __shared__ double red[3][kThreads];
  for (unsigned long long cl = blockIdx.x; cl < nchunks; cl += gridDim.x) {
    const unsigned long long c = cfirst + cl;
    const uint32_t* e = dir_entry(P, c);
    const uint32_t b = e[0];
    if (b > cap || e[1] > max_pages(kc)) {
      if (threadIdx.x == 0) atomicOr(&P.ctl->err, (unsigned)E_CORRUPT);
      return;
    }
    load_image_block(P, c, img, pages, cap);
    if (!decode_block<VPT>(img, b, kc, tile, s, pp) && threadIdx.x == 0) atomicOr(&P.ctl->err, (unsigned)E_CORRUPT);
    const double* v = reinterpret_cast<const double*>(tile);
    double x = 0.0, y = 0.0, z = 0.0;
    for (uint32_t i = threadIdx.x; i < A; i += kThreads) {
      const double pr = v[tile_val(2 * i)], pi = v[tile_val(2 * i + 1)];
      z += __fma_rn(pr, pr, __dmul_rn(pi, pi));
      if (DOT) {
        const double rr = ref[(cl << kc) * 2 + 2 * i], ri = ref[(cl << kc) * 2 + 2 * i + 1];
        x += rr * pr + ri * pi;
        y += rr * pi - ri * pr;
      }
    }
    red[0][threadIdx.x] = x;
    red[1][threadIdx.x] = y;
    red[2][threadIdx.x] = z;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) {
        red[0][threadIdx.x] += red[0][threadIdx.x + h];
        red[1][threadIdx.x] += red[1][threadIdx.x + h];
        red[2][threadIdx.x] += red[2][threadIdx.x + h];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (DOT) {
        out[3 * cl] = red[0][0];
        out[3 * cl + 1] = red[1][0];
        out[3 * cl + 2] = red[2][0];
      } else {
        out[cl] = red[2][0];
      }
    }
    __syncthreads();
  }
}

// Chunks per mode (counts[8]) and, if wide is not null, the images whose header says
// S = 64 (added to *wide).
__global__ void k_mode_counts(const Pool P, unsigned long long nchunks, unsigned long long* counts,
                              unsigned long long* wide) {
  __shared__ unsigned long long sc[9];
  if (threadIdx.x < 9) sc[threadIdx.x] = 0;
  __syncthreads();
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < nchunks; c += stride) {
    const uint32_t* e = dir_entry(P, c);
    uint32_t h = e[4];
    if (e[1] != 0u) h = *reinterpret_cast<const uint32_t*>(P.pages + (unsigned long long)e[4] * kPage);
    atomicAdd(&sc[h & 7u], 1ull);
    if (((h >> 8) & 0xffu) == 64u) atomicAdd(&sc[8], 1ull);
  }
  __syncthreads();
  if (threadIdx.x < 8 && sc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sc[threadIdx.x]);
  if (threadIdx.x == 8 && wide && sc[8]) atomicAdd(wide, sc[8]);
}

__global__ void k_copy_image(const Pool P, unsigned long long chunk, uint8_t* out) {
  const uint32_t* e = dir_entry(P, chunk);
  const uint32_t b = e[0], np = e[1];
  if (b > max_image_bytes(P.kc) || np > max_pages(P.kc)) return;
  for (uint32_t u = threadIdx.x; u < b / 16u; u += blockDim.x) {
    uint4 v;
    if (np == 0) v = reinterpret_cast<const uint4*>(e + 4)[u];
    else v = reinterpret_cast<const uint4*>(P.pages + (unsigned long long)e[4 + u / (kPage / 16)] * kPage)[u % (kPage / 16)];
    reinterpret_cast<uint4*>(out)[u] = v;
  }
}

// ------------------------------------------------------ uncompressed path -- //
__global__ void k_sv_init(double2* psi, unsigned long long amps) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < amps; i += stride)
    psi[i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
}

// rows: bit 0 / 1 = amplitude a / b is written (its row is not a plain copy [1, 0] /
// [0, 1]), bit 2 / 3 = a / b is read (written, or the other row takes it with a nonzero
// coefficient).  An amplitude left out is neither read nor written: T and CZ move half or
// a quarter of the state.  A value not read enters only with an exactly zero
// coefficient, which the kept-term sums leave out, so the results do not change.
__global__ void __launch_bounds__(256) k_sv_gate(double2* psi, unsigned long long npairs, const GateCoef g, int target,
                                                 unsigned long long cmask, unsigned long long cvals, uint32_t rows) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long tb = 1ull << target, lowm = tb - 1ull;
  for (unsigned long long p = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; p < npairs; p += stride) {
    const unsigned long long i0 = ((p & ~lowm) << 1) | (p & lowm);
    if ((i0 & cmask) != cvals) continue;
    double2 a = (rows & 4u) ? psi[i0] : make_double2(0.0, 0.0);
    double2 b = (rows & 8u) ? psi[i0 | tb] : make_double2(0.0, 0.0);
    apply_pair(g, a, b);
    if (rows & 1u) psi[i0] = a;
    if (rows & 2u) psi[i0 | tb] = b;
  }
}

// ----------------------------------------------------------- checkpoint -- //
// Section 3.5: the compressed state is saved as its chunk images and restored by
// rebuilding the directory and the page arena around them.

// Image length of every chunk (directory entry word 0).
__global__ void k_ck_lengths(const Pool P, unsigned long long nchunks, uint32_t* len) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < nchunks; c += stride)
    len[c] = dir_entry(P, c)[0];
}

// Copies every chunk's image to out + off[c] (one warp per chunk; off multiples of 16).
__global__ void k_ck_gather(const Pool P, unsigned long long nchunks, const unsigned long long* off, uint8_t* out) {
  const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x / 32u);
  const uint32_t lane = threadIdx.x & 31u;
  constexpr uint32_t upp = kPage / 16;
  for (unsigned long long c = blockIdx.x * (unsigned long long)(blockDim.x / 32u) + threadIdx.x / 32u; c < nchunks;
       c += warps) {
    const uint32_t* e = dir_entry(P, c);
    const uint32_t units = e[0] >> 4, np = e[1];
    uint4* dst = reinterpret_cast<uint4*>(out + off[c]);
    for (uint32_t u = lane; u < units; u += 32u)
      dst[u] = np == 0u ? reinterpret_cast<const uint4*>(e + 4)[u]
                        : reinterpret_cast<const uint4*>(P.pages + (unsigned long long)e[4 + u / upp] * kPage)[u % upp];
  }
}

// Writes chunk c's image from in + off[c] (len[c] bytes) back: inline in the directory
// entry when it fits, else into pages pbase[c], pbase[c] + 1, ...
__global__ void k_ck_scatter(const Pool P, unsigned long long nchunks, const unsigned long long* off,
                             const unsigned long long* pbase, const uint32_t* len, const uint8_t* in) {
  const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x / 32u);
  const uint32_t lane = threadIdx.x & 31u;
  constexpr uint32_t upp = kPage / 16;
  for (unsigned long long c = blockIdx.x * (unsigned long long)(blockDim.x / 32u) + threadIdx.x / 32u; c < nchunks;
       c += warps) {
    uint32_t* e = dir_entry(P, c);
    const uint32_t bytes = len[c], units = bytes >> 4, np = pages_for(bytes, P.kc);
    const uint4* src = reinterpret_cast<const uint4*>(in + off[c]);
    for (uint32_t u = lane; u < units; u += 32u) {
      if (np == 0u) reinterpret_cast<uint4*>(e + 4)[u] = src[u];
      else reinterpret_cast<uint4*>(P.pages + (pbase[c] + u / upp) * kPage)[u % upp] = src[u];
    }
    if (np) for (uint32_t k = lane; k < np; k += 32u) e[4 + k] = (uint32_t)(pbase[c] + k);
    if (lane == 0) {
      e[0] = bytes;
      e[1] = np;
      e[2] = e[3] = 0u;
    }
  }
}

// After a restore pages [0, used) hold images: the free stack lists the others.
__global__ void k_ck_stack(const Pool P, unsigned long long used) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; used + i < P.npages; i += stride)
    P.stack[i] = (uint32_t)(used + i);
}

// ------------------------------------------------------------- launchers -- //
static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

#define QC_VPT_DISPATCH(kc, ...)                          \
  switch (vpt_for(kc)) {                                  \
    case 1: { constexpr int V = 1; __VA_ARGS__; } break;  \
    case 2: { constexpr int V = 2; __VA_ARGS__; } break;  \
    case 4: { constexpr int V = 4; __VA_ARGS__; } break;  \
    case 8: { constexpr int V = 8; __VA_ARGS__; } break;  \
    case 16: { constexpr int V = 16; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;                \
  }

int gate_ctas_per_sm(int kc) {
  int n = 0;
  const size_t smem = gate_smem_bytes(kc);
  cudaError_t e = cudaSuccess;
  switch (vpt_for(kc)) {
    case 1: prep(k_gate<1>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gate<1>, kThreads, smem); break;
    case 2: prep(k_gate<2>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gate<2>, kThreads, smem); break;
    case 4: prep(k_gate<4>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gate<4>, kThreads, smem); break;
    case 8: prep(k_gate<8>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gate<8>, kThreads, smem); break;
    case 16: prep(k_gate<16>, smem); e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gate<16>, kThreads, smem); break;
  }
  if (e != cudaSuccess || n < 1) n = 1;
  return n;
}

cudaError_t launch_gate(const GateLaunch& L, int grid, cudaStream_t st) {
  const size_t smem = gate_smem_bytes(L.P.kc);
  QC_VPT_DISPATCH(L.P.kc, {
    cudaError_t e = prep(k_gate<V>, smem);
    if (e != cudaSuccess) return e;
    k_gate<V><<<grid, kThreads, smem, st>>>(L);
  });
  return cudaGetLastError();
}

cudaError_t launch_post(const Pool& P, const CtlParams& cp, int grid_ctas, cudaStream_t st) {
  k_post<<<1, 1024, 0, st>>>(P, cp, grid_ctas);
  return cudaGetLastError();
}

cudaError_t launch_gate_batch(const BatchJob* jobs, int njobs, unsigned long long total, int kc, int grid,
                              cudaStream_t st) {
  const size_t smem = gate_smem_bytes(kc);
  QC_VPT_DISPATCH(kc, {
    cudaError_t e = prep(k_gate_batch<V>, smem);
    if (e != cudaSuccess) return e;
    k_gate_batch<V><<<grid, kThreads, smem, st>>>(jobs, njobs, total);
  });
  return cudaGetLastError();
}

cudaError_t launch_post_batch(const BatchJob* jobs, int njobs, int grid_ctas, cudaStream_t st) {
  k_post_batch<<<njobs, 1024, 0, st>>>(jobs, grid_ctas);
  return cudaGetLastError();
}

cudaError_t launch_pool_init(const Pool& P, unsigned long long nchunks, cudaStream_t st) {
  k_pool_init<<<num_sms() * 4, 256, 0, st>>>(P, nchunks);
  return cudaGetLastError();
}

cudaError_t launch_init_chunk0(const Pool& P, unsigned long long nchunks, cudaStream_t st) {
  const size_t smem = codec_smem_bytes(P.kc);
  QC_VPT_DISPATCH(P.kc, {
    cudaError_t e = prep(k_init_chunk0<V>, smem);
    if (e != cudaSuccess) return e;
    k_init_chunk0<V><<<1, kThreads, smem, st>>>(P, nchunks);
  });
  return cudaGetLastError();
}

cudaError_t launch_codec_encode(const double* in, unsigned long long nchunks, int kc, uint32_t S, int force,
                                uint8_t* out, unsigned long long stride, uint32_t* lens, unsigned int* err,
                                cudaStream_t st) {
  return launch_codec_encode(in, nchunks, kc, S, force, kDefaultModes, out, stride, lens, err, st);
}

cudaError_t launch_codec_encode(const double* in, unsigned long long nchunks, int kc, uint32_t S, int force,
                                uint32_t modes, uint8_t* out, unsigned long long stride, uint32_t* lens,
                                unsigned int* err, cudaStream_t st) {
  const size_t smem = codec_smem_bytes(kc);
  const unsigned long long g = nchunks < (unsigned long long)num_sms() * 8 ? nchunks : (unsigned long long)num_sms() * 8;
  QC_VPT_DISPATCH(kc, {
    cudaError_t e = prep(k_codec_encode<V>, smem);
    if (e != cudaSuccess) return e;
    k_codec_encode<V><<<(unsigned)g, kThreads, smem, st>>>(in, nchunks, kc, S, force, modes, out, stride, lens, err);
  });
  return cudaGetLastError();
}

cudaError_t launch_codec_decode(const uint8_t* in, unsigned long long stride, const uint32_t* lens,
                                unsigned long long nchunks, int kc, double* out, unsigned int* err, cudaStream_t st) {
  const size_t smem = codec_smem_bytes(kc);
  const unsigned long long g = nchunks < (unsigned long long)num_sms() * 8 ? nchunks : (unsigned long long)num_sms() * 8;
  QC_VPT_DISPATCH(kc, {
    cudaError_t e = prep(k_codec_decode<V>, smem);
    if (e != cudaSuccess) return e;
    k_codec_decode<V><<<(unsigned)g, kThreads, smem, st>>>(in, stride, lens, nchunks, kc, out, err);
  });
  return cudaGetLastError();
}

cudaError_t launch_decode_range(const Pool& P, unsigned long long first_amp, unsigned long long count, double* out,
                                cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const size_t smem = codec_smem_bytes(P.kc);
  const unsigned long long nch = ((first_amp + count - 1ull) >> P.kc) - (first_amp >> P.kc) + 1ull;
  const unsigned long long g = nch < (unsigned long long)num_sms() * 8 ? nch : (unsigned long long)num_sms() * 8;
  QC_VPT_DISPATCH(P.kc, {
    cudaError_t e = prep(k_decode_range<V>, smem);
    if (e != cudaSuccess) return e;
    k_decode_range<V><<<(unsigned)g, kThreads, smem, st>>>(P, first_amp, count, out);
  });
  return cudaGetLastError();
}

cudaError_t launch_chunk_norms(const Pool& P, unsigned long long cfirst, unsigned long long nchunks, double* out,
                              cudaStream_t st) {
  const size_t smem = codec_smem_bytes(P.kc);
  const unsigned long long g = nchunks < (unsigned long long)num_sms() * 8 ? nchunks : (unsigned long long)num_sms() * 8;
  QC_VPT_DISPATCH(P.kc, {
    cudaError_t e = prep(k_chunk_reduce<V, false>, smem);
    if (e != cudaSuccess) return e;
    k_chunk_reduce<V, false><<<(unsigned)g, kThreads, smem, st>>>(P, cfirst, nchunks, nullptr, out);
  });
  return cudaGetLastError();
}

cudaError_t launch_chunk_dots(const Pool& P, unsigned long long cfirst, unsigned long long nchunks, const double* ref,
                             double* out, cudaStream_t st) {
  const size_t smem = codec_smem_bytes(P.kc);
  const unsigned long long g = nchunks < (unsigned long long)num_sms() * 8 ? nchunks : (unsigned long long)num_sms() * 8;
  QC_VPT_DISPATCH(P.kc, {
    cudaError_t e = prep(k_chunk_reduce<V, true>, smem);
    if (e != cudaSuccess) return e;
    k_chunk_reduce<V, true><<<(unsigned)g, kThreads, smem, st>>>(P, cfirst, nchunks, ref, out);
  });
  return cudaGetLastError();
}

cudaError_t launch_mode_counts(const Pool& P, unsigned long long nchunks, unsigned long long* counts,
                               unsigned long long* wide, cudaStream_t st) {
  const unsigned long long blocks = (nchunks + 255ull) / 256ull;
  const unsigned g = (unsigned)(blocks < (unsigned long long)num_sms() * 8 ? blocks : (unsigned long long)num_sms() * 8);
  k_mode_counts<<<g, 256, 0, st>>>(P, nchunks, counts, wide);
  return cudaGetLastError();
}

cudaError_t launch_copy_image(const Pool& P, unsigned long long chunk, uint8_t* out, cudaStream_t st) {
  k_copy_image<<<1, 256, 0, st>>>(P, chunk, out);
  return cudaGetLastError();
}

cudaError_t launch_sv_init(double* psi, unsigned long long amps, cudaStream_t st) {
  k_sv_init<<<num_sms() * 8, 256, 0, st>>>(reinterpret_cast<double2*>(psi), amps);
  return cudaGetLastError();
}

cudaError_t launch_sv_gate(double* psi, int n, const GateCoef& g, int target, unsigned long long cmask,
                           unsigned long long cvals, uint32_t rows, cudaStream_t st) {
  const unsigned long long npairs = 1ull << (n - 1);
  const unsigned long long want = (npairs + 255ull) / 256ull;
  const unsigned grid = (unsigned)(want < (unsigned long long)num_sms() * 16 ? want : (unsigned long long)num_sms() * 16);
  if ((rows & 3u) == 0u) return cudaSuccess;  // the identity
  k_sv_gate<<<grid, 256, 0, st>>>(reinterpret_cast<double2*>(psi), npairs, g, target, cmask, cvals, rows);
  return cudaGetLastError();
}

cudaError_t launch_checkpoint_lengths(const Pool& P, unsigned long long nchunks, uint32_t* len, cudaStream_t st) {
  const unsigned long long g = (nchunks + 255) / 256;
  k_ck_lengths<<<(unsigned)(g < 65535ull ? g : 65535ull), 256, 0, st>>>(P, nchunks, len);
  return cudaGetLastError();
}
cudaError_t launch_checkpoint_gather(const Pool& P, unsigned long long nchunks, const unsigned long long* off,
                                     uint8_t* out, cudaStream_t st) {
  k_ck_gather<<<num_sms() * 8, 256, 0, st>>>(P, nchunks, off, out);
  return cudaGetLastError();
}
cudaError_t launch_checkpoint_scatter(const Pool& P, unsigned long long nchunks, const unsigned long long* off,
                                      const unsigned long long* pbase, const uint32_t* len, const uint8_t* in,
                                      unsigned long long used, cudaStream_t st) {
  k_ck_scatter<<<num_sms() * 8, 256, 0, st>>>(P, nchunks, off, pbase, len, in);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ck_stack<<<num_sms() * 8, 256, 0, st>>>(P, used);
  return cudaGetLastError();
}

}  // namespace qc
