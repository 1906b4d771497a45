/*
 * qcsim.h -- C ABI of libqcsim: full-state quantum circuit simulation with the state
 * vector kept compressed in GPU memory (one GB300, sm_103a).
 *
 * Method: Wu et al., "Full-State Quantum Circuit Simulation by Using Data
 * Compression" (SC'19).  The state of n qubits is 2^n complex128 amplitudes
 * (Section 2.1, Eq. 2nrep).  It is split into blocks of 2^block_log2 amplitudes
 * (Section 3.1), each stored compressed; a block is coded as independent chunks of
 * 2^chunk_log2 amplitudes.  Every gate decodes the chunks it touches, applies the 2x2
 * unitary to each amplitude pair that differs only in the target bit and satisfies
 * the controls (Section 3.1, Eq. matrix1 and Eq. matrix2), and re-encodes them with
 * the hybrid codec: a lossless stage first, then the error-bounded lossy coder
 * (bit-plane truncation to 12 - EXP(eps) bits, Eq. sigbits, plus XOR leading-zero
 * coding, Section 4.2 Solution C) once the compressed state plus two decompressed
 * blocks (Eq. totalnbBytes) no longer fit in tau * budget (Section 3.7).
 *
 * Conventions
 *  - Every call returns a sim_status.  No exception crosses the ABI.
 *  - Buffers and out-parameters belong to the caller; the library copies what it
 *    keeps.  The sim_t handle owns all device memory it allocates and frees it in
 *    sim_destroy.
 *  - Work is queued on the handle's CUDA stream (sim_set_stream; default: the legacy
 *    default stream).  Calls that return data to the host synchronise that stream.
 *  - Amplitude index bit k is qubit k.  Amplitudes are interleaved (re, im) doubles.
 *  - SIM_ERR_INVALID: bad arguments; the state is unchanged.
 *  - A failure found on the device while a gate runs (SIM_ERR_OOM: the page pool ran
 *    dry; SIM_ERR_CORRUPT: an image failed its checks or a value was not finite)
 *    poisons the handle: that call, or the next call that synchronises, returns the
 *    error and every later call returns SIM_ERR_STATE.
 *  - sim_last_error() returns a message for the last failure on this thread.
 */
#ifndef QCSIM_H
#define QCSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SIM_OK = 0,
  SIM_ERR_INVALID = -1,
  SIM_ERR_OOM = -2,
  SIM_ERR_CUDA = -3,
  SIM_ERR_CORRUPT = -4,
  SIM_ERR_TIMEOUT = -5,
  SIM_ERR_STATE = -6
} sim_status;

/* One gate (Eq. matrix1; with controls, Eq. matrix2).  The unitary acts on the pair
 * (a_i, a_{i | 2^target}) for every index i with bit `target` clear and
 * (i & ctrl_mask) == ctrl_vals.  u = u00r, u00i, u01r, u01i, u10r, u10i, u11r, u11i,
 * computed on the host (the device never evaluates a trigonometric function).
 * `kind` is a hint (0 general, 1 diagonal, 2 permutation) and is ignored.
 * Rejected with SIM_ERR_INVALID: target outside [0, n), a control outside the
 * register or on the target, ctrl_vals outside ctrl_mask, a non-finite entry, or
 * |U^H U - I| > 1e-12 in any entry.  88 bytes, natural alignment. */
typedef struct sim_gate {
  int32_t target;
  int32_t kind;
  uint64_t ctrl_mask;
  uint64_t ctrl_vals;
  double u[8];
} sim_gate;

typedef struct sim sim_t;

/* Run statistics (Table 2 columns: compression ratio, fidelity bound, time split). */
typedef struct sim_stats_t {
  uint64_t gates;             /* gates applied */
  uint64_t encoded_bytes;     /* sum of chunk image bytes now (sum of sizeof(CB_i), Eq. totalnbBytes) */
  uint64_t max_encoded_bytes; /* largest encoded_bytes seen after any gate */
  uint64_t raw_bytes;         /* 2^(n+4) */
  uint64_t inflight_bytes;    /* two decompressed blocks, 2 * 2^(block_log2 + 4) */
  uint64_t chunks_by_mode[8]; /* chunk images by mode: ZERO CONST PERIOD STREAM RAW SPLIT */
  uint64_t pool_bytes;        /* page arena size */
  uint64_t pages_in_use_bytes;/* pages holding images now */
  uint64_t peak_pages_bytes;  /* most pages in use after any gate */
  uint64_t device_bytes;      /* all device memory the handle owns */
  uint64_t amp_updates;       /* amplitudes in chunks decoded and re-encoded, summed over gates */
  double ratio;               /* raw_bytes / encoded_bytes */
  double min_ratio;           /* raw_bytes / max_encoded_bytes (Table 2 "compression ratio") */
  double eps_current;         /* bound used by the last gate; 0 = lossless */
  double fidelity_lb_sum;     /* 1 - sum_i delta_i, delta_i = 2^EXP(eps_i) per lossy gate (provable) */
  double fidelity_lb_prod;    /* prod_i (1 - delta_i) (Section 3.8) */
  int64_t eps_switch_gate;    /* index of the first gate run lossy, -1 if none */
  int32_t sig_bits_current;   /* S of the last gate (64 = lossless) */
  int32_t level;              /* position on the bound ladder, 0 = lossless */
  int32_t chunk_log2, block_log2;
  uint64_t phase_cycles[6];   /* with sim_set_timing(sim, 2): SM cycles of the fused kernel's CTAs in
                                 stage / decode / apply / encode / commit / constant fast paths */
  uint64_t split_trials;      /* chunk encodes that ran the Solution D trial */
  uint64_t cache_lookups;     /* block-cache lookups (work items that consulted it) */
  uint64_t cache_hits;        /* ... that took a cached result */
  uint64_t fast_items;        /* work items the streaming gate kernel wrote (cumulative) */
  uint64_t fast_deferred;     /* work items it left to the general gate kernel (cumulative) */
  uint64_t kernel_launches;   /* kernels the gates enqueued (selector, streaming, general and post kernels) */
  uint64_t palette_trials;    /* chunk encodes that ran the PALETTE trial */
  uint64_t graph_replays;     /* sim_batch_apply calls led by this handle that replayed its kept graph */
  int32_t ladder;             /* the controller's bound ladder (0 jump, 1 the paper's, 2 guarded) */
  uint32_t modes;             /* the mode set of sim_set_modes / sim_set_selector */
  uint64_t wide_images;       /* chunk images coded at 64 bits (the lossless stage, or a subnormal) */
} sim_stats_t;

/* Creates the state |0...0> of n_qubits (1..40) split into blocks of 2^block_log2
 * amplitudes (clamped to n) with lossy bound err_bound (0 = always lossless;
 * otherwise a normal double in [2^-52, 1)).  The budget defaults to 90 % of the free
 * device memory at creation; chunk_log2 defaults to min(10, block_log2).  Allocates
 * the page arena, directory and free-page stack with cudaMalloc.  *out receives the
 * handle.  Errors: SIM_ERR_INVALID, SIM_ERR_OOM (cudaMalloc failed), SIM_ERR_CUDA. */
sim_status sim_create(int n_qubits, int block_log2, double err_bound, sim_t** out);

/* Like sim_create with every setting given: chunk_log2 in [0, 11] (clamped to the
 * block); budget in bytes (> 0): the memory the compressed state may use, against
 * which the controller compares E + two blocks with threshold floor(tau * budget),
 * tau in (0, 1]; ladder 0 = lossless then err_bound, 1 = the paper's ladder 1e-5,
 * 1e-4, ... up to err_bound, one level per gate (Section 3.7); 2 = the same levels,
 * guarded: before each gate the smallest level (never below the current one) at
 * which the largest images the encoder can write on every chunk the gate rewrites
 * still keep the compressed size within floor(tau * budget) -- a gate that rewrites
 * every chunk ends with at most (chunks x largest image) bytes, any other gate grows
 * the size by at most (rewritten chunks x largest image); if no level satisfies that,
 * err_bound.  pool_bytes is the page arena actually allocated (0: budget + 1/8 for
 * page rounding + the per-CTA page caches).  With ladders 0 and 1 the controller acts
 * before a gate, so one gate can grow the state past the threshold; if the images
 * then exceed the arena the gate fails with SIM_ERR_OOM. */
sim_status sim_create_ex(int n_qubits, int block_log2, int chunk_log2, double err_bound, uint64_t budget,
                         double tau, int ladder, uint64_t pool_bytes, sim_t** out);

/* Frees every device allocation of the handle (after synchronising its stream). */
sim_status sim_destroy(sim_t* sim);

/* Puts the handle back to the state sim_create_ex left it in: |0...0> (chunk 0 coded
 * losslessly, every other chunk ZERO), the lossless stage, every statistic of the run
 * and device counter zero (graph_replays counts on), the block-cache lines empty.  Keeps the allocations and the settings
 * (modes, selector, block cache, fast path, stream, budget).  Synchronises the handle's
 * stream.  Lets a serving loop run circuit after circuit on the same handles, and the
 * batched path replay its cached graph. */
sim_status sim_reset(sim_t* sim);

/* Uses `cuda_stream` (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for all later work of this handle.  The caller keeps the stream alive. */
sim_status sim_set_stream(sim_t* sim, void* cuda_stream);

/* Applies one gate (Section 3.1).  Queued on the stream; device-side failures are
 * reported by this call only if they are already known, otherwise by the next
 * synchronising call.  Kernels per gate: the selector's decisions (selector 2 only);
 * at chunk sizes 2^7..2^11 and widths S <= 32 the streaming kernel (a warp pair per
 * work item, STREAM images in and out); the general kernel over the items the
 * streaming kernel left, or the whole gate; the bookkeeping kernel.  Every path writes
 * the same bytes. */
sim_status sim_apply_gate(sim_t* sim, const sim_gate* gate);

/* Applies n_gates gates in order.  All gates are validated first (none runs if one
 * is invalid).  `gates` is a host array.  Synchronises the stream at the end and
 * returns any device-side error. */
sim_status sim_apply_circuit(sim_t* sim, const sim_gate* gates, size_t n_gates);

/* Batched form: runs `count` circuits, circuits[k] (n_gates[k] gates) on handle
 * sims[k], together.  Gate step t applies gate t of every circuit that has one with a
 * single fused-kernel launch covering the work items of all of them (and one
 * bookkeeping launch); with use_graph != 0 the whole launch sequence is captured into a
 * CUDA graph, launched, and kept by sims[0]: a later call whose launches are the same
 * (same handles and settings, same gates; e.g. after sim_reset) replays it without
 * capturing or uploading again (sim_stats_t.graph_replays).  Each handle keeps its own
 * pool, controller and statistics, and ends in exactly the state sim_apply_circuit
 * would give it.  The
 * handles must be distinct and share chunk_log2; launches go to sims[0]'s stream.
 * All gates are validated first.  Synchronises; returns the first device error. */
sim_status sim_batch_apply(sim_t* const* sims, int count, const sim_gate* const* circuits, const size_t* n_gates,
                           int use_graph);

/* Runs n_circ independent circuits (n_qubits[k] qubits, circ[k][0..n_gates[k]) each)
 * through the batched path and writes each one's statistics to out[k].  One setting
 * for the batch, from sim_autotune on the largest circuit when it has at least 4
 * gates and every circuit at least 8 qubits (blocks 2^10..2^16, chunks 2^8..2^10 up to
 * the smallest circuit, ladders 0..2, mode sets Solution C and Solution C + PALETTE);
 * else blocks 2^20, chunks 2^min(10, smallest n), the jump ladder, Solution C.  Bound
 * err_bound after the lossless stage at budget raw/4, page pool raw + 1/8 + 8 MiB, the
 * gates advanced one step at a time across all circuits in one persistent launch
 * replayed from a CUDA graph (sim_batch_apply).  The handles are created and destroyed
 * inside the call.  Errors as sim_create_ex / sim_autotune / sim_batch_apply. */
sim_status sim_batch_run(int n_circ, const int* n_qubits, const sim_gate* const* circ, const size_t* n_gates,
                         double err_bound, sim_stats_t* out);

/* Chunk-size autotuner: for each candidate chunk_log2, creates a handle (budget raw/4,
 * pool raw + 1/8), applies the first half of the probe circuit, then times the fused
 * kernel over the second half; *best receives the candidate with the most amplitude
 * updates per second of kernel time, rates[i] (if not NULL) each candidate's rate. */
sim_status sim_autotune_chunk(int n_qubits, int block_log2, double err_bound, const sim_gate* probe, size_t n_probe,
                              const int* candidates, int n_candidates, int* best, double* rates);

/* One point of the autotuner's search space and what it measured. */
typedef struct {
  int32_t block_log2;      /* blocks of 2^block_log2 amplitudes (Section 3.1; the controller's in-flight bytes) */
  int32_t chunk_log2;      /* the coding tile: 2^chunk_log2 amplitudes decoded and encoded as one unit */
  int32_t ladder;          /* codec schedule: bound ladder 0 jump, 1 the paper's ladder, 2 guarded */
  uint32_t modes;          /* codec schedule: the chunk modes the encoder may choose */
  double rate;             /* amplitude updates per second of gate-kernel time over the probe's second half */
  double ratio;            /* raw bytes over the peak encoded bytes of the probe run */
  double fidelity_lb_sum;  /* the probe run's provable fidelity bound */
} sim_tune_point;

/* Autotuner over block size, tile size and codec schedule: coordinate descent from the
 * first value of each list, sweeping the chunk sizes, then the block sizes, the
 * ladders and the mode sets with the other settings at their best so far, until a
 * sweep changes nothing (3 sweeps at most).  Each point is measured as in
 * sim_autotune_chunk: a fresh handle (budget raw/4, pool raw + 1/8 + 64 MiB) runs the
 * first half of the probe, then the second half with gate-kernel timing; the best
 * point has the highest rate (every point keeps the bound err_bound).  Blocks clamp to
 * n_qubits and chunks to the block, as sim_create_ex does; points that coincide after
 * clamping are measured once.  *best receives the winner; tried (cap_tried entries,
 * may be NULL) every measured point in order, *n_tried (may be NULL) their number. */
sim_status sim_autotune(int n_qubits, double err_bound, const sim_gate* probe, size_t n_probe,
                        const int32_t* block_log2s, int n_b, const int32_t* chunk_log2s, int n_c, const int32_t* ladders,
                        int n_l, const uint32_t* mode_sets, int n_m, sim_tune_point* best, sim_tune_point* tried,
                        size_t cap_tried, size_t* n_tried);

/* Changes the budget the controller compares with (Section 3.7; threshold floor(tau *
 * bytes)) from the next gate on; the page arena keeps the size it was created with.
 * bytes > 0, else SIM_ERR_INVALID. */
sim_status sim_set_budget(sim_t* sim, uint64_t bytes);

/* Named settings, from the next gate on: "modes" (as sim_set_modes), "selector" (0 or
 * 1; the network needs sim_set_selector), "block_cache" (0/1, as sim_set_block_cache),
 * "timing" (0/1/2, as sim_set_timing), "tau_ppm" (tau in millionths, (0, 1e6]),
 * "fast_path" (1 default: gates run the streaming kernel first where it applies, see
 * sim_apply_gate; 0: every item through the general kernel -- same bytes, slower),
 * "ladder" (0/1/2; only before the first gate).  "chunk_log2" and "block_log2" are fixed
 * at creation.  Unknown keys or values out of range: SIM_ERR_INVALID. */
sim_status sim_set_option(sim_t* sim, const char* key, int64_t value);

/* Compressed block cache (Section 3.4): on = 1 allocates 256 lines (each 64 bytes plus
 * room for four images of the largest size, 16.8 MB at chunk_log2 10) and makes later
 * gates look up every work item of two chunks: a line holds the item's two input
 * images and the two images the running gate made of them, so another item of the same
 * gate with byte-identical inputs takes those images instead of decoding, applying and
 * encoding (the result is the same bytes).  Lines are valid for one gate; when 16 gates
 * in a row look up without a hit the cache sits out 64 gates, then probes again.  No
 * lookups while selector training records are being written.  on = 0 frees the lines.
 * Counts in sim_stats_t.cache_lookups / cache_hits. */
sim_status sim_set_block_cache(sim_t* sim, int on);

/* Chunk modes the encoder chooses from for later gates (bit m = mode m).  The default
 * 0x1F is Solution C (Section 4.2) with its Zstd stand-in modes ZERO..RAW; bit 5 adds
 * SPLIT, Solution D (the real parts, then the imaginary parts, XOR-coded); bit 6 adds
 * PALETTE (the lossless stage's dictionary part, Section 3.7: a chunk's at most 256
 * distinct truncated values ascending, then one k-bit index per value,
 * k = max(1, ceil(log2 P))).  The set must contain 0x1F.  With any extra mode every work
 * item runs in the general gate kernel. */
sim_status sim_set_modes(sim_t* sim, uint32_t modes);

/* Learned selector (not from the paper).  selector 0: the mode set of sim_set_modes
 * (default Solution C, 0x1F); 1: every mode (0x7F), each chunk running the SPLIT
 * (Solution D) and PALETTE trials (exhaustive); 2: Solution C's modes, plus the SPLIT /
 * PALETTE trial for a chunk only where a 16 -> 32 -> 32 -> 8 network with bfloat16
 * weights (1864 values, W1[32][16] b1 W2[32][32] b2 W3[8][32] b3, host pointer, copied)
 * grants it.  The network predicts the best mode (outputs 0..6) and a bit budget (output
 * 7: the best image's size over the RAW size) from the chunk's current image header and
 * the gate alone, so one small kernel takes a whole gate's decisions before the gate
 * runs; a trial runs iff its mode's logit + 2 reaches the largest mode logit, and both
 * run when the budget is below half the chunk's current size fraction.  Items none of
 * whose chunks got a trial stay on the streaming kernel.  float32 inference in a fixed
 * order: decisions are reproducible.  The codec enforces the bound whatever the network
 * says.  Selector 2 allocates one decision byte per chunk.  Counts in
 * sim_stats_t.split_trials / palette_trials. */
sim_status sim_set_selector(sim_t* sim, int selector, const uint16_t* bf16_params);

/* Selector training records: with capacity > 0, every chunk a gate encodes appends 20
 * floats (the network's 16 inputs from the chunk's pre-gate image and the gate, the mode
 * the mode set chose, that image's size over the RAW size, 0, 0) until capacity records
 * exist; with selector 1 the chosen mode is the best of all seven.  Gates run in the
 * general kernel while records are written.  0 stops and frees. */
sim_status sim_trace(sim_t* sim, uint64_t capacity);
sim_status sim_trace_read(sim_t* sim, float* out, uint64_t cap_records, uint64_t* n_records);

/* Selector training on the GPU with the library's own kernels: n samples of 16 inputs
 * (x), the exhaustive mode (0..6) and the best size fraction (sizes, one per sample);
 * loss: softmax cross-entropy of outputs 0..6 plus the squared error of output 7;
 * float32 master weights
 * (params, 1864 values, in: initial, out: trained) rounded to bfloat16 for every
 * forward and backward pass; Adam (beta 0.9, 0.999), minibatches from a seeded
 * shuffle.  bf16_out (may be NULL) receives the trained bfloat16 weights, last_loss
 * the mean loss of the last epoch. */
sim_status sim_mlp_train(const float* x, const int32_t* mode, const float* sizes, uint64_t n, int epochs, int batch,
                         float lr, uint64_t seed, float* params, uint16_t* bf16_out, float* last_loss);

/* Loss and its gradient over n samples at the bfloat16 rounding of params (float32
 * arithmetic), for checking the training kernels. */
sim_status sim_mlp_grad(const float* params, const float* x, const int32_t* mode, const float* sizes, uint64_t n,
                        float* grad_out, float* loss_out);

/* Waits for queued work and returns the device error state. */
sim_status sim_sync(sim_t* sim);

/* Decodes amplitudes [first, first + count) into out (2*count doubles, interleaved).
 * out_on_device != 0: `out` is a device pointer; else a host pointer. */
sim_status sim_amplitudes(sim_t* sim, uint64_t first, uint64_t count, double* out, int out_on_device);

/* One measurement of all qubits in the computational basis, without collapsing the
 * state: u = (splitmix64(seed) >> 11) * 2^-53, outcome = smallest index whose running
 * sum of |a_i|^2 reaches u * sum |a|^2; *prob = |a_outcome|^2 / sum |a|^2. */
sim_status sim_measure(sim_t* sim, uint64_t seed, uint64_t* outcome, double* prob);

/* F = |<ref|psi>| (Section 3.8, Eq. idealsim) against a full reference state of
 * 2^n interleaved amplitudes (host pointer, or device pointer if ref_on_device).
 * Also returns <ref|psi> in re_im[2] and |psi|^2 in norm2 (either may be NULL). */
sim_status sim_fidelity(sim_t* sim, const double* ref, int ref_on_device, double* F, double* re_im,
                        double* norm2);

/* Copies the run statistics (synchronises). */
sim_status sim_stats(sim_t* sim, sim_stats_t* out);

/* Copies chunk c's image into out (capacity cap bytes, host memory); *len receives
 * its length.  For checking images against a reference codec. */
sim_status sim_chunk_image(sim_t* sim, uint64_t c, uint8_t* out, size_t cap, size_t* len);

/* Checkpoint / resume (Section 3.5: save the compressed blocks, load them in a later
 * job).  The checkpoint is one flat little-endian buffer: a 256-byte header (magic
 * "QCSIMCK1", version 1, n, block_log2, chunk_log2, err_bound, budget, tau, ladder,
 * mode set, controller level and bits, E, Emax, gates, switch gate, both fidelity-bound
 * accumulators, amplitude updates, peak pages, chunk count, image bytes), then one
 * uint32 image length per chunk, then the chunk images in chunk order (each a multiple
 * of 16 bytes, the chunk image format).  Page ids are not saved; the selector network
 * and timing switches are host settings and are not saved either.
 * sim_checkpoint_size: bytes sim_checkpoint_save writes for the current state.
 * sim_checkpoint_save: writes the checkpoint to out (cap bytes; out on the device if
 *   out_on_device, else host memory); SIM_ERR_INVALID if cap is too small.  The state
 *   is unchanged.
 * sim_checkpoint_load: replaces the state of sim (created with the same n, block_log2,
 *   chunk_log2, err_bound, budget, tau and ladder, else SIM_ERR_INVALID) with the saved
 *   one: images, directory, page arena (pages reassigned in chunk order), controller and
 *   counters, so later gates give the images an uninterrupted run gives.  Lengths and
 *   header fields are checked (SIM_ERR_INVALID); an arena too small for the saved images
 *   gives SIM_ERR_OOM.  Clears a poisoned handle on success.  The caller owns the
 *   buffers; both calls synchronise the handle's stream. */
sim_status sim_checkpoint_size(sim_t* sim, uint64_t* bytes);
sim_status sim_checkpoint_save(sim_t* sim, void* out, uint64_t cap, int out_on_device);
sim_status sim_checkpoint_load(sim_t* sim, const void* in, uint64_t in_len, int in_on_device);

/* Number of chunks and chunk_log2 of the handle. */
sim_status sim_layout(sim_t* sim, uint64_t* n_chunks, int* chunk_log2, int* block_log2);

/* Timing of the fused gate kernel: with timing on (on = 1; on = 2 also counts the
 * SM cycles of each phase of the kernel, see sim_stats_t), every gate-kernel launch is
 * bracketed by CUDA events on the handle's stream.  sim_timing synchronises and
 * returns, since timing was switched on or last read: the summed kernel time in ms,
 * the number of gate-kernel launches, and the chunk-image bytes those launches read
 * and wrote (the compressed traffic of the gates); then it starts counting anew. */
sim_status sim_set_timing(sim_t* sim, int on);
sim_status sim_timing(sim_t* sim, double* gate_kernel_ms, uint64_t* launches, uint64_t* bytes_read,
                      uint64_t* bytes_written);

/* The same figures launch by launch, for the launches sim_timing would sum next (call
 * it before sim_timing, which starts counting anew): *n receives their number; the
 * first min(*n, cap) entries of ms, bytes_read and bytes_written (caller-owned arrays of
 * cap entries) receive each gate-kernel launch's CUDA-event time and the chunk-image
 * bytes it read and wrote, in launch order.  Synchronises the handle's stream.  With
 * timing on, every gate also copies the two traffic counters into a device log that
 * grows by stream-ordered allocation.  Errors: SIM_ERR_INVALID (NULL pointers with
 * cap > 0), SIM_ERR_CUDA. */
sim_status sim_timing_launches(sim_t* sim, uint64_t cap, float* ms, uint64_t* bytes_read, uint64_t* bytes_written,
                               uint64_t* n);

/* Message for the last failure on the calling thread ("" if none). */
const char* sim_last_error(void);

/* ---------------------------------------------------------------------------------
 * Codec entry points: the device encoder and decoder on caller-provided chunks.
 * A chunk is 2^chunk_log2 amplitudes = 2^(chunk_log2+1) doubles.  Image format:
 * 16-byte header [mode, S, log2 P, 0, payload bytes u32, coded values u32,
 * residual bits u32] then the payload (a multiple of 16 bytes); modes 0 ZERO,
 * 1 CONST, 2 PERIOD, 3 STREAM, 4 RAW (Section 4.2 Solution C for the coded streams;
 * the modes stand in for its Zstd stage), 5 SPLIT (Solution D), 6 PALETTE (header byte 2
 * = index bits k, bytes 12..15 = palette size P; payload: the P values ascending as
 * unsigned 64-bit integers, padded to 16 bytes, then the k-bit indices like a residual
 * stream, padded to 16 bytes).  The encoder truncates with
 * S = 12 - EXP(eps) bits (eps = 0: 64 bits), forced to 64 for a chunk holding a
 * nonzero subnormal, and keeps the smallest image (ties: lower mode); force_mode
 * >= 0 selects a mode instead (SIM_ERR_INVALID if it does not apply).
 * ------------------------------------------------------------------------------- */

/* Encodes n_chunks chunks: in = n_chunks * 2^(chunk_log2+1) doubles; image k is
 * written at out + k * out_stride (out_stride >= 16 + 16 * 2^chunk_log2 + 2^chunk_log2/2
 * + 32, a multiple of 16) and its length to out_len[k].  on_device != 0: all three
 * pointers are device pointers; else host pointers. */
sim_status sim_codec_encode(const double* in, uint64_t n_chunks, int chunk_log2, double eps, int force_mode,
                            uint8_t* out, uint64_t out_stride, uint32_t* out_len, int on_device);

/* sim_codec_encode with the automatic choice restricted to the mode set `modes`
 * (see sim_set_modes). */
sim_status sim_codec_encode_ex(const double* in, uint64_t n_chunks, int chunk_log2, double eps, int force_mode,
                               uint32_t modes, uint8_t* out, uint64_t out_stride, uint32_t* out_len, int on_device);

/* Decodes n_chunks images (image k at in + k * in_stride, length in_len[k]) into
 * out = n_chunks * 2^(chunk_log2+1) doubles.  SIM_ERR_CORRUPT if any image fails
 * its checks (its chunk is then zero-filled). */
sim_status sim_codec_decode(const uint8_t* in, uint64_t in_stride, const uint32_t* in_len, uint64_t n_chunks,
                            int chunk_log2, double* out, int on_device);

/* The encoder of sim_codec_encode for callers that must not allocate device memory
 * (the paper has no counterpart; this is a deployment variant).  In, out and out_len
 * are host pointers with the meaning of sim_codec_encode.  Where sim_codec_encode
 * obtains its staging buffer with cudaMalloc on every call, this call stages through
 * one fixed device array of 8 MiB that the library declares (held by every GPU that
 * loads the library until the process exits), so it never calls cudaMalloc, cudaFree
 * or an allocating library routine.  That suits processes whose device memory is
 * already owned by another allocator or bounded by a fixed budget.
 *  - A request whose inputs, images and lengths need more than the array returns
 *    SIM_ERR_INVALID ("request larger than the 8 MiB scratch"): n_chunks *
 *    (16 * 2^chunk_log2 + out_stride) + 4 * n_chunks + 768 bytes must fit in 8 MiB.
 *  - The first call on each device looks up the array's device address (with that
 *    device current, under a lock, so first calls from several host threads are
 *    safe); make that first call before any stream capture.  The address is kept for
 *    the process: after a cudaDeviceReset of a device the call must not be used there.
 *  - All calls on a device share the array: calls that overlap on the same device
 *    (other host threads or streams) race and must be serialised by the caller.
 *    Each call resets the parts it uses, so results never depend on earlier calls.
 *  - Works on the legacy default stream and returns when the images are on the host. */
sim_status sim_codec_encode_noalloc(const double* in, uint64_t n_chunks, int chunk_log2, double eps, int force_mode,
                                    uint8_t* out, uint64_t out_stride, uint32_t* out_len);

/* ---------------------------------------------------------------------------------
 * Uncompressed complex128 state vector on the same GPU (the comparator of the
 * compressed path; same gate arithmetic).  16 * 2^n bytes of device memory.
 * ------------------------------------------------------------------------------- */
typedef struct sim_sv sim_sv_t;
sim_status sim_sv_create(int n_qubits, sim_sv_t** out);
sim_status sim_sv_destroy(sim_sv_t* sv);
sim_status sim_sv_set_stream(sim_sv_t* sv, void* cuda_stream);
sim_status sim_sv_apply_circuit(sim_sv_t* sv, const sim_gate* gates, size_t n_gates);
sim_status sim_sv_amplitudes(sim_sv_t* sv, uint64_t first, uint64_t count, double* out, int out_on_device);
/* Device pointer to the 2^n interleaved amplitudes (valid until sim_sv_destroy). */
sim_status sim_sv_data(sim_sv_t* sv, double** dev_ptr);

#ifdef __cplusplus
}
#endif

#endif /* QCSIM_H */
