/*
 * vibe.h -- C ABI of the GB300 (sm_103a) VibeLSD decoding library, libvibe.so.
 *
 * VibeLSD (arXiv 2508.15743): a batch of syndromes of a detector error model (check matrix H,
 * logical matrix L, priors p_j; Sec. II.B, Eq. 1) is decoded by an ensemble of K serial-schedule
 * min-sum BP members (Sec. III.A-B, Appendix A Algorithm 1), each with its own permutation of the
 * columns (Sec. III.D.1). Once M members converge the rest stop and the most likely candidate is
 * kept (Sec. III.D.2 steps 3-4); when none converges, the normalised average of the members' LLRs
 * (Sec. III.D.2 step 5) drives LSD post-processing (Sec. III.C).
 *
 * Conventions for every entry point:
 *  - All sizes are in elements. Bit-packed vectors are arrays of uint32 words with bit b of word w
 *    holding entry 32*w + b; padding bits past the last entry must be zero on input and are zero
 *    on output.
 *  - Pointers named d_* are device pointers (cudaMalloc or equivalent, on the handle's device);
 *    pointers named h_* or without a prefix are host pointers. The library never frees caller memory.
 *  - Functions return VIBE_OK (0) or a negative VIBE_ERR_* code; vibe_last_error() then describes
 *    the failure for the calling thread. Per-shot outcomes never fail a call: they go in
 *    vibe_shot_stats.status.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 */
#ifndef VIBE_H
#define VIBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VIBE_OK 0
#define VIBE_ERR_INVALID (-1) /* malformed matrix, bad sizes or parameters */
#define VIBE_ERR_NOMEM (-2)   /* a device or host allocation failed */
#define VIBE_ERR_CUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define VIBE_ERR_UNSUPPORTED (-4) /* valid input beyond this build's limits (see vibe_create) */

#define VIBE_STATUS_OK 0
#define VIBE_STATUS_UNSOLVABLE 1 /* syndrome outside the column span of H; correction is zero */
#define VIBE_STATUS_CLUSTER_LIMIT 3 /* LSD met a cluster of more columns than its combination records hold
                                       (32 x 32 x words-per-lane: at least 4096, or all n); correction zero */
#define VIBE_STATUS_BAD_PROBLEM 2 /* vibe_batch_decode: problem index outside 0..count-1; nothing decoded,
                                     correction and logical words zero */

/* Sparse binary matrix in CSR form, host memory; copied by vibe_create. colidx ascending, no
 * duplicates within a row. */
typedef struct {
  int32_t nrows;
  int32_t ncols;
  const int32_t* rowptr; /* nrows + 1 entries, rowptr[0] = 0 */
  const int32_t* colidx; /* rowptr[nrows] entries in [0, ncols) */
} vibe_csr;

/* Decoder parameters (Sec. III.D.1 steps 1-2 and 5; Algorithm 1 inputs). */
typedef struct {
  int32_t max_iter;  /* T: BP iterations per member, >= 1 */
  float alpha;       /* min-sum scaling factor in (0, 1], applied to every check-to-variable message */
  int32_t M;         /* correction limit, 1 <= M <= K and M <= 32 */
  int32_t lsd_order; /* 0 = LSD-0; q > 0 searches the 2^q settings of the first q free columns of each
                        cluster for the lowest prior weight (q <= 10) */
  int32_t msg_fp16;  /* 0: FP32 messages; 1: FP16 storage of variable-to-check messages, FP32 arithmetic */
  uint64_t seed;     /* seeds the schedules when vibe_create gets schedules == NULL */
  int32_t bp_engine; /* BP kernel: VIBE_ENGINE_AUTO, _IMAGE or _SUMMARY (same results) */
  int32_t n_flood;   /* members 0 .. n_flood-1 use Algorithm 1's parallel (flooding) schedule instead of
                        a serial one (their schedules are ignored); 0 <= n_flood <= K. With FP16
                        storage only the stored variable-to-check messages are rounded. Image engine
                        only (the summary engine returns VIBE_ERR_UNSUPPORTED) */
  const float* member_alpha; /* NULL, or K host floats in (0, 1] (copied): member i scales its
                        check-to-variable messages by member_alpha[i] instead of alpha, an ensemble
                        mixing heuristics (Sec. V); results, ranking and LLR average are otherwise
                        unchanged. Both engines, all schedules and storage precisions */
  int32_t pair_mode; /* 0: one warp per shot runs the shot's members one after another (throughput);
                        1: one warp per (shot, member) pair, so a shot's members run at the same time
                        and its BP latency is that of its slowest member, not the sum (latency). The
                        outputs are identical; pair mode does more sweeps in total (members run until
                        they see M earlier candidates) and keeps every member's record per shot */
  int32_t n_layered; /* members n_flood .. n_flood+n_layered-1 use a layered schedule (Sec. V names
                        layered schedules between serial and parallel without defining one; read as
                        row-layered min-sum): the checks are split into layers by greedy colouring in
                        ascending check order (a check joins the smallest layer holding no earlier
                        check that shares a column with it); each iteration takes the layers in order,
                        every check of the layer computes its check-to-variable messages from the
                        current variable-to-check ones, then every column of those checks recomputes
                        its variable-to-check messages from its current check-to-variable messages
                        (zero before a member's first iteration); the posterior follows the last layer.
                        n_flood + n_layered <= K; schedules of these members are ignored. Image engine
                        only, FP32 or FP16 storage (only the variable-to-check messages are rounded) */
} vibe_params;

/* BP engines; both run one warp per shot (per (shot, member) pair in pair mode) and give the same bits.
 * IMAGE: the member's whole message image in shared memory; fast for problems whose image is small
 * (code capacity, phenomenological). SUMMARY: the messages in global memory in schedule order and,
 * per check, a summary in shared memory (smallest and second-smallest magnitude with their holders, a
 * lower bound on the other holders' magnitudes, the sign parity; 16 bytes, 8 with FP16 messages); a
 * check whose summary cannot answer a query exactly is rescanned from the messages
 * (VIBE_CNT_RESCANS). For circuit-level problems whose image does not fit. AUTO takes IMAGE when at
 * least 8 warps per SM fit, else SUMMARY. */
#define VIBE_ENGINE_AUTO 0
#define VIBE_ENGINE_IMAGE 1
#define VIBE_ENGINE_SUMMARY 2

/* Per-shot record, 12 bytes. */
typedef struct {
  uint8_t status;           /* VIBE_STATUS_* */
  uint8_t lsd_invoked;      /* 1 if no member converged and LSD produced the correction */
  uint8_t n_converged;      /* candidates kept: min(M, members converged when BP stopped) */
  uint8_t chosen_member;    /* member whose correction was kept; 255 when LSD decided */
  uint16_t iters;           /* iteration at which the ensemble stopped; T when fewer than M converged */
  uint16_t largest_cluster; /* columns in the largest LSD cluster (0 without LSD) */
  uint32_t n_clusters;      /* final LSD clusters (0 without LSD) */
} vibe_shot_stats;

/* Indices into the optional counters array of vibe_decode (uint64, accumulated, never reset). */
#define VIBE_CNT_SHOTS 0       /* shots decoded */
#define VIBE_CNT_FAILURES 1    /* shots whose L*e differs from the given observables */
#define VIBE_CNT_LSD 2         /* shots sent to LSD */
#define VIBE_CNT_PAIR_ITERS 3  /* BP sweeps executed, summed over (shot, member) pairs */
#define VIBE_CNT_UNSOLVABLE 4
#define VIBE_CNT_BAD_PROBLEM 5 /* vibe_batch_decode shots with an out-of-range problem index */
#define VIBE_CNT_RESCANS 6     /* summary engine: check rows rescanned (a summary could not answer) */
#define VIBE_CNT_LSD_WORDOPS 7 /* LSD: 32-bit words XOR-ed by its GF(2) eliminations (its integer work) */
#define VIBE_NUM_COUNTERS 8

typedef struct vibe_handle vibe_handle;
typedef struct vibe_batch vibe_batch; /* opaque: several handles decoded in one launch */

/*
 * vibe_create -- offline setup (Sec. III.D.1).
 *   H: m x n check matrix (detectors x mechanisms); L: k x n logical matrix (k <= 1024);
 *   priors: n doubles p_j in (0, 0.5); the prior LLRs log((1-p)/p) are evaluated in double on the
 *   host and rounded once to float.
 *   K: ensemble size, 1..255. schedules: K x n uint32 permutations of 0..n-1 (member i processes
 *   columns in the order schedules[i*n .. i*n+n-1]); NULL draws them on the device from params->seed
 *   (member i: SplitMix64 started at seed + (i+1)*0xD1B54A32D192ED03, Durstenfeld shuffle taking
 *   j = high 64 bits of next()*(k+1) for k = n-1 down to 1).
 *   Uses the current CUDA device. Copies everything it is given; the device tables (CSR/CSC of H,
 *   per-member dependency wavefronts, message images) stay resident until vibe_destroy.
 *   Limits of this build (VIBE_ERR_UNSUPPORTED beyond them): n < 2^24, m < 2^24, every row of H has
 *   at most 255 entries, every column at most 32, and one shot's BP state (messages, posteriors,
 *   syndrome) must fit in 200 KB of shared memory.
 *   Errors: VIBE_ERR_INVALID (NULL pointers, malformed CSR, a row with no entry, priors outside
 *   (0, 0.5), bad K/params, schedules not permutations), VIBE_ERR_NOMEM, VIBE_ERR_CUDA.
 *   On error *out is set to NULL and nothing is leaked.
 */
int vibe_create(const vibe_csr* H, const vibe_csr* L, const double* priors, int32_t K,
                const uint32_t* schedules, const vibe_params* params, vibe_handle** out);

/*
 * vibe_decode -- online decoding of B shots (Sec. III.D.2), asynchronous on `stream`.
 *   d_syndromes: B x ceil(m/32) words (device). Outputs (device, caller-owned):
 *   d_corrections: B x ceil(n/32) words, the correction e with H e = s for solvable shots;
 *   d_logical: B x ceil(k/32) words, L e mod 2 (may be NULL); d_stats: B records (may be NULL);
 *   d_soft: B x n floats (may be NULL): the chosen member's final posterior LLRs, or for LSD shots
 *   the normalised LLR average that ranked the columns;
 *   d_observables: B x ceil(k/32) true logical flips (may be NULL) -- with d_counters, counts
 *   shots whose L e differs; d_counters: VIBE_NUM_COUNTERS uint64 accumulators (may be NULL).
 *   The handle's workspace is allocated on the first call and grown when a larger batch needs it;
 *   calls with a batch no larger than an earlier one allocate nothing. Large batches run in chunks.
 *   Calls on one handle must not overlap in time (the workspace is shared); use one handle per stream.
 *   Errors: VIBE_ERR_INVALID (NULL handle/required pointer, B < 0), VIBE_ERR_NOMEM, VIBE_ERR_CUDA.
 *   B = 0 is a no-op.
 */
int vibe_decode(vibe_handle* h, const uint32_t* d_syndromes, int64_t B, uint32_t* d_corrections,
                uint32_t* d_logical, vibe_shot_stats* d_stats, float* d_soft,
                const uint32_t* d_observables, uint64_t* d_counters, void* stream);

/*
 * vibe_decode_host -- the same decoding with host buffers (pageable or pinned). Copies the
 * syndromes (and observables) to the device, decodes, copies the results back and waits for the
 * stream. Device staging buffers belong to the handle and grow like its workspace.
 *   h_counters, if not NULL, receives this call's counters (not accumulated across calls).
 */
int vibe_decode_host(vibe_handle* h, const uint32_t* h_syndromes, int64_t B, uint32_t* h_corrections,
                     uint32_t* h_logical, vibe_shot_stats* h_stats, const uint32_t* h_observables,
                     uint64_t* h_counters, void* stream);

/*
 * vibe_get_wavefronts -- the dependency wavefronts built for one member (Sec. III.D.1 step 4):
 *   level(v) = 1 + max{level(u) : u before v in the member's order and u, v share a check}, so the
 *   columns of one level share no check and may be updated together with results identical to the
 *   serial order. order_out: n column indices grouped by level (host); level_offsets_out: n + 1
 *   entries, level l holds order_out[level_offsets_out[l] .. level_offsets_out[l+1]); *nlevels_out
 *   the level count. Synchronous. Errors: VIBE_ERR_INVALID, VIBE_ERR_CUDA.
 */
int vibe_get_wavefronts(vibe_handle* h, int32_t member, uint32_t* order_out,
                        uint32_t* level_offsets_out, int32_t* nlevels_out);

/*
 * vibe_get_layers -- the check layers of the layered schedule as built on the device (n_layered > 0):
 *   layer_of_check_out (host, m int32, may be NULL) receives each check's layer, *nlayer_out (may be
 *   NULL) the number of layers. Synchronous.
 *   Errors: VIBE_ERR_INVALID (NULL handle, or a handle without layered members), VIBE_ERR_CUDA.
 */
int vibe_get_layers(vibe_handle* h, int32_t* layer_of_check_out, int32_t* nlayer_out);

/*
 * vibe_profile -- start (enable != 0) or stop recording CUDA events around every kernel that
 * vibe_decode launches on the caller's stream; clears the totals. vibe_profile_read waits for the
 * last recorded event and returns the summed device time (ms) of the BP ensemble kernel and of the
 * LSD kernel since the last vibe_profile call, and how many of each were launched. A decode runs in
 * chunks, each one LSD launch after its BP launches; in pair mode a chunk's BP part is several
 * launches (sized by the member records), timed together as the chunk's BP time.
 */
int vibe_profile(vibe_handle* h, int32_t enable);
int vibe_profile_read(vibe_handle* h, double* bp_ms, double* lsd_ms, int64_t* bp_launches, int64_t* lsd_launches);

/*
 * vibe_decode_noalloc -- vibe_decode for callers that must not allocate device memory while they
 * decode: a control loop that has to keep a fixed memory footprint once running, a process sharing
 * the GPU under a hard memory budget, or code running where the CUDA allocator may not be entered.
 * The paper has no counterpart; this is an operational variant of vibe_decode.
 *   It runs the same BP ensemble and LSD kernels but takes all of their scratch from one static
 *   device array of 64 MiB that every GPU loading the library holds until the process exits. It
 *   calls no cudaMalloc/cudaFree and allocates nothing on the host; the handle must already exist.
 *   Inputs and outputs are as for vibe_decode (d_logical and d_stats may be NULL); no soft output,
 *   observables or counters.
 *   Limit: B shots need B*(4n+4) bytes beside a fixed part that depends on the problem
 *   (counters, one n-float accumulator per BP warp, one row set per LSD CTA); a batch that does not
 *   fit returns VIBE_ERR_UNSUPPORTED with the largest batch that does (about 15,000 shots for the
 *   d=9 phenomenological problem) -- split larger batches into several calls.
 *   CUDA loads device code lazily by default (CUDA_MODULE_LOADING=EAGER changes that), so the array is
 *   placed on a device, and its address looked up (cudaGetSymbolAddress, with the handle's device
 *   current), at the first call on that device -- which may need 64 MiB of free device memory. A call
 *   with B = 0 does exactly that set-up and decodes nothing: make one per device while allocation is
 *   still allowed and before any stream capture. The address is kept for the life of the process; do
 *   not use this entry point after cudaDeviceReset.
 *   Every call on a device shares the one array, and its contents persist between calls (the call
 *   clears the counters it needs). Calls whose work overlaps on the GPU -- on different streams or
 *   from different threads without ordering -- race on it and must be serialised by the caller.
 *   Errors: VIBE_ERR_INVALID (NULL handle/pointers, B < 0, handle's device not current),
 *   VIBE_ERR_UNSUPPORTED (batch too large, or a handle on the summary engine, whose per-warp message
 *   arrays leave no useful grid in 64 MiB), VIBE_ERR_CUDA. B = 0 performs only the set-up above.
 *   Always runs one warp per shot, whatever the handle's pair_mode (same results).
 */
int vibe_decode_noalloc(vibe_handle* h, const uint32_t* d_syndromes, int64_t B, uint32_t* d_corrections,
                        uint32_t* d_logical, vibe_shot_stats* d_stats, void* stream);

/*
 * vibe_autotune -- times the decode of a sample batch (d_syndromes: B >= 1 shots, device) and keeps the
 * fastest launch configuration for this handle. For each BP engine the problem fits
 * (VIBE_ENGINE_IMAGE, VIBE_ENGINE_SUMMARY) it searches, one knob after the other: pair or shot mode
 * (one warp per (shot, member) pair, or one warp per shot -- the pair_mode given at creation is only
 * the starting point), the BP kernel's persistent grid (occupancy maximum, 3/4 and 1/2 CTAs per SM),
 * and the LSD kernel's CTA size (64, 128 or 256 threads: warps that reduce the columns of different
 * clusters at the same time) with its grid (maximum and half). Every candidate is timed on a second
 * decode of the sample, unless its first decode took over twice the best time so far (a mode whose
 * first candidate fails that way is dropped). Decoding results do not depend on any of these knobs (shots are
 * independent and each shot's arithmetic is fixed), only the time does. Synchronous; allocates a
 * B-shot output buffer for the duration of the call and grows the workspace. A vibe_batch copies the
 * descriptor (engine) it sees at creation and has its own launch: tune it with vibe_batch_autotune.
 * The choices (engine, BP CTAs per SM, LSD CTAs per SM, LSD threads per CTA) are returned through the
 * pointers that are not NULL; vibe_get_launch reports the whole launch.
 *   Errors: VIBE_ERR_INVALID, VIBE_ERR_NOMEM, VIBE_ERR_CUDA.
 */
int vibe_autotune(vibe_handle* h, const uint32_t* d_syndromes, int64_t B, void* stream, int32_t* engine,
                  int32_t* bp_blocks_per_sm, int32_t* lsd_blocks_per_sm, int32_t* lsd_threads);

/* Launch configuration of a handle or a batch (vibe_get_launch). */
typedef struct {
  int32_t engines;           /* bit 0: the image engine's kernel runs, bit 1: the summary engine's */
  int32_t pair_mode;         /* 1: one warp per (shot, member) pair; 0: one warp per shot */
  int32_t bp_blocks_per_sm;  /* image-engine CTAs per SM of its persistent grid (0 if it does not run) */
  int32_t bpx_blocks_per_sm; /* summary-engine CTAs per SM (0 if it does not run) */
  int32_t lsd_blocks_per_sm; /* LSD CTAs per SM */
  int32_t lsd_threads;       /* threads per LSD CTA */
  int32_t num_sms;           /* the device's SM count (grids are CTAs per SM x this) */
} vibe_launch;

/*
 * vibe_get_launch -- the launch configuration of exactly one of h or b (the other NULL) into *out.
 *   Errors: VIBE_ERR_INVALID.
 */
int vibe_get_launch(const vibe_handle* h, const vibe_batch* b, vibe_launch* out);

/*
 * Mixed batches. The paper decodes one detector error model per run; a decoding service often holds
 * several (code distances, noise models, X and Z memory) and receives shots for all of them. A
 * vibe_batch groups up to 64 handles so that one pair of kernel launches decodes a batch whose shots
 * belong to different problems: every shot names its problem, and each shot's decoding is exactly
 * the decoding vibe_decode gives it with that problem's handle (same members, schedules, limits).
 *
 * vibe_batch_create -- handles[0..count) (1 <= count <= 64, non-NULL, created on the current
 *   device, all with the same msg_fp16) are referenced, not copied: they must outlive the batch and
 *   must not be destroyed first. The batch owns a device copy of their descriptors (each problem keeps
 *   its handle's BP engine) and its own launch and workspace; it starts in handles[0]'s shot or pair
 *   mode with occupancy-maximal grids. Errors: VIBE_ERR_INVALID (bad count/handles, mixed devices or message precisions,
 *   device not current), VIBE_ERR_UNSUPPORTED (the largest problem's state with the batch's
 *   descriptor table does not fit in shared memory), VIBE_ERR_NOMEM, VIBE_ERR_CUDA.
 */
int vibe_batch_create(vibe_handle* const* handles, int32_t count, vibe_batch** out);

/*
 * vibe_batch_decode -- decodes B shots of mixed problems, asynchronous on `stream`.
 *   d_problem: B int32 problem indices into the handles given to vibe_batch_create (device). Shot b's
 *   syndrome is d_syndromes[b * syn_stride ...], its first ceil(m_p/32) words meaningful (padding bits
 *   zero); syn_stride >= the largest ceil(m/32). d_corrections (corr_stride >= the largest
 *   ceil(n/32)) receives ceil(n_p/32) words per shot; words past them are left untouched.
 *   d_logical and d_observables (may be NULL) use log_stride >= the largest ceil(k/32) when given.
 *   d_stats and d_counters as for vibe_decode; no soft output. A shot whose index is outside
 *   0..count-1 is not decoded: its status is VIBE_STATUS_BAD_PROBLEM and its corr_stride correction
 *   words (and log_stride logical words) are zero. Calls on one batch must not overlap in time.
 *   Errors: VIBE_ERR_INVALID (NULL batch/required pointer, B < 0, strides too small), VIBE_ERR_NOMEM,
 *   VIBE_ERR_CUDA. B = 0 is a no-op.
 */
int vibe_batch_decode(vibe_batch* b, const int32_t* d_problem, const uint32_t* d_syndromes, int32_t syn_stride,
                      int64_t B, uint32_t* d_corrections, int32_t corr_stride, uint32_t* d_logical,
                      int32_t log_stride, vibe_shot_stats* d_stats, const uint32_t* d_observables,
                      uint64_t* d_counters, void* stream);

/*
 * vibe_batch_autotune -- vibe_autotune's launch search (shot or pair mode, the persistent grid of each
 * BP engine the batch runs, LSD CTA size and grid) for a batch, timed on a sample of mixed shots
 * (d_problem, d_syndromes, syn_stride as for vibe_batch_decode; B >= 1). Each problem keeps the engine
 * its handle had when the batch was created. Results do not depend on the choice. Synchronous;
 * allocates a B-shot output buffer for the duration of the call. Read the choice with vibe_get_launch.
 *   Errors: VIBE_ERR_INVALID (NULL pointers, B < 1, stride too small), VIBE_ERR_NOMEM, VIBE_ERR_CUDA.
 */
int vibe_batch_autotune(vibe_batch* b, const int32_t* d_problem, const uint32_t* d_syndromes, int32_t syn_stride,
                        int64_t B, void* stream);

/* vibe_batch_destroy -- frees the batch's device memory; the handles stay valid. NULL is accepted. */
int vibe_batch_destroy(vibe_batch* b);

/* vibe_destroy -- frees every device and host resource of the handle. NULL is accepted. */
int vibe_destroy(vibe_handle* h);

/* Message describing the calling thread's most recent error ("" if none). Owned by the library. */
const char* vibe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VIBE_H */
