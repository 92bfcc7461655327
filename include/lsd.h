/*
 * lsd.h -- C ABI of the GB300 (sm_103a) BP + localized statistics decoding library.
 *
 * The library decodes batches of syndromes of one binary check matrix H (m detectors x
 * n faults).  For each shot it runs min-sum belief propagation (BP) over the Tanner
 * graph of H and, when BP's hard decision does not satisfy the syndrome, the localized
 * statistics decoder (LSD) on BP's posterior log-likelihood ratios.  Everything after
 * lsd_create runs in the library's own CUDA kernels on the caller's stream; there is no
 * CPU fallback.
 *
 * The decoding problem (arXiv 2406.18655, Sec. 2.1): given s in F_2^m, find e_hat in
 * F_2^n with H e_hat = s, guided by soft information lambda in R^n in log-likelihood
 * ratio form (lower lambda = more likely faulty, Sec. 4.1).  LSD (Alg. 1, Sec. 4.1)
 * factorizes this into independent local problems on clusters grown in order of
 * reliability, validated and solved by on-the-fly GF(2) elimination (Sec. 4.2), and
 * returns the union of the local solutions (Eq. 2).  BP is the pre-decoder of Sec. 4.3:
 * min-sum, flooding ("parallel") schedule, scaling alpha = 0.625.  LSD-mu (App. D) adds
 * mu growth steps per cluster followed by local exhaustive OSD of order mu, or the
 * combination sweep OSD-CS-w.
 *
 * Beyond batches of one matrix: (w, c) overlapping-window decoding of repeated syndrome
 * rounds (Methods 4.3; lsd_window_*), batch or round by round; one giant shot decoded by
 * the whole GPU with the parallel LSD of App. B (lsd_giant_*); the learned prior
 * (lsd_prior_*) and the continuous-batching server (lsd_server_*), which have no
 * counterpart in the paper.
 *
 * Conventions used by every entry point
 *   - Return value: LSD_OK (0) or a negative LSD_ERR_* code.  lsd_status_string()
 *     names it.  On an error no output is guaranteed to be written.
 *   - "device" pointers are CUDA device (or managed) memory of the current device,
 *     "host" pointers are ordinary host memory.  The caller owns every pointer it
 *     passes; the library never frees or retains them after the call returns.
 *   - All device work of a call is enqueued on the decoder's stream (lsd_options.stream)
 *     and is complete only after that stream is synchronized, except where an entry
 *     point says it synchronizes.
 *   - One decoder must not be used from two host threads at the same time, and calls on
 *     one decoder must not overlap on the GPU (they share the decoder's workspace); the
 *     library enqueues them in order on one stream, which guarantees this.  Separate
 *     decoders are independent.
 *   - Layouts are row-major and shot-major in the sense "one contiguous row per shot":
 *     syndromes [shots][m] bytes, corrections [shots][n] bytes, LLRs [shots][n] float32.
 *     Bytes hold 0 or 1; any nonzero syndrome byte counts as 1.
 */
#ifndef LSD_GB300_H
#define LSD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define LSD_OK 0
#define LSD_ERR_INVALID_ARG (-1) /* bad size, pointer, index, duplicate entry or option */
#define LSD_ERR_CUDA (-2)        /* a CUDA runtime call or kernel launch failed */
#define LSD_ERR_OOM (-3)         /* device allocation failed */
#define LSD_ERR_ADMISSION (-4)   /* the work does not fit in lsd_options.mem_budget */
#define LSD_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define LSD_ERR_UNSUPPORTED (-6) /* matrix shape beyond this build's kernel limits */

/* ---- per-shot status bytes ---- */
#define LSD_SHOT_OK_BP 1      /* BP's hard decision satisfied the syndrome */
#define LSD_SHOT_OK_LSD 2     /* LSD produced the correction */
#define LSD_SHOT_UNSOLVABLE 3 /* s is not in image(H): some cluster exhausted its component */

typedef struct lsd_decoder lsd_decoder; /* opaque; owns device copies of H, priors, workspace */

/* Options.  A zero-initialised struct (or NULL) selects every default. */
typedef struct lsd_options {
  float ms_scaling;       /* min-sum scaling alpha of the check message; 0 -> 0.625 (Sec. 4.3) */
  int32_t bp_method;      /* 0 = min-sum (default); 1 = sum-product (tanh rule) */
  int32_t no_early_exit;  /* 0 = a shot stops BP once H e_hat = s (default); 1 = run all iterations */
  int32_t single_cluster; /* 1 = LSD seeds one cluster holding every detector; it then equals OSD-0 */
  int32_t bp_lanes;       /* threads cooperating on one shot in BP: 0 = auto, else 8, 16 or 32 */
  int32_t lsd_warps;      /* warps per CTA of the LSD kernel: 0 = auto, else 1..16 */
  int32_t bp_kernel;      /* BP kernel: 0 = auto (register tables when a shape fits and,
                             for the CTA-per-shot shapes, the graph has at least as many
                             checks as the shape has threads; else generic), 1 = generic
                             (graph in shared memory, or read through the cache by one CTA
                             per shot for large graphs), 2 = register-resident graph tables
                             (min-sum: a warp group per shot for small regular codes; a CTA
                             per shot for larger graphs whose rows all have 7 edges and
                             columns at most 4, as hypergraph products, or whose rows have
                             at most 8 or 17 edges and columns at most 3, as space-time
                             matrices with or without hook faults; shorter rows are
                             padded), 3 = latency: of the CTA-per-shot register shapes that
                             fit, the one with the most threads (at least one fault per
                             thread), for small batches such as the server's; else as 0 */
  int32_t lsd_kernel;     /* LSD kernel: 0 = auto, 1 = dense (state indexed by detector and
                             fault, m <= 512, n <= 2048), 2 = sparse (state sized by what a shot
                             touches; any m, n < 65536; no single_cluster) */
  int32_t osd_method;     /* local reprocessing of LSD-mu (lsd_order > 0, App. D): 0 = exhaustive
                             OSD-E over the first mu dependent columns of each cluster
                             (lsd_order <= 12; default); 1 = combination sweep OSD-CS-w: no
                             flip, every single dependent column, every pair among the first
                             w, in reliability order, the first least-cost pattern winning
                             (lsd_order <= 65535 extra growth steps) */
  int32_t osd_cs_order;   /* w of OSD-CS-w, 0..8; must be 0 unless osd_method == 1 */
  int32_t reserved;       /* must be zero */
  size_t mem_budget;      /* device bytes the decoder may hold (H, priors, workspace); 0 = no limit */
  void* stream;           /* cudaStream_t used for all work; NULL = the legacy default stream */
} lsd_options;

/* Batch summary, filled only when a non-NULL pointer is passed (the call then synchronizes). */
typedef struct lsd_stats {
  int64_t shots;         /* shots in the call */
  int64_t bp_converged;  /* shots whose BP hard decision satisfied s */
  int64_t lsd_shots;     /* shots handed to LSD */
  int64_t unsolvable;    /* shots with status LSD_SHOT_UNSOLVABLE */
  int64_t bp_iterations; /* BP iterations summed over shots */
  int64_t lsd_steps;     /* LSD growth steps summed over LSD shots */
  int32_t kappa_max;     /* largest final cluster (columns) of any shot (App. A's kappa) */
  int32_t nu_max;        /* most final clusters in one shot (App. A's nu) */
  float ms_bp;           /* device time of the BP kernel, CUDA events on the decoder stream */
  float ms_lsd;          /* device time of the LSD kernel(s) */
  int64_t lsd_spilled;   /* sparse LSD: shots handed to its large-capacity instance */
} lsd_stats;

/*
 * lsd_create -- build a decoder for H and the i.i.d. channel probabilities.
 *   out            receives the decoder (host pointer to a handle).
 *   m, n           H is m x n (detectors x faults); 1 <= m, 1 <= n.
 *   nnz, rows,cols host COO list of the ones of H, any order; an out-of-range index or a
 *                  repeated (row, col) pair is LSD_ERR_INVALID_ARG.
 *   channel_probs  host, n values in (0, 1): fault probabilities p_j.  The priors
 *                  lambda_j = ln((1-p_j)/p_j) (Sec. 4.1's LLR form) are computed on the
 *                  device in double and rounded to float32.
 *   bp_iters       maximum BP iterations, >= 0 (0 = LSD on the priors alone).
 *   lsd_order      mu of LSD-mu (App. D): extra growth steps per cluster before the local
 *                  reprocessing; 0 = LSD-0; at most 12 with OSD-E (opt->osd_method 0), 65535
 *                  with OSD-CS.
 *   opt            nullable; see lsd_options.
 * The decoder copies H and the priors to the device; the caller's arrays may be freed
 * after the call.  Synchronizes its stream before returning.
 */
int lsd_create(lsd_decoder** out, int32_t m, int32_t n, int64_t nnz, const int32_t* rows,
               const int32_t* cols, const float* channel_probs, int32_t bp_iters,
               int32_t lsd_order, const lsd_options* opt);

/*
 * lsd_decode_batch -- BP then LSD on `shots` syndromes (App. C.4: LSD runs only when BP
 * does not converge).  Asynchronous unless stats != NULL.
 *   syndromes    device, [shots][m] bytes.
 *   corrections  device, [shots][n] bytes, written for every shot; H e_hat = s for every
 *                shot whose status is 1 or 2.
 *   status       device, [shots] bytes (LSD_SHOT_*), nullable.
 *   posteriors   device, [shots][n] float32 BP posteriors of the last iteration run, nullable.
 *   stats        host, nullable; filled after the call's work completes.
 */
int lsd_decode_batch(lsd_decoder* dec, int64_t shots, const uint8_t* syndromes,
                     uint8_t* corrections, uint8_t* status, float* posteriors, lsd_stats* stats);

/*
 * lsd_decode_batch_host -- lsd_decode_batch with HOST buffers: copies the syndromes to
 * the decoder's device staging buffers, decodes, copies the corrections (and status)
 * back, and synchronizes.  Pinned host memory makes the copies asynchronous DMA.  A batch
 * of at least 2 x 65536 shots with stats == NULL runs as a pipeline of up to 4 chunks on
 * two internal copy streams (copies of one chunk overlap the decoding of its neighbours);
 * the results are the same as one call per batch.
 *   syndromes    host, [shots][m] bytes.   corrections host, [shots][n] bytes.
 *   status       host, [shots] bytes, nullable.   stats host, nullable.
 */
int lsd_decode_batch_host(lsd_decoder* dec, int64_t shots, const uint8_t* syndromes,
                          uint8_t* corrections, uint8_t* status, lsd_stats* stats);

/*
 * lsd_decode_batch_packed / lsd_decode_batch_host_packed -- lsd_decode_batch and
 * lsd_decode_batch_host with bit-packed syndromes and corrections (the problem statement's
 * s in F_2^m and e in F_2^n, Sec. 2.1, one bit each): element i of a row is bit (i & 31)
 * of 32-bit word i >> 5, rows of W_m = ceil(m/32) and W_n = ceil(n/32) words.
 *   syndromes    [shots][W_m] uint32 (device, or host for _host_packed); bits past m in
 *                the last word of a row are ignored.
 *   corrections  [shots][W_n] uint32; bits past n are written as zero.
 *   status, stats  as for lsd_decode_batch (status: device / host respectively).
 * The kernels read and write the packed rows themselves (no unpacking pass); results are
 * identical to the byte-per-bit calls.  No posteriors output.
 */
int lsd_decode_batch_packed(lsd_decoder* dec, int64_t shots, const uint32_t* syndromes,
                            uint32_t* corrections, uint8_t* status, lsd_stats* stats);
int lsd_decode_batch_host_packed(lsd_decoder* dec, int64_t shots, const uint32_t* syndromes,
                                 uint32_t* corrections, uint8_t* status, lsd_stats* stats);

/*
 * lsd_bp_batch -- BP only (the pre-decoder of Sec. 4.3), for inspection and tests.
 *   syndromes   device [shots][m] bytes.
 *   posteriors  device [shots][n] float32: Lambda of the last iteration run.
 *   converged   device [shots] bytes, nullable: 1 if the hard decision [Lambda < 0]
 *               satisfied s after that iteration.
 *   iterations  device [shots] int32, nullable: iterations run.
 */
int lsd_bp_batch(lsd_decoder* dec, int64_t shots, const uint8_t* syndromes, float* posteriors,
                 uint8_t* converged, int32_t* iterations);

/*
 * lsd_postprocess_batch -- LSD only (Alg. 1 plus LSD-mu when lsd_order > 0) on given soft
 * information, for every shot (no BP, no convergence test).
 *   llrs         device [shots][n] float32 soft information (lower = more likely faulty);
 *                ties are broken toward the lower column index.
 *   syndromes    device [shots][m] bytes.
 *   corrections  device [shots][n] bytes.
 *   status       device [shots] bytes, nullable (LSD_SHOT_OK_LSD or LSD_SHOT_UNSOLVABLE).
 *   shot_info    device [shots][3] int32, nullable: (nu, kappa, growth steps of LSD-0).
 */
int lsd_postprocess_batch(lsd_decoder* dec, int64_t shots, const float* llrs,
                          const uint8_t* syndromes, uint8_t* corrections, uint8_t* status,
                          int32_t* shot_info);

/*
 * lsd_get_stats -- counters and kernel event times of the decoder's most recent
 * lsd_decode_batch / lsd_bp_batch / lsd_postprocess_batch call (stats: host, required).
 * Synchronizes the decoder's stream.  Counts of a call are complete only once that call's
 * work has finished, which this synchronization guarantees.
 */
int lsd_get_stats(lsd_decoder* dec, lsd_stats* stats);

/*
 * lsd_decode_batch_static -- lsd_decode_batch for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant of the same BP + LSD
 * path, with identical results.
 *
 * Who needs it: code that must not call cudaMalloc at decode time -- for example a
 * real-time decoding loop that runs with a fixed device-memory footprint reserved at
 * start-up (cudaMalloc can block on an implicit device synchronization and its latency is
 * unbounded), or a host process whose free device memory is already held by another
 * allocator (a framework's caching allocator), where a further cudaMalloc fails or
 * fragments.  lsd_decode_batch may grow the decoder's workspace with cudaMalloc when a
 * batch is larger than any before; this entry point never allocates or frees anything.
 *
 * Its scratch (the work-queue counters, the queue of unconverged shots and their LLR rows)
 * lives in one file-scope device array of LSD_STATIC_SCRATCH_BYTES bytes inside the
 * library, which every GPU that loads the library holds until the process exits.
 *   dec          a decoder from lsd_create (H and the priors are already on the device).
 *   shots        0 <= shots, and 256 + shots * 4 (rounded up to 256) + shots * n * 4 must
 *                not exceed LSD_STATIC_SCRATCH_BYTES (BB[[144,12,12]]: up to 14,462 shots
 *                per call); a larger batch returns LSD_ERR_ADMISSION and touches nothing.
 *   syndromes    device [shots][m] bytes.  corrections device [shots][n] bytes.
 *   status       device [shots] bytes, nullable.
 * Behaviour:
 *   - Decoders whose LSD runs in the sparse kernel (more than 512 detectors or 2048 faults:
 *     the large HGP and space-time matrices) are refused with LSD_ERR_UNSUPPORTED, since
 *     that kernel's per-warp scratch is not part of the array; so is a decoder without LSD.
 *   - The first call on a device looks up the array's device address on that device (the
 *     current one); make that first call before any stream capture.  Later calls reuse it.
 *     A lookup that fails returns LSD_ERR_CUDA and is retried by the next call.
 *   - Every call, on every decoder, shares the one array; each call clears the counters it
 *     needs at its start.  Calls that overlap on the GPU (different streams, decoders or
 *     threads without ordering between them) race on the array and give wrong results:
 *     order them on one stream or synchronize between them.
 *   - Asynchronous on the decoder's stream, like lsd_decode_batch.
 *   - It keeps no statistics: lsd_get_stats goes on reporting the decoder's last
 *     lsd_decode_batch (or similar) call, not this one.
 */
#define LSD_STATIC_SCRATCH_BYTES ((size_t)8 << 20)
int lsd_decode_batch_static(lsd_decoder* dec, int64_t shots, const uint8_t* syndromes,
                            uint8_t* corrections, uint8_t* status);

/* ------------------------------------------------------------------------------------
 * Learned prior (no counterpart in the paper: an extension that replaces most BP iterations
 * by a small trained network whose per-fault LLRs feed LSD).
 *
 * Model, hidden width LSD_PRIOR_HIDDEN = 32, R rounds, for the decoder's H:
 *   sigma_c = 1 - 2 s_c,  h_v = relu(lambda_v a0 + a1),  h_c = sigma_c u0 + u1
 *   each round:  h_v += sum_{c in N(v)} MLP_cv([h_c, h_v, sigma_c])
 *                h_c += sum_{v in N(c)} MLP_vc([h_v, h_c, sigma_c])
 *   LLR_v = lambda_v + w_o . h_v + b_o,   MLP(x) = W2 relu(W1 x + b1) + b2,
 *   W1: 32 x 65, W2: 32 x 32 (row-major), the two MLPs shared by all rounds.
 * Loss: mean over shots and faults of softplus(LLR_v) - (1 - e_v) LLR_v (binary
 * cross-entropy of P(e_v = 1) = sigmoid(-LLR_v)).
 * Parameters: FP32 master copy, flat in the order a0, a1, u0, u1, W1_cv, b1_cv, W2_cv,
 * b2_cv, W1_vc, b1_vc, W2_vc, b2_vc, w_o, b_o (lsd_prior_num_params() floats).  The
 * matrix products run on the tensor cores with BF16 weights and activations and FP32
 * accumulation; node states and the loss are FP32.  Inference runs on the tcgen05 tensor
 * cores with the per-node projections held in tensor memory when H has at most 8 tiles of
 * 128 node rows (ceil(n/128) + ceil(m/128) <= 8, e.g. BB [[144,12,12]]: 3), else on the
 * per-node mma.sync kernel, whose states of one shot live in one CTA's shared memory (about
 * 384 (n + m) + 64 max(n, m) + 16 KB bytes; BB [[288,12,18]], 201 KB, fits).  Training runs
 * on the mma.sync kernels and takes more (up to m = 96, n = 192); lsd_prior_gradient /
 * lsd_prior_train_step return LSD_ERR_UNSUPPORTED beyond that.
 * ------------------------------------------------------------------------------------ */
#define LSD_PRIOR_HIDDEN 32
typedef struct lsd_prior lsd_prior;

/* Number of FP32 parameters of the model (6497). */
int lsd_prior_num_params(void);

/*
 * lsd_prior_create -- a prior for decoder `dec` (which must outlive it) with `rounds`
 * message-passing rounds (1..8).  params: host, lsd_prior_num_params() floats, or NULL for
 * all zeros.  Uses the decoder's stream; synchronizes.
 */
int lsd_prior_create(lsd_prior** out, lsd_decoder* dec, int32_t rounds, const float* params);

/* Copy the FP32 parameters from / to host memory (synchronizes).  Setting resets Adam. */
int lsd_prior_set_params(lsd_prior* prior, const float* params);
int lsd_prior_get_params(lsd_prior* prior, float* params);

/* lsd_prior_forward -- LLRs of every shot: syndromes device [shots][m] bytes, llrs device
 * [shots][n] float32.  Asynchronous on the mma.sync kernel; on the tensor-memory kernel it
 * synchronizes and returns LSD_ERR_TIMEOUT if a completion wait inside the kernel ran out
 * (after one second; the LLRs are then unspecified). */
int lsd_prior_forward(lsd_prior* prior, int64_t shots, const uint8_t* syndromes, float* llrs);

/* lsd_prior_set_kernel -- the inference kernel: 0 = automatic (the tensor-memory kernel
 * when H fits it), 1 = the per-node mma.sync kernel, 2 = the tensor-memory kernel
 * (LSD_ERR_UNSUPPORTED when H does not fit it).  Both compute the same model; their
 * results differ only in rounding. */
int lsd_prior_set_kernel(lsd_prior* prior, int32_t kernel);

/* lsd_prior_get_kernel -- the inference kernel in use (1 = mma.sync, 2 = tensor-memory) and
 * the number of CTAs of its persistent grid.  No GPU call. */
int lsd_prior_get_kernel(const lsd_prior* prior, int32_t* kernel, int32_t* grid);

/*
 * lsd_prior_gradient -- loss and gradient over a batch without updating the parameters.
 *   syndromes, errors: device [shots][m] / [shots][n] bytes (errors are the targets).
 *   loss: host, the batch's mean loss.  grads: host, lsd_prior_num_params() floats, nullable.
 * Synchronizes.
 */
int lsd_prior_gradient(lsd_prior* prior, int64_t shots, const uint8_t* syndromes,
                       const uint8_t* errors, double* loss, float* grads);

/* lsd_prior_train_step -- gradient of the batch, then one Adam step (beta 0.9, 0.999,
 * eps 1e-8) with learning rate lr.  loss: host, nullable (if given, synchronizes). */
int lsd_prior_train_step(lsd_prior* prior, int64_t shots, const uint8_t* syndromes,
                         const uint8_t* errors, float lr, double* loss);

/*
 * lsd_decode_learned -- decode with the prior in place of BP: LLRs from the prior; if their
 * hard decision satisfies s the shot is done (status 1), otherwise LSD runs on them
 * (status 2).  Shots LSD cannot solve (status 3) are decoded again by the decoder's own
 * BP + LSD, the fallback.  Arguments as lsd_decode_batch, except that `status` is required
 * (the fallback reads it).  Synchronizes (the fallback needs the count of unsolved shots);
 * stats->bp_converged counts the shots the prior's hard decision solved.  LSD_ERR_TIMEOUT:
 * a completion wait of the tensor-memory kernel ran out (after one second).
 */
int lsd_decode_learned(lsd_decoder* dec, lsd_prior* prior, int64_t shots,
                       const uint8_t* syndromes, uint8_t* corrections, uint8_t* status,
                       lsd_stats* stats);

int lsd_prior_destroy(lsd_prior* prior);

/*
 * lsd_sample -- seeded i.i.d. training pairs on the device: fault j of shot k is 1 with the
 * decoder's channel probability p_j, drawn from the xoshiro256** stream of shot first+k
 * (state from splitmix64 applied to seed ^ (first+k+1) * 0xD1B54A32D192ED03, Blackman and
 * Vigna), u = (x >> 11) 2^-53 < p_j in double, columns in ascending order; syndromes = H e.
 *   errors device [shots][n] bytes, syndromes device [shots][m] bytes.  Asynchronous.
 */
int lsd_sample(lsd_decoder* dec, uint64_t seed, int64_t first_shot, int64_t shots,
               uint8_t* errors, uint8_t* syndromes);

/* ------------------------------------------------------------------------------------
 * Overlapping-window decoding of repeated syndrome rounds (Methods 4.3: a (w, c) = (3, 1)
 * window, w rounds decoded, the c oldest committed).  Phenomenological noise on a code H
 * (m x n): d noisy syndrome rounds and one noiseless round.  Detector block t (t = 0..d,
 * m bytes each) is the difference of syndrome rounds t and t-1; the faults of round t
 * (t = 0..d-1, n + m bytes each) are the n data faults (flipping block t through H) and
 * then the m measurement faults (flipping blocks t and t+1).  A shot's syndrome is its
 * (d+1) m detector bytes, block by block; its correction d (n+m) fault bytes, round by round.
 *
 * Windows start at t = 0, c, 2c, ...  A window with t + w - 1 < d holds blocks t..t+w-1 and
 * fault rounds t..t+w-1 (the measurement faults of its last round flip only its last block
 * inside it), is decoded by BP + LSD, and commits its first c rounds: they are written to
 * the correction, and the measurement faults of its round c-1 flip the first block of the
 * next window.  The first window with t + w - 1 >= d (it reaches block d) or t + c >= d (it
 * would commit the last round; only possible when c = w) is the final one: blocks t..d,
 * rounds t..d-1, all committed.  Every window is decoded exactly as lsd_decode_batch decodes
 * its matrix with the channel probabilities of its columns.
 * ------------------------------------------------------------------------------------ */
typedef struct lsd_window lsd_window;

/*
 * lsd_window_create -- a window decoder.
 *   out            receives the handle.
 *   m, n, nnz, rows, cols   H as for lsd_create (host COO).
 *   p_data         host, n probabilities in (0, 1) of the data faults of every round.
 *   q_meas         host, m probabilities in (0, 1) of the measurement faults.
 *   rounds         d >= 1 noisy rounds.
 *   window, commit w >= 1 and 1 <= c <= w.
 *   bp_iters, lsd_order, opt   as for lsd_create, applied to the decoder of every window
 *                  (opt->stream is the stream of all the work).
 * Builds two decoders: the inner window's matrix (w m x w (n+m)) and the final window's
 * ((d - t_f + 1) m x (d - t_f) (n+m), t_f its first round); only the final one when w > d.
 * Errors as lsd_create.
 */
int lsd_window_create(lsd_window** out, int32_t m, int32_t n, int64_t nnz, const int32_t* rows,
                      const int32_t* cols, const float* p_data, const float* q_meas,
                      int32_t rounds, int32_t window, int32_t commit, int32_t bp_iters,
                      int32_t lsd_order, const lsd_options* opt);

/*
 * lsd_window_decode -- decode `shots` shots window by window.  Asynchronous unless
 * stats != NULL.
 *   syndromes    device [shots][(d+1) m] bytes (read only).
 *   corrections  device [shots][d (n+m)] bytes, every byte written.
 *   status       device [shots] bytes, nullable: the largest per-shot status of any window
 *                (LSD_SHOT_UNSOLVABLE if some window's syndrome was outside its image).
 *   stats        nullable: the sums over windows of every window decode's lsd_stats
 *                (shots counts window decodes; kappa_max, nu_max are maxima); synchronizes.
 * Workspace (window syndromes, corrections and status: about shots (w m + w (n+m) + 1)
 * bytes, one more block per shot when c = w) is
 * allocated on first use and kept; the work of one call runs on the decoder's stream, so
 * calls on the same stream are ordered.
 */
int lsd_window_decode(lsd_window* win, int64_t shots, const uint8_t* syndromes,
                      uint8_t* corrections, uint8_t* status, lsd_stats* stats);

/*
 * Streaming: the same windows, decoded as the rounds arrive.  `shots` concurrent streams
 * (for example one per logical block) deliver detector block t = 0, 1, ..., d one push at a
 * time; a push that completes a window (its last block, or block d for the final window)
 * decodes it for every stream and commits its first c rounds (all remaining rounds for the
 * final window).  The committed corrections equal lsd_window_decode's on the same blocks.
 *
 * lsd_window_stream_reset -- start (or restart) `shots` >= 1 streams; allocates the
 *   syndrome history (shots (d+1) m bytes) and the window workspace on first use.
 * lsd_window_stream_push -- the next detector block of every stream.
 *   block        device [shots][m] bytes (read before the call's work completes on the stream).
 *   corrections  device [shots][d (n+m)] bytes, the same buffer for every push of a stream:
 *                a push that commits rounds [first, first + count) writes exactly those.
 *   status       device [shots] bytes, nullable, the same buffer for every push: largest
 *                window status so far (valid once a window has been committed).
 *   first_round, rounds_committed   host, nullable: the committed range (count 0 when the
 *                push completed no window).
 *   Asynchronous on the decoder's stream.  More than d + 1 pushes, or a push before a reset,
 *   is LSD_ERR_INVALID_ARG.  The stream keeps the last window's corrections in the decoder's
 *   workspace: a lsd_window_decode call between two pushes of a stream breaks it (reset it).
 */
int lsd_window_stream_reset(lsd_window* win, int64_t shots);
int lsd_window_stream_push(lsd_window* win, const uint8_t* block, uint8_t* corrections,
                           uint8_t* status, int32_t* first_round, int32_t* rounds_committed);

/* lsd_window_kernel_launches -- kernels launched so far by the window decoder and the
 * decoders of its windows. */
int lsd_window_kernel_launches(const lsd_window* win, int64_t* count);

/* lsd_window_destroy -- free the window decoder; NULL is a no-op.  Synchronizes. */
int lsd_window_destroy(lsd_window* win);

/* ------------------------------------------------------------------------------------
 * One giant shot on the whole GPU (App. B's P-LSD, Alg. 2): a single syndrome of a large
 * code (any m, n below 2^31 and fewer than 2^31 edges; the batch decoder stops at 65535)
 * decoded by BP with one thread per check and per variable, then, if BP does not converge,
 * by LSD with every cluster grown in parallel: clusters take their best candidate at once,
 * merge through a lock-free union-find, and keep their own on-the-fly elimination in
 * blocks of a device arena; with lsd_order = mu > 0, mu more growth steps for every cluster
 * and the local OSD-E or OSD-CS reprocessing of LSD-mu follow.  Corrections and status equal
 * lsd_decode_batch's on the same shot.  Limits: a cluster spans at most 8192 detectors (LSD_ERR_UNSUPPORTED beyond);
 * the arena holds every block a call allocates (LSD_ERR_ADMISSION when it runs out).
 * ------------------------------------------------------------------------------------ */
typedef struct lsd_giant lsd_giant;

typedef struct lsd_giant_info {
  int32_t status;          /* LSD_SHOT_* */
  int32_t bp_iterations;   /* BP iterations run (lsd_giant_decode) */
  int32_t nu, kappa;       /* final clusters; largest cluster in columns (App. A) */
  int32_t steps;           /* LSD-0 growth steps */
  int32_t reserved;
  int64_t arena_bytes_used;
  float ms_bp, ms_lsd;     /* device time of the BP and LSD phases (CUDA events) */
} lsd_giant_info;

/*
 * lsd_giant_create -- decoder of one large check matrix.
 *   m, n, nnz, rows, cols, channel_probs, bp_iters, lsd_order   as lsd_create (host COO, no
 *                  duplicates; lsd_order = mu of LSD-mu, App. D).
 *   arena_bytes    device bytes of the cluster arena; 0 = 256 MiB.
 *   opt            nullable; ms_scaling, osd_method, osd_cs_order and stream are used, the
 *                  other fields ignored.
 * Device memory: about 100 m + 40 n + 20 E bytes plus the arena (640 000 faults, 307 200
 * detectors, 2.15 M edges: 100 MB + 256 MiB).  Synchronizes.
 */
int lsd_giant_create(lsd_giant** out, int32_t m, int32_t n, int64_t nnz, const int32_t* rows,
                     const int32_t* cols, const float* channel_probs, int32_t bp_iters,
                     int32_t lsd_order, size_t arena_bytes, const lsd_options* opt);

/*
 * lsd_giant_decode -- BP (min-sum, flooding, early exit on H e_hat = s, Sec. 4.3), then
 * P-LSD on the posteriors when BP does not converge.  Synchronous (one host round trip per
 * growth step).  BP runs as one cooperative launch whose blocks meet at grid barriers; a
 * barrier that waits past its bound (about a second) makes the call return
 * LSD_ERR_TIMEOUT.
 *   syndrome     device [m] bytes.   correction  device [n] bytes (written).
 *   posteriors   device [n] float32, nullable: the BP posteriors.
 *   info         host, nullable.
 */
int lsd_giant_decode(lsd_giant* dec, const uint8_t* syndrome, uint8_t* correction,
                     float* posteriors, lsd_giant_info* info);

/* lsd_giant_postprocess -- P-LSD alone on given soft information llr (device [n] float32),
 * as lsd_postprocess_batch for one shot.  Synchronous. */
int lsd_giant_postprocess(lsd_giant* dec, const float* llr, const uint8_t* syndrome,
                          uint8_t* correction, lsd_giant_info* info);

/* lsd_giant_test_hold_barrier -- test facility for the timeout path (no counterpart in the
 * paper): with hold != 0, block 0 of every following BP launch withholds its arrival at the
 * first grid barrier, so the other blocks' bounded waits run out after limit_ns and the
 * decode returns LSD_ERR_TIMEOUT with the device still usable; hold = 0 restores normal
 * operation and the one-second bound.  LSD_ERR_UNSUPPORTED when the device cannot run the
 * cooperative launch. */
int lsd_giant_test_hold_barrier(lsd_giant* dec, int32_t hold, int64_t limit_ns);

/* lsd_giant_kernel_launches -- kernels launched so far by the giant-shot decoder. */
int lsd_giant_kernel_launches(const lsd_giant* dec, int64_t* count);

/* lsd_giant_destroy -- free the decoder; NULL is a no-op.  Synchronizes. */
int lsd_giant_destroy(lsd_giant* dec);

/* ------------------------------------------------------------------------------------
 * Serving (no counterpart in the paper): continuous batching of single-shot requests over
 * several codes, and of streams of syndrome rounds decoded in overlapping windows (Methods
 * 4.3).  A scheduler thread keeps `slots_per_code` batches of each code (each window
 * matrix of a window code) in flight, each slot a decoder with its own stream; a batch
 * launches as soon as a slot is idle (or, with max_wait_us > 0, once max_batch requests
 * wait or the oldest has waited max_wait_us), and only as many shots as the memory budget
 * still admits.  A request completes as soon as its own result is written back: the shots
 * (window jobs) that BP solves right after BP, the others after their batch's LSD.  Request buffers are read and written by the GPU directly: they must be
 * page-locked host memory (cudaHostAlloc / cudaHostRegister) or device memory, owned by the
 * caller and valid until the request completes.
 * ------------------------------------------------------------------------------------ */
typedef struct lsd_server lsd_server;

typedef struct lsd_server_code {    /* one code served: the arguments of lsd_create */
  int32_t m, n;
  int64_t nnz;
  const int32_t* rows;
  const int32_t* cols;
  const float* channel_probs;
  int32_t bp_iters, lsd_order;
} lsd_server_code;

typedef struct lsd_server_options { /* zero = defaults */
  int32_t slots_per_code;   /* batches of one code in flight (default 3, at most 16) */
  int32_t max_batch;        /* shots per batch (default 8192) */
  int32_t max_wait_us;      /* 0: an idle slot launches whatever is pending at once; > 0: a partial
                               batch waits for max_batch requests or for its oldest to reach this age */
  int32_t use_graphs;       /* 0: each slot's batch pipeline is captured once as two CUDA graphs
                               (gather, BP, write-back of the rows BP solved; LSD, write-back
                               of the rest) and replayed per batch; -1: plain launches */
  size_t mem_budget;        /* device bytes of in-flight shots (m + 2n + 2 + 4(n+1) each); 0 = no limit */
} lsd_server_options;

typedef struct lsd_server_report {
  int64_t submitted, completed, batches, admission_waits, peak_inflight_bytes, generated;
  double mean_batch;        /* shots per launched batch */
  double seconds;           /* first arrival to last completion */
  double shots_per_s;       /* completed / seconds */
  double p50_us, p99_us, mean_us, max_us;  /* arrival-to-completion latency */
  double offered_rate;      /* lsd_server_run_poisson: the requested arrival rate (shots/s) */
  /* p99 of the latency's parts: arrival to submission (the load generator's lag behind its
   * schedule), submission to batch launch (queueing), launch to completion (service) */
  double p99_lag_us, p99_queue_us, p99_service_us;
  double p99_batch_gpu_us;  /* lsd_server_get_code_report: p99 of a batch's GPU time */
  double p99_launch_call_us;  /* ... and of the host time of a batch's launch calls */
} lsd_server_report;

/* Creates the server and its decoders (each slot's workspace sized for max_batch). */
int lsd_server_create(lsd_server** out, int32_t n_codes, const lsd_server_code* codes,
                      const lsd_server_options* opt);

/*
 * Window codes: streams of repeated syndrome rounds of a code H (m x n) under
 * phenomenological noise, d noisy rounds plus a noiseless one per sequence, decoded in
 * (w, c) overlapping windows exactly as lsd_window_decode decodes them (Methods 4.3: the
 * windows, their matrices and the commit rule are those of lsd_window_create).
 */
typedef struct lsd_server_window_code {
  int32_t m, n;
  int64_t nnz;
  const int32_t* rows;      /* host COO of H (one round), as for lsd_create */
  const int32_t* cols;
  const float* p_data;      /* host, n data-fault probabilities */
  const float* q_meas;      /* host, m measurement-fault probabilities */
  int32_t rounds;           /* d >= 1: noisy rounds per sequence (d + 1 detector blocks) */
  int32_t window, commit;   /* w >= 1, 1 <= c <= w */
  int32_t bp_iters, lsd_order;
  int32_t streams;          /* concurrent streams, 1 .. 2^24 */
} lsd_server_window_code;

/*
 * lsd_server_create_with_windows -- a server of n_codes shot codes (user code ids
 * 0 .. n_codes-1, lsd_server_submit) and n_window_codes window codes (ids n_codes ..
 * n_codes + n_window_codes - 1, lsd_server_submit_round); n_codes + n_window_codes >= 1.
 * Each window code holds two windows' decoders per slot (the inner window's matrix,
 * w m x w (n+m), and the final window's), a pinned host history of 2 (d+1) m bytes per
 * stream and m device bytes per stream (the measurement faults of its last committed round).
 */
int lsd_server_create_with_windows(lsd_server** out, int32_t n_codes, const lsd_server_code* codes,
                                   int32_t n_window_codes, const lsd_server_window_code* wcodes,
                                   const lsd_server_options* opt);

/* Submits one shot: syndrome [m] bytes, correction [n] bytes and status [1] byte (both
 * nullable) in GPU-accessible memory (see above).  Thread-safe; returns at once. */
int lsd_server_submit(lsd_server* s, int32_t code, const uint8_t* syndrome, uint8_t* correction,
                      uint8_t* status, int64_t* id);

/*
 * lsd_server_submit_round -- the next detector block of stream `stream` of window code
 * `code`: [m] bytes of host memory (any; copied before the call returns).  Blocks 0 .. d
 * of a stream form one sequence; after block d the stream's next block starts a new one.
 * The block that completes a window (block t + w - 1 of the window starting at round t, or
 * block d for the final window) makes it a request: once decoded, the corrections of the
 * rounds the window commits -- `*rounds` rounds from `*first_round` on, [rounds][n + m]
 * bytes, data faults then measurement faults per round -- go to `correction` and the
 * window's LSD_SHOT_* status to `status` (both nullable, GPU-accessible as above).  A block
 * that completes no window sets *first_round = -1, *rounds = 0 and leaves both untouched.
 * Windows of one stream are decoded one at a time, in order; different streams batch
 * together and with shot requests.  Returns LSD_ERR_ADMISSION (nothing stored) when block
 * 0 of a sequence arrives while a window of the sequence two before it is still pending.
 * Thread-safe; calls for one stream must come from one thread at a time, in round order.
 */
int lsd_server_submit_round(lsd_server* s, int32_t code, int32_t stream, const uint8_t* block,
                            uint8_t* correction, uint8_t* status, int32_t* first_round,
                            int32_t* rounds, int64_t* id);

/* Blocks until every submitted request has completed. */
int lsd_server_wait_all(lsd_server* s);

/* Throughput, batching and latency since the last reset (reset != 0 clears them).  For
 * window codes a request is one window job (latency from its completing block's submission). */
int lsd_server_get_report(lsd_server* s, lsd_server_report* report, int32_t reset);

/* The same figures for one user code since the last reset (submitted, completed,
 * shots_per_s over the server's whole reporting interval, latency percentiles). */
int lsd_server_get_code_report(lsd_server* s, int32_t code, lsd_server_report* report);

/*
 * lsd_server_run_poisson -- load test: requests arrive as a Poisson process of `rate`
 * shots/s for `seconds`; each picks code c with probability mix[c] / sum(mix) (one entry per
 * user code, window codes included) and the next syndrome of pools[c] ([pool_sizes[c]][m_c]
 * bytes, GPU-accessible, cycled); outputs are discarded.  For a window code an arrival is
 * one detector block of the code's streams in turn, stream s playing the sequences s,
 * s + S, s + 2S, ... of pools[c] ([pool_sizes[c]][(d+1) m] bytes, host memory) and
 * continuing from where the stream stands in the server (successive calls extend the same
 * sequences); blocks
 * refused for a busy history are dropped and counted in admission_waits.  Waits for
 * completion and fills `report` (latency from the scheduled arrival); the per-code reports
 * of the run stay readable until the next reset.
 */
int lsd_server_run_poisson(lsd_server* s, double rate, double seconds, const double* mix,
                           const uint8_t* const* pools, const int64_t* pool_sizes, uint64_t seed,
                           lsd_server_report* report);

/* Stops the scheduler after the outstanding requests and frees everything. */
int lsd_server_destroy(lsd_server* s);

/*
 * lsd_autotune -- time the decoder's launch variants on a sample batch and keep the fastest:
 * every BP kernel variant compatible with H and the BP method (register-resident shapes,
 * generic 8/16/32-lane groups, one CTA per shot), then the LSD kernel's warps per CTA
 * (2, 4, 8, 16 for the dense kernel).  Results of the decoder do not depend on the choice.
 *   syndromes   device [shots][m] bytes, a representative sample (e.g. 10^5 shots).
 *   report      host, nullable: the chosen variants and their times.
 * Allocates temporary device buffers and synchronizes.
 */
typedef struct lsd_tune_report {
  int32_t bp_variant, bp_candidates;   /* chosen BP variant id and how many were timed */
  int32_t lsd_warps, lsd_candidates;
  float ms_bp_best, ms_bp_first;       /* best BP time and the time of the default choice */
  float ms_lsd_best, ms_lsd_first;
} lsd_tune_report;
int lsd_autotune(lsd_decoder* dec, int64_t shots, const uint8_t* syndromes,
                 lsd_tune_report* report);

/* lsd_bp_variant_name -- the BP kernel and template shape behind a variant id of
 * lsd_tune_report.bp_variant, e.g. "bp_reg_kernel<32,3,6,5,3>" (as it appears in profiler
 * launch lists).  Static storage owned by the library; "" for an unknown id.  No GPU call. */
const char* lsd_bp_variant_name(int32_t variant);

/* lsd_get_priors -- copy the n float32 priors lambda_j to host memory; synchronizes. */
int lsd_get_priors(lsd_decoder* dec, float* priors);

/* lsd_workspace_bytes -- device bytes the decoder currently holds (H, priors, workspace). */
int lsd_workspace_bytes(const lsd_decoder* dec, size_t* bytes);

/* lsd_kernel_launches -- number of kernels the decoder has launched so far. */
int lsd_kernel_launches(const lsd_decoder* dec, int64_t* count);

/* lsd_destroy -- free the decoder and its device memory; NULL is a no-op.  Synchronizes. */
int lsd_destroy(lsd_decoder* dec);

/* lsd_status_string -- static description of a return code or per-shot status. */
const char* lsd_status_string(int code);

/* lsd_last_error -- the CUDA error name and message behind the last LSD_ERR_CUDA or
 * LSD_ERR_OOM returned on the calling host thread ("" if none).  The string belongs to the
 * library and stays valid until the thread's next failing call. */
const char* lsd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LSD_GB300_H */
