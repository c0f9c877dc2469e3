/*
 * gakco.h -- C ABI of the GB300-native gapped k-mer string kernel engine.
 *
 * The engine computes the gapped k-mer string kernel of GaKCo (Singh et al.,
 * "GaKCo: a Fast Gapped k-mer string Kernel using Counting",
 * arXiv 1704.07468):
 *
 *   Input (Table 1, Alg. 1 "Require L, g, k"): a dataset D = {x_1 .. x_N} of
 *   strings over an alphabet of sigma symbols and the user parameters g (the
 *   g-mer length) and k (the non-gapped length), 1 <= k <= g; M = g - k.
 *
 *   Mismatch profile (Definition 1, Eq. 7): N_m(x, y) = number of pairs
 *   (i, j), i a window of x and j a window of y, whose g-mers differ in
 *   exactly m positions.  A sequence of length l has max(0, l - g + 1)
 *   windows (Eq. 5).  All ordered pairs count, including i == j for x == y.
 *
 *   Kernel (Eq. 6, Eq. 7; Alg. 1 "Ensure K"): K(x, y) = sum_{m=0}^{M}
 *   h_m N_m(x, y) with h_m = C(g - m, k).
 *
 *   Normalised kernel (not in the paper; part of this interface):
 *   Khat(x, y) = K(x, y) / sqrt(K(x, x) K(y, y)), 0 where K(x, x) or
 *   K(y, y) is 0, and exactly 1.0 on a nonzero diagonal.  Computed in fp64;
 *   relative error below 1e-15.
 *
 * The engine follows the paper's counting route (Section 2.2, Alg. 1): for
 * every level m and every one of the C(g, m) position masks it deletes the
 * masked positions from every g-mer, sorts the (g-m)-mers, counts equal
 * runs, accumulates the cumulative mismatch profile C_m (Eq. 8) and
 * recovers N_m by inclusion-exclusion (Eq. 9).  Integer outputs are exact.
 *
 * Conventions
 *   - Symbols are bytes with values in [0, sigma).  A byte >= sigma makes the
 *     call fail with GAKCO_E_INVALID (mapping unknown characters to an extra
 *     symbol, as Section S:5.2 describes, is the caller's job).
 *   - A dataset is `codes` (all sequences concatenated) plus `offsets`
 *     (int64, n + 1 entries, offsets[0] = 0, non-decreasing; sequence x is
 *     codes[offsets[x] .. offsets[x+1])).  `offsets` is always a HOST
 *     pointer, also in the *_device calls: the host plans the work from it.
 *   - Output matrices are row-major: K[x * n + y]; N_m at Nm[(m * n + x) * n
 *     + y] for m = 0..M.
 *   - Every output pointer except the kernel K may be NULL to skip it.  In
 *     the host-buffer calls K may also be NULL.
 *   - The caller owns every buffer.  The library copies what it needs and
 *     keeps no pointer to caller memory after a call returns (the *_device
 *     calls read and write the caller's device buffers on the given stream).
 *   - Limits: n <= 65535 sequences per dataset; the number of windows of a
 *     dataset below 2^32; g * ceil(log2 sigma) <= 64; M + 1 <= 16; and
 *     max_m C(g, m) * W_max^2 < 2^31 (W_max = most windows of any sequence),
 *     which keeps every C_m and K inside int32.  A call beyond a limit
 *     returns GAKCO_E_OVERFLOW or GAKCO_E_INVALID without touching outputs.
 *   - Errors: every call returns GAKCO_OK (0) or a negative code; the
 *     context's message is available from gakco_last_error.  After an error
 *     the context remains usable.
 *   - Threads: a context is used by one host thread at a time, except that
 *     gakco_submit / gakco_poll may be called concurrently (see below).
 */
#ifndef GAKCO_H
#define GAKCO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GAKCO_OK 0
#define GAKCO_E_INVALID (-1)   /* bad argument or input symbol */
#define GAKCO_E_OOM (-2)       /* device or host allocation failed */
#define GAKCO_E_OVERFLOW (-3)  /* the int32 bound above is exceeded */
#define GAKCO_E_CUDA (-4)      /* a CUDA call failed */
#define GAKCO_E_TIMEOUT (-5)   /* a bounded wait ran out */
#define GAKCO_E_PENDING (-6)   /* asynchronous work not finished yet */
#define GAKCO_E_INTERNAL (-7)  /* an internal consistency check failed */

typedef struct gakco_ctx gakco_ctx;

/*
 * Create a context for alphabet size `sigma` (2..255) and parameters g, k
 * (1 <= k <= g, Table 1).  Selects the current CUDA device.  On success
 * *out receives the context (owned by the caller, freed by gakco_destroy).
 * Returns GAKCO_E_INVALID for parameters outside the limits above,
 * GAKCO_E_CUDA when no usable device is present.
 */
int gakco_create(int sigma, int g, int k, gakco_ctx **out);

/* Free a context and all device memory it holds.  NULL is ignored. */
void gakco_destroy(gakco_ctx *ctx);

/* Message describing the last error on this context ("" if none).  The
 * string is owned by the context and valid until its next call. */
const char *gakco_last_error(const gakco_ctx *ctx);

/*
 * Tuning and engine options (key, value).  Unknown keys return
 * GAKCO_E_INVALID.
 */
#define GAKCO_OPT_ENGINE 1          /* 0 = batched (default), 1 = plain per-mask */
#define GAKCO_OPT_RADIX_BITS 2      /* widest sort digit, 4..11 (default 8) */
#define GAKCO_OPT_CHUNK_ELEMS 3     /* sort elements per batched chunk (>= 4096) */
#define GAKCO_OPT_GRAPH 4           /* 1 = replay batched work from a CUDA graph */
#define GAKCO_OPT_ACCUM_THREADS 5   /* 256, 512 or 1024 */
#define GAKCO_OPT_PROFILE 6         /* 1 = time every kernel launch (no graph) */
#define GAKCO_OPT_SMEM_COLS 7       /* cap on columns per accumulation tile (0 = auto) */
#define GAKCO_OPT_FAIL_ALLOC_AFTER 8 /* fault injection: fail the Nth next device
                                        allocation (0 = off); host side only */
#define GAKCO_OPT_GROUP_BYTES 9     /* entry-array bytes per accumulation mask group */
#define GAKCO_OPT_SERVE_SLOTS 10    /* serving: concurrent batches (streams), 1..16, default 3 */
#define GAKCO_OPT_SERVE_MAX_SEQS 11 /* serving: test sequences per micro-batch (default 512) */
#define GAKCO_OPT_SERVE_MAX_WINDOWS 12 /* serving: test windows per micro-batch (default 2^19) */
#define GAKCO_OPT_SERVE_MEM_BYTES 13 /* serving: device-memory budget of busy slots (0 = none) */
/* Dense levels (batched Gram engine only).  For a level m whose masked
 * keys have at most 16 bits, countAndUpdate (Section 2.2, Alg. 1) can run
 * as a dense contraction C_m += A A^T on the tensor cores, A holding the
 * count of every (mask, (g-m)-mer) per sequence (in e4m3 up to 16; larger
 * counts are corrected exactly on the side).  Results are identical.
 * 0 = never (default), 1 = where a cost model expects it to be faster,
 * 2 = every qualifying level. */
#define GAKCO_OPT_DENSE 14
#define GAKCO_OPT_DENSE_BYTES 15    /* device bytes of the count matrices of one dense
                                       wave (default 16 GiB, at most a quarter of the
                                       device); a level whose one-mask matrix exceeds it
                                       stays sparse */
#define GAKCO_OPT_DENSE_OVERFLOW 16 /* entries of the list of counts above 16 per dense
                                       wave (default 32768); a call that needs more runs
                                       again with every level sparse */
#define GAKCO_OPT_DENSE_RUN_COLS 17 /* columns (masks x keys) of one dense contraction
                                       (default 131072); shorter runs keep concurrent
                                       tiles closer together in L2 */
/* Kernel-only mode (batched Gram engine).  The coefficients of Eq. 6 are
 * those of N_m in Eq. 8 at level M: h_m = C(g-m, k) = C(g-m, M-m), so
 * K = sum_m h_m N_m equals the cumulative profile C_M.  With this option
 * set to 1, a call that requests no N_m output computes the C(g, M) masks
 * of level M alone (K and Khat are identical); a call that asks for N_m
 * computes every level as usual.  This identity is derived here; the paper
 * computes all levels.  Default 0. */
#define GAKCO_OPT_KERNEL_ONLY 18
#define GAKCO_OPT_OVERLAP 19        /* 1 (default): a Gram call runs its dense levels and its
                                       sparse levels as two concurrent branches */
#define GAKCO_OPT_DENSE_SMS 20      /* CTAs of the dense GEMM (0 = one per SM, default) */
/* Heavy features (batched Gram engine, sparse levels).  A feature held by L
 * sequences costs about L^2 / 2 pair updates in the on-chip accumulation,
 * one column (n^2 multiply-adds) in a tensor-core contraction.  After a
 * sparse level's run-length pass, every feature with at least
 * T = ceil(GAKCO_OPT_HEAVY * n / 1000) entries (n = sequences of the
 * dataset, T >= 8, datasets of at least 256 sequences) whose counts are
 * all <= 16 becomes a column of an e4m3 count matrix A of its (dataset,
 * level), and C_m += A A^T runs on the tensor cores beside the
 * accumulation of the remaining features.  Results are identical.
 * GAKCO_OPT_HEAVY: threshold in thousandths (0 = off, the default; 20 to
 * 50 suits strongly skewed inputs).
 * GAKCO_OPT_HEAVY_BYTES: device bytes of those matrices (default 4 GiB,
 * at most 1/16 of the device); features beyond it stay sparse. */
#define GAKCO_OPT_HEAVY 21
#define GAKCO_OPT_HEAVY_BYTES 22
/* Host-buffer outputs: -1 (default) = copy straight into the caller's
 * buffers when the GPU reaches pageable memory through the host page tables
 * (the pages are first touched by host threads while the GPU computes),
 * else through two pinned staging chunks; 0 = always staging; 1 = always
 * direct. */
#define GAKCO_OPT_DIRECT_D2H 23
/* Exact accumulation rounds of the dense GEMM.  Its f32 tensor-memory
 * accumulators hold integer sums of products of counts; a round is closed
 * (and added into the int32 C_m) before any partial sum can pass this bound.
 * Default and maximum 2^24 - 1, where f32 still holds every integer; the
 * test suite drives real partial sums just below it and checks them
 * against the oracle.  Smaller values only split the work into more rounds
 * (results unchanged, slower): the tests use them to run the multi-round
 * path. */
#define GAKCO_OPT_DENSE_ROUND_SUM 24
/* Limit, in GPU clock cycles, of each wait between the dense GEMM's roles
 * (TMA loads, MMA issue, epilogue) before the call gives up with
 * GAKCO_E_TIMEOUT (0 = default, about 2 s).  The wind-down after a timeout
 * (waiting for copies and MMAs already issued) keeps the default limit.
 * For tests of the timeout path: a limit of a few cycles makes an ordinary
 * call run out; the context stays usable. */
#define GAKCO_OPT_DENSE_WAIT_CYCLES 25
/* Sort of the masked keys (Alg. 1 "sort"; the non-swapping LSD radix sort
 * of Section S:1.2), both stable and identical in result: 0 = per pass an
 * upsweep histogram, digit scans and a downsweep scatter; 1 = onesweep:
 * every pass's digit counts in one read of the keys, then one scatter per
 * pass whose tiles find their digit offsets by a decoupled look-back
 * (digits of at most 8 bits; wider digits use 0). */
#define GAKCO_OPT_SORT 26
/* How the sparse accumulation (countAndUpdate, Alg. 1) walks a feature's
 * entries when the range is shorter than a warp: 0 = up to four per lane
 * directly, the rest in rounds of 32 whose owners a shuffle search finds;
 * 1 = ranges shorter than 64 in rounds of 32, owners from a warp-wide OR
 * of range starts;
 * 2 = the direct step of 0, then the rounds of 1.  Identical results; the
 * autotuner picks one per workload (default 0). */
#define GAKCO_OPT_ACCUM_VARIANT 27
/* Elements per thread of the Gram call's run-length kernels: 16 (256-thread
 * blocks, default) or 8 (512-thread blocks, fewer registers per thread). */
#define GAKCO_OPT_RLE_ITEMS 28
/* Sort digit width of one level: value (level << 8) | bits, bits 4..11, or
 * 0 to use GAKCO_OPT_RADIX_BITS for that level (the default).  The
 * autotuner sets these where a level's key width favours another digit. */
#define GAKCO_OPT_LEVEL_RADIX_BITS 29
/* The dense GEMM's persistent CTAs may take the tiles of a partial last
 * wave as K-parts (up to 8 per tile, taken part by part), so that the wave
 * ends sooner: 1 = always, 0 = never, -1 (default) = when the call has no
 * sparse level, whose kernels would otherwise fill the wave's idle SMs.
 * Identical results. */
#define GAKCO_OPT_DENSE_SPLIT 30
/* 1: when a Gram call runs its dense and sparse levels side by side, the
 * dense GEMM starts after the sparse levels' sort and run-length passes (it
 * then runs beside the on-chip accumulation); 0 (default): as soon as its
 * count matrices are built.  Identical results. */
#define GAKCO_OPT_DENSE_LATE 31
int gakco_set_option(gakco_ctx *ctx, int key, int64_t value);

/*
 * Statistics of the last completed call.
 *   GAKCO_STAT_LAUNCHES     kernels launched by the call
 *   GAKCO_STAT_MASK_PASSES  (dataset, mask) passes processed
 *   GAKCO_STAT_DEVICE_BYTES device workspace held by the context
 *   GAKCO_STAT_GRAPH_REPLAY 1 if the call replayed a cached CUDA graph
 *   GAKCO_STAT_PAIR_UPDATES, _ENTRIES_VISITED, _WINDOWS_VISITED: work
 *   counted on the device by the accumulation stage (0 for the plain engine)
 */
#define GAKCO_STAT_LAUNCHES 1
#define GAKCO_STAT_MASK_PASSES 2
#define GAKCO_STAT_DEVICE_BYTES 3
#define GAKCO_STAT_GRAPH_REPLAY 4
#define GAKCO_STAT_PAIR_UPDATES 5     /* batched engine: c_x*c_y additions made */
#define GAKCO_STAT_ENTRIES_VISITED 6  /* batched engine: (feature, sequence) entries visited */
#define GAKCO_STAT_WINDOWS_VISITED 7  /* batched engine: (window, mask) slots read */
#define GAKCO_STAT_SERVED_BATCHES 8   /* serving: micro-batches completed so far */
#define GAKCO_STAT_SERVED_REQUESTS 9  /* serving: requests completed so far */
#define GAKCO_STAT_DENSE_PROBLEMS 10  /* Gram: (dataset, level, mask run) contractions on the tensor cores */
#define GAKCO_STAT_DENSE_FLOPS 11     /* Gram: flops of the dense contractions' upper triangles,
                                         2 per multiply-add, padding excluded */
#define GAKCO_STAT_DENSE_ISSUED_FLOPS 12 /* Gram: flops the tensor cores issued (whole tiles, padding) */
#define GAKCO_STAT_DENSE_BYTES 13     /* Gram: bytes of the dense count matrices written */
#define GAKCO_STAT_SORT_BYTES 14      /* Gram: algorithmic bytes of every sort pass (keys and
                                         payloads read and written once per pass) */
#define GAKCO_STAT_HEAVY_COLUMNS 15   /* Gram: heavy features moved to the tensor cores */
#define GAKCO_STAT_HEAVY_FLOPS 16     /* Gram: flops of their contractions' upper triangles */
#define GAKCO_STAT_MASKS 20           /* c_gk: position masks of all levels (the units a
                                         sharded Gram splits) */
#define GAKCO_STAT_RLE_BYTES 17       /* Gram: algorithmic bytes of the run-length passes (each
                                         element's key and payload read once, its ewin slot
                                         written; 8 bytes per entry emitted) */
#define GAKCO_STAT_PACK_BYTES 18      /* Gram: algorithmic bytes of the g-mer packing (symbols read
                                         once; 8-byte key and 4-byte window id per window) */
#define GAKCO_STAT_COMBINE_BYTES 19   /* Gram: algorithmic bytes of the diagonal and combine tail
                                         (upper triangles of C_0..C_M read once, requested outputs
                                         written in full) */
int gakco_get_stat(const gakco_ctx *ctx, int key, double *value);

/*
 * Per-kernel timing of the last call made with GAKCO_OPT_PROFILE = 1:
 * entry `idx` (0-based) gives the kernel's name, total milliseconds and
 * number of launches.  Returns GAKCO_E_INVALID past the last entry.
 */
int gakco_kernel_timing(const gakco_ctx *ctx, int idx, char *name,
                        int name_len, double *total_ms, int64_t *launches);

/*
 * Autotuner: times the stages of gakco_gram_batch_device on the given
 * datasets (device codes, host offsets), one parameter at a time, and sets
 * the fastest on the context: the sort digit width (6, 8, 10 bits, then
 * per level 7..11), the sort chunk size (2^22..2^26 elements), the
 * run-length items per thread (16, 8), the accumulation block size (256,
 * 512 threads) with the mask-group size (64..512 MiB), the dense-level mode
 * (0, 1, 2) and the accumulation variant (0, 1, 2).  Results are cached per
 * (sigma, g, k, SM count, size buckets) for the life of the process, so a
 * second call for a similar workload returns at once.  `report` (may be
 * NULL) receives the choice.  The options only change speed, never results.
 */
int gakco_autotune(gakco_ctx *ctx, int32_t ndata, const uint8_t *const *codes,
                   const int64_t *const *offsets, const int32_t *n,
                   void *stream, char *report, int report_len);

/*
 * Gram kernel of one dataset, host buffers (Alg. 1 CALCULATEKERNEL).
 *   codes, offsets, n : the dataset (host)
 *   K      : n*n int32 kernel, or NULL
 *   Khat   : n*n fp64 normalised kernel, or NULL
 *   Nm     : (M+1)*n*n int32 mismatch profiles N_0..N_M, or NULL
 * Synchronous: returns after the outputs are written.
 */
int gakco_gram(gakco_ctx *ctx, const uint8_t *codes, const int64_t *offsets,
               int32_t n, int32_t *K, double *Khat, int32_t *Nm);

/*
 * Gram kernels of several independent datasets in one batched pass (all
 * datasets share sigma, g, k).  Arrays have `ndata` entries; per-dataset
 * output pointers follow gakco_gram.  Host buffers; synchronous.
 */
int gakco_gram_batch(gakco_ctx *ctx, int32_t ndata,
                     const uint8_t *const *codes,
                     const int64_t *const *offsets, const int32_t *n,
                     int32_t *const *K, double *const *Khat,
                     int32_t *const *Nm);

/*
 * Device-buffer forms.  `codes`, K, Khat, Nm are device pointers (K is
 * required); `offsets` are host pointers; `stream` is a cudaStream_t (NULL
 * = the legacy default stream).  Work is ordered on `stream`; the call
 * returns after it completes and the device status has been checked.
 */
int gakco_gram_device(gakco_ctx *ctx, const uint8_t *codes,
                      const int64_t *offsets, int32_t n, int32_t *K,
                      double *Khat, int32_t *Nm, void *stream);
int gakco_gram_batch_device(gakco_ctx *ctx, int32_t ndata,
                            const uint8_t *const *codes,
                            const int64_t *const *offsets, const int32_t *n,
                            int32_t *const *K, double *const *Khat,
                            int32_t *const *Nm, void *stream);

/*
 * Cross kernel K(test, train) (Section 3.1: the paper classifies with one
 * kernel over training and test sequences together; K(test, train) is its
 * test-rows x train-columns block, and K(t, t) depends on t alone).
 *
 * gakco_fit makes a training set resident: for every mask its features
 * (distinct (g-m)-mers, in key order) with their entries, and the training
 * diagonal.  Host buffers; synchronous.  The index stays until the next
 * fit or gakco_destroy.  Fails with GAKCO_E_INVALID while served requests
 * are in flight.  gakco_fit_device takes device codes on `stream`.
 */
int gakco_fit(gakco_ctx *ctx, const uint8_t *codes, const int64_t *offsets,
              int32_t n);
int gakco_fit_device(gakco_ctx *ctx, const uint8_t *codes,
                     const int64_t *offsets, int32_t n, void *stream);

/*
 * K and Khat of a test batch (nt sequences) against the fitted training
 * set: row-major nt x n_train int32 K and fp64 Khat (either may be NULL in
 * the host form).  Khat(t, y) = K(t, y) / sqrt(K(t, t) K(y, y)).  The
 * int32 bound uses the longest test and training sequences.
 * gakco_cross_fitted: host buffers; _device: device codes and outputs (K
 * required) on `stream`.  gakco_cross = gakco_fit(train) followed by
 * gakco_cross_fitted(test).
 */
int gakco_cross_fitted(gakco_ctx *ctx, const uint8_t *codes,
                       const int64_t *offsets, int32_t nt, int32_t *K,
                       double *Khat);
int gakco_cross_fitted_device(gakco_ctx *ctx, const uint8_t *codes,
                              const int64_t *offsets, int32_t nt, int32_t *K,
                              double *Khat, void *stream);
int gakco_cross(gakco_ctx *ctx, const uint8_t *test_codes,
                const int64_t *test_offsets, int32_t nt,
                const uint8_t *train_codes, const int64_t *train_offsets,
                int32_t ntrain, int32_t *K, double *Khat);

/*
 * Serving: asynchronous cross-kernel requests against the fitted training
 * set, with continuous batching.  gakco_submit copies the request's host
 * inputs, queues it and returns a ticket at once; K / Khat are the
 * caller's host output buffers (nt x n_train, may be NULL), written before
 * the request is reported done and untouched afterwards.  A dispatcher
 * thread admits queued requests into free slots (one CUDA stream and
 * working memory each) as micro-batches bounded by GAKCO_OPT_SERVE_MAX_SEQS
 * / _MAX_WINDOWS and by the memory budget; batches in different slots
 * overlap on the device, and requests arriving meanwhile are admitted as
 * slots free up.  A request's results do not depend on the batch it ran in.
 *
 * gakco_poll waits up to timeout_ms (0: no wait, < 0: until done) and
 * returns GAKCO_OK when the request is done (the ticket is then released
 * and *latency_ms, if given, receives submit-to-done milliseconds),
 * GAKCO_E_PENDING if it is not done yet, or the request's error.
 * gakco_submit and gakco_poll may be called from several threads.
 */
int gakco_submit(gakco_ctx *ctx, const uint8_t *codes, const int64_t *offsets,
                 int32_t nt, int32_t *K, double *Khat, uint64_t *ticket);
int gakco_poll(gakco_ctx *ctx, uint64_t ticket, int timeout_ms,
               double *latency_ms);

/*
 * SVM decision values on the fitted training set (Eq. 1):
 *   f(x) = sum_i coef[i] * k(x_i, x) + bias,
 * with coef[i] = alpha_i * y_i and the bias supplied by the caller (training
 * the SVM is outside this library) and k = Khat (kind 0) or K (kind 1).
 * The sum runs over the training sequences in a fixed order, so a value does
 * not depend on the batch a request ran in.
 *
 * gakco_set_svm copies n coefficients (n must equal the fitted training
 * set's size) next to the resident training index; a later gakco_fit drops
 * them.  It fails with GAKCO_E_INVALID while served requests are in flight.
 * gakco_decision computes the decision values of nt test sequences (host
 * buffers; `decision` holds nt doubles).  gakco_submit_svm is gakco_submit
 * with the request's decision values as one more output (nt doubles, may
 * be NULL); it fails with GAKCO_E_INVALID when no coefficients are set.
 */
/*
 * Adding sequences to the fitted set (the adaptive training that Section 3.2
 * discusses with Fig. 5(c): the kernel grows as new sequences arrive).
 * Computes the nb new rows of the Gram matrix of the union (old sequences
 * first, then the new ones in order): K_rows and Khat_rows (may be NULL)
 * are nb x (n + nb), row-major; the full matrix is the old one bordered by
 * these rows and their transposes.  The values equal gakco_gram on the
 * union bit for bit.  The new rows against the old sequences come from the
 * resident index (the cross kernel), the new block from a Gram kernel of
 * the new sequences; the fitted set then becomes the union (SVM
 * coefficients are dropped).  Host buffers; fails with GAKCO_E_INVALID
 * while served requests are in flight.
 */
int gakco_extend(gakco_ctx *ctx, const uint8_t *codes, const int64_t *offsets,
                 int32_t nb, int32_t *K_rows, double *Khat_rows);

int gakco_set_svm(gakco_ctx *ctx, const double *coef, int32_t n, double bias,
                  int kind);
int gakco_decision(gakco_ctx *ctx, const uint8_t *codes,
                   const int64_t *offsets, int32_t nt, double *decision);
int gakco_submit_svm(gakco_ctx *ctx, const uint8_t *codes,
                     const int64_t *offsets, int32_t nt, int32_t *K,
                     double *Khat, double *decision, uint64_t *ticket);

/*
 * Sharded Gram computation (Section 2.2, "Parallelization"; S:5.3): every
 * (level m, position mask) pass of countAndUpdate is independent, and C_m
 * (Eq. 8) is the sum of the passes' contributions.  A dataset's c_gk masks
 * (GAKCO_STAT_MASKS; level order, lexicographic within a level) can
 * therefore be split into slices, one per GPU or process:
 *
 * gakco_gram_partial_device computes the contribution of masks
 * [mask_begin, mask_end) to C_0..C_M for one dataset (device codes, host
 * offsets as in gakco_gram_device) into C, a device buffer of (M+1) x n x n
 * uint32 (C[(m n + x) n + y]), upper triangles (y >= x) only; the strict
 * lower triangles are written as 0.  Work is ordered on `stream`; the call
 * returns when it is done.  Batched engine only (GAKCO_OPT_ENGINE = 0).
 *
 * The slices' C buffers are summed element-wise with wrap-around uint32 (or
 * int32) addition, e.g. by an all-reduce across ranks; integer addition is
 * exact and order-independent, and the sum over all c_gk masks is the
 * dataset's C.  gakco_combine_device then applies inclusion-exclusion
 * (Eq. 9), the kernel K = sum_m h_m N_m (Eq. 6, Eq. 7) and the
 * normalisation to a summed C (device pointer, read only), writing K (n x n
 * int32, required), Khat and N_m (optional) exactly as gakco_gram_device
 * does.  The sum must cover every mask exactly once: the combine step
 * cannot tell a missing or repeated slice from a complete sum.
 */
int gakco_gram_partial_device(gakco_ctx *ctx, const uint8_t *codes,
                              const int64_t *offsets, int32_t n,
                              int32_t mask_begin, int32_t mask_end,
                              uint32_t *C, void *stream);
int gakco_combine_device(gakco_ctx *ctx, const uint32_t *C, int32_t n,
                         int32_t *K, double *Khat, int32_t *Nm, void *stream);

/*
 * Measured ceiling of the sparse accumulation: the rate (atomic adds per
 * second, whole device) at which the current GPU retires conflict-free
 * 32-bit shared-memory atomic adds, the operation countAndUpdate (Alg. 1)
 * performs once per pair update on the sparse route.  Runs a probe kernel
 * of a few milliseconds on `stream` (a cudaStream_t, NULL = legacy stream)
 * and waits for it; allocates and frees a small device buffer.  Returns
 * GAKCO_OK and *updates_per_s, or GAKCO_E_CUDA.  Not part of the paper: the
 * denominator of the accumulation's roofline.
 */
int gakco_measure_smem_atomics(void *stream, double *updates_per_s);
/* The same rate with each lane adding at pseudo-random words of a 4096-word
 * row (random_columns = 1), the column pattern of the accumulation: lanes
 * meet in banks as random draws do.  random_columns = 0 is
 * gakco_measure_smem_atomics. */
int gakco_measure_smem_atomics_pattern(void *stream, int random_columns,
                                       double *updates_per_s);

/*
 * Gram kernel of one dataset that allocates nothing.  The paper has no
 * counterpart; this entry point exists for callers that cannot let a
 * library allocate device memory: applications whose GPU memory belongs to
 * a framework's caching allocator or is split into fixed budgets up front,
 * request paths that cannot afford the device-wide synchronisation of
 * cudaMalloc / cudaFree, and plug-ins that are handed buffers but may not
 * own device memory.
 *
 * It computes the same K, Khat and N_m as gakco_gram_device (same layouts,
 * K required, Khat and Nm optional; codes, K, Khat, Nm are device pointers,
 * offsets a host pointer) without a context: sigma, g, k are passed
 * directly.  All intermediate data lives in one static device array of
 * 64 MiB that is part of the library image (every GPU that loads the
 * library holds it until the process exits), and host tables live in a
 * static host array.  The call makes no cudaMalloc, cudaFree or other
 * allocation and creates no stream or event.
 *
 * Limits: at most 1024 position masks (c_gk); the input's scratch need
 * (about 64 bytes per window plus 4 (M+1) n^2 bytes) must fit in 64 MiB;
 * plus the limits of gakco_gram.  Larger inputs return GAKCO_E_OVERFLOW
 * with a message in `err` (caller buffer of `err_len` bytes, may be NULL).
 *
 * Every call made outside stream capture looks up the device address of
 * the static array on the current device (cudaGetSymbolAddress, which
 * allocates nothing) and sets the kernels' attributes, so a device reset
 * leaves no stale address; a call made while `stream` is capturing uses the
 * address of the last call outside capture on that device, so make the
 * first call on each device before any stream capture (otherwise the call
 * returns GAKCO_E_INVALID).  Work is ordered on `stream` and the call
 * returns after it completes.
 *
 * Every call uses the same static arrays: the device array keeps the last
 * call's contents (everything that must start at zero is cleared by each
 * call), and the host tables are shared by every device.  Calls whose work
 * overlaps on the GPU race and corrupt each other's results.  The entry
 * point therefore holds one process-wide lock, for all devices, from start
 * to finish, so concurrent callers in one process (other host threads, on
 * the same or another GPU) are serialised.
 */
int gakco_gram_device_noalloc(int sigma, int g, int k, const uint8_t *codes,
                              const int64_t *offsets, int32_t n, int32_t *K,
                              double *Khat, int32_t *Nm, void *stream,
                              char *err, int err_len);

#ifdef __cplusplus
}
#endif

#endif /* GAKCO_H */
