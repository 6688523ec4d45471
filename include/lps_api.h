/*
 * lps_api.h — C ABI of the GB300 (sm_103a) Priori L+S reconstruction library (liblps.so).
 *
 * Method: Zonoobi, Faghih Roohi, Kassim, "Low-Rank and Sparse Matrix Decomposition with
 * a-priori knowledge for Dynamic 3D MRI reconstruction" (arXiv:1411.6206).
 *   - Each time instance t is a volume nx x ny x nz reshaped to the Casorati matrix
 *     X^(t) in C^{(nx ny) x nz}, one column per slice (Sec. 2), decomposed as L + S.
 *   - Acquisition: d = A(X) + eta (Sec. 2), here the multi-coil Cartesian encode
 *     E = M F C: coil sensitivities C_c, orthonormal unshifted DFT F over (z, x, y) (or over
 *     (x, y) per slice), and a line mask M on the (ky, kz) grid (kx fully sampled).
 *   - Algorithm 1 (Sec. 3): (0) X_0 = E^H d, S_0 = 0; per iteration (1) singular-value
 *     soft-thresholding of X - S, (2) pull of the singular values towards those of L^(t-1),
 *     (3) soft-thresholding of the wavelet coefficients of S off the support of the previous
 *     frame, (4) the data-consistency update X = L + S - E^H(E(L + S) - d).
 *   - Recursion (Sec. 3, Fig. 2): frame 1 runs plain L+S (no prior), frame t >= 2 uses the
 *     support and singular values of frame t-1.
 *
 * Conventions shared by every call:
 *   - Every call returns int: LPS_OK (0) or a negative LPS_ERR_* code. No exceptions or
 *     aborts cross this boundary; lps_status_string() names a code; lps_last_error() gives a
 *     one-line description of the last failure in the calling thread.
 *   - Array arguments are plain pointers to either host or device memory (CUDA unified
 *     addressing decides which); they are owned by the caller. Input arrays are copied
 *     into the plan, in stream order on the plan's stream, before the call returns; a
 *     device input may be reused once that stream has passed the call. Host inputs are
 *     copied synchronously. Outputs are written in stream order; to a host pointer the call
 *     synchronises the stream before returning.
 *   - complex64 = two float32 (re, im), interleaved (the layout of std::complex<float>,
 *     cuComplex, torch.complex64).
 *   - Image arrays are [nz][nx][ny] with y fastest. Coil maps are [ncoil][nz][nx][ny].
 *     Masks are uint8 [nz][ny] (nonzero = sampled), indexed [kz][ky] for the 3D encode
 *     (fft_z = 1) and [z][ky] for the per-slice 2D encode (fft_z = 0). Frequencies are
 *     unshifted DFT indices. k-space samples are [ncoil][nlines][nx], line l being the l-th
 *     nonzero mask entry in raster order (index kz*ny + ky ascending), each line one kx
 *     readout of nx samples.
 *   - Wavelet coefficients (support bitmaps): per slice z the orthonormal J-level 2D Haar
 *     transform splits into independent aligned B x B blocks, B = 2^J <= 8. Coefficients are
 *     numbered by 8 x 8 in-plane tiles:
 *       ((z * (nx/8) + tx) * (ny/8) + ty) * 64 + u*8 + v
 *     where (tx, ty) is the tile and (u, v) the position in the tile's 8 x 8 coefficient
 *     array, in which every aligned B x B sub-block holds that block's own Mallat layout
 *     (approximation at the block origin; the level-j details at offsets B/2^j along v
 *     (x-low, y-high), along u (x-high, y-low) and both). For J = 3 a tile is one block.
 *     With the 3D Haar (wavelet_dims = 3) the same numbering
 *     holds, slice z = bz * B + w standing for 1D position w, in Mallat order inside the
 *     block (approximation at w = 0, the level-j details at B/2^j .. B/2^(j-1) - 1), of the
 *     aligned block bz of B slices. Bit i of a bitmap is bit (i & 31) of 32-bit word i >> 5;
 *     lps_support_words() gives the word count (nx*ny*nz/32).
 *   - Work is issued on the plan's CUDA stream. Only calls that return host-visible results
 *     (stats, host outputs, mask upload) synchronise it.
 */
#ifndef LPS_API_H
#define LPS_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define LPS_OK               0
#define LPS_ERR_INVALID_ARG -1   /* bad size, NULL where required, value out of range      */
#define LPS_ERR_OOM         -2   /* device or pinned-host allocation failed                */
#define LPS_ERR_CUDA        -3   /* a CUDA runtime call or kernel launch failed            */
#define LPS_ERR_TIMEOUT     -4   /* a bounded device-side wait gave up                     */
#define LPS_ERR_NONFINITE   -5   /* NaN/Inf met in the residual or the singular values     */
#define LPS_ERR_ADMISSION   -6   /* refused by a memory budget                             */
#define LPS_ERR_STATE       -7   /* call out of order (e.g. iterate before set_data)       */
#define LPS_ERR_UNSUPPORTED -8   /* size or option this build does not implement           */

/* ---- options ---------------------------------------------------------------------- */
#define LPS_LAYOUT_SLICES      0  /* Casorati columns = the nz slices of a volume (Sec. 2) */
/* Casorati columns = the frames of a segment. 2D frames (frame_slices 1, nx x ny images): nz
 * counts the frames, mask row z holds frame z's ky lines and every frame is encoded by its own
 * 2D DFT (fft_z must be 0). 3D frames (frame_slices = s > 1): nz = frames * s slices, frame t
 * being slices t s .. t s + s - 1 (one Casorati column of s nx ny voxels); mask rows t s + kz
 * hold frame t's (kz, ky) lines and each frame volume is encoded by its own 3D DFT over its s
 * slices (fft_z = 1) or per slice (fft_z = 0). Coil maps are given per frame
 * ([c][slice][x][y] over all nz slices); sigma arrays have one entry per column. With the
 * recursion, the prior of a segment comes from the previous segment of the session. */
#define LPS_LAYOUT_FRAMES      1

#define LPS_FP32               0  /* every stage in float32 (Gram and reprojection on FMA) */
/* Precision modes: the two dense contractions (Casorati Gram and low-rank reprojection) run
 * on the tensor cores with float32 accumulation; each float32 operand x is split into
 * hi = round(x) and lo = round(x - hi) in the operand type and the products keep
 * hi hi + hi lo + lo hi (one refinement step). FFTs, thresholds and the data-consistency
 * step stay in float32; the eigendecomposition follows eig_precision. */
#define LPS_TF32_REFINE        1  /* tf32 operands (11-bit significand)                      */
#define LPS_BF16_REFINE        2  /* bf16 operands (8-bit significand)                       */

#define LPS_EIG_FP32           0  /* Gram eigendecomposition by float32 Jacobi             */
#define LPS_EIG_FP64           1  /* float32 Jacobi refined by a float64 Rayleigh-Ritz step */

#define LPS_SUPPORT_THRESHOLD  0  /* T^(t) = {i : |c_i| > lambda_S} of the last iteration  */
#define LPS_SUPPORT_NONZERO    1  /* T^(t) = supp of the shrunk coefficients (literal)     */

#define LPS_MAX_NC            32  /* largest Casorati column count (slices) supported      */

/* Storage of the coil maps (the acquisition operator's C_c, Sec. 2). With LPS_COILS_FP16 the
 * plan rounds the complex64 maps given to lps_set_coils to half precision (each of Re and Im
 * to the nearest IEEE binary16) and every operator of the plan uses the rounded maps; the
 * per-iteration data-consistency kernels of 128 x 16 planes and the runtime-sized kernel
 * reading coil maps from global memory read them as 4-byte half pairs, half the coil-map
 * bytes of an iteration. |Re|, |Im| must stay below 65504 (maps normalised to unit sum of
 * squares do). Maps that are already half-representable give results equal to LPS_COILS_FP32. */
#define LPS_COILS_FP32         0
#define LPS_COILS_FP16         1
/* Storage of the samples (the data y of Sec. 2, kept in hybrid space d' = F_x^H d). With
 * LPS_DATA_FP16, lps_set_data rounds the plan's hybrid copy to binary16 (each of Re and Im to
 * the nearest value) and keeps a half-pair copy that the per-iteration data-consistency kernels
 * read; every kernel sees the rounded values. |Re|, |Im| of d' must stay below 65504. */
#define LPS_DATA_FP32          0
#define LPS_DATA_FP16          1

typedef struct lps_plan lps_plan;   /* opaque; owns its device workspace */

typedef struct lps_params {
  int nx, ny, nz, ncoil;   /* volume size (nx: fully sampled readout axis) and coils       */
  int layout;              /* LPS_LAYOUT_SLICES | LPS_LAYOUT_FRAMES                         */
  int fft_z;               /* 1: 3D Fourier encode, (ky,kz) line mask; 0: 2D per slice     */
  int wavelet_levels;      /* Haar levels J, 1..3 (nx, ny multiples of 2^J)                */
  int max_iters;           /* iterations of Algorithm 1 per frame (1..4096)                */
  double lambda_L_rel;     /* lambda_L = lambda_L_rel * sigma_max(X_0)                      */
  double lambda_S_rel;     /* lambda_S = lambda_S_rel * max |T(X_0)|                        */
  double lambda_p;         /* prior pull of step (2), in [0, 1]                             */
  double rank_tau;         /* drop directions with sigma_i <= rank_tau * sigma_1            */
  double tol;              /* stop when ||Z_k - Z_{k-1}|| / ||Z_{k-1}|| < tol (0 = never)   */
  int precision;           /* LPS_FP32 | LPS_TF32_REFINE | LPS_BF16_REFINE                  */
  int eig_precision;       /* LPS_EIG_FP32 | LPS_EIG_FP64                                   */
  int support_rule;        /* LPS_SUPPORT_THRESHOLD | LPS_SUPPORT_NONZERO                   */
  int recursive;           /* 1: each lps_reconstruct_frame installs its support and sigma
                              as the prior of the next call (the recursion of Sec. 3)        */
  int coil_format;         /* LPS_COILS_FP32 (default) | LPS_COILS_FP16                      */
  int nx_total;            /* 0: the plan holds the whole volume; else the x extent of the
                              volume of which it holds planes x0 .. x0+nx-1 (lps_slab_*)     */
  int x0;                  /* first plane of the slab (multiple of 8)                       */
  int wavelet_dims;        /* sparsifying transform T: 2 (0 reads as 2) the per-slice 2D Haar;
                              3 the 3D Haar, the 2D pyramid times the J-level 1D Haar along z
                              (nz a multiple of 2^J; the support numbering below)            */
  int frame_slices;        /* LPS_LAYOUT_FRAMES: slices per frame (0 reads as 1). 1: 2D frames
                              (fft_z = 0); > 1: 3D frames, nz / frame_slices columns each a
                              volume of frame_slices slices with its own 3D encode (fft_z = 1)
                              or per-slice encode (fft_z = 0); float32 path, whole volumes   */
  int data_format;         /* LPS_DATA_FP32 (default) | LPS_DATA_FP16                        */
  int reserved[2];         /* must be zero                                                  */
} lps_params;

typedef struct lps_stats {
  int iters;               /* iterations run in the last frame / lps_iterate call          */
  int rank;                /* number of sigma'' > 0 at the last iteration                  */
  long long support_count; /* bits set in the output support                               */
  double lambda_L, lambda_S;
  double sigma_max;        /* sigma_1(X_0)                                                  */
  double resid_norm2;      /* ||E(L + S) - d||^2 after the last iteration                   */
  double nuclear;          /* sum of sigma'' (nuclear norm of L)                            */
  double l1_off_support;   /* sum |c'_i| over coefficients off the prior support           */
  double objective;        /* resid_norm2/2 + lambda_L*nuclear + lambda_S*l1_off_support    */
  double rel_change;       /* ||Z_k - Z_{k-1}|| / ||Z_{k-1}||, Z = L + S                     */
} lps_stats;

/* Per-iteration record returned by lps_get_history (same meaning as lps_stats fields). */
typedef struct lps_iter_record {
  double resid_norm2, nuclear, l1_off_support, objective, rel_change;
  int rank;
  int eig_sweeps;          /* Jacobi sweeps of the Gram eigendecomposition                */
} lps_iter_record;

/* Fill *p with the defaults: layout SLICES, fft_z 1, J 3, 50 iterations, lambda_L_rel 0.01,
 * lambda_S_rel 0.005, lambda_p 0.5, rank_tau 1e-3, tol 0, FP32, threshold support rule,
 * recursive 0. Sizes are left 0. */
int lps_params_init(lps_params* p);

/* Create a plan for one problem shape. Validates *p (LPS_ERR_INVALID_ARG /
 * LPS_ERR_UNSUPPORTED), allocates the device workspace (LPS_ERR_OOM) and binds `stream`
 * (a cudaStream_t; NULL = the legacy default stream). *out is NULL on failure. */
int lps_plan_create(const lps_params* p, void* stream, lps_plan** out);
int lps_plan_destroy(lps_plan* plan);
int lps_set_stream(lps_plan* plan, void* stream);
/* Device bytes the plan holds (workspace + copies of coils, data and state). */
int lps_plan_device_bytes(const lps_plan* plan, size_t* bytes);
/* Bytes lps_plan_create would allocate for *p, without allocating. */
int lps_estimate_device_bytes(const lps_params* p, size_t* bytes);

/* Acquisition operator pieces (Sec. 2). The mask [nz][ny] (host or device) fixes the line
 * list; it synchronises the stream (the line count is needed on the host). A mask with no
 * sampled entry is LPS_ERR_INVALID_ARG. Returns the number of lines via *nlines (nullable). */
int lps_set_mask(lps_plan* plan, const uint8_t* mask, int* nlines);
/* Coil sensitivity maps, complex64 [ncoil][nz][nx][ny]. */
int lps_set_coils(lps_plan* plan, const void* coils);
/* k-space samples y^(t) of the current mask, complex64 [ncoil][nlines][nx]; nlines must
 * equal the count of the last lps_set_mask. Transformed once along kx into the plan's
 * hybrid (x, ky, kz) copy. Resets the iteration state (the next iterate starts at step 0). */
int lps_set_data(lps_plan* plan, const void* kdata, int nlines);
/* Prior of Algorithm 1 from frame t-1: support bitmap of T(S^(t-1)) (lps_support_words
 * words) and sigma'' of L^(t-1) (nz doubles, descending rank order). Either may be NULL:
 * NULL support = empty T^(t-1); NULL sigma = no pull (step 2 skipped). lps_clear_prior()
 * returns the plan to plain L+S (frame t = 1). */
int lps_set_prior(lps_plan* plan, const uint32_t* support, const double* sigma_prev);
int lps_clear_prior(lps_plan* plan);

/* Sliding temporal window (layout LPS_LAYOUT_FRAMES): when the next call reconstructs the
 * window advanced by `shift` frames, the support installed as the prior (the recursion of
 * Sec. 3) must follow its frames. Moves the prior support `shift` Casorati columns towards
 * column 0 (the first `shift` columns are dropped) and repeats the last remaining column in the
 * `shift` freed ones (the newest frame's prior is the support of the frame before it). The
 * prior singular values are kept. 1 <= shift < columns (nz / frame_slices); enqueued on
 * the plan's stream. */
int lps_shift_prior_columns(lps_plan* plan, int shift);

/* Run n iterations of Algorithm 1 on the resident state, starting with step (0) if the
 * state was reset by lps_set_data. Stops early on the tol rule (stats->iters tells). */
int lps_iterate(lps_plan* plan, int n_iters, lps_stats* stats /* nullable */);

/* One full time instance: step (0), max_iters iterations (or until tol), outputs.
 * out_recon = L + S, out_L, out_S: complex64 [nz][nx][ny]; out_support: bitmap words;
 * out_sigma: nz doubles (sigma'' in rank order). All outputs nullable. The per-frame launch
 * sequence is recorded once into a CUDA graph and replayed. */
int lps_reconstruct_frame(lps_plan* plan, void* out_recon, void* out_L, void* out_S,
                          uint32_t* out_support, double* out_sigma, lps_stats* stats);

/* Per-iteration records of the last frame / iterate calls since lps_set_data
 * (at most max records; *count = records written). Synchronises. */
int lps_get_history(lps_plan* plan, lps_iter_record* out, int max, int* count);

/* State access for tests and checkpoints: X (last step-4 output), L, S, complex64 images.
 * lps_set_state loads X, S and L_prev (the L of the previous iteration; NULL = X) together
 * with fixed lambda_L, lambda_S, as if `iters_done` iterations had run. */
int lps_get_state(lps_plan* plan, void* X, void* L, void* S);
/* Support bitmap T^(t) and sigma'' of the last iteration (the prior the next frame would
 * receive); either output may be NULL. */
int lps_get_support(lps_plan* plan, uint32_t* support, double* sigma);
int lps_set_state(lps_plan* plan, const void* X, const void* S, const void* L_prev,
                  double lambda_L, double lambda_S, int iters_done);

/* Standalone operators with the current coils and mask (Sec. 2):
 * forward: image -> k-space samples [ncoil][nlines][nx]; adjoint: samples -> image. */
int lps_forward(lps_plan* plan, const void* image, void* kdata);
int lps_adjoint(lps_plan* plan, const void* kdata, void* image);
/* Step (4) alone on the resident data: X = Z - E^H(E Z - d); *resid_norm2 = ||E Z - d||^2
 * (nullable).
 * The operators (these three, lps_casorati_gram, lps_lowrank_reproject, lps_adjoint_noalloc)
 * carry no status from the device: a bounded wait that runs out in one of their kernels (it
 * records the timeout only in a plan's frame path, or under lps_test_stall_wait) leaves the
 * output incomplete while the call returns LPS_OK. The frame path (lps_reconstruct_frame,
 * lps_iterate, batches, the server) reports it as LPS_ERR_TIMEOUT. */
int lps_data_consistency(lps_plan* plan, const void* Z, void* X, double* resid_norm2);

/* Casorati Gram G = M^H M, M = X - S: the matrix whose eigendecomposition gives the
 * singular values and right singular vectors for the singular-value thresholding of step (1)
 * (Sec. 3; M is N_r x nz with N_r = nx ny, one column per slice). Computed with the plan's
 * precision: float32 FMA for LPS_FP32, tensor cores with split operands otherwise.
 * X, S: device [nz][nx][ny] complex64 (S may be NULL: S = 0). G: device nz x nz complex64,
 * row-major, G[i][j] = sum_r conj(M[r][i]) M[r][j] (exactly Hermitian). Enqueued on the
 * plan's stream; uses the plan's Gram scratch (do not overlap with other work of the plan). */
int lps_casorati_gram(lps_plan* plan, const void* X, const void* S, void* G);
/* Low-rank reprojection L = (X - S) W of steps (1)-(2) (Sec. 3): with W = V diag(sigma''/
 * sigma) V^H from the eigendecomposition of the Gram, L = U diag(sigma'') V^H. Computed with
 * the plan's precision. X, S as above (S may be NULL); W: device nz x nz complex64 row-major;
 * L: device [nz][nx][ny] complex64, L[j][r] = sum_i M[i][r] W[i][j]. Enqueued on the plan's
 * stream. */
int lps_lowrank_reproject(lps_plan* plan, const void* X, const void* S, const void* W, void* L);

/* recon = L + S of the last reconstructed frame (Algorithm 1's output, Sec. 3) into a device
 * or host buffer [nz][nx][ny] complex64 (a host buffer makes the call synchronous). */
int lps_get_recon(lps_plan* plan, void* out);

/* Test hook (not in the paper; exercises the failure path of the bounded waits without
 * faulting or hanging the GPU). Arms a one-shot stall for the next lps_data_consistency call:
 * on the staged-coil runtime-sized kernel (lps_apply_tune dc_variant 1, else LPS_ERR_STATE),
 * every CTA waits for its first coil on an mbarrier that nothing completes, for `polls` polls
 * (1..2^20), records the timeout, lets the coil copies it has in flight land (normal wait
 * budget) and returns. The call then returns LPS_ERR_TIMEOUT with the error flag cleared; the
 * plan and the context stay usable. */
int lps_test_stall_wait(lps_plan* plan, int polls);

/* ---- autotuner ---------------------------------------------------------------------
 * Not in the paper (it fixes no launch shapes): times, on the plan's resident coils, mask and
 * data, the candidate shapes of the two per-iteration kernels whose shape is a free choice,
 * and installs the fastest in the plan (its frame graph is captured again):
 *  - data consistency: the compile-time plane kernel where one exists, the register-transform
 *    coil loop where the plane has one, and the runtime-sized kernel with each candidate
 *    ordering of the FFT radix passes along y and z, coil planes staged in shared memory or
 *    read from global memory;
 *  - sparse update: 8x8 in-plane tiles per CTA.
 * Results are cached per geometry (nx, ny, nz, ncoil, fft_z, precision) for the process.
 * Requires lps_set_coils, lps_set_mask and lps_set_data; synchronises the plan's stream; the
 * plan's state (X, L, S, prior) is not modified. out may be NULL. */
typedef struct lps_tune_result {
  int dc_variant;          /* 0: compile-time plane kernel, 1: runtime-sized kernel with the
                              coil planes staged in shared memory, 2: the same reading coil
                              maps from global memory (half the shared memory); 128 x 16
                              planes also: 3: register-transform kernel, 4 coil groups (the
                              default there), 4: the same with 8 coil groups; planes of
                              ny = 16 Q (Q = 4..10) by nz in {8, 10, ..., 16, 20, 24, 28, 32}:
                              5: the runtime-sized kernel's update with its coil loop on
                              register transforms (the default there)                      */
  int radix_y[8];          /* FFT passes along y of the runtime-sized kernel (0-terminated) */
  int radix_z[8];          /* FFT passes along z                                            */
  int lrs_tiles;           /* 8x8 tiles per CTA of the sparse-step kernel                   */
  int candidates;          /* configurations timed                                          */
  int cached;              /* 1: taken from the cache, nothing timed                        */
  double dc_us, lrs_us;    /* best measured time per launch (microseconds)                  */
} lps_tune_result;
int lps_autotune(lps_plan* plan, lps_tune_result* out);
int lps_autotune_clear_cache(void);
/* Install a launch shape (for instance one measured by lps_autotune in an earlier process):
 * dc_variant, radix_y / radix_z (variants 1 and 2; their products must be ny and nz) and
 * lrs_tiles are used, the other fields ignored. Variants 3 and 4 need a 128 x 16 plane,
 * variant 5 a plane listed beside it. Synchronises the plan's stream; the frame
 * graph is captured again at the next frame. */
int lps_apply_tune(lps_plan* plan, const lps_tune_result* tune);

/* ---- batches of independent problems -------------------------------------------------
 * Not in the paper: many independent problems (sizes, slices and coils may differ) whose
 * frames are reconstructed together. Each member is an ordinary plan (set its coils, mask,
 * data and prior through lps_batch_plan); lps_batch_reconstruct runs one frame of every
 * active member with ONE graph launch on the batch stream: the members' per-frame graphs are
 * parallel branches of one CUDA graph. Inactive members stay in the graph and return at once
 * (their control block starts converged), so members may finish their sequences at
 * different times without a rebuild. Results: lps_get_recon / lps_get_state per member. */
typedef struct lps_batch lps_batch;
int lps_batch_create(const lps_params* params /* [n] */, int n, void* cuda_stream, lps_batch** out);
int lps_batch_destroy(lps_batch* batch);
int lps_batch_size(lps_batch* batch);
int lps_batch_plan(lps_batch* batch, int i, lps_plan** out);   /* owned by the batch */
int lps_batch_set_active(lps_batch* batch, int i, int active);  /* default: active */
int lps_batch_autotune(lps_batch* batch);                       /* lps_autotune per active member */
/* Step (4) alone (operator form, X = Z - E^H(E Z - d), no Gram) on every active member, Z[i] and
 * X[i] device images of member i ([nz][nx][ny] complex64; ignored for inactive members), and
 * the device time of the launch in *ms (may be NULL). persistent = 0: each member's own
 * data-consistency kernel (the one its plan runs), as parallel branches of one graph;
 * 1: one persistent launch over the members' descriptor table, CTAs taking (member, plane) items
 * from a counter and running the runtime-sized kernel's body (planes of at most 6144 elements,
 * else LPS_ERR_UNSUPPORTED). Not in the paper: it measures the batched layout against a single
 * persistent kernel. Synchronises the batch stream. */
int lps_batch_data_consistency(lps_batch* batch, void* const* Z, void* const* X, int persistent, float* ms);
int lps_batch_reconstruct(lps_batch* batch);

/* ---- serving loop -------------------------------------------------------------------
 * Not in the paper (it reconstructs one sequence): real-time recursive reconstruction of many
 * concurrent sessions. A session is a recursive plan on its own CUDA stream whose coil maps,
 * L, S, prior support and singular values stay on the device between frames. Sessions are
 * admitted while the sum of their lps_estimate_device_bytes fits hbm_budget_bytes (else
 * LPS_ERR_ADMISSION; retry after lps_server_close). Frames are submitted as they arrive; a
 * frame goes to the device as soon as fewer than max_inflight frames are there (0 = no limit),
 * after the earlier frames of its session and concurrently with other sessions' frames
 * (single_stream = 1 runs every frame in arrival order on one stream instead). Latency = time at which the frame's
 * L + S is in the session's output buffer minus the arrival time given at submission, both
 * on the server clock (seconds since lps_server_create, lps_server_now). Single-threaded:
 * calls on one server must not overlap. */
typedef struct lps_server lps_server;
typedef struct lps_server_config {
  size_t hbm_budget_bytes;   /* admission budget over all open sessions                    */
  int max_inflight;          /* frames on the device at once (0 = no limit)                */
  int single_stream;         /* 1: every session on one stream, frames run one after another
                                in arrival order (the plain frame-by-frame path)           */
  int autotune;              /* 1: lps_autotune each session on its first frame (cached per
                                geometry; that frame's latency includes the tuning)        */
  int reserved[5];           /* must be zero                                               */
} lps_server_config;
int lps_server_create(const lps_server_config* cfg, lps_server** out);
int lps_server_destroy(lps_server* server);
double lps_server_now(lps_server* server);
/* params->recursive must be 1; coils: device or host [ncoil][nz][nx][ny] complex64. */
int lps_server_open(lps_server* server, const lps_params* params, const void* coils, int* session);
int lps_server_close(lps_server* server, int session);   /* no frames in flight */
int lps_server_plan(lps_server* server, int session, lps_plan** out);
size_t lps_server_bytes_in_use(lps_server* server);
/* mask: host ny*nz bytes (copied); kdata: device or pinned-host samples as for lps_set_data,
 * caller-owned until the frame is done. */
int lps_server_submit(lps_server* server, int session, const uint8_t* mask, const void* kdata,
                      double arrival_s, long long* ticket);
/* 1: done (latency and completion time in seconds, nullable), 0: not yet, < 0: error. */
int lps_server_poll(lps_server* server, long long ticket, double* latency_s, double* completion_s);
int lps_server_wait(lps_server* server, long long ticket, double* latency_s, double* completion_s);
int lps_server_release(lps_server* server, long long ticket);   /* forget a finished frame */
/* L + S of the session's last completed frame into a device or host buffer (synchronous). */
int lps_server_result(lps_server* server, int session, void* out);

/* Kernel timing of the per-frame graph. With profiling on, the graph records CUDA events
 * around every kernel it launches; lps_get_kernel_times synchronises the stream and returns,
 * for the last lps_reconstruct_frame, the launch count and summed device time of each class:
 * [0] data consistency (step 4, with the reprojection L_k = (X - S) W of steps 1-2 in its
 * prologue), [1] sparse step (3), [2] Gram eigendecomposition and singular-value steps
 * (1)-(2), [3] step (0) kernels,
 * [4] Casorati Gram on the tensor cores and [5] reprojection on the tensor cores (precision
 * modes only). */
#define LPS_KERNEL_CLASSES 6
typedef struct lps_kernel_times {
  int launches[LPS_KERNEL_CLASSES];
  double ms[LPS_KERNEL_CLASSES];
} lps_kernel_times;
int lps_set_profiling(lps_plan* plan, int on);
int lps_get_kernel_times(lps_plan* plan, lps_kernel_times* out);

/* Checkpoint of the recursion state (prior support, prior sigma, L, S, lambdas) to a host
 * buffer. With buf NULL, *bytes receives the size needed. */
int lps_session_export(lps_plan* plan, void* buf, size_t* bytes);
int lps_session_import(lps_plan* plan, const void* buf, size_t bytes);

/* ---- x-slab sharding of one problem -------------------------------------------------
 * Not in the paper, which reconstructs each volume whole. Once the samples are moved to the
 * hybrid (x, ky, kz) space, steps (3) and (4) of Algorithm 1 (Sec. 3) act on every x-plane
 * alone (the Haar tiles are 8 planes wide), so a volume splits into slabs of whole tiles held
 * by separate plans (one per GPU): a plan with nx_total > 0 holds planes x0 .. x0+nx-1 of a
 * volume of nx_total planes; its coil maps and outputs are the slab's ([c][z][x0..][y]),
 * lps_set_data takes whole readouts ([ncoil][nlines][nx_total]) and lps_forward returns the
 * slab's share of E x (the slabs' outputs add up to E x). The only sums over all planes are
 * the Casorati Gram of step (1) and a few scalars (residual, change and l1 statistics), plus
 * the maximum of |T(X_0)| that fixes lambda_S: each iteration leaves the slab's share of them
 * in a small record, the caller reduces the records of all slabs (for instance with one
 * all-reduce), and the next iteration repeats the n x n eigendecomposition on every slab from
 * the reduced record. The record is float32, device memory owned by the caller:
 *   [0, sum_floats)  to be summed over the slabs: data-consistency statistics (4), sparse-step
 *                    statistics (2, then 2 zeros), the Gram (2 nz^2, complex row-major);
 *   [sum_floats, sum_floats + max_floats)  to be maximised over the slabs: max |T(X_0)|.
 * Sequence per frame: lps_slab_begin (step 0), reduce; for k = 1..K: lps_slab_iterate(k),
 * reduce; lps_slab_end. Work is enqueued on the plan's stream; the reduction must be ordered
 * after the call that wrote the record and before the next call (same stream, or events).
 * lps_reconstruct_frame and lps_iterate return LPS_ERR_STATE for a plan that holds a slab. */
int lps_slab_reduction_size(const lps_plan* plan, size_t* sum_floats, size_t* max_floats);
/* Step (0) on the slab; needs lps_set_coils, lps_set_mask and lps_set_data. */
int lps_slab_begin(lps_plan* plan, float* rec);
/* Iteration k (1, 2, ... in order, at most max_iters) from the reduced record; leaves the
 * slab's share of iteration k in rec. Stops doing work once the tol rule has stopped the frame
 * (every slab takes the same decision from the same reduced record). */
int lps_slab_iterate(lps_plan* plan, float* rec, int k);
/* After the last iteration and its reduction: statistics of the frame (support_count is the
 * slab's own), outputs settled for lps_get_recon / lps_get_state / lps_get_support, and for a
 * recursive plan the prior of the next frame installed. Synchronises the plan's stream. */
int lps_slab_end(lps_plan* plan, const float* rec, lps_stats* stats);

/* Adjoint operator E^H without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they need the
 * operator -- code running while another component owns the device memory pool, real-time
 * loops that forbid allocation after start-up, callers that must not risk the device-wide
 * synchronisation an allocation can cause. It needs no plan and calls no allocating routine:
 * its scratch (line table, twiddles, samples moved to hybrid space) is one file-scope device
 * array of LPS_NOALLOC_SCRATCH_BYTES, reserved on every GPU that loads the library until the
 * process exits. Sizes whose scratch would exceed it return LPS_ERR_UNSUPPORTED.
 *   mask   host   uint8 [nz][ny] (nonzero = sampled), as for lps_set_mask
 *   coils  device complex64 [ncoil][nz][nx][ny]
 *   kdata  device complex64 [ncoil][nlines][nx], nlines = set entries of mask
 *   image  device complex64 [nz][nx][ny], written
 *   stream cudaStream_t (NULL = legacy default stream); the work is enqueued there.
 * coils, kdata or image not in device memory, or a mask in device memory, is
 * LPS_ERR_INVALID_ARG (checked on the host before anything is enqueued), as are a mask with no
 * sampled entry and an nlines that differs from the mask's count; lps_last_error() says which.
 * The first call on a device looks up the array's device address once (with that device
 * current); make that first call before any stream capture. All calls share the array and
 * it keeps the last call's contents: calls whose work overlaps on the GPU (other streams or
 * other host threads) race on it and must be ordered by the caller; calls queued one after
 * another on the same stream are ordered and need no synchronisation between them. */
#define LPS_NOALLOC_SCRATCH_BYTES (16u << 20)
int lps_adjoint_noalloc(int nx, int ny, int nz, int ncoil, int fft_z, const uint8_t* mask, const void* coils,
                        const void* kdata, int nlines, void* image, void* stream);

size_t lps_support_words(const lps_params* p);
const char* lps_status_string(int status);
const char* lps_last_error(void);
int lps_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LPS_API_H */
