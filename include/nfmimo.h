/*
 * nfmimo — GB300 (sm_103a) library for regularised 3D near-field MIMO imaging
 * with the stochastic proximal gradient method (SPGM).
 *
 * Paper: O. Oral, "Fast Regularized 3D Near-Field MIMO Imaging Using
 * Stochastic Proximal Gradient Method", arXiv 2509.00774.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex vectors are complex64, interleaved (re, im) float pairs.
 *  - Measurement row m = pair * K + k with pair = t * R + r (TX t, RX r,
 *    frequency k).  A minibatch is a list of pair indices; its rows are the
 *    listed pairs in list order, each with all K frequencies.
 *  - Voxel n = (iz * ny + iy) * nx + ix on the regular grid of nfm_grid.
 *  - Unless an entry point says otherwise, vector pointers are DEVICE pointers
 *    on the context's device, owned by the caller, and the call only enqueues
 *    work on the context's stream (asynchronous).  Pointers must be 8-byte
 *    aligned (complex) or 4-byte aligned (int).
 *  - Return value: NFM_OK (0) or a negative nfm_status.  On error no work has
 *    been enqueued, and nfm_last_error() describes the failure.
 *  - Kernels that meet an out-of-range pair index skip it and raise a device
 *    flag; the next synchronising call (nfm_synchronize, nfm_power_iteration,
 *    nfm_objective, nfm_spgm_epoch_host) returns NFM_ERR_ARG and clears it.
 *  - One context must not be used from two host threads at the same time.
 */
#ifndef NFMIMO_H
#define NFMIMO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nfm_ctx nfm_ctx;

typedef enum {
    NFM_OK = 0,
    NFM_ERR_ARG = -1,      /* invalid argument or geometry */
    NFM_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    NFM_ERR_NOMEM = -3,    /* device allocation failed */
    NFM_ERR_STATE = -4,    /* call order (e.g. no geometry set) */
    NFM_ERR_TIMEOUT = -5,  /* a bounded device wait gave up */
    NFM_ERR_NUMERIC = -6   /* non-finite result */
} nfm_status;

/* Regular voxel grid r_n = (x0 + ix dx, y0 + iy dy, z0 + iz dz) in metres. */
typedef struct {
    double x0, y0, z0;
    double dx, dy, dz;
    int nx, ny, nz;
} nfm_grid;

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream stays owned
 * by the caller.  *out receives the context (library-owned). */
int nfm_create(nfm_ctx** out, int device, void* cuda_stream);

/* Free the context and all device memory it owns.  NULL is ignored. */
void nfm_destroy(nfm_ctx* ctx);

/* Human-readable description of the last error on this context (or of the
 * last failed nfm_create when ctx is NULL).  Library-owned string. */
const char* nfm_last_error(const nfm_ctx* ctx);

/* Replace the stream later calls enqueue on (caller-owned). */
int nfm_set_stream(nfm_ctx* ctx, void* cuda_stream);

/* Geometry of the observation model (Sec. II, Eq. 1-2).
 *   tx_xyz [T][3], rx_xyz [R][3]: HOST FP64 antenna positions (the paper puts
 *     them on z = 0; any z is accepted).
 *   freq_hz [K]: HOST FP64 frequencies, 1 <= K <= 128.  Equally spaced lists use
 *     the phasor-recurrence kernels (and allow the tensor-core adjoint); any
 *     other list uses the general-frequency kernels, which evaluate every
 *     element's phase from FP64 per-(antenna, voxel tile, frequency) tables
 *     (slower; FP32 only; nfm_forward_noalloc rejects such a geometry).
 *   pulse_re_im [K][2]: HOST complex p(f_k), or NULL for p = 1.
 *   grid: the voxel grid (HOST struct).  N = nx ny nz < 2^31.
 *   c: propagation speed (m/s), > 0.
 * Every antenna must lie outside the voxel grid's bounding box, at least
 * 1e-6 m from it (the paper's antennas sit on z = 0 in front of the scene).
 * Copies what it
 * needs (the caller may free its arrays on return), builds the per-(antenna,
 * voxel-tile) FP64 tables on the device and synchronises the stream.
 * Errors: NFM_ERR_ARG (sizes, non-finite values, antenna on a voxel),
 * NFM_ERR_NOMEM, NFM_ERR_CUDA. */
int nfm_set_geometry(nfm_ctx* ctx,
                     const double* tx_xyz, int T,
                     const double* rx_xyz, int R,
                     const double* freq_hz, int K,
                     const double* pulse_re_im,
                     const nfm_grid* grid,
                     double c);

/* Geometry with explicit voxel positions (Sec. II, Eq. 2: the r_n are any set
 * of points), otherwise as nfm_set_geometry.
 *   vox_xyz [n_vox][3]: HOST FP64 voxel positions r_n; voxel n is entry n of
 *     the reflectivity vector s (and of g).  1 <= n_vox <= 2^31 - 129.
 * The operator groups the voxels in runs of 128 consecutive entries (n / 128)
 * and expands the frequency dependence about each run's bounding-box centre,
 * so the voxels should be ordered so that each run of 128 is spatially compact
 * (for example 8 x 4 x 4 blocks of a jittered grid); a run whose path-length
 * spread needs more than 32 expansion terms makes this call fail with
 * NFM_ERR_ARG.  Every antenna must lie at least 1e-6 m from every voxel.
 * Supported by the FP32 expansion operator: frequencies must be equally
 * spaced; the direct recurrence, the tensor-core precision modes, the
 * allocation-free forward and the group term of the regulariser need a
 * regular grid and return NFM_ERR_ARG.  Copies what it needs, synchronises.
 * Errors: NFM_ERR_ARG, NFM_ERR_NOMEM, NFM_ERR_CUDA. */
int nfm_set_geometry_points(nfm_ctx* ctx,
                            const double* tx_xyz, int T,
                            const double* rx_xyz, int R,
                            const double* freq_hz, int K,
                            const double* pulse_re_im,
                            const double* vox_xyz, long long n_vox,
                            double c);

/* Sizes of the current geometry (any pointer may be NULL). */
int nfm_dims(const nfm_ctx* ctx, int* T, int* R, int* K, long long* N);

/* Arithmetic of the adjoint A_B^H r (and of every call that contains it:
 * nfm_adjoint, SPGM/PGM steps and epochs, nfm_solve, power iteration,
 * lambda_max):
 *   NFM_FP32       CUDA-core FP32 (default),
 *   NFM_TC_BF16X3  5th-generation tensor cores, operands split x = hi + lo in
 *                  BF16 and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated
 *                  in FP32 (relative error ~1e-5),
 *   NFM_TC_FP16X3  the same with FP16 halves and the residual scaled per pair
 *                  by a power of two (relative error ~1e-6).
 * With the Chebyshev expansion in use (see nfm_set_algorithm) the tensor cores
 * run the adjoint's coefficient contraction C[(tile, pair), l] = sum_k r'_k b_l(k)
 * and the per-voxel Chebyshev sum stays FP32; otherwise they run the
 * frequency-split phasor GEMM.  The forward operator is FP32 in every mode.
 * Errors: NFM_ERR_ARG. */
enum { NFM_FP32 = 0, NFM_TC_BF16X3 = 1, NFM_TC_FP16X3 = 2 };
int nfm_set_precision(nfm_ctx* ctx, int mode);

/* How the FP32 CUDA-core operator evaluates the frequency dependence of Eq. 2
 * for equally spaced frequencies f_k = f0 + k df:
 *   NFM_ALGO_DIRECT     every (row, voxel) term from phasor recurrences over k;
 *   NFM_ALGO_CHEBYSHEV  per (pair, 8x4x4 voxel tile) the factor
 *                       exp(-j 2 pi (k - k_c) df delta/c), delta = D - D_tile_centre,
 *                       k_c = (K - 1)/2 the band centre (the phase
 *                       2 pi (f_0 D_c + f_c delta)/c is evaluated directly),
 *                       is expanded in Chebyshev polynomials of
 *                       t = delta / xi (|t| <= 0.95):
 *                         exp(-j z_k t) = sum_{l<L} (-j)^l b_l(z_k) T_l(t),
 *                       b_0 = J_0, b_l = 2 J_l (Jacobi-Anger), L even in
 *                       [10, 32] chosen at nfm_set_geometry so the dropped tail
 *                       is below 2e-6 at the band edges; per (pair, voxel) the work is
 *                       L recurrence steps instead of K terms (relative error ~2e-6,
 *                       as DIRECT);
 *   NFM_ALGO_AUTO       CHEBYSHEV where the geometry allows it (L <= 32), else
 *                       DIRECT (default).
 * Arbitrary frequency lists always use their own kernels; the tensor-core
 * adjoint modes keep their own generation.  Requesting CHEBYSHEV where L would
 * exceed 32 makes the operator calls fail with NFM_ERR_ARG. */
enum { NFM_ALGO_AUTO = 0, NFM_ALGO_DIRECT = 1, NFM_ALGO_CHEBYSHEV = 2 };
int nfm_set_algorithm(nfm_ctx* ctx, int algo);

/* Which algorithm the operator uses for the current geometry and setting
 * (NFM_ALGO_DIRECT or NFM_ALGO_CHEBYSHEV), the expansion length L (0 if the
 * expansion is not available) and the largest |z_k| (the band edges).  Any pointer
 * may be NULL.  Errors: NFM_ERR_STATE without a geometry. */
int nfm_algorithm_info(nfm_ctx* ctx, int* algo_in_use, int* n_terms, double* z_max);

/* The expansion the FP32 expansion operator (forward and adjoint) uses on this
 * geometry.  On a regular grid with at least as many blocks as the GPU has SMs
 * it runs over blocks of two tiles along z (8 x 4 x 8 voxels) with their own
 * expansion of n_terms terms.  Otherwise (smaller grids, explicit voxel
 * positions, or a span that needs more terms than the block kernels are built
 * for) it runs over the 8 x 4 x 4 tiles, with the length
 * nfm_algorithm_info reports.  The tensor-core modes and the fused batch
 * always use the tiles.  Writes the expansion length and the voxels per block
 * (256 or 128); 0 terms if the expansion is not available.  Any pointer may be
 * NULL.  Errors: NFM_ERR_STATE without a geometry. */
int nfm_expansion_info(nfm_ctx* ctx, int* n_terms, int* block_voxels);

/* Autotuner (no counterpart in the paper) for minibatches of n_pairs pairs of
 * the current geometry.  Every candidate launch shape of the expansion
 * forward (4 or 8 lanes per (pair, tile), 64 or 128 threads per CTA, 4..32
 * pairs per CTA, one, two or four waves of tile chunks, and one wave of
 * (occupancy - 1) or occupancy CTAs on every SM with chunks that may be
 * shorter than a stage of tiles) is timed on a whole
 * operator step as SPGM runs it (forward + residual + adjoint; pairs
 * 0..n_pairs-1, a zero scene, one warm-up and six timed steps), because the
 * shape also decides how the dependent launches overlap; the three fastest are
 * timed again twice over twelve steps and the lowest time decides.
 * With NFM_ALGO_AUTO the same step with the direct recurrence is timed too
 * and the faster algorithm is kept for every later call with n_pairs pairs.
 * The choice changes the order of the FP32 sums, so results are reproducible
 * for a given choice, not across choices; contexts that are never tuned use a
 * fixed default.  Synchronises the stream.  Writes the chosen algorithm
 * (NFM_ALGO_CHEBYSHEV or NFM_ALGO_DIRECT) and forward shape (any pointer may
 * be NULL).  Errors: NFM_ERR_ARG (n_pairs outside [1, P]), NFM_ERR_STATE (no
 * geometry, or the expansion is not in use). */
int nfm_autotune(nfm_ctx* ctx, int n_pairs, int* algorithm, int* threads, int* lanes_per_group, int* pairs_per_cta,
                 int* chunks);

/* Apply a forward launch shape for minibatches of n_pairs pairs without
 * timing anything (for example one that nfm_autotune returned in an earlier
 * run): threads 64 or 128, lanes_per_group 4 or 8, pairs_per_cta a power of
 * two in [4, threads / lanes_per_group], chunks in [1, number of 8x4x4 voxel
 * tiles].  algorithm NFM_ALGO_DIRECT keeps the direct recurrence for that
 * minibatch size under NFM_ALGO_AUTO (the shape is then ignored).  Replaces
 * any earlier shape for n_pairs.  Errors: NFM_ERR_ARG (a value outside those
 * ranges, n_pairs outside [1, P], or a shape that needs more shared memory
 * than the device has), NFM_ERR_STATE (no geometry, or the expansion is not
 * available). */
int nfm_set_forward_shape(nfm_ctx* ctx, int n_pairs, int algorithm, int threads, int lanes_per_group,
                          int pairs_per_cta, int chunks);

/* Host-only helper (no GPU needed): the expansion coefficients
 * out[k*L + l] = b_l((k - k_center) z_step), l < L, k < K, of
 *   exp(-j z t) = sum_l (-j)^l b_l(z) T_l(t)   (b_0 = J_0(z), b_l = 2 J_l(z)),
 * computed in FP64 by Chebyshev-Gauss quadrature with 2L + 64 nodes.  The
 * operator's table is this one with k_center = (K - 1)/2.
 * Errors: NFM_ERR_ARG for K < 1, L outside [1, 256], NULL out, non-finite
 * z_step or k_center. */
int nfm_cheb_coefficients(double z_step, double k_center, int K, int L, double* out);

/* Regulariser of Eq. 3 (Sec. III uses l1 and notes the method extends to
 * other functionals): R(s) = w1 ||s||_1 + (w2/2) ||s||_2^2 (elastic net;
 * default w1 = 1, w2 = 0, the paper's l1; w1 = 0 is Tikhonov).  Its prox,
 * used by every SPGM/PGM step, is
 *   prox(z) = z max(0, 1 - eta lambda w1/|z|) / (1 + eta lambda w2),
 * and nfm_objective adds lambda R(s).  Weights finite, >= 0, not both 0. */
int nfm_set_regularizer(nfm_ctx* ctx, double w1, double w2);

/* Group term of the regulariser (Sec. III allows other convex functionals; default
 * w3 = 0, off): R(s) += w3 sum_g ||s_g||_2 over the 2 x 2 x 1 voxel blocks
 * g = (ix/2, iy/2, iz) (blocks at an odd grid edge hold fewer voxels).  The prox
 * used by every SPGM/PGM step is then the soft threshold at eta lambda w1, the
 * block shrink u_g max(0, 1 - eta lambda w3/||u_g||), and the 1/(1 + eta lambda w2)
 * scaling (the prox of the sparse-group penalty); nfm_objective adds lambda w3
 * sum_g ||s_g|| (FP64).  Steps with w3 > 0 need the Chebyshev-expansion operator
 * (equally spaced frequencies, algorithm auto or chebyshev; FP32 or tensor-core
 * precision) and fail with NFM_ERR_ARG otherwise.  Errors: NFM_ERR_ARG for a
 * negative or non-finite w3. */
int nfm_set_group_weight(nfm_ctx* ctx, double w3);

/* Minibatch forward operator y = A_B s (Eq. 2 rows of the listed pairs).
 *   pairs [n_pairs] int32 (device), s [N] complex64, y [n_pairs*K] complex64.
 * y must not alias s.  Uses library-owned scratch (allocated on first need). */
int nfm_forward(nfm_ctx* ctx, const int* pairs, int n_pairs, const float* s, float* y);

/* Minibatch residual r = A_B s - y_B (the residual inside Eq. 4 and the gradient
 * of Eq. 6): the forward of nfm_forward with the listed pairs' rows of the FULL
 * measurement vector y [P*K] subtracted in the same kernel (no gather pass).
 *   pairs [n_pairs] int32, s [N], y [P*K], r [n_pairs*K] complex64 (device);
 *   r must not alias s or y. */
int nfm_residual(nfm_ctx* ctx, const int* pairs, int n_pairs, const float* s, const float* y, float* r);

/* Minibatch adjoint g = A_B^H r, the operator inside the gradient of Eq. 4/6.
 *   pairs [n_pairs] int32 (device), r [n_pairs*K] complex64, g [N] complex64. */
int nfm_adjoint(nfm_ctx* ctx, const int* pairs, int n_pairs, const float* r, float* g);

/* One SPGM iteration (Sec. IV Eq. 5 with the minibatch gradient of Eq. 6):
 *   s <- prox_{eta*lambda ||.||_1}( s - (eta/B) A_B^H (A_B s - y_B) ),
 * B = n_pairs*K rows; y is the FULL measurement vector [P*K] (device),
 * s [N] is updated in place.  prox(z) = z max(0, 1 - alpha/|z|). */
int nfm_spgm_step(nfm_ctx* ctx, const float* y, float* s, const int* pairs, int n_pairs,
                  float eta, float lambda);

/* One SPGM epoch (Sec. IV-A, Eq. 6, iterated by Eq. 5): the P pair indices in
 * perm [P] (device) are taken in consecutive chunks of pairs_per_batch (the
 * last chunk may be shorter and uses its own B) and nfm_spgm_step runs on each
 * chunk in order, so every pair's rows enter one minibatch gradient per epoch
 * (the paper draws the minibatch index uniformly; the caller supplies the
 * draws as the permutation).  y [P*K], s [N] (in place), perm [P]: device.
 * Errors: NFM_ERR_ARG (pairs_per_batch outside [1, P], bad pointers). */
int nfm_spgm_epoch(nfm_ctx* ctx, const float* y, float* s, const int* perm, int pairs_per_batch,
                   float eta, float lambda);

/* Same as nfm_spgm_epoch (Sec. IV-A, Eq. 6) for n_epochs epochs, but y_host [P*K], s_host [N]
 * (in/out) and perms_host [n_epochs][P] are HOST buffers: the call copies
 * them to library-owned device buffers, runs, copies s back and synchronises.
 * Pinned host memory makes the copies asynchronous-capable and faster. */
int nfm_spgm_epochs_host(nfm_ctx* ctx, const float* y_host, float* s_host, const int* perms_host,
                         int n_epochs, int pairs_per_batch, float eta, float lambda);

/* SPGM iteration on a Cartesian minibatch (Sec. IV-A: B = #f x #Tx x #Rx
 * rows): the rows of the listed pairs at the frequencies k with
 * freq_mask[k] != 0 (device uint8 [K]; n_freq = number of nonzero entries, so
 * B = n_pairs * n_freq).  The forward runs over all K frequencies of the pairs
 * and the residual of unselected rows is set to 0, so the adjoint is exactly
 * A_B^H (A_B s - y_B).  For the paper's composition pass the pairs of #Tx
 * transmitters x #Rx receivers. */
int nfm_spgm_step_freqs(nfm_ctx* ctx, const float* y, float* s, const int* pairs, int n_pairs,
                        const unsigned char* freq_mask, int n_freq, float eta, float lambda);

/* One full-batch PGM iteration (Sec. IV, Eq. 5): nfm_spgm_step with every
 * pair in index order, B = M rows.  y [P*K], s [N] (in place), device. */
int nfm_pgm_step(nfm_ctx* ctx, const float* y, float* s, float eta, float lambda);

/* SPGM with the termination rule of Sec. V: run epochs e = 0, 1, ... with the
 * permutation perms + e*P (device [max_epochs][P]) until the change in
 * reflectivity magnitudes over one epoch, max_n | |s_n(after)| - |s_n(before)| |
 * (FP64), drops below tol, or max_epochs epochs have run.  pairs_per_batch = P
 * with identity permutations is PGM.  Synchronises once per epoch to read the
 * statistic.  Writes *epochs_out (epochs run) and *change_out (last change). */
int nfm_solve(nfm_ctx* ctx, const float* y, float* s, const int* perms, int max_epochs, int pairs_per_batch,
              float eta, float lambda, double tol, int* epochs_out, double* change_out);

/* Gradient step and prox of Eq. 5 as a separate op (used by unrolled SPGM):
 *   out = shrink prox_alpha(s - step g),  prox(z) = z max(0, 1 - alpha/|z|),
 * shrink = 1 for the paper's l1 and 1/(1 + eta lambda w2) for the elastic net
 * R = w1 ||s||_1 + (w2/2) ||s||^2 (alpha = eta lambda w1).
 * s, g, out: device complex64 [n] (out may alias s).  Errors: NFM_ERR_ARG for
 * alpha < 0, shrink <= 0 or non-finite scalars. */
int nfm_prox_step(nfm_ctx* ctx, const float* s, const float* g, float step, float alpha, float shrink, long long n,
                  float* out);

/* Backward of nfm_prox_step for a real loss, with complex gradients as real
 * pairs (d/dRe + j d/dIm, the PyTorch convention).  grad_out [n] is the
 * gradient of the output; writes grad_s [n] and grad_g [n] (either may be
 * NULL) and, to the device buffer grad_scalars [3] (FP64), dL/dstep,
 * dL/dalpha and dL/dshrink.  All pointers device. */
int nfm_prox_step_backward(nfm_ctx* ctx, const float* s, const float* g, float step, float alpha, float shrink,
                           long long n, const float* grad_out, float* grad_s, float* grad_g, double* grad_scalars);

/* The same op with the group term of the sparse-group regulariser (Sec. III
 * allows any convex regulariser with a cheap prox; Eq. 5 with
 * R = w1 ||s||_1 + (w2/2) ||s||^2 + w3 sum_b ||s_b||_2):
 *   u = prox_alpha(s - step g),
 *   out_v = shrink u_v max(0, 1 - alpha_g / ||u_b||_2),
 * where b is the 2 x 2 x 1 voxel block (ix/2, iy/2, iz) of the context's grid that holds voxel v.
 * Blocks at an odd grid edge hold fewer voxels.  alpha = eta lambda w1, alpha_g = eta lambda w3,
 * shrink = 1/(1 + eta lambda w2).  The prox of the whole penalty is the soft threshold, then the
 * block shrink, then the scaling.
 * s, g, out: device complex64 [N] in the grid's x-fastest order (out may alias s).
 * Errors: NFM_ERR_STATE without geometry or with explicit voxel positions (no grid blocks);
 * NFM_ERR_ARG for alpha < 0, alpha_g < 0, shrink <= 0 or non-finite scalars. */
int nfm_prox_group_step(nfm_ctx* ctx, const float* s, const float* g, float step, float alpha, float alpha_g,
                        float shrink, float* out);

/* Backward of nfm_prox_group_step for a real loss (complex gradients as real
 * pairs, as nfm_prox_step_backward).  grad_out [N] is the gradient of the output;
 * writes grad_s [N] and grad_g [N] (either may be NULL) and, to the device
 * buffer grad_scalars [4] (FP64), dL/dstep, dL/dalpha, dL/dalpha_g and
 * dL/dshrink.  All pointers device; errors as nfm_prox_group_step. */
int nfm_prox_group_step_backward(nfm_ctx* ctx, const float* s, const float* g, float step, float alpha, float alpha_g,
                                 float shrink, const float* grad_out, float* grad_s, float* grad_g,
                                 double* grad_scalars);

/* Batched solves of many independent scenes (uneven grids, arrays and K):
 * Sec. IV-A, Eq. 6 with Eq. 5, applied to every scene independently.
 * A batch holds n_scenes contexts (each with its own geometry, set by
 * nfm_set_geometry; the batch does not own them) and enqueues on cuda_stream
 * (caller-owned; NULL = legacy default stream).  nfm_batch_spgm_epoch runs one
 * SPGM epoch of every scene: scene i uses y[i] [P_i*K_i], s[i] [N_i] (in
 * place), perm[i] [P_i] (all device pointers), pairs_per_batch[i], eta[i],
 * lambda[i] (host arrays of length n_scenes).  The first call captures the
 * epochs of all scenes into one CUDA graph with one concurrent branch per
 * scene and later calls replay it while every pointer and parameter is the
 * same as in the captured call (the contents of y, s and perm may change);
 * any change re-captures.  Profiling must be off in the scene contexts.
 * Errors: NFM_ERR_ARG, NFM_ERR_STATE (a scene without geometry), NFM_ERR_CUDA. */
typedef struct nfm_batch nfm_batch;
int nfm_batch_create(nfm_batch** out, nfm_ctx* const* scenes, int n_scenes, void* cuda_stream);
void nfm_batch_destroy(nfm_batch* batch);
int nfm_batch_spgm_epoch(nfm_batch* batch, const float* const* y, float* const* s, const int* const* perm,
                         const int* pairs_per_batch, const float* eta, const float* lambda);
const char* nfm_batch_last_error(const nfm_batch* batch);

/* How nfm_batch_spgm_epoch runs the scenes (the next call re-captures):
 *   NFM_BATCH_BRANCHES (default): the graph holds one concurrent branch per
 *     scene, each the scene's own launches (any operator, precision or
 *     algorithm the scene is set to);
 *   NFM_BATCH_FUSED: for each step index t of the epoch, one launch of the
 *     expansion forward, one of the chunk reduction and one of the expansion
 *     adjoint cover every scene that still has a minibatch at t (each CTA
 *     finds its scene in a table), so an epoch is 3 max_i ceil(P_i/B_i)
 *     launches whatever the number of scenes.  Needs every scene on the FP32
 *     expansion operator with L <= 20; the scenes share the largest L (the
 *     others' coefficient tables are padded with zero columns, which leaves
 *     their results unchanged).
 * Errors: NFM_ERR_ARG for another mode (and, at the next epoch, for scenes the
 * fused mode cannot run). */
enum { NFM_BATCH_BRANCHES = 0, NFM_BATCH_FUSED = 1 };
int nfm_batch_set_mode(nfm_batch* batch, int mode);

/* Largest eigenvalue L of A^H A / M by `iters` power iterations from
 * v0 [N] (device, complex64, not modified), with FP64 norms.  L is the
 * Lipschitz constant of the gradient of D(s) = ||y - A s||^2/(2M) (Eq. 4); the
 * paper states its step eta without saying how it was found, and the step
 * eta = 1/L used here is not in the paper (a standard choice for Eq. 5).
 * The iteration:
 *   v <- A^H A v / ||A^H A v||, then L = ||A v||^2 / (M ||v||^2).
 * Writes *L_out (host) and synchronises.  The SPGM step is eta = 1/L. */
int nfm_power_iteration(nfm_ctx* ctx, int iters, const float* v0, double* L_out);

/* The same for the minibatch of the listed pairs (Sec. IV-A, Eq. 6): the
 * largest eigenvalue L_B of A_B^H A_B / B, B = n_pairs * K, the Lipschitz
 * constant of the minibatch gradient (1/B) A_B^H (A_B s - y_B).  An SPGM step
 * is stable only where eta < 2 / L_B for every minibatch it takes, and L_B can
 * exceed the full-batch L several times (a few pairs see the scene from one
 * viewpoint), so a step of 1/L that suits PGM can make SPGM diverge.
 * pairs [n_pairs] int32 (device), v0 [N] (device, not modified).  Writes
 * *L_out (host) and synchronises.  Errors: NFM_ERR_ARG (n_pairs < 1, bad
 * pointers), NFM_ERR_NUMERIC. */
int nfm_power_iteration_pairs(nfm_ctx* ctx, const int* pairs, int n_pairs, int iters, const float* v0,
                              double* L_out);

/* Objective of Eq. 3 with Eq. 4 and the regulariser, accumulated in FP64:
 *   F(s) = ||y - A s||^2 / (2M) + lambda R(s)   (R = sum_n |s_n| by default).
 * y [P*K], s [N] device.  Writes *F_out (host) and synchronises. */
int nfm_objective(nfm_ctx* ctx, const float* y, const float* s, double lambda, double* F_out);

/* lambda_max = max_n |(A^H y)_n| / M (FP64 result on the host; synchronises):
 * for lambda >= lambda_max the l1 problem of Eq. 3 has s = 0 as a solution
 * (its optimality condition at s = 0; the paper does not state it). */
int nfm_lambda_max(nfm_ctx* ctx, const float* y, double* out);

/* Wait for the context's stream and report device-side flags. */
int nfm_synchronize(nfm_ctx* ctx);

/* Test hooks for the error paths (no counterpart in the paper).  Every wait of
 * the tensor-core kernels on their MMA completion barrier is bounded by
 * wait_ms milliseconds of the GPU's global timer (0 = the default, 1000 ms).
 * When one runs out the kernel stops issuing MMAs, reads no tensor memory,
 * waits once more (bounded) for the MMAs it had committed, releases its tensor
 * memory, raises a device flag and leaves its output (the iterate s, or g)
 * unwritten; the next synchronising call returns NFM_ERR_TIMEOUT and the
 * context stays usable.  flags = NFM_HOOK_TC_SKIP_ISSUE makes those kernels
 * issue no MMA and no commit, so that their first wait runs out on purpose
 * (nothing is left in flight); flags = NFM_HOOK_SHRINK_EXTENTS halves the
 * buffer extents the kernels of the default operator path receive, which only
 * the bounds-checked build (libnfmimo_check.so, compiled with
 * -DNFM_BOUNDS_CHECK) reads: there a checked index past the declared extent
 * raises a device flag and is replaced by 0 (an element inside the real
 * buffer), and the next synchronising call returns NFM_ERR_STATE;
 * flags = 0 is normal operation.  Applies to calls enqueued afterwards.  Errors: NFM_ERR_ARG for unknown flags or
 * wait_ms outside [0, 60000]. */
enum { NFM_HOOK_TC_SKIP_ISSUE = 1, NFM_HOOK_SHRINK_EXTENTS = 2 };
int nfm_set_test_hooks(nfm_ctx* ctx, int flags, int wait_ms);

/* Allocation-free variant of nfm_forward.  The paper has no counterpart; this
 * entry point exists for callers that cannot call cudaMalloc once they are
 * running: a reconstruction loop with a fixed device-memory budget that must
 * not grow after start-up, a process whose device memory is handed out by
 * another allocator, or a latency-bound caller that cannot accept the device
 * synchronisation cudaMalloc/cudaFree can imply.  nfm_forward keeps its chunk
 * partial sums in library-owned scratch that grows with cudaMalloc; this call
 * keeps them instead in one statically sized device array that is part of the
 * loaded library (4 MiB, held on every GPU that loads the library until the
 * process exits), and it allocates nothing.
 *   Arguments, layout and result are those of nfm_forward (y = A_B s).
 *   Limit: ceil(n_pairs / 8) * 8 * K <= 524288 (the scratch holds 524288
 *   complex64 partial sums and one voxel chunk needs that many, the pairs
 *   padded to whole groups of 8; fewer voxel chunks are used when the usual
 *   plan does not fit).  A larger request returns NFM_ERR_ARG and enqueues
 *   nothing.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   All calls in the process share the one array per device and it keeps the
 *   previous call's contents; every partial sum a call reads is written by the
 *   same call, so nothing has to start at zero.  Calls whose work overlaps on
 *   the GPU (different streams or contexts on one device) race on the array
 *   and give wrong results: order them, e.g. on one stream. */
int nfm_forward_noalloc(nfm_ctx* ctx, const int* pairs, int n_pairs, const float* s, float* y);

/* Kernel timing (tracing aid, not part of the paper's method).  While enabled,
 * every kernel the operator entry points enqueue is bracketed by a pair of
 * CUDA events on the context stream.  nfm_profile_report synchronises, adds up
 * the elapsed times per kernel kind since the last report and resets them:
 *   ms_out[i], launches_out[i] for i < n_kinds (host arrays), kinds:
 *   0 = forward partial sums, 1 = forward chunk reduction (+ residual),
 *   2 = adjoint (+ gradient step and prox), 3 = FP64 reductions. */
#define NFM_PROFILE_KINDS 4
int nfm_profile_enable(nfm_ctx* ctx, int enable);
int nfm_profile_report(nfm_ctx* ctx, double* ms_out, long long* launches_out, int n_kinds);

#ifdef __cplusplus
}
#endif

#endif /* NFMIMO_H */
