/*
 * segsalsa_str.h -- C ABI of the GB300 (sm_103a) SegSALSA-STR solver.
 *
 * SegSALSA-STR (Condessa, Bioucas-Dias, Kovacevic, arXiv 1504.07028) computes the marginal MAP
 * hidden field z of problem (7),
 *
 *     min_z  sum_i -ln(p_i^T z_i) + lambda sum_i ||[J z]_i||_{S_p}   s.t. z >= 0, 1_K^T z = 1,
 *
 * by the SALSA/ADMM iteration (12)-(14) on the split G = [I; J; I; I] of eqs. (9)-(11):
 * a linear z-update with G^T G = 3 I + J^T J (cyclic convolutions, Sec. 4), the Moreau
 * proximity operators of g1..g4 (eq. 10, Sec. 4), and the scaled dual update (14). J is the
 * patch-based Jacobian of eq. (4): for a (2M+1)x(2M+1) patch (L = (2M+1)^2 shifts), [Jz]_i is
 * the (L K) x 2 matrix of weighted shifted horizontal / vertical forward differences.
 *
 * Conventions shared by every entry point
 *  - Every call returns an int status (segsalsa_status); 0 is success. The message of the
 *    last failure on a handle is available from segsalsa_str_last_error().
 *  - Arguments are checked on the host before any launch. A failed check changes no state.
 *  - Element type: a handle created with precision SEGSALSA_FP32 takes and returns float
 *    arrays; SEGSALSA_FP64 takes and returns double arrays (the `const void*` / `void*`
 *    arguments below). Labels are always int32.
 *  - on_device = 1 means the pointer is device memory of the handle's device (for instance a
 *    torch tensor's data_ptr()); 0 means host memory (pageable or pinned). Copies to and from
 *    host memory are synchronous with respect to the call.
 *  - Device work runs on the handle's stream: the stream given at creation (borrowed, never
 *    destroyed) or a stream the library creates. Calls return after their work has completed
 *    on that stream unless stated otherwise.
 *  - Device-memory arguments must be ready when the call is made: the handle's stream does not
 *    wait for work the caller queued on other streams (synchronize or order them first).
 *  - A handle is not thread-safe; separate handles are independent.
 *  - Periodic boundary conditions and forward differences throughout (the cyclic
 *    convolutions of Sec. 4).
 *
 * Layouts
 *  - SEGSALSA_LAYOUT_KHW: class-major (K, H, W), the paper's K x n hidden field.
 *  - SEGSALSA_LAYOUT_HWK: pixel-major (H, W, K), the library's own layout.
 *  - Internal state arrays exposed by get_state / set_state are pixel-major:
 *    z, d1, d3, d4, rhs: (H, W, K); d2: (H, W, L, K, 2) with shift j row-major over
 *    (dy, dx) in [-M, M]^2 and the last axis (horizontal, vertical) difference.
 */
#ifndef SEGSALSA_STR_H
#define SEGSALSA_STR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct segsalsa_str segsalsa_str_t; /* opaque; owned by the library */

typedef enum {
  SEGSALSA_OK = 0,
  SEGSALSA_ERR_ARG = -1,     /* invalid argument; nothing was changed */
  SEGSALSA_ERR_OOM = -2,     /* device allocation failed or workspace too small */
  SEGSALSA_ERR_CUDA = -3,    /* a CUDA runtime call failed; the message names it */
  SEGSALSA_ERR_NUMERIC = -4, /* non-finite values appeared in the iterates */
  SEGSALSA_ERR_TIMEOUT = -5, /* a bounded device-side wait gave up (see set_wait_budget) */
  SEGSALSA_ERR_STATE = -6    /* call out of order (e.g. solve before set_probs) */
} segsalsa_status;

enum { SEGSALSA_FP32 = 0, SEGSALSA_FP64 = 1 };
enum { SEGSALSA_LAYOUT_KHW = 0, SEGSALSA_LAYOUT_HWK = 1 };
enum { SEGSALSA_SCHATTEN_INF = 0 }; /* schatten_p value meaning p = infinity */
enum { SEGSALSA_G4_AFFINE = 0, SEGSALSA_G4_SIMPLEX = 1 }; /* segsalsa_str_set_g4 modes */

/* Problem statement of eq. (7) and the SALSA penalty of eq. (13). */
typedef struct {
  int32_t H, W;          /* image size; H, W >= 2M+2. The row transform length (W when its
                            prime factors are at most 103, else the Bluestein length, a
                            7-smooth length >= 2W - 1) must be <= 8192, so W <= 8192 for such
                            W and about W <= 4096 otherwise; the column solve holds H rows of
                            a complex column in shared memory: H <= 25600 (FP32), 12800
                            (FP64). SEGSALSA_ERR_ARG outside these limits.                 */
  int32_t K;             /* number of classes, 2 <= K <= 32                               */
  int32_t M;             /* patch half-width: (2M+1)x(2M+1) patch, 0 <= M <= 5 (1x1 up to
                            the 11x11 patch of Sec. 5's patch-size study). M = 0 is the 1x1
                            patch, i.e. SegSALSA with the VTV prior (Sec. 3). M <= 2 runs the
                            fused one-launch sweep; M >= 3 a three-launch sweep that keeps the
                            prior's dual as the last prox argument and a 2x2 matrix per pixel
                            (get_state writes d2 itself) and needs a second d2-sized scratch
                            buffer (see workspace_bytes)                                    */
  const double* weights; /* L = (2M+1)^2 shift weights omega_j (row-major over (dy, dx)),
                            host memory, copied at creation; NULL selects the Gaussian
                            omega_j = sqrt(g_j), g_j = exp(-|s_j|^2/(2 sigma^2)) / sum        */
  double sigma;          /* Gaussian bandwidth used when weights == NULL, > 0               */
  double lambda;         /* prior weight lambda of eq. (7), >= 0                            */
  double mu;             /* ADMM penalty mu of eq. (13), > 0                                */
  int32_t schatten_p;    /* 1, 2, or SEGSALSA_SCHATTEN_INF (Sec. 3 norm, Sec. 4 MPO of g2)  */
  int32_t precision;     /* SEGSALSA_FP32 or SEGSALSA_FP64                                  */
  void* stream;          /* cudaStream_t to run on (borrowed), or NULL for a library stream */
} segsalsa_str_params;

/* Device bytes a handle with these parameters needs when the caller provides the memory.
 * Returns SEGSALSA_ERR_ARG for invalid parameters. */
int segsalsa_str_workspace_bytes(const segsalsa_str_params* params, size_t* bytes);

/* Create a solver handle. If `workspace` is non-NULL it must be device memory of at least
 * segsalsa_str_workspace_bytes() bytes, 256-byte aligned, owned by the caller and kept alive
 * until destroy; otherwise the library allocates (and later frees) its own. The handle uses
 * the current CUDA device. On failure *out is set to NULL. */
int segsalsa_str_create(const segsalsa_str_params* params, void* workspace,
                        size_t workspace_bytes, segsalsa_str_t** out);

/* Set the class probabilities p_i of eq. (7) and reset the iteration: z^0 = p_i / 1^T p_i,
 * u^0 = G z^0, d^0 = 0 (iteration counter 0). p has H*W*K elements in `layout`. Every entry
 * must be finite and >= 0 and every pixel needs a positive entry, so that p_i^T z_i > 0 is
 * reachable (Sec. 4, feasible set of eq. 7); otherwise SEGSALSA_ERR_ARG and nothing changes.
 * p need not sum to one: the iterates are invariant to a positive per-pixel scale of p. */
int segsalsa_str_set_probs(segsalsa_str_t* h, const void* p, int32_t layout, int32_t on_device);

/* Run `iters` >= 0 SALSA iterations (12)-(14), continuing from the current state.
 * If `trace` is non-NULL (host memory), every `trace_every` iterations (and after the last
 * one) a record of 6 doubles is written:
 *   (k, primal residual ||G z^k - u^k||, dual residual mu ||G^T (u^k - u^{k-1})||,
 *    objective (7) at the simplex projection of z^k, min z^k, max_i |1^T z_i^k - 1|)
 * The caller provides room for floor(iters / trace_every) + 1 records; *n_records (nullable)
 * receives the count. trace_every must be >= 1 when trace is non-NULL. The stopping rule of
 * Sec. 4 (residuals below a threshold) is left to the caller: the solver runs a fixed count.
 * Returns SEGSALSA_ERR_NUMERIC if non-finite values appear in a traced record. */
int segsalsa_str_solve(segsalsa_str_t* h, int32_t iters, double* trace, int32_t trace_every,
                       int32_t* n_records);

/* Residual-based stopping (Sec. 4: the iteration stops once the primal and dual residuals are
 * below a threshold). Runs traced blocks of check_every >= 1 iterations (the last block may be
 * shorter) until the record after a block has primal residual <= tol_primal and dual residual
 * <= tol_dual (the residuals of segsalsa_str_solve's trace records), or max_iters >= 0
 * iterations have run. *iters_done (nullable) receives the iterations run by this call;
 * last_record (nullable, host, 6 doubles) the last trace record (NaN if none was written). The
 * tolerances must be finite and >= 0; 0 runs max_iters iterations unless a residual is 0. */
int segsalsa_str_solve_until(segsalsa_str_t* h, int32_t max_iters, double tol_primal,
                             double tol_dual, int32_t check_every, int32_t* iters_done,
                             double* last_record);

/* Bounded device-side waits. The kernels that wait for their own bulk copies (the sweep and
 * the MLR class model) or for the tensor core give up after `cycles` SM clock cycles (default
 * 2e9, about one second), set the handle's error flag, wait once more with the same limit for
 * their copies in flight, release any tensor memory and return; the call then reports
 * SEGSALSA_ERR_TIMEOUT and the CUDA context stays usable. This is a host-side control, not part
 * of the method (the paper has no counterpart). With probe = 1 the next launches arm their
 * first bulk-copy barrier with 16 bytes that no copy delivers, so that those waits run out by
 * construction: a test of the error path that faults and hangs nothing. After a timeout in
 * solve the iterates are undefined (call set_probs or set_state); a timeout in set_spectra
 * keeps the previous p. Drops the handle's captured graphs. SEGSALSA_ERR_ARG if cycles < 1 or
 * probe is not 0 or 1. */
int segsalsa_str_set_wait_budget(segsalsa_str_t* h, int64_t cycles, int32_t probe);

/* Which set g4 indicates (eqs. 10-11). SEGSALSA_G4_AFFINE (the default): the affine set
 * {1^T xi = 1} as eq. (10) defines g4, whose MPO is the affine projection. SEGSALSA_G4_SIMPLEX:
 * the probability simplex, whose MPO is the simplex projection, as Sec. 4 describes the MPO of
 * g4. With g3 = i_+ in both, the two splittings constrain z to the same simplex and reach the
 * same minimum of (7) by different iterates. Takes effect from the next iteration; the state is
 * kept. SEGSALSA_ERR_ARG for another mode. */
int segsalsa_str_set_g4(segsalsa_str_t* h, int32_t mode);

/* ------------------------------------------------------------------------------------------
 * Differentiable solver: the gradient of the unrolled iteration (12)-(14).
 * ------------------------------------------------------------------------------------------ */

/* Like set_probs, from log-probabilities: p_i = exp(log p_i - max_k log p_ik) (the iterates do
 * not see a per-pixel scale of p). H*W*K values in `layout`, handle precision. */
int segsalsa_str_set_log_probs(segsalsa_str_t* h, const void* log_p, int32_t layout,
                               int32_t on_device);

/* Change lambda of eq. (7) (finite, >= 0) or the L shift weights omega_j of eq. (4) (host,
 * finite) of an existing handle; the state is kept and the change applies from the next
 * iteration. SEGSALSA_ERR_ARG for invalid values. */
int segsalsa_str_set_lambda(segsalsa_str_t* h, double lambda);
int segsalsa_str_set_weights(segsalsa_str_t* h, const double* weights);

/* Reverse pass. With z^T the field after `iters` >= 1 iterations started from the current p
 * (z^0 = p_i / 1^T p_i, u^0 = G z^0, d^0 = 0) and zbar = dLoss/dz^T (H*W*K values in `layout`),
 * writes dLoss/dlog p (same shape and layout; required), dLoss/dlambda (nullable, host) and
 * dLoss/domega_j (nullable, host, L values). The call runs the forward pass itself, keeping a
 * checkpoint of the state every `checkpoint_every` >= 1 iterations, then walks the iterations
 * backwards, recomputing each segment's states from its checkpoint: the adjoint of the z-update
 * is the z-update itself (G^T G is symmetric), the adjoints of the MPOs of g1..g4 are their
 * Jacobians applied per pixel, and the adjoint of J is J^T. Device memory for the checkpoints
 * and one segment's states is allocated for the call and released before it returns. The
 * handle ends at iteration `iters`, as after set_probs + solve(iters).
 * Covers Schatten p = 1, 2 and infinity, g4 on the affine set or on the probability simplex
 * (set_g4), and patches up to 5x5 (M <= 2); SEGSALSA_ERR_ARG for wider patches. The
 * derivative is that of the iteration as written: at points where an MPO switches case (a
 * singular value equal to tau, the two shrunk singular values of p = infinity meeting, a
 * component of v3 equal to 0, a class entering the simplex projection's active set) one
 * side's derivative is taken. */
int segsalsa_str_backward(segsalsa_str_t* h, int32_t iters, const void* zbar, int32_t layout,
                          void* grad_logp, double* grad_lambda, double* grad_weights,
                          int32_t checkpoint_every, int32_t on_device);

/* Label readout argmax_k z_k of every pixel (link p(y_i = k | z_i) = [z_i]_k, Sec. 2; ties to
 * the lowest k), H*W int32 in row-major pixel order. */
int segsalsa_str_get_labels(segsalsa_str_t* h, int32_t* labels, int32_t on_device);

/* Current hidden field z (H*W*K elements in `layout`). */
int segsalsa_str_get_z(segsalsa_str_t* h, void* z, int32_t layout, int32_t on_device);

/* Number of iterations run since the last set_probs / set_state. */
int segsalsa_str_get_iteration(const segsalsa_str_t* h, int32_t* k);

/* Checkpoint: copy out the solver state after k iterations: z^k, d1^k..d4^k and
 * rhs^k = G^T (u^k + d^k) (the right-hand side of the next z-update, eq. 12), in the
 * pixel-major layouts of the header comment. Any pointer may be NULL to skip it. rhs^k is
 * undefined when k = 0 (the next z-update is the identity then). */
int segsalsa_str_get_state(segsalsa_str_t* h, void* z, void* d1, void* d2, void* d3, void* d4,
                           void* rhs, int32_t on_device);

/* Resume: load a state written by get_state (or computed elsewhere) as iteration k >= 0.
 * z, d1..d4 are required; rhs is required when k > 0 and ignored when k = 0. The class
 * probabilities of the last set_probs stay in use. */
int segsalsa_str_set_state(segsalsa_str_t* h, const void* z, const void* d1, const void* d2,
                           const void* d3, const void* d4, const void* rhs, int32_t k,
                           int32_t on_device);

/* The z-update operator alone: z = (3 I + J^T J)^{-1} rhs (eq. 12 with G^T G = 3I + J^T J),
 * rhs and z pixel-major (H, W, K). Leaves the solver state untouched. */
int segsalsa_str_linear_solve(segsalsa_str_t* h, const void* rhs, void* z, int32_t on_device);

/* Class model of the experiments (Sec. 5: the classes are modelled by a multinomial logistic
 * regression, MLR) as the source of p: p_i = softmax_k(w_k^T x_i + b_k), then everything
 * set_probs does (validation, z^0 = p_i, d^0 = 0, iteration counter 0).
 *  - x: H*W*d BF16 values as raw 16-bit patterns, pixel-major (H, W, d); w: K*d BF16 values,
 *    (K, d); bias: K floats, or NULL for zeros. All three in host memory (on_device = 0) or
 *    all in device memory (on_device = 1); they are not kept after the call.
 *  - 1 <= d <= 256 (bands). The contraction runs on the tensor cores (tcgen05, BF16 inputs,
 *    FP32 accumulation), the bias and softmax in FP32; p is stored in the handle's precision.
 *  - Non-finite spectra or weights give non-finite p: SEGSALSA_ERR_ARG, state unchanged.
 *    SEGSALSA_ERR_TIMEOUT if the kernel's bounded wait on the tensor core gave up. */
int segsalsa_str_set_spectra(segsalsa_str_t* h, const void* x, const void* w, const float* bias,
                             int32_t d, int32_t on_device);

/* The class probabilities p of the current solve (set by set_probs or set_spectra), H*W*K
 * elements in `layout`, in the handle's precision. */
int segsalsa_str_get_probs(segsalsa_str_t* h, void* p, int32_t layout, int32_t on_device);

/* Allocation-free z-update. The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory (code running under a fixed memory budget or an outside
 * allocator, or a plug-in without a handle). It solves (3 I + c (D_h^T D_h + D_v^T D_v)) z = rhs
 * with periodic boundaries, which is the z-update operator (3 I + J^T J) of a handle whose shift
 * weights have sum_j omega_j^2 = c_omega (1 for the default normalised Gaussian weights).
 *  - rhs, z: FP32 device memory, pixel-major (H, W, K), owned by the caller; z may not alias rhs.
 *  - Scratch: one file-scope device array (16 MiB spectrum + 512 KiB tables) that every GPU
 *    loading the library holds until exit. Limits: H*(W/2+1)*K <= 2097152, W <= 8192 when W has
 *    no prime factor above 7 and W <= 4096 otherwise, H <= 3200, 2 <= H, W, 1 <= K <= 32.
 *    Sizes beyond them return SEGSALSA_ERR_OOM; other bad arguments SEGSALSA_ERR_ARG.
 *  - No cudaMalloc / cudaFree or other device allocation happens in any call. Every call looks
 *    up the array's device address in the current context (cudaGetSymbolAddress, which
 *    allocates nothing). The first call on a device, and the first call after H, W or c_omega
 *    change or after the device was reset (a new context), builds the tables with two small
 *    kernels on `stream` before the solve; make the first call before any stream capture.
 *  - Runs asynchronously on `stream` (cudaStream_t, NULL = legacy default stream). Calls on one
 *    stream may follow each other with any geometries and no synchronisation in between. Every
 *    call shares the one array, so calls that overlap on the GPU (different streams, other
 *    threads) race; nothing in it needs to start at zero, because each call writes every
 *    spectrum entry it reads. The host-side bookkeeping is locked, but concurrent calls are
 *    still unsupported for that reason. No message is stored: the status code is the error
 *    report. */
int segsalsa_str_linear_solve_static(const float* rhs, float* z, int32_t H, int32_t W, int32_t K,
                                     double c_omega, void* stream);

/* Measurement hooks. set_profiling(1) records CUDA events around each kernel launch of
 * solve() so that kernel_stats() can report, per kernel kind, the launch count and the total
 * device time in milliseconds since the last reset. Kernel kinds (index):
 *   0 fused sweep (prox + dual + rhs partials), 1 row FFT forward (with partial gather),
 *   2 column solve, 3 row FFT inverse, 4 diagnostics (residual / objective), 5 other,
 *   6 MLR class model (set_spectra), 7 reverse-pass kernels (backward), 8 z-update fused
 *   over a thread-block cluster (replaces 1-3 where the tiling selects it).
 * launches and ms point to arrays of at least 9 entries (host memory). kernel_stats works
 * with profiling off too; then ms is not filled. reset_stats zeroes both. */
int segsalsa_str_set_profiling(segsalsa_str_t* h, int32_t on);
int segsalsa_str_kernel_stats(segsalsa_str_t* h, int64_t* launches, double* ms);
int segsalsa_str_reset_stats(segsalsa_str_t* h);

/* Algorithmic device bytes moved by one fused-sweep launch and one full iteration (the
 * minimum traffic model: every array read or written once, no halo or pass overhead). With
 * the affine g4 and patches up to 5x5 the sweep keeps d1 and d4 as one scalar per pixel each
 * (d1 = c1 p, d4 = c4 1, the forms the MPOs of g1 and g4 leave), so the model counts K + 2
 * local-dual values per pixel; with the simplex g4 or 7x7 ... 11x11 patches it counts 3K. */
int segsalsa_str_traffic_model(const segsalsa_str_t* h, double* sweep_bytes,
                               double* iteration_bytes);

/* ------------------------------------------------------------------------------------------
 * Tiling and batches.
 *
 * The paper notes that the whole iteration is per-pixel or per-class independent work apart
 * from the cyclic convolutions (Sec. 4), so many images can share the GPU. A batch runs every
 * image's SALSA iterations (12)-(14) inside one CUDA graph per chunk of iterations: each image's
 * kernels form a chain and the chains of different images run concurrently.
 * ------------------------------------------------------------------------------------------ */

/* Work decomposition of one image. Zero in a field selects the library's default for it. Any
 * tiling gives the same iterates up to the summation order of the rhs partials (FP rounding).
 *   tile_rows   : height of a fused-sweep tile, 4..32 (rounded so that tiles are >= 2M+1 rows)
 *   row_pairs   : class pairs per row-transform CTA, a power of two (capped at what fits)
 *   col_block   : frequency columns per column-solve CTA, a power of two 1..8
 *   row_threads : target threads of a row-transform CTA, 64..1024 (rounded down to a power
 *                 of two; a CTA gets more when a thread would hold over 16 values)
 *   col_rows    : rows per segment of the column recursions, 2..4096
 *   zfuse       : z-update (12) in one launch over a thread-block cluster of this many CTAs,
 *                 each owning a band of rows whose transforms and spectra stay in shared
 *                 memory (2, 4, 8 or 16); 1 = three launches (row transforms, column solves,
 *                 inverse row transforms); 3 = one launch of persistent CTAs that take the
 *                 units of the three passes in order from a ticket counter (a column unit
 *                 waits, bounded, until every row unit is done; an inverse unit until every
 *                 column unit is; results bit-identical to three launches with the same
 *                 tiling; column segments are lengthened where the column pass would need
 *                 more than 512 threads; one-unit row form only; measured slower than the
 *                 three launches chained by programmatic dependent launch: 145x145, K = 16,
 *                 36.3 vs 30.8 us per iteration); 0 = the library's choice (three launches).
 *                 A fused request that the band or the device cannot hold runs three
 *                 launches (get_tiling reports 1).
 *   row_pipe    : form of the two row-transform passes: 1 = one CTA per (row, class block);
 *                 2 = persistent CTAs (one wave) that walk the (row, class block) units and
 *                 copy the next unit's input into shared memory asynchronously while the
 *                 current unit is transformed; 3 = power-of-two rows (W = 256 ... 4096, no
 *                 Bluestein, K a multiple of 2 row_pairs): compile-time transform plan with
 *                 the first stage computed straight from the loaded row (rows that do not
 *                 qualify run form 1; in FP32, CTAs of 1024 first-stage butterflies take
 *                 512 threads and transform in place in one buffer, two CTAs per SM);
 *                 0 = the library's choice (3 for rows of 2048 and more where it applies,
 *                 else 1). All forms give the same results. */
typedef struct {
  int32_t tile_rows;
  int32_t row_pairs;
  int32_t col_block;
  int32_t row_threads;
  int32_t col_rows;
  int32_t zfuse;
  int32_t row_pipe;
} segsalsa_str_tiling;

/* create / workspace_bytes with an explicit tiling (NULL = defaults, same as the plain calls).
 * SEGSALSA_ERR_ARG if a tiling field is out of range or the tile does not fit on chip. */
int segsalsa_str_workspace_bytes_tiled(const segsalsa_str_params* params,
                                       const segsalsa_str_tiling* tiling, size_t* bytes);
int segsalsa_str_create_tiled(const segsalsa_str_params* params, const segsalsa_str_tiling* tiling,
                              void* workspace, size_t workspace_bytes, segsalsa_str_t** out);
/* The tiling a handle runs with (defaults resolved). */
int segsalsa_str_get_tiling(const segsalsa_str_t* h, segsalsa_str_tiling* out);

typedef struct segsalsa_str_batch segsalsa_str_batch_t; /* opaque; owned by the library */

/* Create a batch of n_images >= 1 independent problems (7) of any size, K, M, p and precision.
 * params[i].stream must be NULL (each image gets a library stream; the graphs run on
 * `stream`, a borrowed cudaStream_t, or a library stream when NULL). tiling (nullable) holds
 * n_images entries; when NULL each image takes the tiling that segsalsa_str_batch_autotune
 * chose for its class (precision, M, K, size class floor(log2(H W) / 2)) earlier in this
 * process, else the defaults. Device memory: the sum of the images' workspace_bytes. */
int segsalsa_str_batch_create(int32_t n_images, const segsalsa_str_params* params,
                              const segsalsa_str_tiling* tiling, void* stream,
                              segsalsa_str_batch_t** out);

/* Borrowed handle of image i (0 <= i < n_images), valid until batch_destroy. Every
 * single-image call works on it: set_probs, solve (this image alone), get_labels, get_z,
 * get_state / set_state, linear_solve. Do not destroy it. */
int segsalsa_str_batch_image(segsalsa_str_batch_t* b, int32_t i, segsalsa_str_t** h);

/* Run `iters` >= 0 SALSA iterations on every image (each continues from its own state; every
 * image needs set_probs first, else SEGSALSA_ERR_STATE). Returns when all are done. Each image
 * ends exactly where `iters` single-image iterations (segsalsa_str_solve with no trace) on its
 * handle would, bit for bit. SEGSALSA_ERR_TIMEOUT if a device-side bounded wait gave up. */
int segsalsa_str_batch_solve(segsalsa_str_batch_t* b, int32_t iters);

/* Project-written autotuner. Groups the images by class (see batch_create), and for each
 * class, largest total work first, times `trial_iters` >= 1 batch iterations for every
 * candidate tiling of that class while the other classes keep their current tiling, keeping
 * the fastest (candidates: tile_rows 4..32, then row_pairs, col_block, row_threads,
 * col_rows and row_pipe in turn). The lane count
 * is tuned first the same way (4, 8, 16, 32, n_images). The choice is
 * stored per class in a process-wide cache (used by later batch_create calls with tiling ==
 * NULL) and written to chosen[i] (nullable, n_images entries). The images are rebuilt with
 * the chosen tiling: their state is reset, so call set_probs (again) afterwards. */
int segsalsa_str_batch_autotune(segsalsa_str_batch_t* b, int32_t trial_iters,
                                segsalsa_str_tiling* chosen);

/* Lanes: the batch's concurrent chains of images (streams forked from and joined to the
 * master stream inside each graph). Images are assigned to lanes longest-work-first so that
 * the lanes carry similar work; the images of one lane run one after the other. Default
 * min(n_images, 16); the autotuner also picks it. 1 <= lanes (capped at n_images). */
int segsalsa_str_batch_set_lanes(segsalsa_str_batch_t* b, int32_t lanes);
int segsalsa_str_batch_get_lanes(const segsalsa_str_batch_t* b, int32_t* lanes);

/* Release the batch, its images and everything the library allocated for it. NULL is a
 * no-op. */
void segsalsa_str_batch_destroy(segsalsa_str_batch_t* b);

/* Message of the last failed batch call on `b` ("" if none); for b == NULL, the last failure
 * of segsalsa_str_batch_create in this thread. */
const char* segsalsa_str_batch_last_error(const segsalsa_str_batch_t* b);

/* Release the handle and everything the library allocated for it. NULL is a no-op. */
void segsalsa_str_destroy(segsalsa_str_t* h);

/* Message of the last failed call on `h` ("" if none); for h == NULL, the last failure of
 * segsalsa_str_create / segsalsa_str_workspace_bytes in this process. */
const char* segsalsa_str_last_error(const segsalsa_str_t* h);

#ifdef __cplusplus
}
#endif

#endif /* SEGSALSA_STR_H */
