/*
 * gadi.h -- C ABI of the GB300 GADI / GADI-IR solver library (libgadi.so).
 *
 * Problem (arXiv 2501.04229, §1.2 and §2.1): solve A x = b, A real n x n,
 * nonsingular, split as A = M + N. GADI iterates eq. (gadi):
 *     (aI + M) x^{k+1/2} = (aI - N) x^k + b
 *     (aI + N) x^{k+1}   = (N - (1-w) aI) x^k + (2-w) a x^{k+1/2}
 * for a > 0, w in [0, 2) (Thm 1). GADI-IR (Algorithm 1) runs the same
 * iteration as a refinement loop in three precisions:
 *     r = b - A x                      precision u_f
 *     solve H z = r,   H = aI + M      precision u_r
 *     solve S y = (2-w) a z, S = aI+N  precision u_r
 *     x = x + y                        precision u
 * The default splitting is HSS (§4.1): M = (A + A^T)/2, N = (A - A^T)/2.
 *
 * Conventions for every entry point:
 *   - Every call returns gadi_status. Nothing aborts, exits or prints.
 *   - Arguments are checked before anything is modified; on
 *     GADI_ERR_INVALID_ARG nothing has changed.
 *   - A handle is not thread-safe: use one handle per host thread.
 *   - Device pointers are CUDA device (or managed) addresses on the device
 *     that was current when the handle was created; host pointers are
 *     ordinary (pageable or pinned) host memory. Where both are accepted the
 *     library tells them apart with cudaPointerGetAttributes.
 *   - All device work is ordered on the stream given to gadi_create.
 *   - gadi_last_error(h) returns a NUL-terminated description of the last
 *     failure on h (owned by h, valid until the next call on h).
 */
#ifndef GADI_H
#define GADI_H

#include <stdint.h>

#if defined(__GNUC__)
#define GADI_API __attribute__((visibility("default")))
#else
#define GADI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gadi_solver gadi_solver;   /* opaque, owned by the library */

typedef enum {
    GADI_OK = 0,
    GADI_ERR_INVALID_ARG = 1,    /* bad argument; nothing was modified */
    GADI_ERR_OUT_OF_MEMORY = 2,  /* a device allocation failed */
    GADI_ERR_CUDA = 3,           /* a CUDA runtime call failed; see gadi_last_error */
    GADI_ERR_RANGE = 4,          /* a value cannot be represented in the inner precision
                                    even after power-of-two scaling */
    GADI_ERR_NOT_CONVERGED = 5,  /* max_outer reached; x holds the last iterate */
    GADI_ERR_DIVERGED = 6,       /* NaN/Inf, inner breakdown, or residual growth > 1e3x */
    GADI_ERR_TIMEOUT = 7,        /* a bounded device-side wait expired */
    GADI_ERR_NO_MODEL = 8,       /* no parameter predictor of the requested kind */
    GADI_ERR_UNSUPPORTED = 9     /* valid request this build does not implement */
} gadi_status;

typedef enum { GADI_SPLIT_HSS = 0, GADI_SPLIT_USER = 1 } gadi_splitting;

typedef enum { GADI_F64 = 0, GADI_F32 = 1, GADI_F16 = 2, GADI_BF16 = 3, GADI_E4M3 = 4 } gadi_precision;

typedef enum {
    GADI_STOP_ETA = 0,   /* stop when eta_inf = ||b-Ax||_inf/(||A||_inf ||x||_inf + ||b||_inf) <= tol */
    GADI_STOP_RES = 1    /* stop when RES = ||b-Ax||_2/||b-Ax0||_2 <= tol (§4.1's RES) */
} gadi_stop;

typedef enum {
    GADI_KERNEL_AUTO = 0,     /* stencil kernels when a stencil descriptor was given, else sparse */
    GADI_KERNEL_SPARSE = 1,   /* general sparse (ELL layout built from the CSR) */
    GADI_KERNEL_STENCIL = 2   /* matrix-free 5/7-point stencil; needs a stencil descriptor */
} gadi_kernel;

/* Sparse matrix in CSR form, int32 indices, FP64 values. Column indices of a
 * row must be ascending and the pattern structurally symmetric (a_ij stored
 * iff a_ji stored), which the HSS splitting needs. Caller-owned; gadi_create
 * copies it, so the caller may free it as soon as gadi_create returns.
 * on_device: 0 = the three arrays are host pointers, 1 = device pointers. */
typedef struct {
    int64_t n, nnz;
    const int32_t *row_ptr;   /* n+1 entries, row_ptr[0] = 0, row_ptr[n] = nnz */
    const int32_t *col_idx;   /* nnz entries */
    const double *val;        /* nnz entries */
    int32_t on_device;
} gadi_csr;

/* Optional structure of A for the matrix-free kernels: A is the h^2-scaled
 * centred-difference convection-diffusion operator of §4.1 on an N^dim grid
 * of interior nodes (x fastest), h = 1/(N+1), convection c = beta*h/2: row
 * i has a diagonal entry, -k_f - c towards the lower neighbour along each
 * axis and -k_f + c towards the upper one, k_f the coefficient of the face
 * between them (neighbours on the boundary are omitted).
 *   variable_k = 0: k_f = 1 everywhere (diagonal 2*dim); the kernels use
 *                   scalar coefficients only.
 *   variable_k = 1: k_f varies (dim = 3 only); the kernels keep the diagonal
 *                   and one coupling per axis and node, taken from A.
 * gadi_create checks the CSR pattern and values against this description
 * (pattern exact; values, and the convection part of every entry, within a
 * relative 1e-12) and returns GADI_ERR_INVALID_ARG on a mismatch. The
 * stencil kernels need the HSS splitting. */
typedef struct {
    int32_t dim, N;
    double beta;
    int32_t variable_k;
} gadi_stencil;

typedef struct {
    int32_t outer_iters;        /* completed refinement steps */
    int32_t status;             /* the gadi_status of the solve */
    int64_t inner_iters_H;      /* total CG iterations on H */
    int64_t inner_iters_S;      /* total CGNR iterations on S */
    int64_t spmv_count;         /* operator applications in the solve (A, H, S, S^T) */
    double eta_inf;             /* backward error of the returned x */
    double res_rel;             /* RES of the returned x */
    double t_solve_s;           /* device time of the solve (CUDA events; host wall time of
                                   launch + synchronisation for gadi_solve_stencil_noalloc,
                                   which creates no events) */
    int32_t scale_exp_M;        /* FP16 scale exponent of H (H stored as 2^-s H) */
    int32_t scale_exp_N;        /* FP16 scale exponent of S */
    int32_t kernel;             /* gadi_kernel actually used */
    int32_t grid_blocks;        /* persistent-kernel launch shape used */
    int32_t block_threads;
    int32_t zmarch_planes;      /* planes per z-marching segment (0: grid-stride items) */
} gadi_info;

/* Create a solver for A (copied to the device): the problem statement of
 * §1.2 (A x = b, A nonsingular, A = M + N) and Algorithm 1's inputs (A and
 * its splitting). split: GADI_SPLIT_HSS, the Hermitian/skew-Hermitian
 * splitting §4.1 uses (M = (A + A^T)/2, N = (A - A^T)/2), or
 * GADI_SPLIT_USER with M_user on A's exact pattern (same row_ptr/col_idx,
 * same on_device flag) and N = A - M (eq. (gadi) admits any splitting; Thm
 * 1 states when it converges); M must be symmetric for the CG on
 * H = aI + M to apply. structure: optional stencil descriptor (see above).
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * Errors: INVALID_ARG (n < 1, bad pattern, pattern not symmetric, unsorted
 * columns, non-finite values, stencil mismatch), OUT_OF_MEMORY, CUDA. */
GADI_API gadi_status gadi_create(const gadi_csr *A, gadi_splitting split, const gadi_csr *M_user,
                        const gadi_stencil *structure, void *cuda_stream, gadi_solver **out);

/* Parameters of eq. (gadi) and the precision triple of Algorithm 1.
 * alpha > 0 and omega in [0, 2) (Thm 1). Supported: u = u_f = GADI_F64 with
 * any u_r; other valid triples return UNSUPPORTED.
 * u_r = GADI_F16 means FP16 storage of the inner matrix values and vectors
 * with FP32 arithmetic (one fused multiply-add per product-sum); A, r and z
 * are scaled by powers of two so FP16 stays in range, and (2 - omega) alpha
 * is applied in the FP64 update. u_r = GADI_BF16: the same with bfloat16
 * storage (8 significant bits). u_r = GADI_E4M3: the same with FP8 E4M3
 * storage (4 significant bits, largest finite value 448; stores round to
 * nearest even and saturate at +-448); a precision below the paper's FP16.
 * u_r = GADI_F32: FP32 storage and arithmetic, r and z scaled, the
 * operators not. u_r = GADI_F64 with the default inner tolerance is plain
 * FP64 GADI. RANGE when a nonzero matrix entry of the scaled inner operators
 * rounds to zero in u_r. */
GADI_API gadi_status gadi_set_params(gadi_solver *h, double alpha, double omega,
                            gadi_precision u_r, gadi_precision u, gadi_precision u_f);

/* Inner relative tolerance eps (0 < eps < 1): each inner solve stops when
 * ||rhs - K v||_2 <= eps ||rhs||_2, or after max_inner iterations (>= 1).
 * This is Algorithm 1's inner tolerance on steps 2 and 3 ("tol <= eps
 * ||r^(0)||_2"), read as relative to the current inner right-hand side.
 * max_outer (>= 0) caps the refinement steps (Algorithm 1's outer loop). Defaults: eps 1e-2 (FP32,
 * FP16 and bfloat16 inner precision) / 0.1 (FP8 E4M3) / 1e-10 (FP64 inner),
 * max_inner 200, max_outer 100000. */
GADI_API gadi_status gadi_set_inner(gadi_solver *h, double eps_inner, int32_t max_inner, int32_t max_outer);

/* Stopping criterion kind for gadi_solve's tol (default GADI_STOP_ETA). */
GADI_API gadi_status gadi_set_stop(gadi_solver *h, gadi_stop kind);

/* Kernel family (default GADI_KERNEL_AUTO). STENCIL without a descriptor
 * returns INVALID_ARG. */
GADI_API gadi_status gadi_set_kernel(gadi_solver *h, gadi_kernel kind);

/* FP16 inner scaling (default on = 1). on: the operator, the residual and
 * the first correction are scaled by powers of two so that FP16 stays in
 * range, alpha is added in FP32 and (2 - omega) alpha is folded into the
 * FP64 update (Alg. 1 with the readings stated in the oracle). off = 0: the
 * unscaled FP16 inner precision the paper's FP16 experiments show (Table
 * "3d", the stall at 1e-8 to 1e-10): alpha is rounded into the stored FP16
 * diagonals of aI + M and aI + N, r and z are not scaled, and (2 - omega)
 * alpha multiplies z in FP16 before the second solve. An ablation mode; it
 * only affects u_r = GADI_F16. Other values return INVALID_ARG. */
GADI_API gadi_status gadi_set_scaling(gadi_solver *h, int32_t on);

/* Rows per work item of the stencil kernels (an implementation choice, not
 * part of the paper's method: operator applications are bit-identical for
 * every value; the dot products of a solve sum in another order):
 * 0 = automatic (8 when the grid side N is a multiple of 8, else 4 when a
 * multiple of 4, else 1), or 1, 4, 8 -- used when N is a multiple of it,
 * else 1. An item of R rows is R consecutive nodes of one x-line, read with
 * one 2R-byte FP16 load per vector. Other values return INVALID_ARG. */
GADI_API gadi_status gadi_set_item_rows(gadi_solver *h, int32_t rows);

/* Traversal of the solve kernel's passes (an implementation choice, not
 * part of the paper's method): 0 = automatic (default): solves of the 3D
 * constant-coefficient stencil with FP16 inner vectors and 8-row items use
 * the z-marching kernel, whose residual, demotion, CGNR-start and CGNR-A
 * passes march along z: every thread takes a column of items (the 8-row
 * chunk of an x-line at fixed y) over a segment of at least 4 planes,
 * keeping the values of planes z-1, z, z+1 in registers and requesting
 * plane z+2 while plane z is formed (its CG and CGNR-B passes take
 * grid-stride items); other solves, and launches too small for segments of
 * 4 planes, use grid-stride items in every pass (gadi_info.zmarch_planes =
 * 0). 1 = grid-stride items always. Every row is formed with the same
 * terms in the same order either way; the dot products of a solve sum in
 * another order. Other values return INVALID_ARG. */
GADI_API gadi_status gadi_set_traversal(gadi_solver *h, int32_t mode);

/* Launch shape of the persistent solve kernel: grid_blocks (0 = automatic,
 * else 1 .. the co-resident maximum) and block_threads (0 = automatic, else
 * 128, 256, 512 or 1024). One block runs the solve with block-local barriers
 * only. gadi_apply uses the same shape when set (else one item per thread,
 * 256 threads per block). */
GADI_API gadi_status gadi_set_launch(gadi_solver *h, int32_t grid_blocks, int32_t block_threads);

/* Upper bound, in milliseconds, of every device-side grid-barrier wait
 * (default 2000). An expired wait ends the solve with GADI_ERR_TIMEOUT and
 * leaves the handle usable. */
GADI_API gadi_status gadi_set_wait_limit(gadi_solver *h, double milliseconds);

/* Test hook: when on != 0, the next solves give every grid-barrier wait an
 * arrival target that no block reaches, so the wait limit expires and the
 * solve returns GADI_ERR_TIMEOUT (needs a launch of 2 or more blocks). No
 * fault and no hang: the wait is bounded by gadi_set_wait_limit. */
GADI_API gadi_status gadi_debug_force_timeout(gadi_solver *h, int32_t on);

/* Solve A x = b by Algorithm 1 (GADI-IR): repeat r = b - A x in u_f
 * (step 1), the inner solves with aI + M and aI + N in u_r (steps 2 and 3),
 * x += the correction in u (step 4), until the stopping test holds: eta_inf
 * <= tol (the normwise backward error, Thm 3's measure with infinity norms)
 * or RES <= tol (§4.1's relative residual), as gadi_set_stop selects. With
 * u_r = GADI_F64 this is eq. (gadi)'s plain FP64 GADI. b (n FP64) and x (n
 * FP64; in: x0, Algorithm 1's starting vector, out: the result) are
 * both host or both device pointers. Host buffers are copied to and from
 * library-owned device memory inside the call. Returns after the result is
 * in x (the stream is synchronised). tol > 0 applies to the criterion set
 * by gadi_set_stop. Returns OK, NOT_CONVERGED, DIVERGED (x holds the last
 * iterate), TIMEOUT, INVALID_ARG (tol <= 0, non-finite b, mixed pointer
 * kinds) or CUDA. info may be NULL. */
GADI_API gadi_status gadi_solve(gadi_solver *h, const double *b, double *x, double tol, gadi_info *info);

/* One operator application with the solver's current kernel and parameters,
 * y = K x, for kernel-level tests and bandwidth measurement. which:
 *   0: K = A      (FP64 x, y)
 *   1: K = H' = 2^-sM (aI + M)  in the inner precision
 *   2: K = S' = 2^-sN (aI + N)
 *   3: K = S'^T
 * x, y are device pointers of n elements of the inner precision (FP64 for
 * which = 0; FP16, bfloat16, FP8 E4M3 (one byte each), FP32 or FP64 after
 * gadi_set_params' u_r).
 * Asynchronous on the handle's stream. */
GADI_API gadi_status gadi_apply(gadi_solver *h, int32_t which, const void *x, void *y);

/* Scale exponents (sM, sN) that the inner operators use for the current
 * alpha and inner precision. */
GADI_API gadi_status gadi_get_scales(gadi_solver *h, int32_t *sM, int32_t *sN);

/* Predict (alpha, omega) for h's system (§3.3). features[0] = log n,
 * features[1] = log beta (nfeat >= 2). kind: GADI_MODEL_MLP or
 * GADI_MODEL_GPR use the model attached with gadi_set_model (NO_MODEL when
 * none); omega is clamped to [0, 1.999]. GADI_MODEL_GRID searches 16 alpha
 * (10^-3 .. 10^2) x 4 omega (0, 0.5, 1, 1.5) with solves of h's own system
 * (b = A 1, x0 = 0, the handle's precisions and inner settings, tol 1e-10),
 * each capped at the fewest outer steps of a converged candidate so far,
 * and returns the candidate with the fewest operator applications. */
GADI_API gadi_status gadi_predict_params(gadi_solver *h, const double *features, int32_t nfeat,
                                int32_t kind, double *alpha, double *omega);

/* ---- Parameter predictors (§3.3) ------------------------------------------
 * A model maps features x = (log n, log beta) to targets (log alpha*,
 * omega*). Both are standardised per column before fitting.
 *   GADI_MODEL_GPR: Gaussian-process regression (§3.3.1), squared-exponential
 *     kernel, posterior mean, FP32 arithmetic (the paper fits its GPR in
 *     FP32), host side. hyper: NULL (length scale and noise chosen by the
 *     log marginal likelihood on the grid {0.25,0.5,1,2,4} x {1e-3,1e-2,1e-1})
 *     or {ell, sn}. m <= 4096.
 *   GADI_MODEL_MLP: 2 -> 64 -> 64 -> 2, tanh, trained on the GPU by full-
 *     batch Adam on MSE (BF16 weights into tensor-core MMAs, FP32
 *     accumulation and master weights). hyper: NULL or {epochs [3000],
 *     lr [1e-2], seed [1]}.
 * X: m x 2 row-major features; Y: m x 2 targets (host pointers, copied).
 * The model is owned by the caller (gadi_model_destroy). */
typedef struct gadi_model gadi_model;
#define GADI_MODEL_MLP 0
#define GADI_MODEL_GPR 1
#define GADI_MODEL_GRID 2
GADI_API gadi_status gadi_model_fit(int32_t kind, const double *X, const double *Y, int32_t m,
                                    const double *hyper, int32_t nhyper, void *cuda_stream,
                                    gadi_model **out);
/* Y (count x 2) = model(X (count x 2)), host pointers. */
GADI_API gadi_status gadi_model_predict(const gadi_model *model, const double *X, int32_t count, double *Y);
/* Training loss per epoch of an MLP (count = epochs; copies min(cap, count)). */
GADI_API gadi_status gadi_model_loss(const gadi_model *model, double *loss, int32_t cap, int32_t *count);
/* Gradient of the MLP loss 1/(2m) sum (y - t)^2 at the given parameters on
 * already standardised X, T (m x 2 each), computed by the training kernels
 * (BF16 operands, FP32 accumulation). params and grad: gadi_mlp_param_count()
 * values in the order W1 [64][2], b1 [64], W2 [64][64], b2 [64], W3 [2][64],
 * b3 [2]. */
GADI_API gadi_status gadi_mlp_gradient(const double *params, const double *X, const double *T, int32_t m,
                                       void *cuda_stream, double *grad);
GADI_API int32_t gadi_mlp_param_count(void);
GADI_API void gadi_model_destroy(gadi_model *model);
/* Attach a model (not owned; must outlive its use) to h for
 * gadi_predict_params of the model's kind. NULL detaches. */
GADI_API gadi_status gadi_set_model(gadi_solver *h, int32_t kind, const gadi_model *model);

/* ---- Batched parameter sweep --------------------------------------------
 * Many FP16-inner GADI-IR solves in one persistent launch per size bin
 * (captured in a CUDA graph), for building training sets of optimal (alpha,
 * omega) the way §3.3 builds them: from small systems of the same structure.
 * Each instance is the constant-coefficient convection-diffusion system of
 * gadi_stencil (variable_k = 0) with b = A 1 and x0 = 0 (as in §4.1); each
 * candidate is an (alpha, omega) pair; every instance is solved with every
 * candidate to eta_inf <= tol (inner eps_inner, max_inner, max_outer as in
 * gadi_set_inner). A team of blocks solves one (instance, candidate) item;
 * items of uneven size share the launch of their size bin, largest first.
 * Schedule: instances are binned by rows (n < 2^15, < 2^18, < 2^20, larger);
 * each bin has one team size (blocks per item; tried: 1 / 1, 2, 4 / 2, 4, 8
 * / 4, 8, 16) and one block size (128, 256, 512), chosen by the built-in
 * autotuner from short timed probes (cached per problem class) unless fixed
 * by block_threads (128, 256 or 512; 0 = tuned) and team_blocks (1 .. 64;
 * 0 = tuned). race != 0 stops a solve once it has used more operator
 * applications than a finished candidate of the same instance (raced_out =
 * 1, status NOT_CONVERGED): it cannot be the cheapest.
 * records: host array of ninst * ncand entries, written at
 * [instance * ncand + candidate]. Returns OK when every item ran (items
 * carry their own status), INVALID_ARG (also: a team larger than the blocks
 * that fit the GPU at once), OUT_OF_MEMORY, TIMEOUT (a bounded wait of a
 * team expired) or CUDA. */
typedef struct {
    int32_t dim, N;
    double beta;
} gadi_sweep_instance;

typedef struct {
    double alpha, omega;
} gadi_sweep_candidate;

typedef struct {
    int32_t instance, candidate;
    int32_t status;             /* gadi_status of this solve */
    int32_t raced_out;          /* 1 when stopped by the race */
    int32_t outer_iters;
    int32_t team_blocks;        /* blocks of the team that solved this item */
    int64_t inner_iters_H, inner_iters_S, spmv_count;
    double eta_inf;
    double time_ms;             /* device time of this item */
} gadi_sweep_record;

GADI_API gadi_status gadi_sweep(const gadi_sweep_instance *instances, int32_t ninst,
                                const gadi_sweep_candidate *candidates, int32_t ncand, double tol,
                                double eps_inner, int32_t max_inner, int32_t max_outer, int32_t race,
                                int32_t block_threads, int32_t team_blocks, void *cuda_stream,
                                gadi_sweep_record *records);

/* Allocation-free solve (the paper has no counterpart: this is a library
 * convenience). Some callers cannot allocate device memory: code that runs
 * under a fixed memory budget or inside a framework that owns all device
 * memory through its own pool (where a raw cudaMalloc may fail or fragment
 * the pool), and latency-critical loops where cudaMalloc's implicit device
 * synchronisation is not acceptable. gadi_solve_stencil_noalloc serves them:
 * it solves the constant-coefficient convection-diffusion stencil system of
 * gadi_stencil (variable_k = 0, HSS splitting, right-hand side b) with
 * FP16-inner GADI-IR, stopping on eta_inf <= tol, and calls no cudaMalloc,
 * cudaFree or other allocating routine. No handle is involved.
 *   dim, N, beta: the operator (as in gadi_stencil); n = N^dim must not
 *                 exceed GADI_NOALLOC_MAX_N (larger n: GADI_ERR_INVALID_ARG).
 *   alpha, omega, eps_inner, max_inner, max_outer: as in gadi_set_params and
 *                 gadi_set_inner.
 *   b, x:         device pointers of the current device (or managed
 *                 pointers) to n FP64 values, owned by the caller; x holds
 *                 x0 on entry and the result on return. Memory of another
 *                 GPU, or host memory, gives GADI_ERR_INVALID_ARG.
 *   cuda_stream:  stream of the work; the call returns after the result is
 *                 in x (the stream is synchronised).
 * Its scratch is one library-owned device array of fixed size (about 9.5 MB),
 * present on every GPU that loads the library until the process exits; the
 * first call on a device looks up that array's address (a one-time set-up
 * done with the device current).
 * Every call uses the same array and leaves its contents behind: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. Returns as gadi_solve; info->t_solve_s is the
 * host wall time of the launch and the synchronisation. */
#define GADI_NOALLOC_MAX_N 262144
GADI_API gadi_status gadi_solve_stencil_noalloc(int32_t dim, int32_t N, double beta, double alpha,
                                                double omega, double eps_inner, int32_t max_inner,
                                                int32_t max_outer, const double *b, double *x,
                                                double tol, void *cuda_stream, gadi_info *info);

/* Release all device memory of h (the copies of A and its splitting that
 * gadi_create made for Algorithm 1, and the solve's work vectors). NULL is
 * accepted. */
GADI_API void gadi_destroy(gadi_solver *h);

GADI_API const char *gadi_status_str(gadi_status s);
GADI_API const char *gadi_last_error(const gadi_solver *h);

/* ------------------------------------------------------------------------
 * GADI-AB for the Sylvester equation A X + X B = C (§4.3): Algorithm 1
 * with the operator X -> A X + X B split into X -> A X and X -> X B. A
 * (m x m) and B (n x n) are tridiagonal: lo[i] = T[i][i-1] (lo[0]
 * ignored), diag[i] = T[i][i], up[i] = T[i][i+1] (up[last] ignored). The
 * residual is R = C - A X - X B in FP64; the two inner systems per outer
 * step, (aI + A) Z = R^ column by column and Y (aI + B) = Z^ row by row,
 * are tridiagonal and solved directly in the inner precision u_r (FP16 and
 * bfloat16 with the power-of-two scaling of the vector method, FP32, or
 * FP64); X is updated in FP64. Stop: eta = max|R| / (||L||_inf max|X| +
 * max|C|) <= tol, with ||L||_inf the largest row sum of I (x) A + B^T (x) I.
 * ------------------------------------------------------------------------ */
typedef struct gadi_sylv gadi_sylv;

/* Copies the host arrays (m >= 1, n >= 1, m n <= 2^31, finite values).
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
GADI_API gadi_status gadi_sylv_create(int64_t m, int64_t n, const double *a_lo, const double *a_diag,
                                      const double *a_up, const double *b_lo, const double *b_diag,
                                      const double *b_up, void *cuda_stream, gadi_sylv **out);

/* alpha > 0, omega in [0, 2) (Thm 1), u_r = GADI_F64, GADI_F32, GADI_F16
 * or GADI_BF16 (GADI_E4M3: UNSUPPORTED). */
GADI_API gadi_status gadi_sylv_set_params(gadi_sylv *s, double alpha, double omega, gadi_precision u_r);

/* Solve in place: C and X are device pointers to row-major m x n FP64
 * arrays (X: in x0, out the result). Returns OK, NOT_CONVERGED (max_outer
 * reached; X holds the last iterate), DIVERGED, INVALID_ARG or CUDA. info
 * (may be NULL) gets outer_iters, eta_inf (also in res_rel), t_solve_s
 * (host wall time of the solve, synchronised), scale_exp_M / _N = the
 * exponents of A's and B's inner operators. */
GADI_API gadi_status gadi_sylv_solve(gadi_sylv *s, const double *C, double *X, double tol, int32_t max_outer,
                                     gadi_info *info);

GADI_API const char *gadi_sylv_last_error(const gadi_sylv *s);

/* Release all device memory of s. NULL is accepted. */
GADI_API void gadi_sylv_destroy(gadi_sylv *s);

#ifdef __cplusplus
}
#endif

#endif /* GADI_H */
