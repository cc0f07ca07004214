/*
 * stab.h -- C ABI of the GB300 matrix-free global stability library.
 *
 * The library computes eigenvalues of the Jacobian J(q0) of the discretised
 * compressible Navier-Stokes right-hand side N(q) in primitive (p, u_i, s)
 * form (Sec. "Governing equations", Eq. navier_stokes), applied matrix-free
 * as the epsilon-quotient of Eq. frechet, by the Cayley-transformed
 * implicitly restarted Arnoldi method (Algorithm iram, Eq. cayley_transform)
 * with GMRES inner solves (Sec. "Iterative solvers") and local block-Jacobi
 * preconditioning (Sec. "Preconditioning").
 *
 * Conventions shared by every entry point:
 *  - Vectors are complex128, interleaved (re, im), laid out [var][z][y][x]
 *    with x fastest; n = nvars * nx * ny * nz, nvars = dim + 2 (p, u, v, [w], s).
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device (a torch tensor's data_ptr() qualifies); all device work is
 *    ordered on the stream given to stab_create.
 *  - Every call returns a stab_status and never aborts; the message of the
 *    last failure is returned by stab_last_error.  A handle is used by one
 *    host thread at a time.
 *  - The handle owns its copies of the base state, its tables, its
 *    workspace and its preconditioner; the caller owns every buffer it
 *    passes in.
 */
#ifndef STAB_H
#define STAB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stab_handle_s* stab_handle;

typedef enum {
  STAB_OK = 0,
  STAB_ERR_INVALID_ARG = 1,   /* bad size, pointer or option */
  STAB_ERR_OOM = 2,           /* device allocation failed */
  STAB_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  STAB_ERR_NOT_CONVERGED = 4, /* iteration limit reached; partial results returned */
  STAB_ERR_BREAKDOWN = 5,     /* Krylov breakdown (invariant subspace found early) */
  STAB_ERR_NUMERIC = 6,       /* NaN / Inf met in a reduction or the Hessenberg matrix */
  STAB_ERR_TIMEOUT = 7,       /* a bounded device-side wait ran out */
  STAB_ERR_BUSY = 8,
  STAB_ERR_UNSUPPORTED = 9    /* a valid option this build does not implement */
} stab_status;

/* Grid: x (and z) periodic with lengths lx (lz); y bounded on [ly0, ly1]
 * with non-reflective boundaries (Sec. "Model problem").  stretch = 0 gives
 * uniform y; beta > 0 places y(eta) = yc + (ly1-ly0)/2 sinh(beta(2 eta-1))/sinh(beta),
 * eta uniform on [0, 1].  dim = 2 requires nz = 1.  Lines need nx, ny >= 6
 * (nz >= 6 in 3-D). */
typedef struct {
  int dim;
  int nx, ny, nz;
  double lx, ly0, ly1, lz;
  double stretch;
} stab_grid;

typedef struct {
  double gamma;           /* ratio of specific heats, default 1.4 */
  double sutherland_S;    /* Sutherland constant over the reference temperature, default 110.4/273.15 */
  double bulk_visc_ratio; /* mu_v / mu, default 0 */
  int eps_mode;           /* J v form: 0 = epsilon-quotient of Eq. frechet evaluated without
                             cancellation (default); 2 = exact tangent (epsilon -> 0).
                             1 (literal double quotient) returns STAB_ERR_UNSUPPORTED. */
  double eps;             /* 0: eps = sqrt(eps_m)(1 + ||q0||_2)/||v||_2 per call; > 0: fixed */
  int gmres_m;            /* inner GMRES restart length, default 30 */
  int gmres_max_restarts; /* default 200 */
  double gmres_tol;       /* inner relative residual tolerance, default 1e-10 */
  int precond;            /* 0 none, 1 block-Jacobi (exact tile blocks of J), 2 block-Jacobi of the reduced
                             operator (Sec. "Numerical experiments", Conclusions: the right-hand side
                             discretised with second-order explicit differences, f' = (f+1 - f-1)/(2h),
                             f'' = (f+1 - 2f + f-1)/h^2, second-order one-sided at the y boundaries; its tile
                             blocks are block tridiagonal in levels of two y lines, factorised by block
                             Thomas elimination and stored as three level blocks per level, so tiles may
                             span the whole y range: ty even, nv * 2 * tx * tz <= 256 unknowns per level;
                             precond_prec 64 or 32 (16: STAB_ERR_UNSUPPORTED); single-handle solves only) */
  int tile[3];            /* block-Jacobi tile in grid points (x, y, z), default 8 x 8 x 1 */
  int precond_prec;       /* block-Jacobi inverse storage: 64 (FP64), 32 (FP32, default) or 16 (BF16:
                             inverted in FP32, stored in bfloat16, applied with FP32 accumulation) */
  int max_restarts;       /* IRAM restart limit, default 300 */
  unsigned long long seed;/* start vector seed when no v0 is given, default 0x5EED */
  int gmres_basis_prec;   /* GMRES Krylov basis and its orthogonalisation: 64 (FP64 flexible GMRES,
                             default) or 32 (FP32 basis, non-flexible right preconditioning; J v, the
                             solution update and the true residual of every restart stay FP64, so the
                             restarts refine the solution to the FP64 tolerance) */
  int stencil_prec;       /* right-hand sides B f of the compact schemes inside J v: 64 (FP64, default) or
                             48 (interior rows in FP32 pair arithmetic on exactly power-of-two-scaled
                             inputs, ~2^-47 relative; the Thomas sweeps, the closure rows and the set-up
                             stay FP64) */
  int lgmres_k;           /* inner solver: 0 = GMRES(gmres_m) (default); k in [1, min(8, gmres_m - 1)] =
                             LGMRES (Sec. "Iterative solvers", after Baker, Jessup and Manteuffel): every
                             cycle spans gmres_m directions, gmres_m - k Krylov directions of the residual
                             followed by the k latest error approximations x_{c+1} - x_c of earlier cycles,
                             which enter without a J v (their products are the residual differences).
                             Needs gmres_basis_prec = 64 (else STAB_ERR_UNSUPPORTED) */
  int precond_factor;     /* inversion of the FP32 block-Jacobi blocks (precond_prec 32 or 16): 0 = Gauss-Jordan
                             with partial pivoting on the CUDA cores (default); 1 = the same elimination blocked
                             in panels of 32 columns (16 above 640 rows) staged in shared memory, every panel's update of the other
                             columns one batched complex GEMM on the tensor cores with FP32 inputs emulated in
                             BF16 (FP32 accuracy); 2 = the same with TF32 inputs (about 1e-3 relative).
                             precond_prec 64 always uses the CUDA cores */
  int gmres_inner_m;      /* nested inner solver (mixed precision): 0 = none (default); k in [1, 100] = every
                             step of the FP64 flexible GMRES(gmres_m) takes as its direction z_j an inner
                             GMRES(k) approximation of (J - sigma I)^{-1} v_j with an FP32 Krylov basis and FP32
                             orthogonalisation, right preconditioned with the block-Jacobi inverses (opts.precond),
                             run until its residual is below gmres_inner_tol ||v_j|| or k steps; J v stays FP64.
                             Needs gmres_basis_prec = 64 and lgmres_k = 0 (else STAB_ERR_UNSUPPORTED) */
  double gmres_inner_tol; /* relative tolerance of each inner solve, default 1e-3 */
} stab_opts;

typedef struct {
  long long jv_calls;         /* matrix-free operator applications (the paper's matvec count) */
  long long gmres_iterations; /* inner iterations over all solves */
  long long gmres_solves;     /* Cayley applications */
  long long arnoldi_steps;
  long long restarts;         /* IRAM restarts */
  long long precond_builds;
  double seconds_total;
  double seconds_precond;
} stab_stats;

/* Fill *o with the defaults listed above. */
void stab_default_opts(stab_opts* o);

/* Create a handle for one problem.
 *  base_flow : q0, FP64 [var][z][y][x] (n doubles), on the host
 *              (base_on_device = 0) or device (1); copied.
 *  Ma, Re, Pr: Mach, Reynolds (Re <= 0: inviscid, Re -> infinity) and Prandtl numbers,
 *              nondimensionalised by the layer thickness, u_inf, rho_inf, T_inf.
 *  opts      : NULL for defaults.   cuda_stream: a cudaStream_t or NULL (legacy stream).
 * Errors: INVALID_ARG for bad sizes, OOM, CUDA; *h is NULL on failure. */
stab_status stab_create(stab_handle* h, const double* base_flow, int base_on_device,
                        const stab_grid* grid, double Ma, double Re, double Pr,
                        const stab_opts* opts, void* cuda_stream);

void stab_destroy(stab_handle h);

/* Message of the last failed call on h (h may be NULL for stab_create failures). */
const char* stab_last_error(stab_handle h);

/* Number of complex unknowns n. */
long long stab_size(stab_handle h);

/* Jv = J(q0) v - shift v   (Eq. frechet; with shift = tau it is the Cayley
 * right-hand side of Eq. cayley_arnoldi).  v, Jv: device complex128, n
 * entries each, must not overlap.  The J v form follows opts.eps_mode.
 * Range: parts of the operator run in FP32 pair arithmetic and in FP32
 * warm-ups, so entries of v (and of its derivative fields) keep full FP64-class
 * accuracy between about 2^-74 and 2^100 in magnitude; smaller entries are
 * resolved to FP32 precision relative to themselves, entries below 2^-126 are
 * dropped, and v with entries above 2^100 is outside the supported range.  The
 * solvers always pass normalised vectors. */
stab_status stab_apply_J(stab_handle h, const void* v, void* Jv, double shift_re, double shift_im);

/* Batched J v over several problems with uneven grids, on one stream.  Every
 * phase of Eq. frechet's J v (epsilon norm, temperature differences, the y,
 * z and x compact-derivative passes, the pointwise assembly) is one launch
 * for all instances (one per kernel variant in use), each instance with its
 * own options and tuned line-pass shapes, so each result equals what its
 * handle's stab_apply_J returns, bit for bit.
 *   create: handles distinct, created on the current device, each with a base
 *           flow that depends on y only (else STAB_ERR_UNSUPPORTED); count in
 *           [1, 4096]; cuda_stream runs every call of the batch.  The batch
 *           keeps the handle pointers (not ownership).
 *   apply:  v[i], Jv[i]: device complex128 vectors of handle i's size, not
 *           overlapping each other; shifts: NULL or 2*count doubles
 *           (re, im of each instance's shift).  Returns when the work is
 *           queued.  Every batch call is ordered after the work already
 *           queued on each handle's own stream, and each handle's stream is
 *           ordered after the batch call's kernels, so single-handle calls
 *           before and after a batch call never race with it.
 * A batch is used by one host thread at a time; its messages are in
 * stab_jv_batch_last_error.  destroy waits for all of the batch's work
 * (its kernels read the handles' memory) and then releases its buffers;
 * destroy a batch before any of its handles. */
typedef struct stab_jv_batch_s* stab_jv_batch;
stab_status stab_jv_batch_create(stab_jv_batch* b, const stab_handle* handles, int count, void* cuda_stream);
stab_status stab_jv_batch_apply(stab_jv_batch b, const void* const* v, void* const* Jv, const double* shifts);
/* z[i] = M_i^-1 q[i] for every handle of the batch (block-Jacobi inverses of
 * each handle's last stab_precond_build): one launch per inverse storage
 * layout for all instances; each result equals its handle's own
 * stab_precond_apply bit for bit.  q[i], z[i]: device complex128 vectors
 * of handle i's size, not overlapping.  INVALID_ARG when a handle has no
 * preconditioner built. */
stab_status stab_jv_batch_precond_apply(stab_jv_batch b, const void* const* q, void* const* z);
/* CGS2 (as stab_orthogonalize) of w[i] against the k[i] orthonormal columns
 * of V[i] for every handle of the batch: one launch per step for all
 * instances; each result equals its handle's own stab_orthogonalize bit for
 * bit.  V[i]: device complex128 n_i x k[i]; w[i]: device complex128 n_i,
 * updated in place; 1 <= k[i] <= 1536.  hcoef (host, may be NULL): the
 * coefficients of all instances one after the other (k[0] complex, then
 * k[1], ...); norms (host, may be NULL): ||w[i]|| after.  Uses each handle's
 * orthogonalisation scratch; synchronises the batch's stream. */
stab_status stab_jv_batch_orthogonalize(stab_jv_batch b, const void* const* V, const int* k, void* const* w,
                                        double* hcoef, double* norms);
const char* stab_jv_batch_last_error(stab_jv_batch b);
void stab_jv_batch_destroy(stab_jv_batch b);

/* epsilon used by the last stab_apply_J call (0 for the exact tangent).  Synchronises the stream. */
stab_status stab_last_eps(stab_handle h, double* eps);

/* Solve (J - sigma I) x = b by restarted, right-preconditioned (flexible)
 * GMRES to ||b - (J - sigma I) x|| <= opts.gmres_tol ||b|| with x0 = 0
 * (Sec. "Iterative solvers").  b, x: device complex128 n.  Uses the
 * block-Jacobi preconditioner when opts.precond = 1 or 2 (built on first use
 * for this sigma).  iters (host, may be NULL) receives the iteration count.
 * NOT_CONVERGED if the restart limit is reached (x holds the last iterate). */
stab_status stab_solve(stab_handle h, double sigma_re, double sigma_im, const void* b, void* x, int* iters);

/* Build the block-Jacobi preconditioner for shift sigma (Sec.
 * "Preconditioning"): one dense block per tile of opts.tile grid points with
 * all variables, the principal submatrix of (J_tangent - sigma I) over the
 * tile's unknowns (local order [var][lz][ly][lx]), inverted by LU with partial
 * pivoting and stored in opts.precond_prec precision.  With opts.precond = 2
 * the blocks are those of the reduced operator's tangent, factorised level by
 * level (S_l = D_l - L_l S_{l-1}^{-1} U_{l-1}, each S_l inverted with partial
 * pivoting inside the level).  INVALID_ARG if the tile does not fit the grid
 * (or, for precond 2, ty is odd or a level exceeds 256 unknowns); NUMERIC if a
 * block (a level) is singular. */
stab_status stab_precond_build(stab_handle h, double sigma_re, double sigma_im);

/* z = M^{-1} q with the block-Jacobi preconditioner (built before).  Device complex128 n. */
stab_status stab_precond_apply(stab_handle h, const void* q, void* z);

/* Copy the assembled (unfactored) block of tile t, b x b complex128 row-major, to host memory
 * `out`; assembles it on demand for sigma (diagnostics and tests).  With opts.precond = 2 the
 * reduced operator's block (b = nv * tile points, any size the caller can hold). */
stab_status stab_precond_block(stab_handle h, double sigma_re, double sigma_im, long long t, double* out);

/* Orthogonalise w against the k orthonormal columns of V by classical
 * Gram-Schmidt applied twice (CGS2): h = V^H w (both passes summed) and
 * w <- w - V h; returns ||w|| after.  V: device complex128 n x k, column j at
 * V + j*n; w: device complex128 n (updated in place); hcoef: host complex128 k
 * (may be NULL); norm: host (may be NULL). */
stab_status stab_orthogonalize(stab_handle h, const void* V, int k, void* w, double* hcoef, double* norm);

/* Cayley-transformed IRAM (Algorithm iram on C = (J - sigma I)^{-1}(J - tau I),
 * Eqs. cayley_transform and cayley_arnoldi): nev wanted Ritz values of largest
 * |theta|, ncv Arnoldi vectors (nev < ncv <= n), Ritz estimate of Eq.
 * ritz_estimate with tolerance tol.
 *  v0     : device complex128 start vector or NULL (splitmix64 from opts.seed).
 *  lambda : host complex128 nev (interleaved), eigenvalues of J, ordered by
 *           decreasing |theta|, ties by larger Re then Im of lambda.
 *  vecs   : device complex128 n x nev unit eigenvectors, or NULL.
 *  resid  : host nev true residuals ||J x - lambda x|| / ||x|| (exact tangent J), or NULL.
 *  nconv  : host, number of converged wanted pairs.   stats: may be NULL.
 * NOT_CONVERGED if max_restarts is reached (partial results are returned). */
stab_status stab_eigs(stab_handle h, double sigma_re, double sigma_im, double tau_re, double tau_im,
                      int nev, int ncv, double tol, const void* v0, double* lambda, void* vecs,
                      double* resid, int* nconv, stab_stats* stats);

/* Counters accumulated over the handle's lifetime. */
stab_status stab_get_stats(stab_handle h, stab_stats* stats);

/* The CGS2 step of stab_orthogonalize for callers that cannot allocate device
 * memory (their device memory belongs to another framework's pool, or they run
 * under a fixed device budget reserved up front), so they can neither call
 * cudaMalloc nor create a handle.  The paper has no counterpart: this is a
 * deployment variant.  No handle; no allocation of any kind: the reduction
 * scratch is a file-scope device array of about 1.3 MB that every device
 * loading the library keeps until exit.
 *  V, w   : device complex128, V = k columns of n (column j at V + j*n), w updated in place.
 *  hcoef  : host complex128 k (may be NULL);  norm: host (may be NULL).
 *  stream : cudaStream_t or NULL; the call synchronises it.
 * Limits: 0 <= k <= 128, 1 <= n <= 2^28; larger sizes return INVALID_ARG with
 * a message in stab_last_error(NULL).  All calls share the scratch array, so
 * calls whose GPU work overlaps race: serialise them.  The first call on a
 * device looks up the array's device address (with that device current);
 * make that first call before any stream capture.  The address is kept for
 * the life of the process, so resetting the device (cudaDeviceReset) after
 * the first call is not supported. */
stab_status stab_orthogonalize_noalloc(const void* V, int k, long long n, void* w, double* hcoef, double* norm,
                                       void* stream);

/* Per-kernel device timing (measurement aid; the paper has no counterpart).
 * While enabled, every entry point records a CUDA event pair on the handle's
 * stream around each of the phases below, so a phase's time is its kernels'
 * device time plus the launch gaps inside it.  Work replayed from a captured
 * CUDA graph (the GMRES cycles of stab_solve and stab_eigs) is not split into
 * phases.  Phases: */
typedef enum {
  STAB_PHASE_EPS = 0,        /* ||v|| reduction that fixes epsilon (Eq. frechet) */
  STAB_PHASE_TEMPERATURE = 1,/* temperature perturbation field for the heat flux */
  STAB_PHASE_LINE_Y = 2,     /* compact-derivative line pass along y (first, second derivatives) */
  STAB_PHASE_LINE_Z = 3,     /* line pass along z (3-D only), with the yz mixed derivatives */
  STAB_PHASE_LINE_X = 4,     /* line pass along x, with the xy (xz) mixed derivatives */
  STAB_PHASE_POINTWISE = 5,  /* pointwise assembly of J v - shift v */
  STAB_PHASE_CGS2 = 6,       /* one CGS2 orthogonalisation (all its kernels) */
  STAB_PHASE_PRECOND_APPLY = 7, /* one block-Jacobi apply */
  STAB_PHASE_COUNT = 8
} stab_phase;

/* enable = 1 starts recording (discarding anything recorded), 0 stops.  At
 * most 65536 phase intervals are kept; later ones are counted as dropped. */
stab_status stab_timing(stab_handle h, int enable);

/* Synchronise the stream and return, per phase, the summed milliseconds
 * (ms[STAB_PHASE_COUNT]) and the number of intervals (count[STAB_PHASE_COUNT]);
 * either may be NULL.  dropped (may be NULL) receives the intervals not kept.
 * The record is cleared; recording continues if enabled. */
stab_status stab_timing_read(stab_handle h, double* ms, long long* count, long long* dropped);

/* Autotuner of the compact-derivative line pass (performance only; the paper
 * has no counterpart).  For every axis of h, times each admissible launch
 * shape (C = 16, 32 or 64 points per sweep chunk; L = 1..32 lines per CTA;
 * the first and second derivatives side by side in 6 planes of shared memory
 * per line, or one after the other in 4 or 2)
 * with CUDA events on the handle's stream and keeps the fastest, in h and in a
 * process-wide cache keyed by device, line length, line count, job count and
 * boundary type; stab_create applies cached shapes to new handles.  force = 0
 * reuses a cached shape without timing.  cfg (host int[9], may be NULL)
 * receives (C, L, kinds) per axis (x, y, z; zeros for an absent z), ms (host
 * double[3], may be NULL) the tuned pass time per axis (-1 when cached).
 * The chunk length moves where the sweeps' warm-up starts, so results may
 * change at the rounding level (about 1e-16 relative); L and kinds change nothing.
 * Allocates one temporary vector; synchronises the stream. */
stab_status stab_autotune(stab_handle h, int force, int* cfg, double* ms);

/* Pin the line-pass launch shape of one axis (0 x, 1 y, 2 z): C points per
 * sweep chunk (16, 32 or 64), L lines per CTA (1..32), kinds = 2 to sweep the
 * first and second derivatives side by side, 1 to do them one after the
 * other with 4 instead of 6 planes of shared memory per line, 3 one after the
 * other with 2 planes (the input reloaded per kind and turned into right-hand
 * sides in place); all zero restores the built-in default.
 * INVALID_ARG when the shape does not fit the line (more than 1024 threads,
 * 512 with kinds 3, or the shared-memory limit). */
stab_status stab_set_line_config(stab_handle h, int axis, int C, int L, int kinds);

/* Handles take device memory from a library-owned, stream-ordered pool (one
 * per device; allocation and release are ordered on the handle's stream, so
 * handles on different streams never wait for each other's frees).  Memory a
 * destroyed handle released stays cached for later handles; this returns it
 * to the device.  Returns the number of pools trimmed. */
int stab_trim_memory(void);

/* Write / read the process-wide tuning cache as text ("n nlines njobs
 * periodic C L kinds" per line; loaded entries apply to the current device).
 * Return the number of entries, or -1 if the file cannot be opened. */
int stab_autotune_save(const char* path);
int stab_autotune_load(const char* path);

/* ---------------------------------------------------------------------------
 * Many problems on one GPU (the paper solves one problem at a time; these
 * entry points have no counterpart there).
 * ------------------------------------------------------------------------- */

/* Device memory a handle for this grid and options needs, in bytes, through
 * a full stab_eigs(nev, ncv) including the preconditioner (an upper estimate
 * for the viscous case; yonly = 1 when the base flow varies in y only).
 * -1 for a bad grid. */
long long stab_estimate_bytes(const stab_grid* grid, const stab_opts* opts, int yonly, int nev, int ncv);

/* One solve of a batch: the arguments of stab_eigs, then its outputs. */
typedef struct {
  double sigma_re, sigma_im, tau_re, tau_im;
  int nev, ncv;
  double tol;
  const void* v0;     /* device start vector or NULL */
  double* lambda;     /* host complex128 nev */
  void* vecs;         /* device n x nev or NULL */
  double* resid;      /* host nev or NULL */
  int nconv;          /* out */
  stab_status status; /* out: the solve's own status */
  stab_stats stats;   /* out */
} stab_eig_job;

/* Solver-level batching: GMRES of every instance of the batch in lockstep,
 * (J_i - sigma_i I) x_i = rhs_i (Sec. "Iterative solvers", each handle's
 * options: restart length, tolerance, block-Jacobi preconditioner, built for
 * sigma_i on first use).  Each phase of a GMRES cycle (block apply, J v,
 * CGS2, Givens update, scaling, solution update, true residual) is one
 * launch for all instances; an instance that converges is skipped by the
 * following launches through a device-side flag, and the host reads one
 * report per cycle for all instances.  The orthogonalisation is CGS2 at
 * every size (stab_solve switches to selective reorthogonalisation from
 * 16,384 unknowns), so below that size each x_i equals stab_solve's bit for
 * bit.  sigmas: 2*count doubles (re, im); rhs[i], x[i]: device complex128 of
 * handle i's size; iters (host, count, may be NULL): iterations per instance.
 * Handles with gmres_basis_prec = 32, lgmres_k > 0 or gmres_inner_m > 0: STAB_ERR_UNSUPPORTED.
 * NOT_CONVERGED when an instance reached its restart limit (its x holds the
 * last iterate).  Synchronises the batch's stream. */
stab_status stab_jv_batch_solve(stab_jv_batch b, const double* sigmas, const void* const* rhs, void* const* x,
                                int* iters);
/* Cayley-IRAM (Algorithm iram) of every instance of the batch in lockstep:
 * jobs[i] holds the arguments and receives the outputs of a stab_eigs call on
 * handle i (vecs: device).  The Arnoldi steps of all unfinished instances run
 * as one launch per phase (J v - tau v, the lockstep GMRES above, CGS2, the
 * Hessenberg entries) and the implicit restarts as one launch with one CTA
 * per instance; instances finish independently.  Eigenvalues agree with a
 * lone stab_eigs to rounding (bit for bit below 16,384 unknowns).  Returns
 * STAB_OK, NOT_CONVERGED when a job reached its restart limit, or the first
 * error; each job's own status is in jobs[i].status.  Same restrictions as
 * stab_jv_batch_solve. */
stab_status stab_jv_batch_eigs(stab_jv_batch b, stab_eig_job* jobs);

/* Run stab_eigs(handles[i], jobs[i]) for i < count side by side: up to
 * `concurrency` host threads (<= 0: count), each handle on a private stream
 * for the duration (ordered after the handle's stream; the handle's stream is
 * restored and idle on return).  The handles must be distinct.  Each job gets
 * exactly the result a lone stab_eigs call would give.  Returns STAB_OK or the
 * first failing job's status. */
stab_status stab_eigs_batch(stab_handle* handles, stab_eig_job* jobs, int count, int concurrency);

/* Continuous-batching server: requests of any grid and flow parameters are
 * queued first come, first served; a request starts when one of `slots`
 * worker threads is free and its estimated memory (stab_estimate_bytes) fits
 * in what the running requests leave of mem_budget_bytes.  Each running
 * request has its own handle and stream on the device current at creation,
 * so requests overlap on the GPU; a slot takes the next request as soon as
 * its solve ends.  autotune = 1 tunes (or takes from the cache) the line-pass
 * shapes of each new grid before solving. */
typedef struct stab_server_s* stab_server;

typedef struct {
  const double* base_flow;  /* host FP64 [var][z][y][x]; copied at submit */
  stab_grid grid;
  double Ma, Re, Pr;
  const stab_opts* opts;    /* NULL: defaults; copied at submit */
  double sigma_re, sigma_im, tau_re, tau_im;
  int nev, ncv;
  double tol;
  void* vecs;               /* host complex128 n x nev (vector q at vecs + q n) receiving the unit
                               eigenvectors, or NULL; must stay valid until the request has finished */
} stab_request;

typedef struct {
  stab_status status;       /* the solve's stab_eigs status */
  int nconv;
  double queued_s;          /* submit -> start */
  double run_s;             /* start -> end */
  double latency_s;         /* submit -> end */
  long long est_bytes;      /* admission estimate */
  stab_stats stats;
} stab_request_info;

stab_status stab_server_create(stab_server* server, int slots, long long mem_budget_bytes, int autotune);

/* Lockstep cohorts (default 1): a free worker takes the queue's head and up to
 * cohort - 1 requests queued behind it whose memory fits, and solves those
 * that can be batched (base flow varying in y only, FP64 GMRES basis, no
 * LGMRES) together with stab_jv_batch_eigs, every phase one launch for the
 * cohort; the others run one after the other on the worker.  Each request of
 * a cohort finishes when the cohort does.  Applies to cohorts formed after the
 * call. */
stab_status stab_server_set_cohort(stab_server server, int cohort);

/* Queue a request; *id identifies it.  OOM if its estimate exceeds the whole budget. */
stab_status stab_server_submit(stab_server server, const stab_request* request, long long* id);

/* Wait until request id has finished (timeout_s < 0: no limit).  TIMEOUT if it
 * has not finished in time; INVALID_ARG for an unknown id. */
stab_status stab_server_wait(stab_server server, long long id, double timeout_s);

/* Results of a finished request: lambda (host complex128 nev, eigenvalues as
 * stab_eigs orders them), resid (host nev), info; any may be NULL.  The
 * request is forgotten afterwards.  BUSY if it has not finished. */
stab_status stab_server_result(stab_server server, long long id, double* lambda, double* resid,
                               stab_request_info* info);

/* Peak admitted memory estimate and peak concurrent requests since creation; current queue and running counts. */
stab_status stab_server_stats(stab_server server, long long* peak_bytes, int* peak_running, int* queued, int* running);

/* Stop: requests not yet started finish with status BUSY; running ones complete; threads are joined. */
void stab_server_destroy(stab_server server);

#ifdef __cplusplus
}
#endif
#endif /* STAB_H */
