/*
 * fde.h -- C ABI of the GB300 (sm_103a) Strang-preconditioned BVM/GMRES solver
 * for one-dimensional two-sided space-fractional diffusion equations.
 *
 * Method: X.-M. Gu, T.-Z. Huang, X.-L. Zhao, H.-B. Li, L. Li, "Strang-type
 * preconditioners for solving fractional diffusion equations by boundary value
 * methods" (arXiv:1305.6653).  Equation numbers are the paper's labels.
 *
 *   Problem (Sec. 2, eq. (1.1)):
 *     u_t = d+(x) D^alpha_+ u + d-(x) D^alpha_- u + f(x,t),  x in (xL,xR), t in (t0,T],
 *     u(xL,t) = u(xR,t) = 0,  u(x,t0) = u0(x),  1 < alpha < 2,  d+, d- >= 0, d+ + d- != 0.
 *   Space (Sec. 2.1, eqs. (1.2)-(1.5)): m interior points, dx = (xR-xL)/(m+1),
 *     J = dx^-alpha (D+ G + D- G^T), G the shifted-Grunwald Toeplitz matrix.
 *   Time (Sec. 2.2, eqs. (1.7)-(1.10)): s steps, h = (T-t0)/s, a mu-step BVM with
 *     nu initial and mu-nu final conditions; all time levels at once:
 *     M u = (A (x) I - h B (x) J) u = b.
 *     The given u_0 is eliminated, so the unknowns are u_1..u_s (n = s*m values),
 *     stored time-major: x[(t-1)*m + (i-1)] = u_i at time level t.
 *   Preconditioner (Sec. 3.1, eq. (1.11)): S = s(A) (x) I - h s(B) (x) J, applied as
 *     a length-s FFT along time, s/2+1 dense complex solves with
 *     phi_k I - h psi_k J (LU factored once), and an inverse FFT (Sec. 3.2).
 *   Solver (Sec. 3.2, Sec. 4): restarted GMRES; here the flexible, right-
 *     preconditioned form with FP64 Arnoldi (CGS2), FP64 Givens least squares and
 *     an FP64 true-residual check at every restart.
 *
 * Conventions for every entry point:
 *   - Return value: FDE_OK (0) on success, a negative FDE_ERR_* code otherwise.
 *     The message of the last error on the calling thread is fde_last_error().
 *   - Pointers marked "device" are CUDA device pointers of the current device;
 *     pointers marked "host" are ordinary host memory.  Pointers in a
 *     fde_problem_desc are host or device according to desc->device_ptrs.
 *   - All work is enqueued on the CUDA stream given to fde_problem_create (NULL =
 *     the legacy default stream).  Entry points that return results to the host
 *     (pgmres_solve's stats, fde_last_error) synchronise that stream.
 *   - Calls on one fde_problem are not thread-safe; distinct problems are
 *     independent.  No entry point falls back to a CPU implementation: if the
 *     GPU path cannot run, the call fails with FDE_ERR_CUDA.
 */
#ifndef FDE_H_
#define FDE_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define FDE_OK 0
#define FDE_ERR_ARG (-1)           /* invalid argument (message says which) */
#define FDE_ERR_ALLOC (-2)         /* device allocation failed */
#define FDE_ERR_CUDA (-3)          /* a CUDA runtime call or kernel failed */
#define FDE_ERR_SINGULAR (-4)      /* zero / non-finite pivot in a block LU */
#define FDE_ERR_NOT_CONVERGED (-5) /* maxit reached before the tolerance */
#define FDE_ERR_NAN (-6)           /* non-finite residual or Hessenberg entry */
#define FDE_ERR_STATE (-7)         /* call order violated (e.g. solve before factor) */
#define FDE_ERR_TIMEOUT (-8)       /* a bounded device wait ran out */

/* ---- BVM families (Sec. 2.2; Sec. 4 uses the fifth-order GAM, mu = 4) ---- */
#define FDE_GBDF 1 /* generalised BDF: beta = e_nu, order mu */
#define FDE_GAM 2  /* generalised Adams: rho(z) = z^nu - z^(nu-1), order mu+1 */
#define FDE_ETR 3  /* extended trapezoidal rule: the GAM with odd mu (symmetric) */

/* ---- precision of the preconditioner (block LU, its solves, the time FFT) */
#define FDE_FP64 0 /* everything in FP64: the plain method */
#define FDE_FP32 1 /* FP32 factors computed on CUDA cores */
#define FDE_TF32 2 /* FP32 factors, trailing updates on tcgen05 tensor cores (TF32 in, FP32 acc) */
#define FDE_BF16 3 /* FP32 factors, trailing updates on tcgen05 tensor cores (BF16 in, FP32 acc) */
#define FDE_TF32X3 4 /* as FDE_TF32 with split operands (hi + lo): three TF32 products, FP32-level accuracy */

/* Limits of this implementation. */
#define FDE_MAX_MU 6      /* BVM steps */
#define FDE_MAX_S 1024    /* time steps; s must be a power of two, s >= 2*mu */
#define FDE_MAX_M 4095    /* interior points; the Toeplitz FFT length is <= 8192 */

/* Problem description (eq. (1.1) on the grid of Sec. 2.1/2.2).  Copied by
 * fde_problem_create; the caller may free its buffers afterwards. */
typedef struct {
    int m;          /* interior spatial points N (Sec. 2.1), 1 <= m <= FDE_MAX_M */
    int s;          /* time steps (Sec. 2.2), power of two, 2*mu <= s <= FDE_MAX_S */
    double alpha;   /* fractional order, 1 < alpha < 2 */
    double xL, xR;  /* spatial interval, xL < xR */
    double t0, T;   /* time interval, t0 < T */
    const double* dplus;  /* length m: d+(x_i), i = 1..m, or NULL to use dplus_c */
    const double* dminus; /* length m: d-(x_i), or NULL to use dminus_c */
    double dplus_c, dminus_c; /* constant coefficients used when the arrays are NULL */
    int family;     /* FDE_GBDF, FDE_GAM or FDE_ETR */
    int mu;         /* number of steps, 1 <= mu <= FDE_MAX_MU (ETR: odd) */
    const double* u0; /* length m: u0(x_i) */
    const double* f;  /* length (s+1)*m, row-major [n][i]: f(x_i, t_n), n = 0..s */
    int device_ptrs;  /* 0: dplus/dminus/u0/f/dplus_t/dminus_t are host pointers, 1: device pointers */
    /* Coefficients that vary in time, d+-(x_i, t_n) (eq. (1.1) allows them): NULL, or
     * length (s+1)*m, row-major [n][i], n = 0..s.  Both or neither are given; when
     * given, dplus/dminus/dplus_c/dminus_c are ignored, the matvec applies J_n =
     * dx^-alpha (D+(t_n) G + D-(t_n) G^T) at each time level (the BVM on
     * u' = J(t) u + f), and the Strang / BCCB preconditioners use the means of d+-
     * over n = 1..s.  Not supported by fde_batch_create (FDE_ERR_ARG). */
    const double* dplus_t;
    const double* dminus_t;
} fde_problem_desc;

/* Options of pgmres_solve. */
typedef struct {
    double tol;    /* stop when ||b - M x||_2 <= tol * ||b||_2 (true FP64 residual) */
    int restart;   /* Krylov subspace size per cycle (the paper uses 20) */
    int maxit;     /* cap on the total number of inner iterations */
    int reorth;    /* 1: classical Gram-Schmidt with one re-orthogonalisation (CGS2); 0: CGS */
    int matvec_precision; /* FDE_FP64 (0): every product M z in FP64.  FDE_FP32: the Arnoldi
                   * products w = M z_j apply the Toeplitz part J (Sec. 2.1, the FFT of the
                   * circulant embedding) in FP32 while the cycle's Givens estimate of
                   * ||r|| / ||b|| is above `relax`, in FP64 below it (an inexact-Krylov
                   * relaxation: early products may be inexact, late ones may not); the
                   * restart's true residual is always FP64. */
    double relax;  /* the switch-over for FDE_FP32 (0: FP32 in every Arnoldi product) */
} fde_pgmres_opts;

/* Statistics returned by pgmres_solve. */
typedef struct {
    int status;          /* FDE_OK or the FDE_ERR_* code also returned */
    int iterations;      /* total inner (Arnoldi) iterations, the paper's ITS */
    int restarts;        /* completed restart cycles */
    int precision;       /* precision of the factors used */
    double rel_residual; /* final ||b - M x|| / ||b|| (FP64, recomputed) */
    double rel_residual_estimate; /* final Givens estimate of the last cycle */
    double ms_solve;     /* device time of the solve (CUDA events) */
    int x0_rejected;     /* 1: the initial guess had ||b - M x0|| > ||b|| and x = 0 was used */
    int matvecs_fp32;    /* Arnoldi products that used the FP32 Toeplitz apply */
} fde_stats;

typedef struct fde_problem fde_problem;

/* Validate desc (alpha in (1,2), d+/d- >= 0 with d+ + d- != 0 at every point,
 * sizes, scheme, finite inputs), copy its arrays to the device and derive the BVM
 * coefficients of eqs. (1.7)-(1.9) (exact rationals) and the Strang symbols.
 * stream: a cudaStream_t (NULL = default stream).  *out receives the handle, owned
 * by the caller and released with fde_problem_destroy.  Errors: FDE_ERR_ARG,
 * FDE_ERR_ALLOC, FDE_ERR_CUDA. */
int fde_problem_create(const fde_problem_desc* desc, void* stream, fde_problem** out);

/* Assemble the space-time system (eqs. (1.2)-(1.5), (1.10)): Grunwald weights
 * g_0..g_{m+1} (eq. (1.2) recurrence), the FFT symbol of the circulant embedding
 * of G, and the right-hand side b = -A[:,0] (x) u0 + h B[:,0] (x) (J u0 + f_0)
 * + h (B[:,1:] (x) I) f_{1:s}.  M itself is never formed.  Errors: FDE_ERR_CUDA. */
int bvm_assemble(fde_problem* p);

/* Form and factor the s/2+1 distinct Strang blocks phi_k I - h psi_k J
 * (eq. (1.11), Sec. 3.2) by blocked complex LU without pivoting (the blocks are
 * strictly row diagonally dominant), in the given precision (FDE_FP64, FDE_FP32,
 * FDE_TF32, FDE_BF16, FDE_TF32X3).  The library owns the factors (FP64: 16*(s/2+1)*mp^2
 * bytes, otherwise 8*(s/2+1)*mp^2, mp = m rounded up to 64).  The tensor-core
 * precisions (FDE_TF32, FDE_BF16, FDE_TF32X3) with mp a multiple of 128 also write a
 * copy of the factors in the order the block solves stream them (32-column strips,
 * rows contiguous), in the storage fde_factor_storage selects: 8*(s/2+1)*mp^2 bytes
 * more (FP32) or 4*(s/2+1)*mp^2 (bfloat16); when that memory cannot be had, the
 * block solves read the factors themselves.  Requires bvm_assemble.  Errors:
 * FDE_ERR_ARG, FDE_ERR_ALLOC, FDE_ERR_SINGULAR, FDE_ERR_STATE, FDE_ERR_CUDA. */
int strang_precond_factor(fde_problem* p, int precision);

/* Storage of the copy of the factors that the block solves of the preconditioner
 * (Sec. 3.2: one forward and one backward triangular solve per Strang block and
 * application) read after a tensor-core factorisation:
 *   FDE_STORAGE_FP32  (default) the FP32 factor values;
 *   FDE_STORAGE_BF16  the factor values rounded to bfloat16 (8-bit significand, to
 *                     nearest even): half the bytes each application streams.  The
 *                     block solves still compute in FP32 and the diagonal 32 x 32
 *                     tiles enter through their FP32 inverses; the preconditioner is
 *                     then the exact inverse of slightly perturbed factors, which the
 *                     flexible outer iteration in FP64 (true residual) tolerates.
 * Takes effect at the next strang_precond_factor, or fde_batch_factor for an instance
 * of a batch (fde_batch_problem; there only FDE_STORAGE_BF16 makes a copy, and the
 * instances of a shared operator read the factors themselves); the factors
 * themselves (fde_get_factor_block) stay FP32.  Errors: FDE_ERR_ARG. */
#define FDE_STORAGE_FP32 0
#define FDE_STORAGE_BF16 1
int fde_factor_storage(fde_problem* p, int storage);

/* Set up the Strang-type BCCB preconditioner S^(2) = s(A) (x) I - h s(B) (x) s(J)
 * (eq. (x1), Sec. 3.1), or with modified != 0 the preconditioner S~^(2) of eq. (xc),
 * whose eigenvalue phi_0 = 0 of s(A) is replaced by Re(phi_{s-1}).  s(J) =
 * dx^-alpha (mean(d+) s(G) + mean(d-) s(G)^T), s(G) the Strang circulant of G with
 * first column [g_1, .., g_K, 0, .., 0, g_0], K = floor((m+1)/2).  It is applied by
 * the two-dimensional Fourier diagonalisation of Sec. 3.3: the FFT along time, one
 * circulant solve per time frequency (a length-L FFT convolution with the first
 * column of the circulant inverse), the inverse FFT along time.  precision:
 * FDE_FP64 or FDE_FP32 arithmetic of the apply (the set-up is FP64).  After this
 * call pgmres_solve and fde_precond_apply use S^(2) (or S~^(2)) until
 * strang_precond_factor selects S again; no block LU is formed.  The library owns
 * the spectra (16 (s/2+1) L + 8 (s/2+1) L bytes, L = the power of two >= 2m).
 * Requires bvm_assemble.  Errors: FDE_ERR_ARG, FDE_ERR_STATE, FDE_ERR_ALLOC,
 * FDE_ERR_SINGULAR (a zero eigenvalue of the preconditioner), FDE_ERR_CUDA. */
int bccb_precond_setup(fde_problem* p, int modified, int precision);

/* Select no preconditioner (the column "I" of Tables 1-2, Sec. 4): pgmres_solve then
 * runs plain restarted GMRES on M u = b (z_j = v_j).  Requires bvm_assemble.
 * strang_precond_factor or bccb_precond_setup select a preconditioner again.
 * Errors: FDE_ERR_ARG, FDE_ERR_STATE. */
int fde_precond_none(fde_problem* p);

/* Solve M u = b by flexible GMRES(restart) right-preconditioned with S (or with the
 * BCCB preconditioner after bccb_precond_setup, or none after fde_precond_none).
 * x0: length s*m initial guess (u_1..u_s of eq. (1.10), time-major), or NULL for
 * zero; a guess whose residual exceeds ||b|| (or is not finite) is replaced by zero
 * (stats->x0_rejected).  x_out: length s*m (may alias x0).  Both are device pointers
 * when the problem was created with desc->device_ptrs = 1 and host pointers when it
 * was created with 0; in the host case the library copies x0 in and the solution out
 * on the problem's stream (a device copy of n doubles, allocated at the first such
 * solve, is owned by the problem) and the call returns after the copy.  st: host,
 * may be NULL.  On FDE_ERR_NOT_CONVERGED x_out holds the last iterate.  Requires strang_precond_factor or bccb_precond_setup.  Errors: FDE_ERR_ARG,
 * FDE_ERR_STATE, FDE_ERR_NOT_CONVERGED, FDE_ERR_NAN, FDE_ERR_CUDA. */
int pgmres_solve(fde_problem* p, const fde_pgmres_opts* opts, const double* x0, double* x_out,
                 fde_stats* st);

/* Release the handle and every device buffer it owns.  NULL is ignored. */
void fde_problem_destroy(fde_problem* p);

/* Message of the last error on this thread ("" if none).  Owned by the library. */
const char* fde_last_error(void);

/* ---- batches of independent problems -------------------------------------- */

/* A batch of independent instances of eq. (1.1) (uneven m, s, alpha, d and BVM
 * scheme) solved together: the Strang-block LUs of all instances run as one set of
 * launches per panel step, and flexible GMRES runs in lock-stepped restart rounds
 * whose kernels cover all active instances at once (Sec. 3.2 per instance). */
typedef struct fde_batch fde_batch;

/* Create count problems (each validated and copied as by fde_problem_create) on
 * one stream.  Errors: as fde_problem_create (message names the instance). */
int fde_batch_create(const fde_problem_desc* descs, int count, void* stream, fde_batch** out);

/* bvm_assemble for every instance.  Errors: as bvm_assemble. */
int fde_batch_assemble(fde_batch* b);

/* Factor the Strang blocks of every instance in FDE_FP32, FDE_TF32, FDE_BF16 or
 * FDE_TF32X3 (FP32 factor storage; with the tensor-core precisions an instance set to
 * FDE_STORAGE_BF16 by fde_factor_storage also gets the bfloat16 copy of its factors
 * and the FP32 inverses of their diagonal 32 x 32 tiles for its block solves).  Errors: FDE_ERR_ARG, FDE_ERR_STATE, FDE_ERR_ALLOC,
 * FDE_ERR_SINGULAR, FDE_ERR_TIMEOUT, FDE_ERR_CUDA. */
int fde_batch_factor(fde_batch* b, int precision);

/* Solve every instance from a zero initial guess.  x_out: host array of count
 * pointers, entry i of length s_i*m_i, written with u_1..u_s: a device pointer when
 * instance i was created with device_ptrs = 1, a host pointer when with 0 (copied
 * out on the batch's stream before the call returns).  stats: host
 * array of count entries (may be NULL); ms_solve is the batch's total time.
 * Returns FDE_OK when every instance met the tolerance, else the first failing
 * code (each instance's own code is in stats[i].status). */
int fde_batch_solve(fde_batch* b, const fde_pgmres_opts* opts, double* const* x_out, fde_stats* stats);

/* Declare that every instance has the same operator M and preconditioner (m, s, alpha,
 * interval, BVM scheme and coefficients d+, d- equal; only u0 and f differ): many
 * right-hand sides of one problem.  fde_batch_factor then factors the Strang blocks
 * once (instance 0, through strang_precond_factor) and the block solves of every
 * Arnoldi step take the right-hand sides in groups per CTA (one CTA per Strang block
 * and group; fde_batch_block_solver), so each factor plane is streamed from HBM once
 * per group instead of once per right-hand side.  Call after
 * fde_batch_create and before fde_batch_factor.  Errors: FDE_ERR_ARG (an instance has
 * another operator), FDE_ERR_STATE, FDE_ERR_CUDA.  (The paper solves one right-hand
 * side; the factors depend on J, A and B only, Sec. 3.2.) */
int fde_batch_share_operator(fde_batch* b);

/* Block solves of a shared-operator batch (Sec. 3.2: every right-hand side reuses the
 * factors of the s/2+1 Strang blocks).
 *   FDE_BLOCK_SOLVE_CUDA_CORES    groups of 8 right-hand sides per CTA, FP32 arithmetic
 *                                 on CUDA cores with the FP32 factors.
 *   FDE_BLOCK_SOLVE_TENSOR_CORES  groups of 16 per CTA as tcgen05 products in TF32, in
 *                                 strips of 128 rows: the off-diagonal blocks of L and U
 *                                 from the factor planes, the diagonal blocks through
 *                                 their inverses kept by the tensor-core LU (extra
 *                                 device memory: (s/2+1) m_p^2 x 16 bytes).  Needs
 *                                 FDE_TF32 factors and 256 <= m_p <= 2048.
 *   FDE_BLOCK_SOLVE_AUTO          (default) tensor cores where they apply, else CUDA cores.
 * The TF32 products make the preconditioner coarser than the FP32 block solves, which
 * may cost an iteration; the solution is held to the same true FP64 residual.  Call
 * after fde_batch_share_operator and before fde_batch_factor (the choice is taken at
 * the factorisation).  Errors: FDE_ERR_ARG (unknown solver; tensor cores requested
 * where they do not apply: reported by fde_batch_factor), FDE_ERR_STATE. */
#define FDE_BLOCK_SOLVE_AUTO 0
#define FDE_BLOCK_SOLVE_CUDA_CORES 1
#define FDE_BLOCK_SOLVE_TENSOR_CORES 2
int fde_batch_block_solver(fde_batch* b, int solver);

/* Number of instances, and the problem handle of instance i (owned by the
 * batch; usable with the step-level entry points; NULL if out of range). */
int fde_batch_size(const fde_batch* b);
fde_problem* fde_batch_problem(fde_batch* b, int i);

/* Release the batch and all its instances.  NULL is ignored. */
void fde_batch_destroy(fde_batch* b);

/* ---- learned warm start ----------------------------------------------------
 * A 1-D convolutional neural operator (the paper has no counterpart) that predicts
 * a space-time initial guess for pgmres_solve.  It works with sine-series
 * coefficients c_j = 2/(m+1) sum_i v(x_i) sin(j pi i/(m+1)), j = 1..modes: the
 * convolution runs along the mode index over s+6 input channels [c_j(u0),
 * c_j(f(.,t_n)) for n = 0..s, (alpha-1.5)/0.4, (mean d+ - 1.25)/0.75,
 * (mean d- - 1.25)/0.75, j/modes] and its s output channels are the coefficients
 * of u_1..u_s (v(x_i) = sum_j c_j sin(j pi i/(m+1))).  Layers:
 * `layers` convolutions of odd size `ksize` (<= 7), zero padding, width `width`,
 * ReLU after all but the last.  Parameters (FP32, flat, per layer W (C_out, C_in,
 * K) then b (C_out)) start He-uniform from `seed` (counter-based splitmix64).
 * Activations are [batch][channel][mode] float arrays on the device. */
typedef struct fde_nop fde_nop;
int fde_nop_create(int m, int s, int modes, int width, int layers, int ksize, unsigned long long seed, void* stream,
                   fde_nop** out);
long long fde_nop_num_params(const fde_nop* n);
int fde_nop_in_channels(const fde_nop* n);
/* Copy the flat parameter vector from / to host memory. */
int fde_nop_set_params(fde_nop* n, const float* params);
int fde_nop_get_params(fde_nop* n, float* params);
/* FP32 forward of `batch` samples: in (device, batch x (s+6) x modes) -> out (device, batch x s x modes). */
int fde_nop_forward(fde_nop* n, const float* in, float* out, int batch);
/* Forward, mean-squared-error loss against target (device, batch x s x modes) and
 * backpropagated gradients (kept on the device for fde_nop_adam_step; also copied
 * to grad_host when not NULL).  *loss (host) receives the loss. */
int fde_nop_loss_grad(fde_nop* n, const float* in, const float* target, int batch, double* loss, float* grad_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradients. */
int fde_nop_adam_step(fde_nop* n, float lr);
/* Input channels of problem p (device, (s+6) x modes); p must have the network's m and s. */
int fde_nop_features(fde_nop* n, fde_problem* p, float* in);
/* Sine coefficients (device, s x modes) of a space-time vector x (device, s*m): training targets. */
int fde_nop_coefficients(fde_nop* n, const double* x, float* coef);
/* Space-time vector x (device, s*m) from sine coefficients (device, s x modes). */
int fde_nop_synthesize(fde_nop* n, const float* coef, double* x);
/* Predict the initial guess for p (device, s*m doubles): features, FP16 inference
 * (FP16 weights and activations, FP32 accumulation), synthesis on the grid. */
int fde_nop_warm_start(fde_nop* n, fde_problem* p, double* x0);
void fde_nop_destroy(fde_nop* n);

/* ---- step-level entry points (the same kernels the solver runs) ---------- */

/* y = M z (eq. (1.10), u_0 eliminated) in FP64 on the device: the band of A and B
 * along time and J applied to all s time columns through the FFT of the Toeplitz
 * circulant embedding (Sec. 2.1).  z, y: device, length s*m, must not alias.
 * Requires bvm_assemble.  Errors: FDE_ERR_STATE, FDE_ERR_CUDA. */
int fde_matvec(fde_problem* p, const double* z, double* y);

/* y = M z like fde_matvec, with the Toeplitz apply J w of every time row in FP32
 * (Sec. 2.1: both FFTs of the circulant embedding and the symbol product); the BVM
 * band sums, the A-band part and y are FP64.  The product pgmres_solve uses for the
 * relaxed Arnoldi steps of opts->matvec_precision = FDE_FP32.  Problems with time-
 * dependent coefficients use the FP64 product.  z, y: device, length s*m, must not
 * alias.  Requires bvm_assemble.  Errors: FDE_ERR_STATE, FDE_ERR_CUDA. */
int fde_matvec_fp32(fde_problem* p, const double* z, double* y);

/* z = S^{-1} r with the current factors (Sec. 3.2): FFT along time, the s/2+1
 * block solves, inverse FFT.  r, z: device, length s*m (may alias).  Requires
 * strang_precond_factor.  Errors: FDE_ERR_STATE, FDE_ERR_CUDA. */
int fde_precond_apply(fde_problem* p, const double* r, double* z);

/* z = S^{-1} r like fde_precond_apply, for callers that cannot allocate device
 * memory at the time of the call: applications whose memory manager owns the
 * whole device after start-up, or code that must not risk the implicit device
 * synchronisation of cudaMalloc.  The paper has no counterpart; this is a
 * deployment variant.  It allocates nothing: the frequency-domain scratch (the
 * s/2+1 transformed right-hand sides, (s/2+1) * mp complex values in the factor
 * precision) lives in a file-scope static device array of 8 MiB that every GPU
 * loading the library holds until exit.  Problems whose scratch would exceed
 * 8 MiB are rejected with FDE_ERR_ARG (FP64: (s/2+1)*mp <= 524288, FP32/TF32/BF16:
 * <= 1048576).  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the last
 * call's contents (each call overwrites everything it reads), so calls whose GPU
 * work overlaps -- on different streams or problems -- race and must be
 * serialised by the caller.  r, z: device, length s*m (may alias).  Requires
 * strang_precond_factor (checked first: FDE_ERR_STATE before the size check, which
 * uses the factor precision).  Errors: FDE_ERR_ARG, FDE_ERR_STATE, FDE_ERR_CUDA. */
int fde_precond_apply_noalloc(fde_problem* p, const double* r, double* z);

/* Copy the assembled right-hand side b (device, length s*m).  Requires
 * bvm_assemble.  Errors: FDE_ERR_STATE, FDE_ERR_CUDA. */
int fde_get_rhs(fde_problem* p, double* b);

/* Copy the packed LU factors of Strang block k (0 <= k <= s/2) to host memory as
 * FP64 complex: re and im, each m*m row-major (unit-lower L below the diagonal,
 * U on and above it).  Requires strang_precond_factor.  Errors: FDE_ERR_ARG,
 * FDE_ERR_STATE, FDE_ERR_CUDA. */
int fde_get_factor_block(fde_problem* p, int k, double* re, double* im);

/* Copy the Grunwald weights g_0..g_{m+1} (host, m+2 values) computed on the
 * device by the recurrence of eq. (1.2).  Errors: FDE_ERR_STATE, FDE_ERR_CUDA. */
int fde_get_grunwald(fde_problem* p, double* g);

/* Sizes of a created problem: n = s*m unknowns, number of Strang blocks s/2+1. */
int fde_problem_sizes(const fde_problem* p, int* m, int* s, int* nblocks);

/* ---- measurement ---------------------------------------------------------- */

/* Stages timed by the per-problem profiler. */
#define FDE_STAGE_ASSEMBLE 0   /* Grunwald weights, twiddles, symbols, J u0, b */
#define FDE_STAGE_FORM 1       /* forming the Strang blocks phi_k I - h psi_k J */
#define FDE_STAGE_LU_DIAG 2    /* LU of the diagonal blocks (NB x NB; 128 x 128 with inverses on tensor-core paths) */
#define FDE_STAGE_LU_PANEL 3   /* panel triangular solves */
#define FDE_STAGE_LU_UPDATE 4  /* complex rank-32 updates on CUDA cores */
#define FDE_STAGE_TFFT_FWD 5   /* FFT along time */
#define FDE_STAGE_TRSV 6       /* block forward / backward substitution */
#define FDE_STAGE_TFFT_INV 7   /* inverse FFT along time */
#define FDE_STAGE_MATVEC 8     /* M z */
#define FDE_STAGE_KRYLOV 9     /* Gram-Schmidt, norms, Givens, updates */
#define FDE_STAGE_LU_TC 10     /* rank-128 trailing updates on tcgen05 (FDE_TF32 / FDE_BF16) */
#define FDE_STAGE_LU_PACK 11   /* packing panels into tensor-core operand tiles (tensor-core paths) */
#define FDE_STAGE_LU_PANEL_TC 12 /* panel products L21 = A21 U11^-1, U12 = L11^-1 A12 on tcgen05 */
#define FDE_NUM_STAGES 13

/* on != 0: record a CUDA event pair around every kernel launch of this problem
 * (on its stream) and clear previous records; on == 0: stop recording.
 * Errors: FDE_ERR_ARG. */
int fde_profile_enable(fde_problem* p, int on);

/* Time only the stages whose bit (1 << FDE_STAGE_x) is set in stage_mask, without
 * changing how the solver runs: the GMRES inner iterations keep replaying their
 * CUDA graphs, and the event pairs around the selected stages are recorded inside
 * those graphs (event-record nodes) and read after each replay.  Clears previous
 * records and turns fde_profile_enable's full profiler off; stage_mask 0 stops
 * recording.  Errors: FDE_ERR_ARG (NULL problem, bits beyond FDE_NUM_STAGES). */
int fde_profile_select(fde_problem* p, unsigned stage_mask);

/* Total device time (ms, summed over launches) and number of launches recorded
 * for one stage since fde_profile_enable or fde_profile_select.  Synchronises the problem's stream.
 * Errors: FDE_ERR_ARG, FDE_ERR_CUDA. */
int fde_profile_read(fde_problem* p, int stage, double* total_ms, int* launches);

/* Number of kernels this library has launched in this process (all problems). */
long long fde_launch_count(void);

/* ---- launch-shape autotuner ----------------------------------------------
 * Two kernel families have variants that compute bit-identical results and differ
 * only in how the work is spread over threads: the space-time matvec (threads per
 * time row: 1024, 512, 256, i.e. one, two or more CTAs per SM) and the block
 * triangular solves (512 threads with 4 rows per register buffer, 384 with 8, 640
 * with 2 -- reading a bfloat16 factor copy: 4, 7 and 3 -- or 512 threads fed by bulk
 * asynchronous copies through a ring of shared-memory stages, which reads the FP32
 * factors; with a bfloat16 copy that fourth setting launches the first shape, and the
 * tuner times the three register shapes).  By default the first use of a shape (the matvec in bvm_assemble, the
 * block solves at the end of strang_precond_factor) times every variant with CUDA
 * events on the problem's stream and keeps the fastest for that shape (m_p, s or
 * s/2+1 blocks, precision) in a process-wide table, which is also appended to a text
 * file ($FDE_TUNE_CACHE, default $HOME/.cache/libfde_tune.txt; FDE_TUNE_CACHE=""
 * keeps it in memory) and read back by later processes. */
#define FDE_TUNE_MATVEC 0
#define FDE_TUNE_TRSV 1
/* The interior trailing update of the tensor-core block LU (FDE_TF32 / FDE_BF16 /
 * FDE_TF32X3): 0 row-pair tiles, 1 warp-specialized CTAs of four tiles with two TMEM
 * accumulators (one tile's epilogue overlaps the next tile's MMAs), 2 warp-specialized
 * CTAs of eight tiles whose C tiles stream through a ring of tensor-map copies (m_p a
 * multiple of 128, else row pairs); bit-identical.  Not timed automatically (a
 * factorisation is too long to repeat at first use): variant 2 unless fde_tune_set
 * selects one. */
#define FDE_TUNE_LU 2
#define FDE_TUNE_KERNELS 3
/* variant -1: autotune (the default); 0 .. n-1: always launch that variant.
 * Before a shape is measured the built-in default runs (block solves with FP32
 * factors: 1, the 384 x 8 shape; with the bfloat16 copy: 0, 512 threads; LU interior
 * update: 2; otherwise 0); measuring keeps the default unless
 * another variant is faster by more than 2 % (median of five interleaved rounds).
 * Process-wide.  Errors: FDE_ERR_ARG. */
int fde_tune_set(int kernel, int variant);
/* Use `path` for the tuning table (NULL or "": memory only), dropping the table in
 * memory and loading the file's entries.  Errors: none. */
int fde_tune_cache(const char* path);
/* The variant the table holds for a shape (nb: s for the matvec, s/2+1 for the block
 * solves), the forced variant when one is set, or -1 if the shape is not tuned yet.
 * precision: FDE_FP64 or FDE_FP32 for the matvec; for the block solves the storage of
 * the factors they read: FDE_FP64, FDE_FP32, or FDE_BF16 for the bfloat16 copy
 * (fde_factor_storage).  Errors: FDE_ERR_ARG. */
int fde_tune_query(int kernel, int mp, int nb, int precision, int* variant);

/* Return the library's cached device memory to the CUDA driver.  Buffers freed by
 * fde_problem_destroy / fde_batch_destroy (and replaced workspaces) are kept in a
 * process-wide cache of at most 16 GiB, keyed by exact size, so that the next
 * problem of the same shape reuses them without cudaMalloc / cudaFree; the cache
 * is also emptied for a device when an allocation on it fails.  This call frees
 * every cached block on every device; buffers of live problems are not touched.
 * Thread-safe.  Makes no CUDA call when the cache is empty.  Errors: FDE_ERR_CUDA
 * (a cudaFree failed; the cache is emptied all the same). */
int fde_release_cached_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* FDE_H_ */
