/*
 * fde.h - C ABI of the GB300 (sm_103a) ADMM / Toeplitz-FFT library.
 *
 * The library solves the box-constrained convex quadratic program of
 * Pougkakiotis, Pearson, Leveque, Gondzio, "Fast Solution Methods for Convex
 * Fractional Differential Equation Optimization" (arXiv:1907.13428):
 *
 *   min 1/2 (y - ybar)^T J1 (y - ybar) + 1/2 u^T J2 u
 *   s.t. B y + psi u = psi g,  ya <= y <= yb,  ua <= u <= ub          (Sec. 4, Eq. FDEOpt)
 *
 * with B = psi (C_t (x) I - I (x) (X (x) I + I (x) Y)) the psi-scaled three-level
 * Toeplitz operator of Eq. (FDE constraint matrix) and Section 5, where
 * X = d+ L_x + d- L_x^T and Y = e+ L_y + e- L_y^T are built from shifted
 * Gruenwald-Letnikov matrices (Eq. RL_GL), C_t is the Gruenwald-Letnikov time
 * matrix (Eq. Caputo matrix; alpha_t = 1 is implicit Euler) and J1 = diag(w),
 * J2 = gamma diag(w) (Eq. discretized Objective function).
 *
 * Conventions shared by every entry point:
 *  - Vectors have N = nt*nx*ny entries laid out [t][x1][x2] (x2 fastest; the
 *    lexicographic ordering of Section 2), interior points only, times
 *    t_1..t_nt (t = 0 is the zero initial state).
 *  - Unless stated otherwise, array arguments are DEVICE pointers owned by
 *    the caller, contiguous, of element type double (FDE_FP64 / FDE_MIXED /
 *    FDE_MIXED_DF) or float (FDE_FP32). They must stay valid until the work queued on `stream`
 *    has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). All GPU work is queued on it; calls return when the work is
 *    queued, except where a call must read a convergence scalar back (PCG,
 *    ADMM), which synchronises `stream`.
 *  - The library owns its workspace: fde_setup allocates it (cudaMalloc),
 *    fde_destroy frees it. A problem handle must not be used by two host
 *    threads at once, nor on two streams concurrently.
 *  - Every int-returning call returns FDE_OK (0) or a negative FDE_E* code;
 *    nothing throws across the ABI. fde_strerror gives a static message.
 *    On error, outputs are unspecified except where stated.
 */
#ifndef FDE_H
#define FDE_H

#ifdef __cplusplus
extern "C" {
#endif

enum fde_status {
  FDE_OK = 0,
  FDE_EINVAL = -1,       /* argument outside its domain                                   */
  FDE_ENOMEM = -2,       /* device allocation failed                                      */
  FDE_ECUDA = -3,        /* a CUDA call failed (see fde_last_cuda_error)                   */
  FDE_ENOCONV = -4,      /* iteration cap reached; outputs hold the last iterate           */
  FDE_EBREAKDOWN = -5,   /* PCG breakdown (p^T S p <= 0)                                   */
  FDE_ENONFINITE = -6,   /* NaN or Inf met in a reduction                                  */
  FDE_EUNSUPPORTED = -8, /* size or mode the library does not handle                      */
  FDE_ETIMEOUT = -9      /* a bounded device-side wait of the persistent batch solve ran out */
};

/* Arithmetic of an operator application or of a solve. */
enum fde_precision {
  FDE_FP64 = 0,   /* everything in double                                                   */
  FDE_FP32 = 1,   /* operator/preconditioner in float, float arrays (fde_matvec/fde_precond) */
  FDE_MIXED = 2,  /* solves only: float operator+preconditioner inside a double-precision
                     iterative-refinement loop; double arrays at the interface               */
  FDE_MIXED_DF = 3, /* as FDE_MIXED, but the double products of the refinement (residuals,
                     B y) run their FFTs in double-float arithmetic (a pair of floats,
                     about 48 significand bits, relative error ~1e-14) instead of double;
                     vectors, scalars and epilogues stay double. In fde_matvec: B or B^T
                     (not S) on double arrays with that arithmetic. Not in the paper:
                     a GB300 choice, its float rate is 58x its double rate               */
  FDE_MIXED_DFV = 4 /* solves only: as FDE_MIXED_DF for the refinement evaluations that
                     cannot be the last one (the next float correction cannot reach the
                     target: rel * inner_tol_mixed > tol), double for the others; an
                     evaluation that meets the target in double-float is repeated in
                     double. The accepted residual of every sub-problem and the B y that
                     feeds the ADMM step are double products. The first evaluation of a
                     warm-started sub-problem, which only steers the first correction,
                     runs in float while the warm starts are far from the solutions
                     (relative residual >= 1e-3). Batches: every evaluation but the last
                     in double-float, the last in double.                                */
};

enum fde_op {
  FDE_OP_B = 0,   /* y = B x                                                                */
  FDE_OP_BT = 1,  /* y = B^T x (left and right GL matrices swapped, time reversed)          */
  FDE_OP_S = 2    /* y = S x = M1 x + B^T M2^-1 B x (Eq. generic ADMM normal equations)      */
};

/* Problem description (Sections 4 and 6.1). */
typedef struct fde_params {
  int nx, ny, nt;            /* interior points along x1, x2 and time steps; each in [1, 4096]  */
  double T;                  /* final time (h_t = T/nt when time_step_mode == 0)                 */
  double beta_x, beta_y;     /* spatial orders, each in (1, 2)                                   */
  double alpha_t;            /* time order in (0, 1]; 1 = implicit Euler                         */
  double dp, dm;             /* coefficients of L_x and L_x^T (x1 axis), >= 0                     */
  double ep, em;             /* coefficients of L_y and L_y^T (x2 axis), >= 0                     */
  double gamma;              /* control regularisation, > 0                                      */
  int weights;               /* 0: trapezoid in time (last slice weight 1/2), 1: uniform         */
  int time_step_mode;        /* 0: h_t = T/nt, 1: h_t = h_x = 1/(nx+1) (Section 6.1)             */
} fde_params;

/* ADMM options (Algorithm 1, Section 6.1). */
typedef struct fde_admm_opts {
  double delta;              /* penalty parameter: the penalty term is 1/(2 delta), > 0          */
  double rho;                /* dual step length in (0, (1+sqrt 5)/2)                            */
  double tol_admm;           /* infinity-norm tolerance on the three residuals of Section 6.1    */
  int max_admm;              /* iteration cap                                                     */
  int fixed_iters;           /* 1: run exactly max_admm iterations (no residual test)             */
  int max_pcg;               /* PCG iteration cap per sub-problem (per refinement step in MIXED)  */
  int inner_tol_mode;        /* 0: Section 6.1 rule 0.05 max{min residuals, tol_admm}; 1: fixed   */
  double inner_tol;          /* relative residual target of each sub-solve when inner_tol_mode=1  */
  int precision;             /* FDE_FP64, FDE_MIXED or FDE_MIXED_DF                              */
  double inner_tol_mixed;    /* MIXED: relative residual target of the float PCG per refinement   */
  int max_refine;            /* MIXED: cap on refinement steps per sub-problem                    */
  int algorithm;             /* 0 or 1: Algorithm 1. 2: generalized ADMM (Section 3.3.2,
                                Algorithm 2) with the proximal matrices R_y = c_y I - J1 and
                                R_u = c_u I - J2 (1/2 on both proximal terms); it needs rho in
                                (0, 1], c_y >= 1 (the largest weight of J1) and c_u >= gamma
                                (of J2). Its M1, Q and M2 are multiples of the identity and the
                                preconditioner uses them exactly.                                  */
  double c_y, c_u;           /* Algorithm 2 only                                                  */
  int inner_solver;          /* 0: PCG on the normal equations S y = rhs (Section 3.1) with
                                S-tilde. 1: MINRES on the saddle-point system of y, u, p (Eq.
                                generic ADMM subproblems 1and3 optimality conditions, Section
                                3.3.1) with K-tilde = blkdiag(M1, Q, Sigma-tilde), Sigma-tilde =
                                m2 I + C3 C3^T / m1. FP64 stops on the K-tilde^-1-norm of the
                                residual, MIXED on its 2-norm (double residuals, float MINRES);
                                max_pcg caps the MINRES iterations. Allocates 30N doubles (and
                                30N floats in MIXED) on first use. fde_admm_solve only.             */
  int precond;               /* PCG preconditioner (also fde_precond). 0: S-tilde (Eq. first schur
                                complement preconditioner) with C3 and scalar m1, m2. 1: the
                                matching approximation S-hat (Eq. second schur complement
                                preconditioner, Section 3.2.2) with D-tilde = C3: D-hat = C3^T +
                                sqrt(m1 m2) I is circulant, so S-hat is applied by the same FFTs
                                with sigma = m1 + |Lambda|^2/m2 + 2 sqrt(m1/m2) Re(Lambda).         */
  int warm_start;            /* 1: fde_admm_solve starts from the iterates (y, u, z_y, z_u, p, w_y,
                                w_u) the previous fde_admm_solve on this problem ended with, instead
                                of zero (FDE_EINVAL if there is none); the options and the data
                                may differ between the calls. Batches: FDE_EUNSUPPORTED.          */
  int inner_x0;              /* initial guess of each sub-solve: 0 the previous ADMM iterate (PCG:
                                y^j; MINRES: (y^j, u^j, p^j)); 1 zero, as MATLAB's pcg does by
                                default (the paper's runs, Section 6.1). fde_admm_solve only.     */
} fde_admm_opts;

typedef struct fde_admm_stats {
  int admm_iters;            /* iterations performed                                             */
  int pcg_iters;             /* PCG iterations summed over all sub-problems                      */
  int refine_steps;          /* MIXED: refinement corrections summed over sub-problems           */
  int fp64_matvecs;          /* B or B^T applications on double vectors (double or, in the
                                MIXED_DF / MIXED_DFV refinement, double-float arithmetic)        */
  double res_eq;             /* ||B y + psi (u - g)||_inf at exit                                */
  double res_y;              /* ||y - z_y||_inf at exit                                          */
  double res_u;              /* ||u - z_u||_inf at exit                                          */
  double objective;          /* 1/2 (y-ybar)^T J1 (y-ybar) + 1/2 u^T J2 u at exit                */
  double max_sub_relres;     /* largest final relative residual ||b - S y||/||b|| of a sub-solve */
  int recursive_steers;      /* MIXED_DFV: corrections steered by the float PCG's recursive
                                residual instead of an evaluated one                              */
  double copy_in_ms;         /* fde_admm_solve_host: device time of the host-to-device copies     */
  double copy_out_ms;        /* fde_admm_solve_host: device time of the device-to-host copies     */
  int float_steers;          /* MIXED_DFV: first evaluations of a warm-started sub-problem run in
                                float (they only steer the first correction; never accepted)      */
} fde_admm_stats;

typedef struct fde_problem fde_problem;

/* Create a problem: validate params, allocate the workspace and run the set-up
 * kernels (Gruenwald-Letnikov weights of Eq. C_GL, circulant-embedding symbols
 * of the Toeplitz factors, T. Chan circulants of Eq. (level 1 circulant
 * optimization problem) and their DFTs; Section 5). `*out` receives the handle.
 * Errors: FDE_EINVAL (orders outside their intervals, n < 1, gamma <= 0,
 * negative coefficients), FDE_EUNSUPPORTED (an axis above 4096), FDE_ENOMEM,
 * FDE_ECUDA. Synchronises `stream` before returning. */
int fde_setup(const fde_params* params, fde_problem** out, void* stream);

/* Release a problem and its workspace (NULL is allowed). */
void fde_destroy(fde_problem* prob);

/* Number of vector entries N = nt*nx*ny (0 for NULL). */
long long fde_size(const fde_problem* prob);

/* psi = min{h_t^alpha_t, h_x^beta_x, h_y^beta_y} (Section 5). */
double fde_psi(const fde_problem* prob);

/* Operator application y = op(x) (Eq. FDE constraint matrix scaled by psi;
 * FDE_OP_S adds the normal-equation diagonals of Eq. (generic ADMM normal
 * equations) for the given ADMM options). Toeplitz products run by circulant
 * embedding and FFT (Table "Complexity table", d-level Toeplitz row).
 * precision: FDE_FP64 (x, y double*), FDE_FP32 (float*) or FDE_MIXED_DF
 * (double*, ops B and B^T only). `opts` is read only for FDE_OP_S (delta,
 * rho) and may be NULL otherwise. x and y must not overlap. Errors: FDE_EINVAL. */
int fde_matvec(fde_problem* prob, int op, const fde_admm_opts* opts, int precision,
               const void* x, void* y, void* stream);

/* One Kronecker factor of B alone, one kernel launch: axis 1: y = -psi (I (x) X (x) I) x,
 * axis 2: y = -psi (I (x) I (x) Y) x, with X = d+ L_x + d- L_x^T and Y = e+ L_y + e- L_y^T
 * (Eq. FDE constraint matrix); op FDE_OP_BT applies the transposed factor. No
 * time term. precision FDE_FP64 (double*), FDE_FP32 (float*) or FDE_MIXED_DF
 * (double*, double-float transforms); x and y must not overlap. Errors: FDE_EINVAL. */
int fde_apply_factor(fde_problem* prob, int axis, int op, int precision, const void* x, void* y, void* stream);

/* FFT tile autotuning: times the float, double-float and double transform
 * passes of this problem with each tile configuration (threads per CTA, hence
 * lines per CTA, and the split-halves variant) on the problem's own sizes and
 * keeps the fastest for all later products of `prob` in that arithmetic.
 * Without it a fixed default is used.
 * fde_batch_setup calls it for every instance. Synchronises `stream`. Errors:
 * FDE_EINVAL, FDE_ECUDA. */
int fde_autotune(fde_problem* prob, void* stream);

/* Current tile choice of the x2 pass and x1 pass, for precision FDE_FP32 (the
 * float passes), FDE_MIXED_DF (the double-float passes) or FDE_FP64 (the double
 * passes): threads per CTA of the kernel that holds both embedding halves of a
 * line pair in each thread (float x2: 128, 256 or 512, x1: 256 or 512; double-float
 * and double: 128 or 256; 128 applies to lines of up to 2048, longer ones keep 256),
 * or, negated, of the double-float or double split-halves
 * kernel whose two thread groups hold one half each (x2: 256 or 512, x1: 512). */
int fde_tiles(const fde_problem* prob, int precision, int* rows_threads, int* axis_threads);

/* Sets the tile choice (values as fde_tiles reports them; 0 keeps the current
 * one). Errors: FDE_EINVAL (another precision, a value outside the lists above,
 * 128 and -256 for the x2 pass when ny > 2048). */
int fde_set_tiles(fde_problem* prob, int precision, int rows_threads, int axis_threads);

/* Preconditioner z = S~^-1 r with S~ = m1 I + C_3(B)^T C_3(B) / m2 (Eq. first
 * schur complement preconditioner with C_3 of Eq. multilevel circulant
 * preconditioner, J replaced by I): FFT, divide by m1 + |Lambda|^2/m2,
 * inverse FFT; with opts->precond = 1 the matching approximation S^ (divide by
 * m1 + |Lambda|^2/m2 + 2 sqrt(m1/m2) Re Lambda). m1, m2 follow opts (Algorithm 2:
 * exact scalars). precision: FDE_FP64 (double*) or FDE_FP32 (float*). r and z
 * may be the same array. Errors: FDE_EINVAL, FDE_EUNSUPPORTED (an axis length
 * with a prime factor above 7). */
int fde_precond(fde_problem* prob, const fde_admm_opts* opts, int precision,
                const void* r, void* z, void* stream);

/* ADMM (Algorithm 1 with the sub-problem merged with the p update, Section 3.1,
 * and the psi scaling of Section 6.1). Sub-problems S y = rhs are solved by
 * PCG preconditioned with S~; in FDE_MIXED the operator and preconditioner run
 * in float inside a double iterative-refinement loop, with the Krylov scalars,
 * inner products, refinement residuals and ADMM residuals in double.
 * Inputs (double, device, length N): ybar; g (NULL = 0); bounds ya, yb, ua, ub
 * (NULL = unbounded on that side). Scalar bounds are passed as
 * ya_s/yb_s/ua_s/ub_s and are used where the matching array pointer is NULL;
 * give -INFINITY/+INFINITY for no bound. Outputs (double, device, length N):
 * y, u (required), p, z_u (NULL = not returned). Iterates start at zero, or
 * with opts->warm_start where the previous solve on `prob` ended.
 * stats may be NULL. Errors: FDE_EINVAL, FDE_ENOCONV (cap reached: outputs
 * and stats hold the last iterate), FDE_EBREAKDOWN, FDE_ENONFINITE,
 * FDE_ECUDA. Synchronises `stream`. */
int fde_admm_solve(fde_problem* prob, const fde_admm_opts* opts,
                   const double* ybar, const double* g,
                   const double* ya, const double* yb, const double* ua, const double* ub,
                   double ya_s, double yb_s, double ua_s, double ub_s,
                   double* y, double* u, double* p, double* zu,
                   fde_admm_stats* stats, void* stream);

/* fde_admm_solve on HOST buffers: the same solve, with every array argument
 * (ybar, g, ya, yb, ua, ub in; y, u, p, zu out; same NULL rules and lengths) in
 * host memory. The inputs are copied to device buffers that `prob` keeps for
 * later calls (allocated on first use, N doubles per input given), the solve
 * runs, and the outputs are copied back before it returns. Pinned host memory
 * (cudaHostAlloc, cudaHostRegister) is read and written by a copy kernel through
 * its mapped device address; pageable memory goes through cudaMemcpyAsync.
 * stats->copy_in_ms / copy_out_ms report the device time of the two copy
 * phases. The host arrays must not be touched until the call returns. Errors:
 * those of fde_admm_solve; the outputs are written for FDE_OK and FDE_ENOCONV
 * only. Synchronises `stream`. */
int fde_admm_solve_host(fde_problem* prob, const fde_admm_opts* opts,
                        const double* ybar, const double* g,
                        const double* ya, const double* yb, const double* ua, const double* ub,
                        double ya_s, double yb_s, double ua_s, double ub_s,
                        double* y, double* u, double* p, double* zu,
                        fde_admm_stats* stats, void* stream);

/* The iterates of Algorithm 1 (Section 3.1, psi-scaled as in Section 6.1) that
 * the last fde_admm_solve / fde_admm_solve_host on `prob` ended with (also
 * after FDE_ENOCONV), or that fde_admm_set_iterates loaded: the state y and
 * control u, their projected copies z_y and z_u, the multiplier p of
 * B y + psi u = psi g and the multipliers w_y, w_u of y = z_y and
 * psi u = psi z_u. At a converged solution w_y is the state-box multiplier
 * that the adjoint equation of fde_admm_grad needs. Each output is a DEVICE
 * array of N doubles or NULL (not copied). Errors: FDE_EINVAL (no solve has
 * left iterates on `prob`, or the last one failed), FDE_ECUDA. Synchronises
 * `stream`. */
int fde_admm_get_iterates(const fde_problem* prob, double* y, double* u, double* zy, double* zu, double* p,
                          double* wy, double* wu, void* stream);

/* Load the iterates a solve with opts->warm_start = 1 starts from (same
 * arrays as fde_admm_get_iterates, DEVICE, N doubles each; NULL = zero), for
 * instance the end of a solve of a neighbouring problem (continuation in the
 * coefficients). Computes B y of the given y for the first ADMM step.
 * Errors: FDE_EINVAL, FDE_ECUDA. Synchronises `stream`. */
int fde_admm_set_iterates(fde_problem* prob, const double* y, const double* u, const double* zy, const double* zu,
                          const double* p, const double* wy, const double* wu, void* stream);

/* Gradient of the optimal value J* at a converged solution (envelope theorem
 * on the Lagrangian of Eq. (Generic ADMM aug Lagrangian)):
 *   d(J^*)/dybar = -J1 (y* - ybar)                      -> dJ_dybar (device, N, may be NULL)
 *   d(J^*)/d{d+, d-, e+, e-} = -psi p*^T (I (x) L (x) I) y* with L = L_x, L_x^T on x1
 *                           and L_y, L_y^T on x2       -> dJ_dcoef[4] (HOST doubles)
 * p* is obtained by solving the adjoint equation B^T p = -J1 (y* - ybar) - w_y
 * (w_y: the state-box multiplier of the converged solve, fde_admm_get_iterates;
 * NULL = 0, correct only when no state bound is active) with CG on B B^T preconditioned by
 * C_3 C_3^T, to relative residual `tol` (<= 0 selects 1e-12); p_out (device, N,
 * may be NULL) receives it. Double precision throughout. Errors: FDE_EINVAL,
 * FDE_ENOCONV, FDE_ECUDA. Synchronises `stream`. */
int fde_admm_grad(fde_problem* prob, const double* y, const double* ybar, const double* wy,
                  double tol, double* dJ_dybar, double* dJ_dcoef, double* p_out, void* stream);

/* Largest problem (nt*nx*ny points) fde_matvec_noalloc accepts. */
#define FDE_NOALLOC_MAX_N 1048576LL

/* y = B x (op FDE_OP_B) or y = B^T x (FDE_OP_BT) in double precision, without
 * any device allocation. The paper has no counterpart to this entry point: it
 * exists for callers that cannot call cudaMalloc, such as a plug-in running
 * inside a framework whose caching allocator owns the device memory, or a
 * latency-critical serving path that must not allocate (cudaMalloc can
 * synchronise the device and can fail under memory pressure). It computes the
 * same product as fde_matvec, with no fde_problem: the caller passes `params`
 * and its own x and y (device, double, length N). All other buffers (the
 * intermediates of the transform passes and the symbol/twiddle tables, rebuilt
 * from `params` on every call) live in one fixed device array of about 18 MB
 * that every GPU loading this library holds until the process exits.
 * Errors: FDE_EINVAL (as fde_setup, or op not B/B^T, or x == y),
 * FDE_EUNSUPPORTED (N > FDE_NOALLOC_MAX_N or an axis above 4096), FDE_ECUDA.
 * The first call on each device looks up the array's device address and sets
 * kernel attributes; make it before any stream capture. All calls share the
 * array: calls whose GPU work overlaps (two streams or host threads) race and
 * must be serialised by the caller. The work is queued on `stream`. */
int fde_matvec_noalloc(const fde_params* params, int op, const double* x, double* y, void* stream);

/* A batch of independent problems of different sizes and parameters (one
 * fde_setup per instance; every axis of every instance must factor into 2, 3,
 * 5 and 7). Errors: as fde_setup for any instance, FDE_EUNSUPPORTED. */
typedef struct fde_batch fde_batch;
int fde_batch_setup(const fde_params* params, int count, fde_batch** out, void* stream);
void fde_batch_destroy(fde_batch* batch);
/* N of instance i (0 when out of range). */
long long fde_batch_instance_size(const fde_batch* batch, int i);

/* Solve every instance of the batch with MIXED ADMM (Algorithm 1, Section 6.1
 * psi scaling) in one CUDA-graph launch. Unlike fde_admm_solve, nothing is read
 * back during the solve: each instance runs exactly opts->max_admm ADMM
 * iterations; each sub-problem gets opts->max_refine double residual
 * evaluations/float corrections (the last evaluation has no correction) and
 * each correction exactly opts->max_pcg float PCG iterations, with
 * convergence decided on the device (converged PCG iterations and corrections
 * do no work on the iterates). opts->inner_tol is the sub-problem relative
 * residual target, opts->inner_tol_mixed the float PCG target; tol_admm,
 * fixed_iters and inner_tol_mode are ignored. The solve of the whole batch is
 * captured into one CUDA graph (one independent branch per instance, run
 * concurrently) on the first call and replayed while the arguments stay the
 * same. Inputs: ybar[i] (device, N_i doubles); scalar bounds ya/yb/ua/ub
 * (HOST arrays of `count` doubles, NULL = unbounded). Outputs: y[i], u[i]
 * (device, N_i doubles); stats (HOST array of `count`, may be NULL;
 * max_sub_relres is the largest final relative residual over the
 * sub-problems). Synchronises `stream`. Errors: FDE_EINVAL (opts->precision
 * not FDE_MIXED, FDE_MIXED_DF or FDE_MIXED_DFV, NULL pointers, NaN bounds),
 * FDE_EUNSUPPORTED (opts->inner_solver, warm_start or inner_x0 set),
 * FDE_ENONFINITE, FDE_ECUDA. */
int fde_batch_admm_solve(fde_batch* batch, const fde_admm_opts* opts, const double* const* ybar,
                         const double* ya, const double* yb, const double* ua, const double* ub,
                         double* const* y, double* const* u, fde_admm_stats* stats, void* stream);

/* Configuration of the persistent batch solve. Zero fields take the defaults. */
typedef struct fde_persist_cfg {
  int group_ctas;    /* CTAs that solve one instance together (an instance group);
                        0: the resident CTAs divided into 16 groups (one group for a
                        batch of one); clamped to the resident CTAs                       */
  double timeout_s;  /* limit of every device-side wait (0: 1 s)                          */
  int replay;        /* 0: the persistent kernel; 1: the same recorded launches issued
                        one by one on `stream` (the reference executor of the tests)      */
  int stall_group;   /* test hook, 0: off. k > 0: the first CTA of instance group k - 1
                        (lockstep: of the grid) never arrives at its first barrier, so
                        that every wait of that group runs out                            */
  int schedule;      /* 0: lockstep when every instance recorded the same number of
                        launches (else instance groups); 1: instance groups               */
} fde_persist_cfg;

/* What a persistent solve ran (HOST struct, filled on return). */
typedef struct fde_persist_info {
  long long commands;     /* recorded launches over all instances                        */
  int groups;             /* instance groups                                             */
  int group_ctas;         /* CTAs per group                                              */
  int ctas_per_sm;        /* resident CTAs per SM of the persistent kernel               */
  int smem_bytes;         /* dynamic shared memory per CTA                               */
  int timeout_group;      /* on FDE_ETIMEOUT: the group whose wait ran out, else -1      */
  long long timeout_command; /* ... and the last command (lockstep: step) it had finished,
                                -1 if none                                                 */
  int schedule;           /* 0: lockstep, 1: instance groups                             */
} fde_persist_info;

/* The batch solve of fde_batch_admm_solve (same arguments, options and fixed
 * iteration budgets; opts->precision must be FDE_MIXED: the executor has no
 * double-float transforms) run by ONE persistent cooperative kernel.
 * The launches that fde_batch_admm_solve would capture into its graph are
 * recorded instead (every launch with 256 threads: the register-resident float
 * passes and preconditioner transforms; the double passes and the lines
 * shorter than 16 in the generic shared-memory transforms); the kernel keeps ctas_per_sm x SMs CTAs resident,
 * split into instance groups of cfg->group_ctas CTAs. A group takes the next
 * instance from a device-side queue (largest instances first), runs the
 * bodies of that instance's recorded launches one after another (each launch's
 * blocks spread over the group's CTAs) with a group barrier after each, and
 * takes the next instance until the queue is empty. Lockstep schedule (the
 * default when every instance recorded the same number of launches, as the
 * fixed budgets make them): step k runs launch k of every instance, the blocks
 * of all of them spread over all CTAs, then one barrier of all CTAs; instances
 * of very different sizes then share the whole GPU. Every barrier wait is
 * bounded by cfg->timeout_s: when one runs out the kernel records the group
 * and command, every CTA returns within about one more limit, and the call
 * returns FDE_ETIMEOUT with the context usable. cfg may be NULL (defaults);
 * info may be NULL. Every axis length (nx, ny, nt) must be a power of two
 * (the executor holds the power-of-two transforms of lengths up to 2048).
 * Synchronises `stream`. Errors: FDE_EINVAL (as fde_batch_admm_solve;
 * precision not FDE_MIXED; a negative cfg field), FDE_EUNSUPPORTED (an axis
 * that is not a power of two or above 2048, a command the executor cannot
 * replay), FDE_ETIMEOUT, FDE_ENONFINITE, FDE_ENOMEM, FDE_ECUDA. */
int fde_batch_admm_solve_persistent(fde_batch* batch, const fde_admm_opts* opts, const double* const* ybar,
                                    const double* ya, const double* yb, const double* ua, const double* ub,
                                    double* const* y, double* const* u, const fde_persist_cfg* cfg,
                                    fde_admm_stats* stats, fde_persist_info* info, void* stream);

/* Arithmetic peak of this GPU measured with independent fused multiply-add
 * chains (precision FDE_FP64 or FDE_FP32), in TFLOP/s, best of three runs of
 * about 70 ms (double) or 5 ms (float); a diagnostic used as the roofline of
 * the arithmetic-bound double transforms. Synchronises `stream`. */
int fde_alu_peak_probe(int precision, double* tflops, void* stream);

/* Static message for a status code. */
const char* fde_strerror(int status);

/* Text of the last CUDA error seen by this library in the calling thread. */
const char* fde_last_cuda_error(void);

/* Number of kernel launches this library has issued in this process (all
 * problems, all threads); a diagnostic counter for profiling and benchmarks. */
long long fde_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* FDE_H */
