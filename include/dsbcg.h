/*
 * dsbcg.h -- C ABI of the GB300 (sm_103a) implementation of the deflated
 * shifted block CG method (DSBlockCG) of Birk & Frommer, "A CG Method for
 * Multiple Right Hand Sides and Multiple Shifts in Lattice QCD Calculations"
 * (Lattice 2011, arXiv:1205.0359).
 *
 * Problem (Sec. 1, Eqs. 1.1 and 1.2):
 *     (sigma_j I + A) X_j = B,   j = 1..s,   B = [b_1 | ... | b_m],
 * with A = D^H D, D the Wilson-Dirac operator on a 4D lattice, and
 * sigma_j >= 0 real so that sigma_j I + A is hermitian positive definite.
 *
 * Conventions shared by every entry point:
 *   site index   site = x + Lx*(y + Ly*(z + Lz*t))
 *   vector index site*12 + spin*3 + colour, complex128 (n = 12 * volume)
 *   gauge field  complex128 [site][mu = x,y,z,t][row][col]
 *   D psi(x) = psi(x) - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                      + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu) ],
 *   chiral gamma basis (gamma_5 = diag(-1,-1,1,1)), periodic in space, and
 *   antiperiodic in time when t_antiperiodic != 0.  D^H = gamma_5 D gamma_5.
 *
 * Pointers: "device or host" arguments may point to device memory or to host
 * memory (pageable or pinned); the library detects which.  Page-locked host
 * memory mapped into the device address space is read and written in place
 * by the library's kernels; other host memory is staged through device
 * buffers on the context's stream.  The caller owns every buffer it passes;
 * the library never frees them.  A context owns its workspace (including
 * the streams of its concurrent restarts) and its packed copies of the gauge
 * field.
 *
 * Errors: every call returns a dsbcg_status; nothing is thrown across the
 * ABI.  After DSBCG_ERR_CUDA the context should be destroyed.
 * Thread safety: one context must not be used by two host threads at once.
 */
#ifndef DSBCG_H
#define DSBCG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dsbcg_ctx dsbcg_ctx;

typedef enum {
    DSBCG_OK = 0,
    DSBCG_NOT_CONVERGED = 1,   /* iteration or restart cap reached; X holds the best iterate */
    DSBCG_ERR_ARG = -1,        /* invalid argument (size, null pointer, negative shift, ...) */
    DSBCG_ERR_NOT_HPD = -2,    /* a pivot d_k of sigma_j I + T was <= 0 */
    DSBCG_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    DSBCG_ERR_OOM = -4,        /* device allocation failed */
    DSBCG_ERR_NONFINITE = -5,  /* NaN or Inf in an input */
    DSBCG_ERR_UNSUPPORTED = -6 /* option not supported by this build */
} dsbcg_status;

/* Storage precision of spinor fields and links inside the Krylov iteration.
 * Arithmetic on FP32/BF16/FP16 storage is FP32.  The m x m block
 * coefficients, deflation, per-shift recurrences, true residuals and
 * accumulated solutions are IEEE FP64 by default (dsbcg_params.fp64_residuals
 * = 1); for the reduced storages dsbcg_params.fp64_residuals = 0 selects
 * double-float arithmetic for them instead.
 * DSBCG_PREC_DF32 ("double-float"): each real number is an unevaluated sum
 * hi + lo of two FP32 words (48-bit significand, FP32 exponent range,
 * arithmetic on the FP32 pipes through error-free transformations).  It is
 * the arithmetic of the true residuals of reduced-precision solves, offered
 * to dsbcg_apply / dsbcg_apply_static; it is not a Krylov storage (dsbcg_solve
 * rejects it). */
typedef enum {
    DSBCG_PREC_FP64 = 0,
    DSBCG_PREC_FP32 = 1,
    DSBCG_PREC_BF16 = 2,
    DSBCG_PREC_FP16 = 3,
    DSBCG_PREC_DF32 = 4
} dsbcg_prec;

/* The operator a context solves with (dsbcg_set_operator). */
#define DSBCG_OPERATOR_NORMAL 0     /* A = D^H D on full-lattice fields, n = 12 V (default) */
#define DSBCG_OPERATOR_SCHUR 1      /* Ahat = Dhat^H Dhat on odd-site fields, n = 6 V */

/* Operators for dsbcg_apply. */
typedef enum {
    DSBCG_OP_D = 0,      /* D */
    DSBCG_OP_DDAG = 1,   /* D^H = gamma_5 D gamma_5 */
    DSBCG_OP_A = 2       /* A = D^H D */
} dsbcg_op;

typedef struct {
    int storage;            /* dsbcg_prec of the inner Krylov iteration (default FP32) */
    double dtol;            /* deflation threshold relative to a direction's norm when
                               created; <= 0 selects the default for the precision */
    int max_block_steps;    /* cap on block Lanczos steps over the whole solve */
    int max_restarts;       /* cap on true-residual restarts */
    double restart_drop;    /* an inner solve stops once every estimated residual has
                               dropped by this factor (mixed precision only) */
    int poll_every;         /* block steps between host reads of the convergence flags */
    int freeze_converged;   /* stop updating converged (i, j) systems (Sec. 4) */
    int refine;             /* 1: after the joint solve, restart each unconverged shift
                               separately (block CG) until its true residual meets tol */
    int fp64_residuals;     /* reduced storages only.  1 (default): true residuals,
                               accumulated solutions and the m x m coefficient work in
                               IEEE FP64, as with FP64 storage; 0 (opt-in): all of them
                               in double-float arithmetic (DSBCG_PREC_DF32) on the FP32
                               pipes, about 1.2x faster on GB300, where FP64 runs at
                               1/64 of the FP32 rate */
    int x0;                 /* 1: X's input is an initial guess X_0 for every system (a
                               resumed solve): the joint block solve is skipped and
                               each shift is restarted from its own true residual
                               b_i - (sigma_j + A) x0_ij; 0 (default): X's input is
                               ignored and X_0 = 0 */
} dsbcg_params;

typedef struct {
    int block_steps;        /* block Lanczos steps, all inner solves */
    long long mvms;         /* A applications to single vectors (one D plus one D^H each) */
    int deflations;         /* directions dropped by deflation */
    int restarts;           /* true-residual restarts */
    int final_rank;         /* block width m_k at the end of the last inner solve */
    double seconds;         /* wall time of the call */
    double* true_relres;    /* caller-provided [s][m] or NULL: final true
                               residual ||b_i - (sigma_j + A) x_ij|| / ||b_i|| */
    int* conv_step;         /* caller-provided [s][m] or NULL: block step at which
                               (i, j) met its inner target (-1: never) */
    double kernel_ms[8];    /* if profiling is on: summed CUDA-event time per kernel
                               class (see DSBCG_KCLASS_*) */
    long long kernel_launches[8];   /* kernels launched per class */
    double kernel_bytes[8]; /* algorithmic HBM bytes per class: each operand field,
                               link and coefficient block read or written once per
                               launch, counted from the block widths of every step */
    double kernel_flops[8]; /* algorithmic floating-point operations per class
                               (a complex multiply-add counts 8), for the classes
                               that are counted: the shift update; 0 elsewhere */
} dsbcg_stats;

/* kernel classes reported in dsbcg_stats.kernel_ms */
#define DSBCG_KCLASS_DSLASH 0       /* Wilson hopping stencil */
#define DSBCG_KCLASS_GRAM 1         /* tall-skinny Gram products */
#define DSBCG_KCLASS_UPDATE 2       /* block update W = Y - V a - V' b^H and V' = W S */
#define DSBCG_KCLASS_SHIFT 3        /* shift update of P_j, X_j over a chunk of steps */
#define DSBCG_KCLASS_SMALL 4        /* FP64 m x m kernels */
#define DSBCG_KCLASS_RESIDUAL 5     /* true residuals (FP64 or double-float) */
#define DSBCG_KCLASS_OTHER 6

/* Fill *p with the defaults (FP32 storage, FP64 reliable updates and m x m
 * work, automatic dtol, freezing on). */
void dsbcg_params_default(dsbcg_params* p);

/* Create a context for one lattice and gauge field.
 *   dims:  {Lx, Ly, Lz, Lt}, each >= 2 (the problem of Sec. 1 on a 4D lattice)
 *   gauge: device or host complex128 [site][4][3][3]; copied and packed
 *   kappa: hopping parameter of D
 *   stream: cudaStream_t to run on (NULL = legacy default stream)
 * Returns DSBCG_ERR_NONFINITE if the gauge field has NaN/Inf. */
dsbcg_status dsbcg_create(dsbcg_ctx** out, const int dims[4], const void* gauge,
                          double kappa, int t_antiperiodic, void* stream);

/* Replace the gauge field of an existing context (same dims).  The new field
 * is checked for NaN/Inf (DSBCG_ERR_NONFINITE) and packed again for every
 * precision on first use.  After any failed update the context holds no
 * gauge field: dsbcg_solve, dsbcg_apply, dsbcg_apply_static and dsbcg_force
 * return DSBCG_ERR_ARG until an update succeeds. */
dsbcg_status dsbcg_update_gauge(dsbcg_ctx* ctx, const void* gauge);

/* Solve (sigma_j I + A) X_j = B for j = 1..s with one block Lanczos process
 * (Sec. 3).  The paper's iterate X^(k) = V (sigma I + T)^{-1} V^H B (Eq. 3.2)
 * is advanced by short recurrences from a root-free (block) Cholesky
 * factorisation of sigma_j I + T per shift; directions that become linearly
 * dependent are deflated (Sec. 1, Sec. 3).  With FP32/BF16/FP16 storage the
 * Krylov iteration runs in reduced precision inside a loop that recomputes
 * true residuals in FP64 (double-float arithmetic, DSBCG_PREC_DF32, with
 * params->fp64_residuals = 0) and restarts (reliable updates); with FP64
 * storage residuals are FP64.  A double-float residual carries an absolute
 * error of roughly 2^-44 |A| |x|, so it certifies tol down to about 1e-13
 * times the condition number of sigma_j I + A.
 *   m:     number of right-hand sides, 1 <= m <= 32
 *   B:     device or host complex128 [m][n]
 *   s:     number of shifts, 1 <= s <= 64
 *   sigma: HOST double[s], each >= 0
 *   tol:   target ||b_i - (sigma_j + A) x_ij|| <= tol ||b_i|| for every (i, j)
 *   X:     device or host complex128 [s][m][n]; output (its input value is the
 *          initial guess with params->x0, otherwise ignored)
 *   params: NULL for defaults
 *   stats: NULL or caller-owned
 * Returns DSBCG_OK when every true relative residual meets tol,
 * DSBCG_NOT_CONVERGED (X still written) when a cap is hit. */
dsbcg_status dsbcg_solve(dsbcg_ctx* ctx, int m, const void* B, int s, const double* sigma,
                         double tol, const dsbcg_params* params, void* X, dsbcg_stats* stats);

/* Solve the shifted systems as dsbcg_solve does and write their rational
 * combination
 *     Y = alpha0 B + sum_j alpha_j X_j   (= r(A) B for the partial fraction
 *                                          r(x) = alpha0 + sum_j alpha_j / (x + sigma_j)),
 * the use of the shifted solves named in Sec. 1 (rational approximations in
 * RHMC).  Y is formed on the device in one pass over the final solutions,
 * shifts summed in index order, in FP64 arithmetic.  Every (i, j) system meets
 * tol as in dsbcg_solve, so ||y_i - r(A) b_i|| <= tol ||b_i|| sum_j |alpha_j| /
 * lambda_min(sigma_j I + A).
 *   alpha0: real; alpha: HOST double[s], finite
 *   Y:      device or host complex128 [m][n], output
 *   X:      NULL (the per-shift solutions are not written: the caller's
 *           output is s times smaller) or device or host [s][m][n]
 * Other arguments, results and status codes as dsbcg_solve; params->x0 needs X. */
dsbcg_status dsbcg_solve_rational(dsbcg_ctx* ctx, int m, const void* B, int s, const double* sigma,
                                  double alpha0, const double* alpha, double tol, const dsbcg_params* params,
                                  void* Y, void* X, dsbcg_stats* stats);

/* Backward pass of dsbcg_solve: gradients of a real loss L through
 * X_j = (sigma_j I + A)^{-1} B, given the incoming gradients G_j = dL/dX_j.
 * Not in the paper (its motivation is the RHMC force, Sec. 1).  With
 * sigma_j I + A hermitian, the adjoint solutions are Lambda_j =
 * (sigma_j I + A)^{-1} G_j, and
 *     dL/dB       = g_direct G + sum_j Lambda_j
 *     dL/dsigma_j = -Re tr(Lambda_j^H X_j)
 *     dL/dU       = the force of dsbcg_force on (X_j, Lambda_j) with unit weights
 * (complex gradients in the dL/dRe + i dL/dIm convention).  Every step runs
 * in the library's kernels:
 *   - g_weights != NULL: G is ONE block [m][n] and G_j = g_weights[j] G (the
 *     gradient of a loss of Y = sum_j g_weights[j] X_j, the RHMC case): one
 *     joint DSBlockCG solve of G for all shifts, Lambda_j scaled by w_j;
 *   - g_weights == NULL: G is [s][m][n] (one block per shift): all s shifts
 *     are solved in this one call, each shift's block CG on its own stream
 *     (the restart lanes of dsbcg_solve), concurrently;
 *   - X == NULL: the solutions are recomputed from B by a dsbcg_solve
 *     (memory instead of storage); otherwise X holds them and B may be NULL.
 * Each adjoint system meets tol like a forward system.
 *   B:         device or host complex128 [m][n] (needed only when X == NULL)
 *   X:         NULL or device or host complex128 [s][m][n]
 *   G:         device or host complex128 [m][n] or [s][m][n], see above
 *   g_weights: NULL or HOST double[s]
 *   g_direct:  0, or (with g_weights) the weight of B's direct term in the
 *              forward output, e.g. alpha0 for dsbcg_solve_rational's Y
 *   gB:        NULL or device or host complex128 [m][n], output
 *   gsigma:    NULL or HOST double[s], output
 *   gU:        NULL or device or host complex128 [site][4][3][3], output
 *              (computed in FP64 for FP64 storage, else from FP32 fields)
 *   Lambda:    NULL or device or host complex128 [s][m][n], output
 *   params:    as dsbcg_solve (x0 is ignored)
 *   stats:     block steps, mvms, restarts and deflations summed over the
 *              solves of the call; true_relres and conv_step (if given) are
 *              those of the adjoint systems; kernel_* are not written.
 * Returns DSBCG_NOT_CONVERGED if a solve hit a cap (outputs still written). */
dsbcg_status dsbcg_backward(dsbcg_ctx* ctx, int m, const void* B, int s, const double* sigma, const void* X,
                            const void* G, const double* g_weights, double g_direct, double tol,
                            const dsbcg_params* params, void* gB, double* gsigma, void* gU, void* Lambda,
                            dsbcg_stats* stats);

/* Select the operator of the context's solves and applications.
 *   DSBCG_OPERATOR_NORMAL: A = D^H D of the Wilson operator (Sec. 1), the
 *     paper's setting; fields have n = 12 V complex entries.
 *   DSBCG_OPERATOR_SCHUR: the even-odd preconditioned (Schur complement)
 *     operator on the odd sites.  With D = 1 - kappa H (H the hopping term,
 *     which connects only sites of opposite parity x + y + z + t mod 2 when
 *     every extent is even),
 *         Dhat = 1 - kappa^2 H_oe H_eo,   Dhat^H = gamma_5 Dhat gamma_5,
 *         Ahat = Dhat^H Dhat,
 *     and sigma_j I + Ahat is hpd for sigma_j > 0, so the method applies to it
 *     unchanged (Sec. 3).  The paper itself uses no such structure (Sec. 4):
 *     this is a preconditioned variant.  Fields are then odd-site half
 *     fields of n = 6 V complex entries: the odd sites in increasing
 *     canonical site order (half index = site / 2), 12 entries each.  D x = b
 *     follows from the odd-site system Dhat x_o = b_o + kappa H_oe b_e and
 *     x_e = b_e + kappa H_eo x_o.
 * dsbcg_solve, dsbcg_solve_rational, dsbcg_apply (D -> Dhat, D^H -> Dhat^H,
 * A -> Ahat) and the B / sigma gradients of dsbcg_backward act on the
 * selected operator; dsbcg_force, the link gradient of dsbcg_backward and
 * dsbcg_apply_static support the normal operator only (DSBCG_ERR_UNSUPPORTED).
 * Changing the operator frees the context's solver workspace.  Returns
 * DSBCG_ERR_ARG for an unknown operator, or SCHUR on a lattice with an odd
 * extent. */
dsbcg_status dsbcg_set_operator(dsbcg_ctx* ctx, int op);

/* Apply D, D^H or A to m fields: out_i = op(in_i).  The fields are converted
 * to `storage` precision (any dsbcg_prec, including DSBCG_PREC_DF32), the
 * stencil runs in that precision (FP32 arithmetic for FP32/BF16/FP16,
 * double-float for DF32), and the result is converted back.
 *   in, out: device or host complex128 [m][n]; they may not overlap. */
dsbcg_status dsbcg_apply(dsbcg_ctx* ctx, int op, int storage, int m, const void* in, void* out);

/* Size of the library's static device scratch used by dsbcg_apply_static. */
#define DSBCG_STATIC_SCRATCH_BYTES (32u << 20)

/* dsbcg_apply without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc at the time
 * of the call, e.g. code whose memory pool has already reserved the whole GPU,
 * or latency-critical loops where cudaMalloc's implicit device
 * synchronisation is not acceptable.  Same operation, arguments and result as
 * dsbcg_apply, with these differences:
 *   - in and out must be device pointers (host buffers would need staging);
 *   - the packed working fields live in one static device array of
 *     DSBCG_STATIC_SCRATCH_BYTES (32 MiB) that every GPU which loads the library
 *     holds until the process exits.  op = A needs 3 * m * (n rounded up to a
 *     multiple of 128) * (16, 8 or 4 bytes for FP64 or DF32, FP32, or
 *     FP16/BF16) bytes,
 *     D and D^H need 2/3 of that; larger requests return DSBCG_ERR_ARG and do
 *     nothing;
 *   - storage precisions other than FP64 need the context's links for that
 *     precision to exist already (packed by an earlier dsbcg_apply or
 *     dsbcg_solve with that precision); otherwise DSBCG_ERR_UNSUPPORTED, since
 *     packing them would allocate;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture;
 *   - all calls share the array and it keeps the last call's contents; every
 *     element a call reads is first written by the same call, so nothing needs
 *     clearing, but calls that overlap on the GPU (different streams or
 *     contexts in flight at once) race on it.
 * The call synchronises the context's stream before returning. */
dsbcg_status dsbcg_apply_static(dsbcg_ctx* ctx, int op, int storage, int m, const void* in, void* out);

/* Gauge-link gradient ("fermion force") of a real loss through the solves
 * X_j = (sigma_j + A)^{-1} B, given adjoint solutions Lambda_j =
 * (sigma_j + A)^{-1} G_j of the incoming gradients G_j = dL/dX_j:
 *   dU_mu(y) = kappa sum_j w_j sum_i [F(D x_ij, lambda_ij) + F(D lambda_ij, x_ij)]_mu(y),
 *   F(a, b)_mu(y) = sum_spin [(1-gamma_mu) a(y)] (x) conj(b(y+mu))
 *                 + sum_spin [(1+gamma_mu) b(y)] (x) conj(a(y+mu)),
 * with the time-boundary sign on the hop.  Complex gradients follow the
 * dL/dRe + i dL/dIm convention.  Not in the paper (its motivation is the RHMC
 * force, Sec. 1).
 *   X, Lambda: device or host complex128 [s][m][n]
 *   weights:   HOST double[s] (NULL = all ones)
 *   dU:        device or host complex128 [site][4][3][3], overwritten
 *   storage:   precision of the fields inside the kernel (FP64 or FP32) */
dsbcg_status dsbcg_force(dsbcg_ctx* ctx, int m, int s, const void* X, const void* Lambda,
                         const double* weights, int storage, void* dU);

/* Test hook for the failure path of the device-side waits; not for
 * production use.  Every shared-memory wait in the library's kernels is
 * bounded: a kernel whose wait gives up drains its own bulk copies, records
 * a timeout in the solve's control block and returns, and the call returns
 * DSBCG_ERR_CUDA with the GPU still usable.  With polls >= 0, the first wait
 * of every consumer warp of the staged block Gram kernel (the product
 * V_k^H A V_k of each block step) gives up after `polls` non-blocking tests
 * (0: at once), so a test can take that path without any fault.  polls < 0
 * restores the normal limit (the default). */
dsbcg_status dsbcg_debug_first_wait(dsbcg_ctx* ctx, int polls);

/* Test hook for the chunked shift update; not for production use.  The
 * per-shift recurrences x_j += p_j u_j, p_j <- v - p_j l_j (Sec. 3) run over
 * chunks of up to 16 block steps with p_j and x_j held on chip, and give
 * bitwise the same result for every chunk length.  steps in 1..16 caps the
 * chunk length of the following inner solves (1: one launch per block step);
 * 0 restores the automatic length (the default).  Other values:
 * DSBCG_ERR_ARG. */
dsbcg_status dsbcg_debug_shift_chunk(dsbcg_ctx* ctx, int steps);

/* Per-kernel CUDA-event timing inside dsbcg_solve (off by default). */
dsbcg_status dsbcg_set_profiling(dsbcg_ctx* ctx, int on);

/* Per-class CUDA-event time (ms, classes as in dsbcg_stats.kernel_ms) and
 * launch counts accumulated while profiling was on, since the last read or
 * the start of the last dsbcg_solve; resets them.  Either pointer may be
 * NULL.  Serves calls without a stats argument (dsbcg_force, dsbcg_apply). */
dsbcg_status dsbcg_read_profile(dsbcg_ctx* ctx, double kernel_ms[8], long long kernel_launches[8]);

void dsbcg_destroy(dsbcg_ctx* ctx);
const char* dsbcg_error_string(dsbcg_status status);

/* Library build identification: "dsbcg <version> sm_103a". */
const char* dsbcg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DSBCG_H */
