/*
 * qcdgb -- clover Wilson-Dirac operator, Schwarz-preconditioned mixed-precision
 * FGCR solver and fermion force on one NVIDIA GB300 (sm_103a).
 *
 * Every function below is a plain C entry point of libqcdgb.so.  Pointers are
 * host or device pointers as stated; sizes are element counts; no C++ or torch
 * types cross this boundary.  Every function returns an int status: QCD_OK (0)
 * or a negative QCD_ERR_* code (see qcd_status_string); no exception and no
 * exit() ever crosses the ABI.  A context is not thread-safe; separate contexts
 * are independent.
 *
 * Method: "Solving the Dirac equation on QPACE" (A. Nobile, Lattice 2010,
 * arXiv:1109.4279).  The solver inverts the Wilson-Dirac operator with clover
 * term (abstract; Sec. 1: the inversions feed the HMC fermion force) by flexible
 * GCR with restarts (Sec. 4), preconditioned by the Schwarz alternating
 * procedure with minimal-residual block solves on chessboard-coloured blocks
 * (Sec. 4), in mixed precision by iterative refinement (Sec. 4), with block
 * fields laid out block-contiguously and split into even and odd sites
 * (Sec. 5).
 *
 * Field conventions at the boundary (all complex numbers are interleaved
 * (re, im) FP64 pairs, C order):
 *   lattice   dims[4] = {L0 = T (time), L1, L2, L3}; V = L0 L1 L2 L3;
 *             site index ((x0 L1 + x1) L2 + x2) L3 + x3 (x0 slowest);
 *   spinor    (V, 4 spin, 3 colour) complex128; nrhs fields back to back;
 *   gauge     (V, 4 mu, 3, 3) complex128; U_mu(x) is the link x -> x + mu,
 *             which must lie in SU(3) (the reduced-precision copies store two
 *             rows and rebuild the third);
 *   force     (V, 4 mu, 8) float64: dL/dtheta_a for U_mu(x) ->
 *             exp(i theta_a lambda_a / 2) U_mu(x), Gell-Mann lambda_a.
 * Gamma matrices: chiral basis, g5 = g0 g1 g2 g3 = diag(1, 1, -1, -1),
 * g0 = [[0, -1], [-1, 0]], g_k = [[0, -i s_k], [i s_k, 0]] (2x2 blocks).
 *
 * D psi(x) = A(x) psi(x) - 1/2 sum_mu [ eta_mu(x) U_mu(x) (1 - g_mu) psi(x+mu)
 *                                    + eta_mu(x-mu) U_mu(x-mu)^+ (1 + g_mu) psi(x-mu) ]
 * A(x) = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_{mu nu} Fhat_{mu nu}(x),
 * sigma_{mu nu} = (i/2)[g_mu, g_nu], Fhat_{mu nu} = (Q_{mu nu} - Q_{nu mu}) / 8
 * with Q the sum of the four counter-clockwise plaquette leaves at x;
 * eta_mu(x) = bc[mu] on the hop from x_mu = L_mu - 1 to 0, else 1.
 */
#ifndef QCDGB_H
#define QCDGB_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define QCD_OK 0
#define QCD_ERR_ARG -1              /* invalid argument (null pointer, bad value) */
#define QCD_ERR_GEOMETRY -2         /* block extents must be even, divide L, and give an even block count per direction */
#define QCD_ERR_CUDA -3             /* a CUDA runtime call failed (message in qcd_last_error) */
#define QCD_ERR_NOMEM -4            /* device allocation failed */
#define QCD_ERR_STATE -5            /* call out of order (e.g. solve before load_gauge / build_clover) */
#define QCD_ERR_NOT_SU3 -6          /* a link deviates from SU(3) by more than 1e-10 */
#define QCD_ERR_SINGULAR_CLOVER -7  /* a 6x6 clover block could not be inverted */
#define QCD_NOT_CONVERGED -8        /* max_restarts reached; x and info hold the best iterate */
#define QCD_STAGNATED -9            /* a restart cycle failed to reduce the true residual */
#define QCD_NAN -10                 /* a NaN/Inf appeared in the recursion */
#define QCD_ERR_UNSUPPORTED -11     /* the requested precision/shape combination is not available */
#define QCD_ERR_TOO_LARGE -12       /* size beyond a fixed limit of the called entry point */
#define QCD_ERR_TIMEOUT -13         /* a kernel's bounded wait ran out (the kernel skipped its work and returned) */

/* storage/arithmetic precisions */
#define QCD_PREC_F64 0   /* FP64 storage and arithmetic */
#define QCD_PREC_F32 1   /* FP32 storage and arithmetic */
#define QCD_PREC_F16 2   /* IEEE FP16 storage with a per-site FP32 scale, FP32 arithmetic */
#define QCD_PREC_BF16 3  /* bfloat16 storage with a per-site FP32 scale, FP32 arithmetic */
#define QCD_PREC_DF64 4  /* double-float: pairs of FP32 values (hi + lo, a 48-bit significand) computed
                            with error-free transformations on the FP32 units; for the FGCR recursion
                            (outer_prec) and qcd_apply_D only */

/* preconditioners */
#define QCD_PRECOND_NONE 0  /* plain GCR */
#define QCD_PRECOND_SAP 1   /* Schwarz alternating procedure with MR block solves */

/* Krylov solver of qcd_solve (qcd_solver_params.solver) */
#define QCD_SOLVER_FGCR 0       /* flexible GCR with plain restarts (Sec. 4) */
#define QCD_SOLVER_FGMRES_DR 1  /* flexible GMRES with deflated restarts (Sec. 4) */
#define QCD_SOLVER_CG 2         /* CG on the normal equations D^+ D x = D^+ b, FP64 (Sec. 4: CG for the
                                   most difficult cases) */
#define QCD_SOLVER_CG_EO 3      /* even/odd-preconditioned CG, FP64: CG on Dhat^+ Dhat x_e = Dhat^+ bhat_e with
                                   the Schur complement Dhat = A_ee - D_eo A_oo^-1 D_oe on the even sites,
                                   bhat_e = b_e - D_eo A_oo^-1 b_o, then x_o = A_oo^-1 (b_o - D_oe x_e) */

typedef struct qcd_ctx qcd_ctx;

/* Lattice, action and Schwarz-block parameters (fixed for the life of a context). */
typedef struct {
    int dims[4];     /* L0 = T, L1, L2, L3 (each even) */
    int block[4];    /* Schwarz block extents: even, dividing dims, dims[mu]/block[mu] even */
    double m0;       /* bare mass; kappa = 1 / (2 m0 + 8) */
    double csw;      /* clover coefficient */
    double bc[4];    /* sign of the hop that wraps direction mu: {-1, 1, 1, 1} = antiperiodic time */
} qcd_params;

/* Solver parameters (Sec. 4: FGCR restart length, SAP cycles, MR steps). */
typedef struct {
    double tol;        /* stop when the true FP64 residual |b - D x| / |b| <= tol */
    int nkv;           /* FGCR restart length (Krylov vectors per cycle), 1..64 */
    int max_restarts;  /* maximum number of restart cycles */
    int precond;       /* QCD_PRECOND_SAP or QCD_PRECOND_NONE */
    int ncy;           /* SAP cycles per preconditioner application */
    int nmr;           /* MR steps per block solve */
    int sap_prec;      /* precision of the SAP block fields: QCD_PREC_F64/F32/F16/BF16 */
    int outer_prec;    /* precision of the FGCR recursion (Sec. 4):
                          QCD_PREC_F64 (default): rho, phi_k, chi_k = D phi_k, Gram-Schmidt and dots in FP64;
                          QCD_PREC_DF64: rho, phi_k, chi_k = D phi_k (links and clover as pairs too), the
                          Gram-Schmidt dots and updates and the solution increment in double-float arithmetic
                          on the FP32 units (GB300 runs FP64 at 1/64 of its FP32 rate); the solution in FP64
                          and the restart residual r = b - D x as residual_prec says;
                          QCD_PREC_F32: iterative refinement -- each restart cycle runs the whole recursion
                          in FP32 on the normalised residual r / |r| until its residual has dropped by
                          inner_tol (or the target is met), then the FP32 correction is added to the FP64
                          solution and r = b - D x is recomputed in FP64 */
    double inner_tol;  /* QCD_PREC_F32 recursion only: residual reduction per restart cycle (default 1e-5) */
    int solver;        /* QCD_SOLVER_FGCR (default) or QCD_SOLVER_FGMRES_DR: flexible GMRES whose restarts keep
                          the harmonic Ritz vectors of the ndefl smallest values (Sec. 4, deflated restarts);
                          FP64 recursion (outer_prec must be QCD_PREC_F64), nkv = cycle length m */
    int ndefl;         /* QCD_SOLVER_FGMRES_DR: deflated vectors k, 0 <= k < nkv (default 4) */
    int cg_fallback;   /* when FGCR or FGMRES-DR stagnates or exhausts max_restarts, continue from its
                          iterate with 1: CG on the normal equations, 2: even/odd-preconditioned CG
                          (QCD_SOLVER_CG_EO); 0 (default): no fallback */
    int cg_max_iter;   /* iteration limit of CG (either form), as solver or fallback (default 20000) */
    int zero_guess;    /* 1: start from x = 0 and ignore the input content of x (a host x is then not
                          uploaded, only written); 0 (default): x holds the initial guess */
    int residual_prec; /* QCD_PREC_DF64 recursion only -- the restart residual r = b - D x:
                          QCD_PREC_DF64 (default): D x in double-float arithmetic on the FP32 units from the
                          split of x, the difference and |r|^2 in FP64 (about 1e-13 |x| of rounding in r, far
                          below any tolerance in |r|: 2.4 times faster than the FP64 operator on GB300);
                          QCD_PREC_F64: everything in FP64 */
} qcd_solver_params;

/* Solver report, always filled (also on failure). */
typedef struct {
    int status;            /* same value as the call's return code */
    int iterations;        /* total FGCR iterations (FGMRES-DR: Arnoldi steps) */
    int restarts;          /* restart cycles performed */
    double true_residual;  /* final |b - D x| / |b| recomputed from the solution (FP64; see residual_prec) */
    double time_ms;        /* wall time of the solve on the stream (CUDA events) */
    double sap_ms;         /* time inside the SAP preconditioner (profiling only, else 0) */
    double dirac_ms;       /* time inside the outer operator applies (profiling only, else 0) */
    double blas_ms;        /* time inside the FP64 vector algebra (profiling only, else 0) */
    int cg_iterations;     /* CG iterations (QCD_SOLVER_CG, or the fallback after FGCR / FGMRES-DR) */
} qcd_solve_info;

/* Default solver parameters: tol 1e-10, nkv 16, max_restarts 100, SAP with
 * ncy 4 and nmr 4 in FP32, FP64 outer operator, initial guess read from x. */
void qcd_solver_defaults(qcd_solver_params* sp);

/*
 * Create a context for one lattice.  Validates dims/blocks (Sec. 4: "the local
 * lattice sizes are only constrained to be multiples of the block sizes"; the
 * chessboard colouring additionally needs an even number of blocks per
 * direction, and the even/odd split inside blocks even block extents),
 * uploads the layout tables and returns *out (caller frees with qcd_destroy).
 * Device memory for fields is allocated on first use.  Errors: QCD_ERR_ARG,
 * QCD_ERR_GEOMETRY, QCD_ERR_CUDA, QCD_ERR_NOMEM.
 */
int qcd_create(qcd_ctx** out, const qcd_params* p);

/* Release every device allocation of the context. */
void qcd_destroy(qcd_ctx* ctx);

/*
 * Load the gauge field U ((V, 4, 3, 3) complex128, lexicographic; host pointer
 * if is_device = 0, device pointer otherwise) into the context: reorders into
 * the block-major even/odd layout (Sec. 5) and checks that every link is in
 * SU(3) to 1e-10 (QCD_ERR_NOT_SU3).  The caller keeps ownership of U.
 * stream: a cudaStream_t (NULL = default stream); the call is synchronous on
 * return.
 */
int qcd_load_gauge(qcd_ctx* ctx, const double* U, int is_device, void* stream);

/*
 * Build the clover term A(x) in FP64 from the loaded links (abstract/Sec. 1:
 * "Wilson-Dirac solver with Clover term"), and the per-site inverses of its
 * two 6x6 chiral blocks used by the even/odd block solver (Sec. 5, Table 1).
 * Errors: QCD_ERR_STATE (no gauge field), QCD_ERR_SINGULAR_CLOVER.
 */
int qcd_build_clover(qcd_ctx* ctx, void* stream);

/*
 * out = D in (dagger = 0) or D^+ in (dagger = 1, computed directly; equal to
 * g5 D g5) for nrhs spinor fields (Sec. 4: the matrix-vector product).
 * in/out: device pointers to nrhs * (V, 4, 3) complex128 (must not alias).
 * prec: QCD_PREC_F64 applies in FP64; F32/F16/BF16 convert the input to that
 * storage, apply with FP32 arithmetic and convert the result back;
 * QCD_PREC_DF64 converts the input to double-float pairs and applies the
 * double-float operator of the df64 recursion (FP32 units, about 2^-46
 * relative rounding), converting the result back.
 * Errors: QCD_ERR_STATE, QCD_ERR_ARG.
 */
int qcd_apply_D(qcd_ctx* ctx, const double* in, double* out, int dagger, int prec, int nrhs, void* stream);

/*
 * Solve D x = b for nrhs right-hand sides by SAP-preconditioned FGCR (Sec. 4)
 * to |b - D x| / |b| <= sp->tol in the true residual (see residual_prec).
 * b, x: nrhs * (V, 4, 3) complex128, both host or both device pointers
 * (detected); x holds the initial guess on entry (zeros for none, or any
 * content with sp->zero_guess) and the solution on return.  The call returns
 * when x is complete; while it runs, a single-right-hand-side FGCR solve may
 * write x more than once (each restart's iterate is handed over while the
 * residual is checked), so x must not be read or written concurrently.
 * sp = NULL uses qcd_solver_defaults.  info (may be NULL) receives one
 * qcd_solve_info per right-hand side.  Returns QCD_OK when every right-hand
 * side converged, else the first failing status (QCD_NOT_CONVERGED,
 * QCD_STAGNATED, QCD_NAN, ...).
 */
int qcd_solve(qcd_ctx* ctx, const double* b, double* x, int nrhs, const qcd_solver_params* sp,
              qcd_solve_info* info, void* stream);

/*
 * Solve the adjoint system D^+ x = b (one right-hand side) through
 * D^+ = g5 D g5: x = g5 D^-1 g5 b, with the same solver as qcd_solve.  b, x:
 * device (V, 4, 3) complex128; x holds the initial guess on entry.  This is
 * the adjoint solve of the gradient (Sec. 1: force from the inversions).
 */
int qcd_solve_dagger(qcd_ctx* ctx, const double* b, double* x, const qcd_solver_params* sp, qcd_solve_info* info,
                     void* stream);

/*
 * Solve one right-hand side on each of n contexts (lattices of possibly
 * different sizes, Sec. 4 "flexibility in the choice of lattice sizes")
 * together: the lattices iterate in lock step, each on its own context stream
 * (forked from and joined to `stream`) so that their launches run
 * concurrently on the GPU, every FGCR iteration of a lattice replayed from a
 * captured CUDA graph, with one host synchronisation per iteration for all of
 * them.  Each lattice keeps its own Krylov basis and convergence test, and a
 * converged one stops iterating while the others continue.  b[i], x[i]: device
 * pointers for ctxs[i] (distinct contexts).  info: n entries (may be NULL).
 */
int qcd_solve_batch(qcd_ctx** ctxs, int n, const double* const* b, double* const* x,
                    const qcd_solver_params* sp, qcd_solve_info* info, void* stream);

/*
 * Gradient of L = Re(phi^+ x), x = D^-1 phi (Sec. 1: the inversions feed the
 * HMC fermion force):
 *   dL_dphi   = x + y with y = D^-+ phi = g5 D^-1 g5 phi (adjoint solve), the
 *               torch convention dL/dRe + i dL/dIm; device (V, 4, 3) complex128;
 *   dL_dtheta = -Re(y^+ dD/dtheta_a x) for every link and generator
 *               (hopping and clover parts); device (V, 4, 8) float64.
 * Either output may be NULL.  x_out/y_out (may be NULL) receive the two
 * solutions.  Both solves use sp (tolerance included).
 */
int qcd_gradient(qcd_ctx* ctx, const double* phi, double* dL_dphi, double* dL_dtheta,
                 double* x_out, double* y_out, const qcd_solver_params* sp, void* stream);

/*
 * Force kernel alone: F_a(x, mu) = -Re(y^+ dD/dtheta_a x) for given device
 * spinors x, y ((V, 4, 3) complex128), written to F ((V, 4, 8) float64).
 */
int qcd_force(qcd_ctx* ctx, const double* x, const double* y, double* F, void* stream);

/* ---- Hybrid Monte Carlo molecular dynamics (Sec. 1: the inversions feed the
 * HMC fermion force), two degenerate clover flavours, one pseudofermion.
 * Gauge fields U here are lexicographic device arrays (V, 4, 3, 3) complex128
 * (qcd_load_gauge's layout, periodic links); momenta pi and forces F are
 * device (V, 4, 8) float64 with P(x, mu) = sum_a pi_a lambda_a / 2, and every
 * derivative is taken for U_mu(x) -> exp(i theta_a lambda_a / 2) U_mu(x).
 * Errors: QCD_ERR_ARG (null pointer, nsteps < 1, eps <= 0), QCD_ERR_NOMEM,
 * and the status of any solve of the trajectory. */
typedef struct {
    int accepted;             /* Metropolis: u_accept < exp(-dH) */
    double dH;                /* H1 - H0 */
    double H0, H1;            /* H = kin + S_g + S_f at the start and the end */
    double kin0, S_g0, S_f0;  /* kin = 1/2 sum pi^2; S_g plaquette action; S_f = |D^-+ phi|^2 */
    double kin1, S_g1, S_f1;
    int solves;               /* linear solves of the trajectory */
    int iterations;           /* Krylov (and CG) iterations summed over the solves */
    double time_ms;           /* CUDA-event time of the trajectory */
} qcd_hmc_info;

/* Wilson plaquette action S = beta sum_{x, mu<nu} (1 - Re tr U_munu(x) / 3),
 * written to *S (host).  U: device, ctx's lattice. */
int qcd_gauge_action(qcd_ctx* ctx, const double* U, double beta, double* S, void* stream);

/* Its force F_a(x, mu) = dS/dtheta_a = (beta / 6) Im tr(lambda_a U_mu(x) V_mu(x)),
 * V_mu(x) the sum of the six staples; U, F device. */
int qcd_gauge_force(qcd_ctx* ctx, const double* U, double beta, double* F, void* stream);

/* U_mu(x) <- exp(i eps P(x, mu)) U_mu(x) for every link, in place (exponential
 * by a scaled Taylor series, exact to rounding). */
int qcd_update_links(qcd_ctx* ctx, double* U, const double* pi, double eps, void* stream);

/* One HMC trajectory: pseudofermion phi = D(U)^+ eta (eta: device (V, 4, 3)
 * complex128, a Gaussian draw); leapfrog of nsteps steps of size eps on
 * H = 1/2 sum pi^2 + S_g + S_f with S_f = phi^+ (D^+ D)^-1 phi: pi -= eps/2 F,
 * then nsteps times {U <- exp(i eps P) U; pi -= eps F} with a final half step,
 * F = dS_g/dtheta - 2 Re(Y^+ dD/dtheta X), Y = D^-+ phi, X = D^-1 Y (solved
 * with sp).  Metropolis with the caller's uniform u_accept in [0, 1): on
 * acceptance U holds the new links, on rejection the starting links; pi holds
 * the final momenta either way.  The context is left loaded with the returned
 * links (clover rebuilt). */
int qcd_hmc_trajectory(qcd_ctx* ctx, double* U, double* pi, const double* eta, double beta, double eps,
                       int nsteps, double u_accept, const qcd_solver_params* sp, qcd_hmc_info* info,
                       void* stream);

/*
 * Pick, by timing on the device, the fastest launch shape of the operator
 * kernel for each storage precision of this context (double-float included)
 * -- CTA size, and for 16-bit storage one or two threads per site -- and, for
 * nrhs > 1, the right-hand-side tile of the batched SAP sweep (timed on FP16
 * block fields);
 * keep the choices in the context (see qcd_set_launch, qcd_set_sap_tile).
 * nrhs: right-hand sides per call the tuning should reflect (the operator
 * timing applies that many operators back to back).  cache_path (may be
 * NULL): a JSON file read before tuning (a matching entry is applied without
 * timing) and rewritten after it, keyed by GPU name, dims, block and nrhs.
 * Needs qcd_load_gauge and qcd_build_clover first.
 */
int qcd_autotune(qcd_ctx* ctx, int nrhs, const char* cache_path);

/*
 * Choose the Schwarz block shape (Sec. 4/5: the block size is the main SAP
 * tuning parameter; local lattice sizes need only be multiples of it) by
 * timing complete solves of b on the given gauge field: for each candidate a
 * temporary context is created with p's action parameters, the field is
 * loaded, the clover term built and D x = b solved with sp.  candidates: n
 * shapes (4 ints each); NULL enumerates shapes with even extents, an even
 * number of blocks per direction and 64..512 sites.  U, b: (V,4,3,3) and
 * (V,4,3) complex128, host (is_device = 0) or device pointers.  out_block
 * receives the fastest shape; times_ms (may be NULL, n entries, or 64 when
 * candidates is NULL) the time-to-solution of each candidate (negative when a
 * candidate failed).  Returns the number of candidates tried, or a negative
 * status.
 */
int qcd_tune_block(const qcd_params* p, const double* U, const double* b, int is_device, const qcd_solver_params* sp,
                   const int* candidates, int n, int out_block[4], double* times_ms);

/*
 * Launch shapes (what qcd_autotune chooses), for callers that pin them:
 * qcd_set_launch sets, for storage precision prec (QCD_PREC_F64 .. DF64), the
 * operator kernel's CTA size `threads` (a multiple of 32, 32..1024; at most
 * 256 for DF64) and its threads per site `tps`: 1, or 2 for 16-bit storage
 * (QCD_PREC_F16 / BF16: two threads share a site, each taking two of the four
 * directions and half of the spin components, in CTAs of 256;
 * QCD_ERR_UNSUPPORTED otherwise).  qcd_get_launch reads the current shape.
 * qcd_set_sap_tile sets how many right-hand sides one CTA of a batched SAP
 * sweep solves with one staging of its block's fields (1..64; 0
 * restores the default: the largest tile that keeps four CTAs per SM);
 * qcd_get_sap_tile returns the tile a solve of nrhs right-hand sides uses.
 * Results do not depend on any of these.
 */
int qcd_set_launch(qcd_ctx* ctx, int prec, int threads, int tps);
int qcd_get_launch(const qcd_ctx* ctx, int prec, int* threads, int* tps);
int qcd_set_sap_tile(qcd_ctx* ctx, int rt);
int qcd_get_sap_tile(qcd_ctx* ctx, int nrhs);

/* Static description of a status code. */
const char* qcd_status_string(int status);

/* Message of the last CUDA error seen by this thread (empty if none). */
const char* qcd_last_error(void);

/* ------------------------------------------------------------------------
 * Resident fields and instrumentation (used by benchmarks and tests)
 * ------------------------------------------------------------------------ */

typedef struct qcd_field qcd_field;

/*
 * Allocate a device spinor field of the context's lattice in internal layout
 * (block-major, even/odd split inside blocks, Sec. 5) with the given storage
 * precision.  Free with qcd_field_free.
 */
int qcd_field_create(qcd_ctx* ctx, int prec, qcd_field** out);
/* Same for nrhs fields back to back (a multi-right-hand-side field: import,
 * export and qcd_apply_D_field then treat nrhs * (V, 4, 3) complex128, and the
 * operator reads each site's links and clover once for all right-hand sides). */
int qcd_field_create_n(qcd_ctx* ctx, int prec, int nrhs, qcd_field** out);
void qcd_field_free(qcd_field* f);

/* Convert a device (V, 4, 3) complex128 lexicographic spinor into / out of a field. */
int qcd_field_import(qcd_ctx* ctx, qcd_field* f, const double* in, void* stream);
int qcd_field_export(qcd_ctx* ctx, const qcd_field* f, double* out, void* stream);

/*
 * out = D in (or D^+ in) on resident fields of the same precision: one kernel
 * launch, no layout conversion (the operator whose HBM traffic the benchmark
 * reports).  Errors: QCD_ERR_STATE, QCD_ERR_ARG (precision mismatch).
 */
int qcd_apply_D_field(qcd_ctx* ctx, const qcd_field* in, qcd_field* out, int dagger, void* stream);

/*
 * out = D in (dagger = 0) or D^+ in (dagger = 1) in FP64, like qcd_apply_D with
 * prec = QCD_PREC_F64 and nrhs = 1, but without allocating device memory.  The
 * paper has no counterpart: this entry point exists for callers that must not
 * have a library allocate or free device memory -- programs whose own pool
 * allocator owns all device memory within a fixed budget, and latency-bound
 * loops where cudaFree's device-wide synchronisation would stall other
 * streams.  The two staging fields live in one static device array of the
 * library instead, so:
 *   - the lattice may have at most 65536 sites (QCD_ERR_TOO_LARGE beyond);
 *   - the array (24 MiB) is held on every GPU that loads the library until exit;
 *   - all calls share the array; calls that overlap on the GPU race;
 *   - the first call on each device looks up the array's address; make it
 *     before any stream capture;
 *   - the address is kept for the life of the process: do not call this entry
 *     point again after cudaDeviceReset in the same process;
 *   - kernel profiling (qcd_profile_enable) must be off (QCD_ERR_STATE
 *     otherwise: the profiler creates CUDA events on demand).
 * in/out: device (V, 4, 3) complex128, must not alias.  The call is
 * asynchronous: out is ready when the stream reaches the call's end.  Needs
 * qcd_load_gauge and qcd_build_clover first (QCD_ERR_STATE).
 */
int qcd_apply_D_noalloc(qcd_ctx* ctx, const double* in, double* out, int dagger, void* stream);

/*
 * psi = M_SAP eta: one application of the Schwarz preconditioner (Sec. 4) with
 * ncy cycles of nmr MR steps per block, block fields in sap_prec.  eta, psi:
 * device (V, 4, 3) complex128 lexicographic.
 */
int qcd_sap_apply(qcd_ctx* ctx, const double* eta, double* psi, int ncy, int nmr, int sap_prec, void* stream);

/*
 * The same for nrhs right-hand sides at once (Sec. 4 applies the
 * preconditioner to one residue at a time; applying it to several shares the
 * staging of each Schwarz block's links and clover): each CTA of a colour
 * sweep solves one block for rt right-hand sides in turn (rt = 0: the
 * library's default tile).  eta, psi: device nrhs * (V, 4, 3) complex128,
 * lexicographic.  psi_q = M_SAP eta_q for every q, identical to nrhs calls of
 * qcd_sap_apply.  Allocates and frees its work fields on every call.
 */
int qcd_sap_apply_n(qcd_ctx* ctx, const double* eta, double* psi, int nrhs, int rt, int ncy, int nmr, int sap_prec,
                    void* stream);

/*
 * Test hooks for failure detection without a GPU fault.  The SAP kernel waits
 * for its staging copies with a bounded spin (about a second); when the
 * budget runs out the kernel records it, lets the copies in flight land and
 * returns, and the calling solve or qcd_sap_apply reports QCD_ERR_TIMEOUT
 * with the context still usable.  qcd_debug_set lets a test make that happen:
 *   QCD_DEBUG_SAP_WAIT_CYCLES: budget of the staging wait in clock cycles,
 *                              1 .. 2^31 (default 2^31);
 *   QCD_DEBUG_SAP_EXTRA_TX:    bytes the staging barrier expects beyond the
 *                              copies, 0 .. 4096 (default 0; any other value
 *                              makes every wait run out).
 * Returns QCD_ERR_ARG for an unknown setting or a value out of range.
 */
#define QCD_DEBUG_SAP_WAIT_CYCLES 0
#define QCD_DEBUG_SAP_EXTRA_TX 1
int qcd_debug_set(qcd_ctx* ctx, int what, long long value);

/*
 * Precision codecs (Sec. 4: single-precision preconditioner inside a double
 * precision solver).  The kernels that move fields between the FP64 recursion
 * and the FP32 preconditioner (the first and last Schwarz sweeps, the
 * refinement updates) convert with integer operations instead of GB300's
 * FP64 conversion unit; this entry point exposes those conversions so that
 * they can be checked against the hardware ones:
 *   out32[i] = in64[i] rounded to FP32 (nearest, ties to even),
 *   out64[i] = in32[i] widened to FP64 (exact),  i < n.
 * All four are device pointers of n elements (n >= 0); the call is
 * asynchronous on `stream`.  Returns QCD_ERR_ARG for n < 0 or a null pointer.
 */
int qcd_convert_check(const double* in64, const float* in32, float* out32, double* out64, long long n, void* stream);

/*
 * Kernel timing: when enabled, each launch of the instrumented kernels is
 * bracketed by CUDA events on its stream.  qcd_profile_get returns, for a
 * kernel id (QCD_KERNEL_*), the launch count and summed device time (ms), and
 * the algorithmic bytes and flops per launch averaged over those launches (a
 * conditional second Gram-Schmidt pass counts as no work).
 */
#define QCD_KERNEL_DIRAC 0      /* full-lattice operator apply (any precision) */
#define QCD_KERNEL_SAP 1        /* one SAP colour sweep */
#define QCD_KERNEL_BLAS 2       /* FP64 vector algebra kernels */
#define QCD_KERNEL_RESIDUAL 3   /* fused true residual r = b - D x */
#define QCD_KERNEL_COUNT 4
int qcd_profile_enable(qcd_ctx* ctx, int on);
/*
 * Measured arithmetic peaks of the current GPU (the denominators of the ALU
 * rooflines): throughput of fused multiply-adds with eight independent
 * register chains per thread on eight CTAs per SM, in TFLOP/s (2 flops per
 * multiply-add and lane): scalar FP32, packed FP32x2 (the form the operator
 * and block-solver kernels use for SU(3) products) and FP64.  Any output may
 * be NULL (that form is not timed).  Takes some tens of milliseconds;
 * synchronous.
 */
int qcd_measure_alu_peaks(double* fp32_tflops, double* fp32x2_tflops, double* fp64_tflops, void* stream);

/* Number of kernels this library has launched since it was loaded (all contexts). */
long long qcd_launch_count(void);
int qcd_profile_reset(qcd_ctx* ctx);
int qcd_profile_get(qcd_ctx* ctx, int kernel, long long* launches, double* total_ms,
                    double* bytes_per_launch, double* flops_per_launch);

#ifdef __cplusplus
}
#endif

#endif /* QCDGB_H */
