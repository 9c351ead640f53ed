/*
 * mg.h -- C ABI of the GB300 adaptive-multigrid solver for the 2D U(1)
 * Wilson-Dirac normal equations A = D^dagger D.
 *
 * Method: Brannick, Brower, Clark, Osborn, Rebbi, "Adaptive Multigrid
 * Algorithm for the QCD Dirac-Wilson Operator" (Lattice 2007):
 *   Sec. 1   Wilson operator D (display after Eq. 1), normal operator A = D^dagger D
 *   Sec. 2   Galerkin coarse operator (Eq. Galerkin), five-step V-cycle
 *   Sec. 3   adaptive setup: relaxation on A e = 0 (Eq. relax), geometric
 *            blocks S_j, normalised block vectors (Eq. P1), index s over
 *            vector sets
 *   Sec. 4   frozen two-step MR smoother, setup reuse across masses, MG-CG
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice: Lx x Lt sites, site index x + Lx * t; x periodic, t antiperiodic
 * for the fermion field, gauge field periodic.  gamma_1 = sigma_1 (x links),
 * gamma_2 = sigma_2 (t links), gamma_5 = sigma_3; diagonal 2d + m = 4 + m.
 *
 * Levels are numbered as in the paper: 1 = finest ... nlevels = coarsest.
 * A level-l vector is [nrhs][Lt_l][Lx_l][n_l] complex, n_1 = 2 (spin),
 * n_{l+1} = 2 * Nv_l.  Coarse dof s = c * Nv + k: vector k restricted to
 * chirality c (c = 0: gamma_5 = +1).  On level 1 chirality c is spin c; on
 * level l > 1 the first n_l/2 components have chirality 0.
 *
 * Coarse operator A_l (l >= 2): 9-point stencil of dense n_l x n_l blocks,
 * stored [Lt_l][Lx_l][9][n_l][n_l] (row-major blocks), displacement index
 * d = (dx + 1) + 3 (dt + 1); (A_l v)(j) = sum_d A_l[j][d] v(j + d).
 *
 * Precision codes: MG_PREC_F64 -> complex128 buffers (double re, double im);
 * MG_PREC_F32 -> complex64 buffers; MG_PREC_BF16 -> complex64 vectors with
 * the coarse blocks held in bfloat16 and FP32 accumulation.
 *
 * Pointers: every vector, gauge and noise pointer is a DEVICE pointer on the
 * handle's device; the caller owns it.  Input and output buffers must not
 * alias.  All work is enqueued on the handle's CUDA stream (the stream passed
 * to mg_setup); calls returning data in host memory synchronise that stream.
 * Errors: every call returns an mg_status, never aborts and never throws;
 * mg_last_error() gives a message.  A handle is not thread-safe.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_MAX_LEVELS 5
#define MG_MAX_REFINE 16                /* adaptive passes made by mg_setup      */

typedef struct mg_handle mg_handle;

typedef enum {
  MG_OK = 0,
  MG_ERR_ARG = 1,        /* invalid argument (sizes, pointers, divisibility) */
  MG_ERR_NOMEM = 2,      /* device allocation failed                          */
  MG_ERR_CUDA = 3,       /* a CUDA call failed                                */
  MG_ERR_NOCONV = 4,     /* solver stopped at maxiter above tolerance         */
  MG_ERR_BREAKDOWN = 5,  /* <p,Ap> <= 0, non-finite residual, or rank-deficient
                            block Gram-Schmidt                                 */
  MG_ERR_TIMEOUT = 6     /* reserved for bounded device-side waits            */
} mg_status;

typedef enum { MG_PREC_F64 = 0, MG_PREC_F32 = 1, MG_PREC_BF16 = 2 } mg_precision;

typedef enum {
  MG_SOLVER_MGCG_FP64 = 0,  /* MG-CG, everything in FP64 (Sec. 4)                */
  MG_SOLVER_MGCG_MIXED = 1, /* FP64 flexible CG (Krylov recursion, residual and
                               solution in FP64) preconditioned by the FP32
                               V-cycle: FP32 smoother, restriction, prolongation
                               and coarse applies (coarse blocks FP32, or BF16
                               with FP32 accumulation), coarsest solve in FP64 */
  MG_SOLVER_CG_FP64 = 2,    /* plain CG on A, FP64 (the paper's baseline)        */
  MG_SOLVER_MGCG_RELIABLE = 3 /* flexible CG preconditioned by the same FP32
                               V-cycle, with the iteration itself in FP32 (A p
                               by the FP32 stencil, residual, search direction
                               and solution increment in FP32; inner products
                               summed in FP64 across thread blocks) and FP64
                               reliable updates: when the iterated |r| falls
                               below reliable_delta times its largest value
                               since the last update, the increment is added
                               to the FP64 solution and r = b - A x is
                               recomputed with the FP64 stencil.  The solution
                               and the final true residual are FP64 as in
                               MG_SOLVER_MGCG_MIXED; per iteration no FP64
                               arithmetic runs on fine-lattice vectors        */
} mg_solver;

typedef struct {
  int Lx, Lt;                           /* fine lattice                          */
  int nlevels;                          /* 1 .. MG_MAX_LEVELS; 1 = fine operator
                                           only (apply calls and plain CG)       */
  int block[MG_MAX_LEVELS - 1][2];      /* (bx, bt) blocking level l -> l+1      */
  int Nv[MG_MAX_LEVELS - 1];            /* vectors per chirality, level l -> l+1 */
  int setup_sweeps;                     /* nu of Eq. relax (default 8)           */
  int power_iters;                      /* iterations for lambda_max (30)        */
  double omega_mr;                      /* MR under-relaxation, Sec. 4 (0.8)     */
  const void* setup_noise;              /* device complex128, mg_setup_noise_len
                                           entries; layout below                 */
  double coarsest_tol;                  /* FP64 refinement target of the coarsest
                                           solve, relative (1e-13)               */
  int coarsest_refine_max;              /* cap on refinement steps (12)          */
  int inner_coarsest_refine;            /* mixed solver: FP64 refinement steps of
                                           the coarsest solve inside the FP32
                                           V-cycle (1)                           */
  int vcycle_coarse_bf16;               /* mixed solver: 1 = coarse blocks of the
                                           FP32 V-cycle in BF16 (FP32 accumulate),
                                           0 = FP32 (1)                          */
  int max_rhs;                          /* right-hand sides solved together by
                                           mg_solve, 1..64 (1); work memory
                                           scales with it                        */
  int profile;                          /* nonzero: per-kernel-family event
                                           timing (mg_profile_enable) from the
                                           start of mg_setup (0)                 */
  int coarsest_dense_max;               /* coarsest levels with at most this
                                           many unknowns use the dense FP32
                                           inverse with FP64 refinement; larger
                                           ones FP64 CG on the coarsest stencil
                                           (16384; at most 24576)               */
  int coarsest_gj_tcgen05;              /* rank-64 updates of the dense inverse
                                           on tcgen05 tensor cores (TMEM
                                           accumulator, 1) or with mma.sync
                                           (0, default: measured faster at 4096
                                           unknowns)                            */
  int refine_levels[MG_MAX_REFINE];     /* adaptive refinement by V-cycles made
                                           by mg_setup after the first pass
                                           (Sec. 3): the level (1 .. nlevels-1)
                                           refined by each pass, in order, ended
                                           by 0 or by the array's end; levels
                                           must not decrease.  Nv above is the
                                           first-pass set; each pass adds one
                                           vector per chirality to its level
                                           (all 0: no refinement)              */
  int refine_cycles;                    /* V-cycles per adaptive pass (30)      */
  int autotune;                         /* nonzero: mg_setup times the launch
                                           shapes of the fused fine A (FP32 and
                                           FP64, 1 and max_rhs right-hand
                                           sides) once per process and shape
                                           and keeps the fastest whose output
                                           is bit-identical to the default
                                           shape's (1)                          */
  int remass_quadratic;                 /* nonzero: keep G0_l and G1_l with
                                           A_l(m) = G0_l + m G1_l + m^2 I on
                                           every coarse level (A(m) = A0 +
                                           m (D0 + D0^dagger) + m^2 and
                                           P^dagger P = I), so a new mass is one
                                           combination per level instead of the
                                           Galerkin products; two more FP64
                                           copies of each coarse operator (1)   */
  double smooth_omega;                  /* smoothed aggregation of the first
                                           coarsening (Sec. 3): the columns of
                                           P (fine level -> level 2) become
                                           P_s = (1 - omega A) P, and level 2 is
                                           P_s^dagger A P_s.  0: off (default);
                                           > 0: this omega; < 0: the omega in
                                           [0, 2 / lambda~max(A)] minimising
                                           the condition number of level 2
                                           (two-level hierarchies with a dense
                                           coarsest level only).  Needs level-1
                                           blocks of at least 4 x 4 and coarse
                                           extents of at least 3; excludes
                                           refine_levels; remass_quadratic is
                                           ignored (each mass is probed anew) */
  double reliable_delta;                /* MG_SOLVER_MGCG_RELIABLE: residual
                                           reduction between FP64 reliable
                                           updates, in (0, 1); default 0.1   */
  int coarsest_reuse;                   /* mg_set_mass with a dense coarsest
                                           level: 0 (default) inverts the new
                                           coarsest operator; k > 0 first tries
                                           the FP32 inverse of the previous
                                           mass inside the FP64 refinement and
                                           keeps it when both test vectors reach
                                           coarsest_tol within
                                           min(k, coarsest_refine_max - 1)
                                           steps (the coarsest solve stays exact
                                           to coarsest_tol; the refinement count
                                           grows instead of a new inversion);
                                           the FP32 V-cycle then refines until
                                           the test vectors reach 1e-6 */
} mg_params;

typedef struct {
  int iterations;             /* Krylov iterations (inner iterations summed)   */
  int refinements;            /* restarts from the true FP64 residual          */
  double true_residual;       /* |b - A x| / |b| recomputed in FP64            */
  long long fine_applies;     /* applications of the fine A = D^dagger D        */
  long long vcycles;          /* V-cycles applied                               */
  double milliseconds;        /* wall time of the call                          */
} mg_solve_info;

/* One launch shape picked by the stencil autotuner (mg_params.autotune). */
typedef struct {
  int precision;              /* MG_PREC_F64 or MG_PREC_F32                    */
  int Lx, Lt, nrhs;           /* the launch it serves                          */
  int tx, ty, rows_per_thread;/* tile of the fused A; 0 x 0 = the streaming
                                 kernel (one warp per strip)                   */
  int tried, admitted;        /* shapes timed / shapes bit-identical to the
                                 default shape (only those may be chosen)      */
  double us_chosen;           /* microseconds per launch of the chosen shape   */
  double us_default;          /* microseconds per launch of the default shape  */
} mg_stencil_tuning;

/* Critical mass m_crit (the mass gap m - m_crit of Sec. 4): the heaviest
 * mass below m_hi at which D(m) is singular, i.e. at which an eigenvalue of the
 * Hermitian H(m) = sigma_3 D(m) crosses zero.  Spectral-flow scan: every
 * eigenvalue of H moves by at most |dm| (dH/dm = sigma_3), so
 * mu(m) = min |eig H(m)| is 1-Lipschitz and no crossing lies within mu(m) of
 * m; from m_hi the scan steps down by safety * mu(m).  mu(m) and the signed
 * eigenvalue lam come from inverse iteration with H^-1 = A^-1 D^dagger
 * sigma_3 (FP64 MG-CG solves on h, re-massed as the scan goes; warm-started
 * from the previous eigenvector), dlam/dm = <v, sigma_3 v>.  Once mu <
 * newton_below, Newton steps aimed at |lam| = newton_floor (never closer,
 * where the solves lose accuracy) bring m near the crossing; there the
 * eigenvalue lam_D of D(m) nearest zero is found by inverse iteration with
 * D^-1 = A^-1 D^dagger, and since D(m) = D_0 + m shifts every eigenvalue by m
 * exactly, m_crit = m - lam_D when lam_D is real (|Im| <= 1e-8 |Re|) and
 * agrees with the cubic Hermite interpolant of the last two (lam, dlam/dm)
 * points; otherwise that interpolant's root is returned.
 *   v0:  device complex128 fine vector, the first inverse-iteration start.
 *   *m_crit, *slope (dlam/dm there, may be NULL), *evals (eigen-solves
 *   made, may be NULL).  h is left at the last mass evaluated.
 * MG_ERR_NOCONV when no crossing is found above m_lo within max_evals
 * eigen-solves; MG_ERR_ARG for invalid arguments or nlevels < 2. */
mg_status mg_critical_mass(mg_handle* h, double m_hi, double m_lo, const void* v0, double safety,
                           double newton_below, double newton_floor, int max_evals,
                           double* m_crit, double* slope, int* evals);

/* Quenched U(1) gauge field on the device (the paper's gauge ensembles,
 * Sec. 4: Wilson plaquette action S = -beta sum_p Re U_p): checkerboard
 * Metropolis sweeps first_sweep .. first_sweep + sweeps - 1 on the link angles
 * theta (device float64 [2][Lt][Lx], x links then t links), updated in place.
 * One sweep visits direction 0 then 1, each in two halves by the parity of
 * the other coordinate; proposal theta' = theta + eps (2 u - 1), accepted
 * when u' < exp(-dS); accepted angles are mapped to [-pi, pi).  The uniforms
 * are Philox4x32-10 (Salmon et al., SC'11) at counter (t Lx + x,
 * 4 sweep + 2 mu + parity as two 32-bit words, 0) and key (seed low 32 bits,
 * seed high 32 bits): u from words 0, 1 and u' from words 2, 3, each
 * (w0 >> 5) 2^-27 + (w1 >> 6) 2^-53.  Lx, Lt even and >= 2.  accepted (host,
 * may be NULL) receives the number of accepted proposals.  Synchronises the
 * stream. */
mg_status mg_gauge_metropolis(double* theta, int Lx, int Lt, double beta, double eps, int sweeps,
                              long long first_sweep, unsigned long long seed, void* stream,
                              long long* accepted);

/* Gauge links U = exp(i theta) (device complex128 [2][Lt][Lx], the layout
 * mg_setup takes) from the angles of mg_gauge_metropolis. */
mg_status mg_gauge_links(const double* theta, void* U, int Lx, int Lt, void* stream);

/* The shapes tuned so far in this process: up to max records into out (host,
 * may be NULL with max = 0); returns the number of records. */
int mg_stencil_tunings(mg_stencil_tuning* out, int max);

/* Fill *p with the defaults listed above for an Lx x Lt lattice (no levels). */
mg_status mg_params_default(mg_params* p, int Lx, int Lt);

/* Number of complex128 entries of params->setup_noise.  For each level
 * l < nlevels (finest first): Nv_l start vectors for the relaxation of
 * Eq. relax, then one start vector for the power iteration that sets the
 * relaxation step 1/lambda_max(A_l), then one start vector for the two MR
 * steps that fix the smoother (Sec. 4).  Each is a level-l vector.  Then,
 * for each adaptive pass p on level l (refine_levels), its random error e0
 * (a level-l vector) followed by the random starts of every level below l
 * for the Nv after pass p, in the per-level layout above.
 * Returns 0 for invalid parameters and for nlevels = 1 (no noise needed). */
size_t mg_setup_noise_len(const mg_params* p);

/* Adaptive setup (Sec. 3, Eq. relax, Eq. P1, Eq. Galerkin; Sec. 4 smoother).
 * gauge: device complex128 [2][Lt][Lx], mu = 0 x links, mu = 1 t links,
 *   |U| = 1 (checked to 1e-12); copied, the caller keeps ownership.
 * mass: m of D (the setup mass; the paper sets up at the lightest mass).
 * stream: cudaStream_t to use (NULL: the legacy default stream).
 * Validation: Lx, Lt even; each extent divisible by its block; every coarse
 *   extent >= 2; blocks >= 2 x 2; 1 <= Nv_l <= (bx * bt * n_l / 2);
 *   1 <= nlevels <= MG_MAX_LEVELS; 0 <= coarsest_dense_max <= 16384;
 *   refine_levels in [1, nlevels - 1], not decreasing, with refine_cycles
 *   >= 1, and the Nv limits holding after every pass.
 *   MG_ERR_ARG otherwise.  With refine_levels set, the first pass is followed
 *   by the adaptive passes of mg_refine, made in place (the handle then has
 *   the refined Nv; mg_get_level reports it).  With nlevels = 1 no
 *   hierarchy is built and setup_noise may be NULL.
 * On success *out owns all device memory of the hierarchy. */
mg_status mg_setup(const void* gauge, double mass, const mg_params* params, void* stream,
                   mg_handle** out);

/* Reuse the setup's vectors at another mass (Sec. 4): rebuilds every
 * Galerkin operator, the smoothers and the coarsest inverse. */
mg_status mg_set_mass(mg_handle* h, double mass);

/* Device memory of a set-up, before making it (no device work): *resident =
 * the bytes mg_setup allocates and keeps (equal to mg_device_bytes of the
 * handle it returns), *peak = an upper bound of what the set-up holds at
 * once (resident + its temporary relaxation vectors; with adaptive passes,
 * also the hierarchy being replaced and the pass's scratch).  Either pointer may be NULL.  MG_ERR_ARG for invalid params. */
mg_status mg_setup_bytes(const mg_params* params, long long* resident, long long* peak);

/* Device bytes currently owned by the handle. */
mg_status mg_device_bytes(const mg_handle* h, long long* bytes);

/* A second hierarchy at another mass from the same set-up (Sec. 4: the
 * vectors of the set-up reused at other masses): the gauge field, the block
 * vectors of every level and the smoother start vectors are copied from src
 * (device to device, on `stream`), then the Galerkin operators, smoothers and
 * coarsest solver are built at `mass`.  The result equals mg_set_mass(src,
 * mass) without changing src, and owns as much device memory as src.  src
 * may be in use on another thread meanwhile (it is only read). */
mg_status mg_clone(const mg_handle* src, double mass, void* stream, mg_handle** out);

/* Adaptive refinement by V-cycles (Sec. 3, the adaptive step that follows the
 * first vector set), one pass on `level` (1 = finest .. nlevels - 1).
 * The V-cycle of that level (FP64, the preconditioner of MG_SOLVER_MGCG_FP64
 * from that level down) is applied `ncycles` times to the error e0 with no
 * source: e <- e - V_l(A_l e).  The error e'' that survives becomes one more
 * vector of the level: restricted to each block, made orthogonal there (per
 * chirality, modified Gram-Schmidt) to the block's current vectors and
 * normalised.  *out receives a new hierarchy at src's mass and parameters
 * with Nv[level - 1] + 1: finer levels copied from src, the level's vectors
 * extended by e'', the Galerkin operators below rebuilt, the coarser levels'
 * vectors set up again by relaxation (Eq. relax) on the new coarse operators
 * from `noise`, then the smoothers and the coarsest solver.  mg_setup makes
 * the same passes when mg_params.refine_levels asks for them.
 *   e0:     device complex128 level vector [Lt_l][Lx_l][ndof_l], read only.
 *   noise:  device complex128: the random starts of the levels below
 *           `level` only, for the refined Nv, each level laid out as in
 *           mg_params.setup_noise (Nv_k starts, power-iteration start,
 *           smoother start).  May be NULL when level = nlevels - 1 (nothing
 *           below is relaxed).
 *   rho:    (host, may be NULL) (|e''|_A / |e0|_A)^(1 / ncycles), the measured
 *           error reduction per cycle of src's V-cycle on that level.
 *   e_out:  (device, may be NULL) receives e''.
 * src is not changed but its stream and work vectors are used (no concurrent
 * use of src); the new handle runs on `stream` and owns its memory (free with
 * mg_destroy).  The scratch (Nv + 3 level vectors and Nv coarse vectors) is
 * allocated and freed inside the call.  MG_ERR_ARG on a bad level, ncycles < 1
 * or an Nv above the limits of mg_setup; MG_ERR_BREAKDOWN when e'' lies in the
 * span of the current vectors on some block (Gram-Schmidt breakdown) or
 * |e0|_A = 0. */
mg_status mg_refine(mg_handle* src, int level, const void* e0, int ncycles, const void* noise,
                    void* stream, mg_handle** out, double* rho, void* e_out);

/* The measured rho of each adaptive pass mg_setup made (see mg_refine), in
 * pass order: up to `max` values into rho (host), their number into *count. */
mg_status mg_get_refine_rho(const mg_handle* h, double* rho, int max, int* count);

/* Solve A x = b for nrhs right-hand sides (Sec. 4, MG-CG), x_0 = 0.
 * b, x: device complex128 [nrhs][Lt][Lx][2].  Right-hand sides are solved in
 * batches of params->max_rhs that share one Krylov loop (one operator and
 * V-cycle launch per iteration for the whole batch, per-RHS scalars; a
 * converged RHS is frozen).  Stops each RHS when the true FP64
 * |b - A x| / |b| <= tol.  b = 0 gives x = 0.  info (host, may be NULL)
 * receives nrhs records.  Synchronises the stream.  MG_ERR_NOCONV when
 * maxiter iterations are exhausted. */
mg_status mg_solve(mg_handle* h, const void* b, void* x, int nrhs, double tol, int maxiter,
                   int solver, mg_solve_info* info);

/* D (dagger = 0) or D^dagger (dagger = 1) on nrhs fine vectors (Sec. 1).
 * precision MG_PREC_F64 (complex128) or MG_PREC_F32 (complex64). */
mg_status mg_apply_D(mg_handle* h, const void* in, void* out, int nrhs, int dagger, int precision);

/* A = D^dagger D on nrhs fine vectors, fused (one pass over memory). */
mg_status mg_apply_A(mg_handle* h, const void* in, void* out, int nrhs, int precision);

/* Coarse operator A_level (2 <= level <= nlevels) on nrhs level vectors
 * (Eq. Galerkin).  precision F64, F32 or BF16 (coarse blocks in bf16). */
mg_status mg_apply_coarse(mg_handle* h, int level, const void* in, void* out, int nrhs,
                          int precision);

/* Tensor-core kernel of the multi-right-hand-side BF16 coarse apply (Eq.
 * Galerkin at every coarse level of the FP32 V-cycle; 8 .. 64 right-hand
 * sides): 0 = tcgen05.mma with the accumulator in tensor memory (default;
 * coarse levels with 2Nv = 16 or 24 dof per site, the others use 1), 1 =
 * mma.sync (the earlier tensor-core path, kept for comparison).  Both
 * compute with the stored BF16 blocks and X carried as two BF16 parts, FP32
 * accumulation.  Process-wide; takes effect for launches (and CUDA graphs)
 * made after the call.  The tcgen05 kernel's completion waits are bounded: one
 * that runs out sets a process-wide flag, and the next mg_solve returns
 * MG_ERR_TIMEOUT and leaves its handle unusable.  MG_ERR_ARG for other
 * values. */
mg_status mg_set_coarse_tensor_kernel(int kind);

/* Restriction P^dagger from level `level` to level+1 (Sec. 2 step 2) and
 * prolongation P from level+1 to `level` (Sec. 2 step 4), 1 <= level < nlevels.
 * precision F64 or F32.  On a handle with smoothed aggregation, level 1 uses
 * P_s = (1 - omega A) P and P_s^dagger (then nrhs <= max_rhs). */
mg_status mg_restrict(mg_handle* h, int level, const void* fine_in, void* coarse_out, int nrhs,
                      int precision);
mg_status mg_prolong(mg_handle* h, int level, const void* coarse_in, void* fine_out, int nrhs,
                     int precision);

/* One V-cycle from the finest level (Sec. 2, five steps, recursive), on one
 * fine vector.  precision F64 (complex128) or F32 (complex64; the mixed
 * solver's preconditioner: FP32 vectors, BF16 coarse blocks, FP64 coarsest). */
mg_status mg_vcycle(mg_handle* h, const void* in, void* out, int precision);

/* Coarsest-level solve A_L x = b (FP64, complex128 level-L vectors): FP32
 * explicit inverse refined in FP64 to coarsest_tol, or, when the level has
 * more than coarsest_dense_max unknowns, FP64 CG on the coarsest stencil for
 * the iteration count fixed at set-up (the count at which a test vector
 * reaches coarsest_tol, times 1.25 plus 4). */
mg_status mg_coarsest_solve(mg_handle* h, const void* in, void* out);

/* The coarsest solve fixed at set-up (Sec. 2: exact solve on the coarsest
 * level).  *dense: 1 = FP32 explicit inverse refined in FP64, 0 = FP64 CG on
 * the coarsest stencil; *steps: FP64 refinement steps, or CG iterations, of
 * one coarsest solve; *test_residual: the largest relative residual the
 * set-up's test vectors (two seeded complex Gaussian vectors) reached with
 * that count (<= coarsest_tol).  mg_setup / mg_set_mass fail with
 * MG_ERR_NOCONV, and say what they reached, when a test vector does not reach
 * coarsest_tol within coarsest_refine_max refinement steps (the coarsest
 * operator's condition number is too close to 1/eps of FP32 for the dense
 * inverse: use a larger coarsest_tol or coarsest_dense_max = 0, the CG path)
 * or within 5000 CG iterations.  Any output pointer may be NULL; MG_ERR_ARG
 * when h has one level. */
mg_status mg_get_coarsest_info(const mg_handle* h, int* dense, int* steps, double* test_residual);

/* Dense coarsest level: *inner = FP64 refinement steps of the FP32 V-cycle's
 * coarsest solve, *reuses = re-masses of this handle that kept the previous
 * FP32 inverse (mg_params.coarsest_reuse).  Any output pointer may be NULL. */
mg_status mg_get_coarsest_reuse(const mg_handle* h, int* inner, int* reuses);

/* Smoothed aggregation of the first coarsening (mg_params.smooth_omega):
 * *omega the damping in use (0 when off) and *cond the condition number of
 * the level-2 operator at that omega as the search estimated it (power
 * iterations on A_2 and on its inverse; 0 when omega was given).  Any output
 * pointer may be NULL. */
mg_status mg_get_smoothing(const mg_handle* h, double* omega, double* cond);

/* Level geometry: extents and dof per site; Nv of the blocking below it
 * (0 on the coarsest).  Any output pointer may be NULL. */
mg_status mg_get_level(const mg_handle* h, int level, int* Lx, int* Lt, int* ndof, int* Nv);

/* Copy the block-orthonormal vectors of level l < nlevels into out:
 * device complex128 [Nv][Lt_l][Lx_l][n_l] (v_k on every block, both
 * chiralities; P e_{j,(c,k)} = Pi_c v_k restricted to S_j). */
mg_status mg_get_null_vectors(const mg_handle* h, int level, void* out);

/* Copy the FP64 coarse operator A_level (2 <= level <= nlevels) into out
 * (device complex128, layout above). */
mg_status mg_get_coarse_op(const mg_handle* h, int level, void* out);

/* Smoother and relaxation scalars of level l < nlevels, host doubles:
 * out4 = {c0, c1, lambda_max, omega_relax}; R = c0 + c1 A_l. */
mg_status mg_get_smoother(const mg_handle* h, int level, double* out4);

/* Block map of Sec. 3 computed by the device index functions the kernels use:
 * coarse[i] = (t / bt) * (Lx / bx) + x / bx, offset[i] = (t % bt) * bx + x % bx,
 * for i = x + Lx t.  Device int32 arrays of Lx * Lt entries.  stream may be NULL. */
mg_status mg_block_map(int Lx, int Lt, int bx, int bt, int32_t* coarse, int32_t* offset,
                       void* stream);

/* Kernel launches made by this library in this process so far (all handles). */
unsigned long long mg_kernel_launches(void);

/* Per-family device timing for roofline reporting.  When enabled, every call
 * of a family is bracketed by CUDA events on the handle's stream (adds a few
 * microseconds per call); mg_profile_read synchronises and returns the summed
 * device time and the number of calls since the last enable. */
typedef enum {
  MG_KF_FINE_A = 0,     /* fused A = D^dagger D on the fine lattice            */
  MG_KF_COARSE = 1,     /* coarse stencil apply in FP32 or BF16 weights        */
  MG_KF_TRANSFER = 2,   /* restriction and prolongation                        */
  MG_KF_COARSEST = 3,   /* coarsest solve (GEMV + FP64 refinement)             */
  MG_KF_INVERSE = 4,    /* coarsest dense inverse (Gauss-Jordan)               */
  MG_KF_GALERKIN = 5,   /* Galerkin coarse-operator build                      */
  MG_KF_FINE_A64 = 6,   /* A = D^dagger D on the fine lattice in FP64 (MG_KF_FINE_A
                           counts the FP32 applications)                        */
  MG_KF_DENSE = 7,      /* the tile kernel of the coarsest-level packed
                           Hermitian GEMV (part of MG_KF_COARSEST)              */
  MG_KF_GJ_UPDATE = 8,  /* the rank-64 tensor-core update kernel of the dense
                           inverse, one call per pivot block (part of
                           MG_KF_INVERSE)                                       */
  MG_KF_COARSE64 = 9,   /* coarse stencil apply in FP64                         */
  MG_KF_COUNT = 10
} mg_kernel_family;
mg_status mg_profile_enable(mg_handle* h, int on);
mg_status mg_profile_read(mg_handle* h, int family, double* total_ms, long long* calls);

/* Allocation-free variant of mg_apply_A (FP64, one right-hand side) that also
 * returns <x, A x>.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- code that records its work into a
 * CUDA graph under stream capture, where allocation is not allowed, or code
 * that runs under a fixed device-memory budget.  out = A in (complex128
 * [Lt][Lx][2], device) and *xAx (device double[2]: real, imaginary part of
 * <in, A in>, deterministic) are written with the same fused kernel as
 * mg_apply_A; its reduction scratch lives in a 10 KB array inside the library
 * (every GPU that loads the library keeps it until exit) instead of the
 * handle's workspace.  Maximum size: 608 thread blocks of the fused kernel,
 * counted as B = ceil(Lx/32) * ceil(Lt/8) when B >= 304, otherwise
 * ceil(Lx/16) * ceil(Lt/8) (so 155648 sites for lattices that are multiples of
 * 32 x 8, e.g. 608 x 256; 384 x 384 takes 576); larger lattices get
 * MG_ERR_ARG and a message with their block count.  The first call on a
 * device looks up the array's device address, with that device current (make
 * that call before any stream capture); the address is cached per device
 * ordinal for the life of the process's CUDA context.  Calls share the array
 * and leave their partial sums in it: calls whose kernels overlap on the GPU
 * race and must be ordered by the caller. */
mg_status mg_apply_A_dot_noalloc(mg_handle* h, const void* in, void* out, double* xAx);

/* Message of the last error on h (h == NULL: last mg_setup / mg_block_map
 * error of the calling thread). */
const char* mg_last_error(const mg_handle* h);

/* Frees everything owned by h; NULL is allowed.  Synchronises the stream. */
void mg_destroy(mg_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
