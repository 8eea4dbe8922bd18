/*
 * fe2.h -- C ABI of the GB300 RVE block of monolithic FE^2
 * (Hesch, Schmidt & Schuss, "Variational formulation and monolithic solution
 * of computational homogenization methods", arXiv 2312.12771).
 *
 * One RVE sits at each macro Gauss point (Dirac test basis, Section 3,
 * Eqs. (fluctVaria_dirac), (fluctSolution)).  For every RVE the library
 * assembles the micro Hessian blocks of Section 4 (Eqs. (discreteSys_K),
 * (discreteSys_D), (discreteSys_L)), reduces the periodic fluctuation DOFs by
 * the discrete null space of periodicity with one pinned corner (Section 2.2,
 * Eq. (Con)(iii); Section 5.2), factorises the condensed micro stiffness and
 * forms the Schur complement of Section 4.2, Eq. (solution2):
 *
 *   Cbar      = (K_MM - K_Mm K_mm^-1 K_mM) / |Omega|
 *   sigma_eff = (Pint - K_Mm K_mm^-1 r_m)  / |Omega|
 *   dw        = -(x_r + X_M : dFbar)        (update below Eq. (solution2))
 *
 * Conventions (all calls):
 *  - RVE = unit cell [0,1]^d, N^d equal elements (Q4 in 2D, Hex8 in 3D), N >= 3,
 *    element e = ex + N*ey (+N*N*ez); full 2^d Gauss quadrature.
 *  - Second-order tensors are row-major d x d (F_iJ, J fastest); tangents
 *    are d^2 x d^2 with Cbar[iJ][kL] = d sigma_iJ / d Fbar_kL.
 *  - Materials per RVE and phase: double[4] = (model, p1, p2, p3):
 *    FE2_MODEL_LINEAR (p1 = E, p2 = nu, plane strain in 2D, strain
 *    sym(F - I)); FE2_MODEL_NEOHOOKE (p1 = mu, p2 = kappa; energy
 *    mu/2 (F:F - 3) - mu ln J + kappa/2 (J-1)^2, Eq. (MR) with beta = 0);
 *    FE2_MODEL_MOONEY_RIVLIN (p1 = alpha, p2 = beta, p3 = kappa; energy
 *    alpha (F:F - 3) + beta (H:H - 3) + kappa/2 (J-1)^2 - 2 (alpha + 2 beta) ln J,
 *    Eq. (MR) with the f(J) of the Section 5.2 membrane; plane strain, 2D only,
 *    where H:H = F:F + J^2).
 *  - Pointers marked [device] are CUDA device pointers, borrowed for the
 *    duration of the work queued on the context's stream; [host] pointers are
 *    read before the call returns.  rve_ids are always [host].
 *  - Calls enqueue work on cfg.cuda_stream and return without synchronising
 *    unless stated.  A context is used by one host thread at a time.
 *  - Errors: every call returns an fe2_status and never aborts;
 *    fe2_last_error() gives a message.  Per-RVE numerical failures are
 *    reported in rve_status and do not fail the call.
 */
#ifndef FE2_H
#define FE2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe2_ctx fe2_ctx;

typedef enum {
    FE2_OK = 0,
    FE2_ERR_ARG = 1,      /* invalid argument (sizes, ids, pointers)            */
    FE2_ERR_CUDA = 2,     /* a CUDA runtime call failed                          */
    FE2_ERR_BUDGET = 3,   /* admission refused: the HBM budget would be exceeded */
    FE2_ERR_NOT_PD = 4,   /* per RVE: non-positive pivot in the factorisation    */
    FE2_ERR_NAN = 5,      /* per RVE: NaN/Inf in input or result                 */
    FE2_ERR_NO_CONV = 6,  /* per RVE: refinement did not reach the tolerance     */
    FE2_ERR_TIMEOUT = 7   /* a bounded device wait gave up                       */
} fe2_status;

enum { FE2_ELEM_Q4 = 0, FE2_ELEM_HEX8 = 1 };
enum { FE2_PREC_FP64 = 0, FE2_PREC_MIXED = 1 };
enum { FE2_MODEL_LINEAR = 0, FE2_MODEL_NEOHOOKE = 1, FE2_MODEL_MOONEY_RIVLIN = 2 };
/* Band factor (Section 4: K_mm factorised once per RVE and Newton iteration).
 * FE2_FACTOR_CUDA_CORE: shared-memory band Cholesky on the CUDA cores, two
 * RVEs per SM, panel phases (diagonal block, panel rows, trailing update)
 * separated by block barriers with a one-panel look-ahead (FP32 on the mixed
 * path, FP64 on the FP64 path).  FE2_FACTOR_CUDA_CORE_PIPELINED: the same
 * factorisation with the panel chain pipelined: warp 0 factors each 32 x 32
 * diagonal block and publishes it column by column (one mbarrier per column)
 * to the threads that solve the panel rows below it, while the other warps
 * take the previous panel's trailing update blocks from a shared counter
 * (2D bands with 32 + kd + d*d+1 <= 224; measured slower on GB300, kept as an
 * option).  FE2_FACTOR_TENSOR_CORE (mixed path): the dense trailing updates as
 * tcgen05 MMAs (3xTF32, fp32 accumulation in tensor memory); two RVEs per SM
 * (a window ring of kd columns, 256 tensor-memory columns each) for 2D bands
 * with kd >= 64 and kd + d*d+1 <= 256 whose layout fits two CTAs per SM, else
 * one RVE per SM for 2D bands with 32 + kd + d*d+1 <= 192 whose shared memory
 * fits; other bands take the CUDA-core kernel.  FE2_FACTOR_AUTO is the library's choice,
 * currently FE2_FACTOR_CUDA_CORE (measured fastest on GB300 for these bands).
 * 3D (Hex8) bands always take the wide-band kernel. */
enum { FE2_FACTOR_AUTO = 0, FE2_FACTOR_CUDA_CORE = 1, FE2_FACTOR_TENSOR_CORE = 2, FE2_FACTOR_CUDA_CORE_PIPELINED = 3 };
/* Macro interpolation of the fluctuation w~ (Section 3).  FE2_BASIS_DIRAC: Dirac
 * pulses at the macro Gauss points, one RVE per Gauss point (Eqs.
 * (fluctVaria_dirac), (fluctSolution)).  FE2_BASIS_CONST: piecewise constant
 * per macro element, one RVE per element whose micro residual and stiffness
 * are integrated over the element's nq = 4 macro Gauss points (Eqs.
 * (constSolution1), (constSolution2)); 2D only.  With FE2_BASIS_CONST every
 * per-RVE array below that has a Gauss-point dimension carries nq of them:
 * Fbar/dFbar [n][nq][d][d], sigma_eff and Pbar [n][nq][d*d],
 * Cbar [n][nq*d*d][nq*d*d] with Cbar[(q,iJ)][(q',kL)] = d sigma_{q,iJ} / d Fbar_{q',kL}. */
enum { FE2_BASIS_DIRAC = 0, FE2_BASIS_CONST = 1 };

typedef struct {
    int dim;                 /* 2 or 3                                            */
    int elem;                /* FE2_ELEM_Q4 (dim 2) or FE2_ELEM_HEX8 (dim 3)      */
    int precision;           /* FE2_PREC_FP64 or FE2_PREC_MIXED                   */
    size_t hbm_budget_bytes; /* device bytes the context may hold; 0 = no limit   */
    void* cuda_stream;       /* cudaStream_t the work is queued on; NULL = default */
    double refine_tol;       /* mixed path: accepted relative error estimate      */
    int max_refine;          /* mixed path: correction sweeps (>= 0), see below   */
    int factor_kernel;       /* FE2_FACTOR_AUTO, _CUDA_CORE, _TENSOR_CORE, _PIPELINED */
    int macro_basis;         /* FE2_BASIS_DIRAC or FE2_BASIS_CONST                */
} fe2_config;

/* Mixed-path accuracy (Section 4.2 with an FP32 factor): sigma_eff and Cbar
 * come from the Schur complement corrected with the FP64 residual R of the
 * FP32 solve, whose error is second order in the solve error.  With
 * max_refine >= 1 every RVE (Dirac basis) also gets one refinement step,
 * dX = (L L^T)^-1 R from the FP32 factor, and the second-order correction
 * Cbar = K_MM - K_Mm X - (X + dX)_M^T R_M (sigma_eff alike, X advanced to
 * X + dX): the remaining error is the FP32 solve's relative error times the
 * second-order term.  Each further sweep (up to max_refine in all) refines the
 * RVEs whose estimate still exceeds refine_tol (X += dX, new FP64 residual);
 * element RVEs take every sweep this way.  An RVE still above refine_tol after
 * the last sweep gets FE2_ERR_NO_CONV.  With max_refine = 0 only the
 * first-order correction runs; its error estimate can understate the error of
 * high-contrast RVEs by four orders of magnitude (measured on Neo-Hooke
 * inclusion RVEs of 32^2 and 48^2: errors up to 1e-7). */

/* Create a context on the current CUDA device.  Allocates nothing large. */
fe2_status fe2_create(const fe2_config* cfg, fe2_ctx** out);
/* Free every device and host resource of the context (synchronises). */
void fe2_destroy(fe2_ctx* ctx);
/* Last error message of the context (never NULL; "" when none). */
const char* fe2_last_error(const fe2_ctx* ctx);
/* Block until all work queued by the context has finished. */
fe2_status fe2_sync(fe2_ctx* ctx);

/* Device bytes one RVE of mesh size N holds while registered (persistent
 * state) and while in a condensation batch (transient workspace). */
size_t fe2_rve_bytes(const fe2_ctx* ctx, int N);

/*
 * Register nrve RVEs (setup step, Section 5.2: periodic nodal coupling and a
 * pinned corner).  N[nrve] [host] mesh sizes (>= 3, may differ per RVE);
 * phase [host] uint8 per element, RVEs concatenated; mat [host]
 * double[nrve][nphase][4]; rve_ids_out[nrve] [host] receives the ids.
 * The fluctuation w~ of each RVE starts at zero.  Returns FE2_ERR_BUDGET,
 * registering nothing, if the context's HBM budget would be exceeded, and
 * FE2_ERR_ARG, registering nothing, for N outside [3, 256], an unknown material
 * model (Mooney-Rivlin is 2D only), a phase index >= nphase, or a band too wide
 * for the solve kernels' shared memory (both paths take every 2D mesh up to
 * N = 62 and Hex8 RVEs up to 8^3).
 */
fe2_status fe2_rve_register(fe2_ctx* ctx, int nrve, const int* N, const uint8_t* phase,
                            int nphase, const double* mat, int* rve_ids_out);
/* Release RVEs and their device memory. */
fe2_status fe2_rve_release(fe2_ctx* ctx, int n, const int* rve_ids);

/*
 * RVEs whose device state comes and goes within the HBM budget (no counterpart
 * in the paper; the serving loop's admission, config 4).  fe2_rve_define takes
 * the arguments of fe2_rve_register (Dirac basis) but allocates nothing: the
 * definition (mesh size, phases, materials) stays on the host, w~ starts at
 * zero.  A defined RVE is resident while its persistent state occupies a
 * device slot; slots have one size (the persistent bytes of the largest RVE of
 * the first fe2_rve_define call; a later call with a larger RVE returns
 * FE2_ERR_ARG), come from slabs of up to 16 slots allocated within the budget,
 * and are recycled, not freed.  fe2_rve_admit makes RVEs resident, evicting
 * other defined RVEs by least recent use when no slot is free and no slab fits
 * (FE2_ERR_BUDGET if still none; synchronises).  fe2_rve_evict copies w~ of
 * idle RVEs to the host and frees their slots (synchronises).  Every other
 * call on a defined RVE that is not resident returns FE2_ERR_ARG, except
 * fe2_rve_set_w (kept on the host until admission) and fe2_rve_release.
 * fe2_rve_resident: 1 resident, 0 not, -1 unknown id.  The server admits
 * defined RVEs by itself (fe2_server_*).
 */
fe2_status fe2_rve_define(fe2_ctx* ctx, int nrve, const int* N, const uint8_t* phase, int nphase,
                          const double* mat, int* rve_ids_out);
fe2_status fe2_rve_admit(fe2_ctx* ctx, int n, const int* rve_ids);
fe2_status fe2_rve_evict(fe2_ctx* ctx, int n, const int* rve_ids);
int fe2_rve_resident(const fe2_ctx* ctx, int rve_id);

/*
 * S1 + S2 (Section 2.2 Eqs. (microdefo), (microGrad); Section 3 Eqs. (linSys3),
 * (linSys4)): at F~ = Fbar + grad w~ evaluate P~ and A = dP~/dF~ at every
 * micro Gauss point and integrate, per element, the rows of the element
 * Hessian k_e, the element residual f_e, the coupling k_eM and the element
 * parts of K_MM = int A and Pint = int P~.  Fbar [device] double[n][d][d].
 * Results stay in a context-owned element workspace until the next call.
 */
fe2_status fe2_micro_assemble(fe2_ctx* ctx, int n, const int* rve_ids, const double* Fbar);

/*
 * S3: reduce the element data of the last fe2_micro_assemble by the discrete
 * null space of periodicity with the pinned corner: K_mm = T^T K T,
 * r_m = T^T f, K_mM = T^T k_M; K_MM and Pint summed over elements.
 * rve_ids must be a subset of the last assembled batch.
 */
fe2_status fe2_nullspace_reduce(fe2_ctx* ctx, int n, const int* rve_ids);

/*
 * S4 - S6 (Section 4.2, Eq. (solution2)): factorise K_mm (band Cholesky in
 * the folded periodic ordering; FP64, or FP32 factor with FP64 residual
 * refinement and a residual-corrected Schur complement on the mixed path),
 * solve X_M = K_mm^-1 K_mM and x_r = K_mm^-1 r_m, and write
 *   sigma_eff [device] double[n][d*d],  Cbar [device] double[n][d^2][d^2],
 *   rve_status [device] int[n] (fe2_status per RVE),
 *   err_est [device] double[n]: estimated relative error of Cbar (may be NULL).
 * X_M and x_r stay resident for fe2_macro_step.
 */
fe2_status fe2_condense(fe2_ctx* ctx, int n, const int* rve_ids, double* sigma_eff, double* Cbar,
                        int* rve_status, double* err_est);

/*
 * Fused S1 - S6: the production path (assembly and periodic reduction in one
 * kernel, then condensation).  Same inputs/outputs as the three calls above.
 */
fe2_status fe2_rve_solve(fe2_ctx* ctx, int n, const int* rve_ids, const double* Fbar,
                         double* sigma_eff, double* Cbar, int* rve_status, double* err_est);

/*
 * S7 micro part (update below Section 4.2, Eq. (solution2)):
 * w~ <- w~ - (x_r + X_M : dFbar), with X_M, x_r of the last condensation
 * of each RVE (no new factorisation).  dFbar [device] double[n][d][d].
 */
fe2_status fe2_macro_step(fe2_ctx* ctx, int n, const int* rve_ids, const double* dFbar);

/*
 * Macro Q4 (dim 2) or Hex8 (dim 3) problem of Section 3, Eq. (linSys2),
 * solved with the condensed tangent of Section 4.2, Eq. (solution2):
 *   K = sum_b eta_b B_b^T Cbar_b B_b,   R = sum_b eta_b B_b^T s_b,
 * over the macro Gauss points b = 2^d e + q (q = qx + 2 qy [+ 4 qz], 2^d Gauss
 * points), with B_b dq = sum_A dq_A (x) grad N^A(X_b).  Dirichlet DOFs are held
 * at their prescribed positions; the free block (natural DOF order, half
 * bandwidth from the element couplings) is factorised on the device by a
 * blocked FP64 band Cholesky (32-column panels: diagonal block, panel rows,
 * trailing update as separate kernels).  The macro state (nodal positions q,
 * starting at X) is owned by the context.  Element RVEs (FE2_BASIS_CONST) are
 * 2D only.
 *
 * fe2_macro_setup [host]: nodes X[nnode][d], connectivity conn[nelem][2^d]
 * (local node a = ax + 2 ay [+ 4 az] on the reference square / cube, positive
 * Jacobian), fixed[d*nnode] (1 = prescribed DOF).  Returns FE2_ERR_ARG for an
 * inverted element.
 */
fe2_status fe2_macro_setup(fe2_ctx* ctx, int nnode, const double* X, int nelem, const int* conn,
                           const uint8_t* fixed);
/* Overwrite nodal positions from q_host [host] double[nnode][d]: every DOF, or
 * only those with which[t] != 0 when `which` [host] is not NULL (e.g. the
 * Dirichlet DOFs at the start of a load step).  Synchronises. */
fe2_status fe2_macro_set_positions(fe2_ctx* ctx, const double* q_host, const uint8_t* which);
/* FE2_BASIS_CONST: the weights of the nq macro Gauss points of each element
 * RVE, wq [host] double[n][nq] (eta_q / sum_q eta_q of its macro element, see
 * fe2_macro_gradients; they sum to 1).  Registration sets 1/nq.  Returns
 * FE2_ERR_ARG with the Dirac basis or for weights that are not positive. */
fe2_status fe2_rve_set_quad_weights(fe2_ctx* ctx, int n, const int* rve_ids, const double* wq);
/* Copy the current nodal positions to q_host [host] double[nnode][d].  Synchronises. */
fe2_status fe2_macro_get_positions(fe2_ctx* ctx, double* q_host);
/* Nodal external forces of the current load, fext_host [host] double[nnode][d]
 * (the surface-load term of Eq. (weakMech), e.g. the Section 5.2 membrane
 * traction scaled to the load step; NULL = no load).  fe2_macro_residual and
 * fe2_macro_solve then use R = (internal) - fext on the free DOFs.  Returns
 * FE2_ERR_NAN for a non-finite entry.  Synchronises. */
fe2_status fe2_macro_set_load(fe2_ctx* ctx, const double* fext_host);
/* The same surface load from a constant traction T [host] double[2] on the
 * polyline of macro boundary nodes nodes [host] int[n] (n >= 2, consecutive
 * nodes joined by straight bilinear element edges; 2D only), multiplied by
 * `scale` (the load-step factor k / n_l of Section 5.2): every edge of length l
 * gives T l scale / 2 to each of its two nodes (the consistent nodal forces of
 * the Neumann term of Eq. (weakMech) for linear edge shape functions).  It
 * replaces the current load.  FE2_ERR_ARG for a node out of range, a 3D
 * context or no macro problem; FE2_ERR_NAN for a non-finite T or scale.
 * Synchronises. */
fe2_status fe2_macro_set_edge_load(fe2_ctx* ctx, int n, const int* nodes, const double* T, double scale);
/* Fbar_b = sum_A q_A (x) grad N^A(X_b) into Fbar [device] double[2^d nelem][d][d];
 * eta [device] double[2^d nelem] receives the quadrature weights (may be NULL). */
fe2_status fe2_macro_gradients(fe2_ctx* ctx, double* Fbar, double* eta);
/* R_macro on the free DOFs for the stress s_b = stress [device]
 * double[2^d nelem][d][d] (Pbar for the equilibrium residual); rnorm [device]
 * double[1] = ||R_free||_2. */
fe2_status fe2_macro_residual(fe2_ctx* ctx, const double* stress, double* rnorm);
/* One monolithic macro update: assemble K from Cbar [device]
 * double[2^d nelem][d*d][d*d] (element RVEs: double[nelem][16][16]) and R from
 * sigma [device] (sigma_eff: condensed right-hand side), solve K dq = -R,
 * update q += dq and write dFbar [device] double[2^d nelem][d][d] = B_b dq,
 * rnorm [device] double[1] = ||R_free||, status [device] int[1] (may be NULL):
 * FE2_ERR_NOT_PD if the macro tangent had a non-positive pivot. */
fe2_status fe2_macro_solve(fe2_ctx* ctx, const double* sigma, const double* Cbar, double* dFbar, double* rnorm,
                           int* status);
/*
 * The same macro update in steps, for a macro Newton whose RVEs are spread
 * over several processes (one GPU each; paper Section 4.1: L is block diagonal
 * over the macro Gauss points, so only the macro system couples them).  Each
 * process assembles the contributions of its own Gauss points (the rows of
 * sigma / Cbar of the others set to zero), the processes sum K and R (e.g. one
 * NCCL all-reduce of each buffer), and every process solves the same reduced
 * system, so all keep the same nodal positions.
 *
 * fe2_macro_system_size [host out]: free DOFs nfree and half bandwidth kd.
 * fe2_macro_assemble: K [device] double[nfree][kd+1] (lower band, column-
 *   major, caller-owned; overwritten) and R [device] double[nfree] from sigma
 *   [device] double[2^d nelem][d][d] and Cbar (layout as fe2_macro_solve);
 *   Cbar = NULL assembles R only (K untouched, may be NULL).  R includes the
 *   current external load (-fext), so exactly one process should hold a load.
 * fe2_macro_norm: rnorm [device] double[1] = ||R||_2 of a (summed) R.
 * fe2_macro_solve_assembled: rnorm = ||R||, factorise K in place (blocked FP64
 *   band Cholesky, K becomes its factor, R the solution), dq = -K^-1 R,
 *   q += dq, dFbar [device] double[2^d nelem][d][d] = B_b dq, status as in
 *   fe2_macro_solve.  fe2_macro_assemble + fe2_macro_solve_assembled on one
 *   process equals fe2_macro_solve bit for bit.
 */
fe2_status fe2_macro_system_size(const fe2_ctx* ctx, int* nfree, int* kd);
fe2_status fe2_macro_assemble(fe2_ctx* ctx, const double* sigma, const double* Cbar, double* K, double* R);
fe2_status fe2_macro_norm(fe2_ctx* ctx, const double* R, double* rnorm);
fe2_status fe2_macro_solve_assembled(fe2_ctx* ctx, double* K, double* R, double* dFbar, double* rnorm, int* status);
/* Volume-averaged stress Pbar = Pint / |Omega| (Section 2.2, Eq. (averageStress))
 * of each RVE at its last assembly: Pbar [device] double[n][d*d]. */
fe2_status fe2_rve_average_stress(fe2_ctx* ctx, int n, const int* rve_ids, double* Pbar);
/* ||r_m||_2 of each RVE's reduced micro residual at its last assembly (the
 * micro part of the Newton stop test, Section 4): rnorm [device] double[n]. */
fe2_status fe2_rve_residual_norm(fe2_ctx* ctx, int n, const int* rve_ids, double* rnorm);

/*
 * Test/diagnostic export of one RVE in the natural periodic numbering
 * (node p = i + N j (+N^2 k), reduced DOF d*(p-1)+c):  what = 0: dense K_mm
 * [nm][nm] (2D only); 1: r_m [nm]; 2: K_mM [nm][d*d]; 3: w~ [nm]; 4: K_MM
 * [d^2][d^2] then Pint [d^2].  host_out [host] must hold the stated doubles.
 * Synchronises the stream.
 */
fe2_status fe2_rve_export(fe2_ctx* ctx, int rve_id, int what, double* host_out);
/* Copy w~ of n RVEs (folded order) to row k of buf [device] double[n][ld]
 * (to_buf = 1) or back (to_buf = 0): a device-side snapshot of the micro
 * states, e.g. the classical scheme's restart of every inner Newton from the
 * last converged load step (Section 4.1; the reading of Table 2).  ld >= the
 * largest n_m. */
fe2_status fe2_rve_w_copy(fe2_ctx* ctx, int n, const int* rve_ids, double* buf, int ld, int to_buf);
/* Set w~ of one RVE from the natural numbering ([host] double[nm]). */
fe2_status fe2_rve_set_w(fe2_ctx* ctx, int rve_id, const double* host_w);

/*
 * Fused RVE solve that allocates nothing (the paper has no counterpart: this is
 * an integration entry point).  For callers that cannot call cudaMalloc /
 * cudaFree: code running inside another framework's memory pool or a plugin
 * host that owns the device allocator, or real-time loops that must not touch
 * the allocator.  Same computation as fe2_rve_solve on the mixed path (FP32
 * band factor, FP64 residual, residual-corrected Schur complement, no
 * refinement sweeps, rve_status FE2_ERR_NO_CONV when the error estimate
 * exceeds 1e-10), for n RVEs of one mesh size N (2D Q4, zero fluctuation w~).
 *
 * Inputs [device]: phase uint8[n][N*N], mat double[n][nphase][4],
 * Fbar double[n][2][2].  Outputs [device]: sigma_eff double[n][4],
 * Cbar double[n][4][4], rve_status int[n], err_est double[n] (may be NULL).
 * Work is queued on cuda_stream (NULL = default stream); no context is used.
 * The inputs are checked on the device: an RVE with a phase index >= nphase,
 * an unknown material model or a non-finite material parameter gets
 * rve_status FE2_ERR_ARG (a non-finite Fbar FE2_ERR_NAN) and meaningless
 * outputs, and no kernel reads beyond its rows of phase and mat.
 *
 * All intermediate data live in one library-owned __device__ array of
 * FE2_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits.  Limits: N >= 3, 1 <= nphase <= 8, and the n RVEs
 * must fit the array (1.69 MB per RVE at N = 32, i.e. 39 RVEs; 0.29 MB at
 * N = 16, 230 RVEs); larger requests return FE2_ERR_BUDGET without running anything.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; until one call on the
 * device has passed it, a call also waits for its stream and reads the set-up
 * descriptors back to check them (FE2_ERR_CUDA if they are not as written), so
 * make the first call on each device before any stream capture.  Every call
 * reuses the same array and leaves the previous call's data in it: calls that
 * overlap on the GPU (other streams, other host threads) race and corrupt each
 * other -- serialise them.
 */
#define FE2_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
fe2_status fe2_rve_solve_noalloc(int N, int n, int nphase, const uint8_t* phase, const double* mat,
                                 const double* Fbar, double* sigma_eff, double* Cbar, int* rve_status,
                                 double* err_est, void* cuda_stream);
/* Reason of the last failed fe2_rve_solve_noalloc call on any thread ("" after
 * a call that succeeded); the string is owned by the library. */
const char* fe2_noalloc_last_error(void);

/*
 * Serving: continuous batching of RVE solve requests (S1 - S6 per request) as
 * macro Newton iterations emit them.  RVE state stays resident in the context
 * between requests.  Requests may name defined RVEs that are not resident
 * (fe2_rve_define): a batch admits them as device memory allows within the
 * context's HBM budget (the lanes' buffers and workspaces count against it),
 * evicting idle defined RVEs (not in flight, least recently served first,
 * w~ kept on the host); a request that cannot be admitted stays queued until
 * memory frees up.  The server runs `nlanes` execution lanes, each with its
 * own CUDA stream, factorisation workspace, pinned staging and completion
 * event: a batch formed while another runs is launched at once and overlaps it
 * on the device.  A batch takes up to max_batch queued requests of one mesh
 * size (that of the oldest request; any sizes with fe2_server_mixed_sizes)
 * whose RVE is not already in flight, in submission order.  Results are bit-identical to solving the RVE alone.
 *
 * fe2_server_submit: queue n requests (rve_ids [host], Fbar [host]
 *   double[n][d][d]); tickets [host] long long[n] receives their ids.
 * fe2_server_pump: harvest finished lanes and launch batches on idle lanes;
 *   returns immediately (busy_lanes [host], may be NULL).  Call it repeatedly.
 * fe2_server_take: move up to max finished results to the caller ([host]
 *   arrays: tickets, sigma [max][d*d], Cbar [max][d^4], status, latency_ms
 *   = completion - submission time); returns the number taken (-1 on error).
 * fe2_server_pending: requests queued or in flight.
 * fe2_server_use_graphs: a lane captures its launch sequence (input copies,
 *   S1 - S6 kernels, result copies) as a CUDA graph once per batch shape
 *   (batch size and the batch's maximum mesh sizes) and replays it for later
 *   batches of that shape; on by default, enable = 0 launches every kernel
 *   from the host instead.  The results are the same either way.
 * fe2_server_graph_stats: captures and replays so far ([host], may be NULL).
 * fe2_server_mixed_sizes: enable = 1 lets a batch take the oldest queued
 *   requests whatever their mesh sizes (one launch of uneven RVEs, shared
 *   memory and workspace sized for the largest); default 0 (one size per batch).
 * fe2_server_bucket: with graphs on, round each batch down to a power of two
 *   or 1.5 times one (the rest stay at the head of the queue) so that
 *   captured graphs are replayed (default on).
 * fe2_server_memory_stats: defined RVEs admitted and evicted so far, requests
 *   passed over for lack of memory, device bytes held against the budget
 *   ([host], may be NULL).
 */
typedef struct fe2_server fe2_server;
fe2_status fe2_server_create(fe2_ctx* ctx, int max_batch, int nlanes, fe2_server** out);
void fe2_server_destroy(fe2_server* srv);
fe2_status fe2_server_submit(fe2_server* srv, int n, const int* rve_ids, const double* Fbar, long long* tickets);
fe2_status fe2_server_pump(fe2_server* srv, int* busy_lanes);
int fe2_server_take(fe2_server* srv, int max, long long* tickets, double* sigma, double* Cbar, int* status,
                    double* latency_ms);
int fe2_server_pending(const fe2_server* srv);
fe2_status fe2_server_use_graphs(fe2_server* srv, int enable);
fe2_status fe2_server_graph_stats(const fe2_server* srv, long long* captures, long long* replays);
fe2_status fe2_server_bucket(fe2_server* srv, int enable);
fe2_status fe2_server_mixed_sizes(fe2_server* srv, int enable);
fe2_status fe2_server_memory_stats(const fe2_server* srv, long long* admitted, long long* evicted,
                                   long long* deferred, size_t* device_bytes);

/*
 * Self-test of the bounded device waits used by the TMA streams of the solve
 * kernels (no counterpart in the paper): one kernel waits on an mbarrier that
 * nothing arrives on; after about a second (2^31 SM cycles) the wait gives up
 * and status [device] int[1] receives FE2_ERR_TIMEOUT.  The context stays
 * usable.  Failure detection is exercised this way without faulting the GPU.
 */
fe2_status fe2_selftest_wait_timeout(fe2_ctx* ctx, int* status);

/* Number of kernel launches the context has issued so far. */
long long fe2_launch_count(const fe2_ctx* ctx);

/*
 * Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch.  fe2_profile(ctx, 1) enables it and clears the totals;
 * fe2_profile(ctx, 0) disables it.  fe2_profile_read synchronises the stream
 * and writes, for up to max kernels, the name (names [host] char[max][48],
 * NUL-terminated), the summed milliseconds (ms [host]) and the launch count
 * (count [host]); it returns the number of kernels (or -1 on error).
 */
fe2_status fe2_profile(fe2_ctx* ctx, int enable);
int fe2_profile_read(fe2_ctx* ctx, int max, char* names, double* ms, long long* count);

#ifdef __cplusplus
}
#endif
#endif /* FE2_H */
