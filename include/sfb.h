/*
 * sfb.h - C ABI of the GB300 stochastic multiscale flux basis library.
 *
 * The library computes, on one GPU, the hot path of Method S3 of
 * Ambartsumyan, Khattatov, Wang, Yotov, "Stochastic multiscale flux basis for
 * Stokes-Darcy flows" (arXiv 1802.06263, Section 5.4): for every Darcy
 * subdomain and every local realization of its KL region the log-normal
 * permeability (Section 2.1, Eq. 2.13), the lowest-order RT / cell-centred
 * operator, its block-tridiagonal factorization and the multiscale flux basis
 * (Section 5.3); then the interface problem Eq. 5.10 for a batch of global
 * collocation points (Section 5.4, Steps 3-5) and the moments (Step 6,
 * Eq. 2.1).
 *
 * Conventions shared by every entry point:
 *  - The status is the return value; no C++ exception crosses the ABI.
 *    sfb_last_error() returns the message of the last failing call.
 *  - Descriptors passed in are deep-copied; the caller keeps ownership of
 *    every pointer it passes.
 *  - Device memory comes only from the caller: sfb_workspace_size() says how
 *    much, sfb_set_workspace() hands it over (the caller frees it after
 *    sfb_destroy). The one exception is the allocation-free entry point
 *    sfb_build_basis_item_noalloc, whose scratch is a static array of the
 *    library. All device work is ordered on the stream given to
 *    sfb_create() / sfb_set_stream(); entry points that return host data
 *    synchronise that stream.
 *  - "host or device" arguments are detected with cudaPointerGetAttributes;
 *    host buffers are copied inside the call.
 *  - Call order: sfb_create; sfb_kl_setup (or sfb_kl_setup_regions);
 *    sfb_collocation_setup; sfb_workspace_size and sfb_set_workspace; then,
 *    per basis build, sfb_build_stochastic_basis; per batch of points,
 *    sfb_interface_solve_batch (after sfb_moments_reset for a new
 *    accumulation); sfb_moments at any time after a solve; sfb_destroy. A
 *    call out of order returns SFB_ERR_STATE.
 *  - Geometry: the Darcy box is tiled by px x py subdomains (s = iy*px + ix,
 *    bottom row first); one Stokes subdomain sits on top. Global mortar DOFs:
 *    Stokes-Darcy edges left to right, then vertical Darcy-Darcy edges row by
 *    row, then horizontal Darcy-Darcy edges row by row; inside an interface
 *    element by element along increasing coordinate, then local node. A
 *    subdomain's local mortar DOFs are its global DOFs in increasing order.
 */
#ifndef SFB_H
#define SFB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SFB_OK = 0,
  SFB_ERR_ARG = 1,            /* bad argument or descriptor                     */
  SFB_ERR_STATE = 2,          /* call out of order (e.g. moments before solve)  */
  SFB_ERR_CUDA = 3,           /* a CUDA runtime call failed                     */
  SFB_ERR_WORKSPACE = 4,      /* no workspace set, or it is too small           */
  SFB_ERR_NONFINITE = 5,      /* non-finite permeability or solution            */
  SFB_ERR_NOT_CONVERGED = 6,  /* some point did not converge (outputs filled)   */
  SFB_ERR_NOT_SPD = 7,        /* a non-positive pivot in a factorization        */
  SFB_ERR_UNSUPPORTED = 8,    /* size beyond a compiled limit                   */
  SFB_ERR_TIMEOUT = 9         /* a bounded wait inside a kernel gave up         */
} sfb_status;

typedef enum {
  SFB_FP64 = 0,          /* factor and solve in FP64                                  */
  SFB_MIXED = 1,         /* FP32 factor/solves with diagonal scaling, refined by FP64 */
                         /* residuals of the 5-point operator                          */
  SFB_FP32_NOREFINE = 2, /* FP32 factor/solve only: diagnostics of the unrefined error */
  SFB_FACTOR_FP64 = 3    /* Method S1's set-up (Section 5.2): the FP64 block factor of  */
                         /* every item and its particular solution, so g; no flux     */
                         /* basis (Phi) is formed. Needs an SFB_FP64 workspace; only  */
                         /* SFB_CG_DTN solves from it.                                */
} sfb_precision;

/* Interface Krylov solver (Section 5.4 Step 5, reading of Eq. 5.10 as an SPD
 * coefficient system).
 * SFB_CG:       CG in FP64 throughout.
 * SFB_CG_MIXED: CG whose products S p use the bases rounded to FP32, with FP64
 *               inner products, updates and iterates. The recursive residual
 *               is replaced by the FP64 residual g - S lambda whenever it has
 *               dropped by cg_replace_ratio since the last replacement, and
 *               before a point is declared converged, so the stopping test
 *               ||g - S lambda|| <= rtol ||g|| holds in FP64 (residual
 *               replacement in the manner of reliable-update Krylov methods).
 *               Not in the paper: an operator-precision choice for GPUs whose
 *               FP64 rate is a small fraction of FP32.
 * SFB_GMRES:    restarted GMRES(m) in FP64 (m = option "gmres_restart",
 *               default 30), right-preconditioned with the CG's
 *               preconditioner (option "cg_precond", applied in FP64) so that
 *               its residual is the unpreconditioned one; classical
 *               Gram-Schmidt with one re-orthogonalization pass, Givens
 *               rotations; a cycle ends when the least-squares residual
 *               reaches rtol ||g|| or after m steps, and a point is accepted
 *               only on its FP64 true residual ||g - S lambda|| <= rtol ||g||
 *               (otherwise the next cycle starts from it). The iteration
 *               count is the number of Arnoldi steps.
 * SFB_GMRES_MIXED: the same GMRES with the Arnoldi products S p on the bases
 *               rounded to FP32 and the Arnoldi process itself in FP32 (the
 *               Krylov basis stored in FP32, the Gram-Schmidt sums and
 *               updates on the FP32 pipe, the preconditioner applied in
 *               FP32); the Hessenberg matrix, the rotations, the iterate and
 *               its update stay FP64. A cycle also ends once it has reduced
 *               its initial residual by 1e-5, and every cycle starts from,
 *               and every point is accepted on, the FP64 true residual:
 *               restarted GMRES as the inner solver of FP64 iterative
 *               refinement. Not in the paper, like SFB_CG_MIXED.
 * SFB_CG_DTN:   Method S1 (Section 5.2): unpreconditioned CG in FP64 whose
 *               product S p applies every Darcy subdomain's Dirichlet-to-
 *               Neumann map by one subdomain solve per iteration (Eqs. 5.5-
 *               5.6 with the data R_i p, then -<u.n, xi> on its mortar DOFs),
 *               with the point's own block factor from an SFB_FP64 or
 *               SFB_FACTOR_FP64 build; the Stokes subdomain, whose operator
 *               is the same for every point, is applied by its basis. The
 *               Darcy moments then come from one more subdomain solve per
 *               point (the recovery of Section 5.2, Eqs. 5.7-5.8). Per Darcy
 *               subdomain the point's solves number its iterations plus two
 *               (the right-hand side, folded into the build, and the
 *               recovery). */
typedef enum {
  SFB_CG = 0,
  SFB_CG_MIXED = 1,
  SFB_GMRES = 2,
  SFB_GMRES_MIXED = 3,
  SFB_CG_DTN = 4
} sfb_krylov;

typedef enum {
  SFB_FIELD_DARCY_P = 0,     /* cell pressures, subdomain by subdomain, c = iy*nx+ix    */
  SFB_FIELD_DARCY_FLUX = 1,  /* per subdomain: x-face normal velocities (ny x (nx+1)), */
                             /* then y-face ones ((ny+1) x nx), +x / +y orientation    */
  SFB_FIELD_STOKES_U = 2,    /* P2 nodes: all u_x then all u_y, node j*(2Sx+1)+i       */
  SFB_FIELD_STOKES_P = 3     /* P1 vertices J*(Sx+1)+I                                 */
} sfb_field;

/* Problem geometry and data (Section 3.1 decomposition, Section 6 set-up). */
typedef struct {
  double darcy_box[4];        /* x0, x1, y0, y1                                   */
  double stokes_box[4];       /* x0, x1, y1, y2 (same x extent, directly above)   */
  int32_t px, py;             /* Darcy subdomain array                            */
  const int32_t* darcy_nx;    /* [px*py] cells in x                               */
  const int32_t* darcy_ny;    /* [px*py] cells in y                               */
  int32_t stokes_sx, stokes_sy;
  int32_t mortar_degree;      /* 1 or 2, discontinuous                            */
  const int32_t* mortar_sd;   /* [px] elements on each Stokes-Darcy edge          */
  const int32_t* mortar_dd_v; /* [py*(px-1)] vertical Darcy-Darcy edges           */
  const int32_t* mortar_dd_h; /* [(py-1)*px] horizontal Darcy-Darcy edges         */
  double nu_s, nu_d, alpha;   /* viscosities, BJS friction (Eqs. 2.2, 2.5, 2.10)  */
  double u_in;                /* peak of the parabolic Stokes inflow              */
  double bottom_pressure;     /* Dirichlet pressure on the Darcy bottom           */
  const double* source;       /* [px*py] constant q_d per subdomain, or NULL      */
} sfb_problem;

/* One KL region, covariance Eq. 6.1 on its rectangle (sfb_kl_setup: one per
 * Darcy subdomain, on the subdomain; sfb_kl_setup_regions: on given rectangles). */
typedef struct {
  double sigma2;              /* multiplies the kernel (the variance of Y)         */
  double eta1, eta2;          /* correlation lengths                               */
  double mean_y;              /* E[Y]                                              */
  int32_t n_term;             /* kept modes: the n_term largest products           */
  int32_t n_modes_x;          /* > 0 with n_modes_y > 0: keep instead the tensor  */
  int32_t n_modes_y;          /* set of the n_modes_x largest 1-D modes in x      */
                              /* times the n_modes_y largest in y (the paper's    */
                              /* "N_term = 2 x 1" form, Section 6.1); n_term must */
                              /* equal their product. Modes are ordered by        */
                              /* decreasing eigenvalue, ties by (a + b, a). Both  */
                              /* 0: the n_term largest products                   */
} sfb_kl_region;

/* Collocation (Section 4): tensor grid of m-point rules, or the Smolyak
 * combination formula of level lmax with 1-D rule sizes rule[p]
 * (n_rule == 0: the paper's 2^(p+1)-1). local_tensor = 1 builds every
 * region's basis on the full local tensor grid of the largest 1-D rule (of
 * the region's own rules for an anisotropic tensor grid); 0 on the distinct
 * projections of the global grid (Method S3, Section 5.4); 2 on the
 * projection of every global point, repeats kept, so that every point gets
 * its own basis items (Method S2, Section 5.3: a multiscale flux basis per
 * global point, no reuse). m_dim (tensor only, nullable, host): the
 * anisotropic tensor rule of Section 4.1, m_dim[kappa] points in global
 * stochastic dimension kappa (sum of n_term entries, regions in order, each
 * in [1, 32]); NULL: m points in every dimension. */
typedef struct {
  int32_t kind;               /* 0 tensor, 1 Smolyak */
  int32_t m;
  int32_t lmax;
  int32_t n_rule;
  const int32_t* rule;
  int32_t local_tensor;
  const int32_t* m_dim;
} sfb_collocation;

typedef struct {
  int64_t n_items;            /* (subdomain, local realization) pairs            */
  int64_t n_flux_responses;   /* sum over items of the subdomain's mortar DOFs    */
  int32_t max_refine_steps;   /* mixed form: largest refinement count             */
  int32_t n_not_converged;    /* mixed form: items that stopped above tolerance   */
  double max_rel_residual;    /* final ||B - A X||_F / ||B||_F over items         */
  double max_first_correction;/* mixed form: max ||dX_1||_F / ||X||_F: the        */
                              /* relative error of the unrefined FP32 solve       */
  double max_error_estimate;  /* mixed form: max predicted relative error of X    */
                              /* from the contraction of successive corrections   */
  double ms;                  /* device time of the build (CUDA events)           */
  double phase_cycles[16];    /* mean SM cycles per item in: permeability and     */
                              /* assembly, factorization, forward sweeps,         */
                              /* backward sweeps (clock64 in the kernel); then    */
                              /* sub-phases of the row steps up to each barrier:  */
                              /* factor [4] row set-up [5] block inversion [6]    */
                              /* G store and right-hand side [7] product;         */
                              /* forward [8] set-up [12] residual (thread 0's     */
                              /* loop) [9] G and store waits [10] product;        */
                              /* backward [11] set-up and copies issued [13] z    */
                              /* and G waits [14] product [15] X update with the  */
                              /* next row's product input                         */
  double kernel_ms;           /* device time of the basis kernel alone            */
  double flops_fp32;          /* algorithmic flops of the build by precision, per */
  double flops_fp64;          /* item: factor (7/3) nx^3 ny (block Cholesky       */
                              /* count), each multi-RHS solve 6 nx^2 ny (R+1),    */
                              /* each FP64 refinement pass 11 nx ny (R+1)         */
                              /* (5-point residual and update). FP64 form: all in */
                              /* flops_fp64; mixed: factor and 1 + n_refine       */
                              /* solves in flops_fp32, the passes in flops_fp64   */
  int32_t launch_shape[2];    /* launch shape of the basis kernel per size class: */
                              /* [0] grids wider than 64 cells, [1] the rest     */
                              /* (sfb_basis_launch_shape); -1: class is empty     */
  int32_t graph;              /* 1: the launches of all size classes ran as one   */
                              /* replayed CUDA graph                              */
  int32_t persistent;         /* 1: every item of both size classes ran in one    */
                              /* persistent launch (factor tasks, then chunk      */
                              /* tasks; launch_shape then gives the per-class     */
                              /* choices it was timed against)                    */
  double tune_ms[2][4];       /* autotuner, per size class and launch shape: the  */
                              /* shorter of two timed launches of the class's     */
                              /* items (ms); 0: not timed                         */
  double mean_refine_steps;   /* mixed form: refinement passes, mean over items   */
} sfb_basis_stats;

typedef struct sfb_ctx sfb_ctx;

/* Creates a context for one problem on the current CUDA device; stream is a
 * cudaStream_t (NULL = legacy default stream). Copies the descriptor and
 * assembles the host-side geometry (interfaces, mortar DOF maps, face
 * projections of Section 5.2 step 1). It loads the library's device module on
 * the current device, which reserves the static array of
 * sfb_build_basis_item_noalloc there (a caller that reserves its own device
 * memory pool should create its contexts first); no other device memory is
 * touched. Without a usable device this step is skipped. */
sfb_status sfb_create(const sfb_problem* prob, void* stream, sfb_ctx** out);
void sfb_destroy(sfb_ctx* ctx);
const char* sfb_last_error(const sfb_ctx* ctx);
sfb_status sfb_set_stream(sfb_ctx* ctx, void* stream);

/* Sizes of the problem: total mortar DOFs, Darcy subdomains, the mortar DOF
 * count of a subdomain (sub = -1: the Stokes subdomain), and field lengths. */
sfb_status sfb_sizes(const sfb_ctx* ctx, int64_t* n_lambda, int32_t* n_darcy);
sfb_status sfb_subdomain_dofs(const sfb_ctx* ctx, int32_t sub, int32_t* n_dof,
                              int64_t* global_dofs /* nullable [n_dof] */);
sfb_status sfb_field_size(const sfb_ctx* ctx, int32_t field, int64_t* n);

/* KL eigenpairs of Eq. 2.11 for the covariance Eq. 6.1 of every region (one
 * per Darcy subdomain, in subdomain order), from the 1-D transcendental
 * equations of the exponential kernel. eigvals_out (nullable, host) receives
 * sum(n_term) eigenvalues, region by region, in decreasing order. */
sfb_status sfb_kl_setup(sfb_ctx* ctx, const sfb_kl_region* regions, int32_t n_regions,
                        double* eigvals_out);

/* The same on KL regions that may each cover several Darcy subdomains
 * (Section 2.1: the Darcy region is split into statistically independent KL
 * regions, each a union of subdomains; the paper's Case 1, Section 6.1, has
 * two regions of two subdomains each). Region r is regions[r] on the
 * rectangle rects[4r .. 4r+3] = (x0, x1, y0, y1); region_of[s] (length: the
 * Darcy subdomain count) is subdomain s's region, and the subdomain must lie
 * inside it. Every region needs at least one subdomain. The modes are those
 * of the region's rectangle, evaluated at each subdomain's cell centres in
 * the region's centred coordinates. Region r's stochastic dimensions follow
 * those of regions 0..r-1, and all subdomains of a region share its local
 * realizations. eigvals_out (nullable, host) receives sum(n_term) eigenvalues,
 * region by region. SFB_ERR_ARG on an empty region, a subdomain outside its
 * region or a bad region. sfb_kl_setup is this call with one region per
 * subdomain on the subdomain's own rectangle. All arrays are host memory. */
sfb_status sfb_kl_setup_regions(sfb_ctx* ctx, const sfb_kl_region* regions, int32_t n_regions,
                                const double* rects, const int32_t* region_of, double* eigvals_out);

/* Global grid (Section 4.1 / 4.2) and every region's local realizations
 * (Section 5.4 Steps 1-2). n_pts_out receives the global point count. */
sfb_status sfb_collocation_setup(sfb_ctx* ctx, const sfb_collocation* spec, int64_t* n_pts_out);
/* Copies the global grid to host buffers y_out [n_pts x n_dim] and w_out [n_pts]. */
sfb_status sfb_collocation_points(const sfb_ctx* ctx, double* y_out, double* w_out);
/* Read-back of the KL tables that the basis kernel evaluates for Darcy
 * subdomain `sub` (set-up data of Eq. 2.13, no realization): sqrt_lambda
 * [n_term], and the 1-D eigenfunction factors at the subdomain's cell
 * centres, fx [n_term x nx] and fy [n_term x ny], so that mode j at cell
 * (ix, iy) is fx[j][ix] * fy[j][iy]. Host buffers, each nullable.
 * SFB_ERR_STATE before sfb_kl_setup. */
sfb_status sfb_kl_tables(const sfb_ctx* ctx, int32_t sub, double* sqrt_lambda, double* fx, double* fy);

/* Local realization count and coordinates [n_local x n_term] of the KL region
 * of Darcy subdomain `region` (its own region unless sfb_kl_setup_regions
 * gave it a shared one; the items of the subdomain are these realizations). */
sfb_status sfb_local_points(const sfb_ctx* ctx, int32_t region, int32_t* n_local, double* y_out);

/* Device bytes needed for precision `prec` and batches of up to max_pts
 * points, and the hand-over of that memory (256-byte aligned). A KL or
 * collocation set-up call made after sfb_set_workspace outdates the
 * workspace's layout and tables: sfb_build_stochastic_basis then returns
 * SFB_ERR_STATE until sfb_workspace_size and sfb_set_workspace run again. */
sfb_status sfb_workspace_size(const sfb_ctx* ctx, int32_t prec, int64_t max_pts, size_t* bytes);
sfb_status sfb_set_workspace(sfb_ctx* ctx, void* dev_ptr, size_t bytes);

/* Section 5.4 pre-computation loop for every (Darcy subdomain, local
 * realization) item: permeability, assembly, block-tridiagonal
 * factorization, R+1 right-hand sides (R mortar DOFs plus the particular
 * problem Eqs. 5.7-5.8), and the flux basis Phi[l][j] = -<u*(xi_j).n, xi_l>
 * with g[l] = <u_bar.n, xi_l>; also the deterministic Stokes basis (Section
 * 5.4: N_real = 1 for Stokes subdomains). stats_out is nullable.
 * prec = SFB_FACTOR_FP64 (Method S1, Section 5.2) stops after the FP64 factor
 * and the particular solution: g is formed, Phi and the mortar responses are
 * not (no autotuning and no captured graph: one plain launch per size class);
 * SFB_ERR_WORKSPACE unless the workspace was sized for SFB_FP64. */
sfb_status sfb_build_stochastic_basis(sfb_ctx* ctx, int32_t prec, sfb_basis_stats* stats_out);

/* Launch shapes of the basis kernel (no counterpart in the paper: how the
 * items of Section 5.4 Steps 1-2 map onto the GPU). The items fall into two
 * size classes, grids more than 64 cells wide (wide = 1) and the rest; each
 * class is one launch (a pipeline of launches for a split shape), the two
 * classes run concurrently. prec selects the factor precision (SFB_FP64: one
 * narrow and two wide shapes; SFB_MIXED, SFB_FP32_NOREFINE: four narrow and
 * three wide). Writes the shape's threads per CTA, the CTAs per SM its
 * register budget is compiled for, its number of shared-memory G_b buffers
 * (2: the next block row's inverse is prefetched), whether it runs the
 * block-row products on the tensor cores (tcgen05 = 1: SFB_MIXED /
 * SFB_FP32_NOREFINE narrow shape 2; tcgen05.mma kind::tf32 with every operand
 * split into two TF32 parts and FP32 accumulation, the block inverses fed by
 * TMA tensor copies), and whether it is split (split = 1: narrow shape 3 and
 * wide shape 2 of the FP32 factor). A split shape factors every item in one
 * launch (narrow class: 128-thread CTAs, wide class: 256) and solves and
 * refines every chunk of at most 24 of an item's right-hand sides in a CTA
 * of its own, in a second launch; option "basis_pipe_groups" splits the
 * items into groups whose chunk launches follow their own factor launch on a
 * second stream.
 * The other outputs describe the solve launch. Pointers are host memory and
 * nullable. SFB_ERR_ARG for a shape that the precision and class do not
 * have. By default the first build of each precision times every shape of
 * each class on that class's own items and keeps the fastest (option
 * "basis_autotune"). */
sfb_status sfb_basis_launch_shape(int32_t prec, int32_t wide, int32_t shape, int32_t* threads,
                                  int32_t* ctas_per_sm, int32_t* g_buffers, int32_t* tcgen05,
                                  int32_t* split);

/* Read-back of one stored basis item (host or device buffers): phi [R x R]
 * row-major, g [R], x [(R+1) x n_cells] (pressure responses, column j is the
 * response to xi_j, column R the particular solution; nullable). sub = -1 and
 * k = 0 return the Stokes basis (x must be NULL). After an SFB_FACTOR_FP64
 * build a Darcy item has g and the particular solution (column R of x) only:
 * phi must be NULL and the response columns of x are left unwritten. */
sfb_status sfb_get_basis(sfb_ctx* ctx, int32_t sub, int32_t k, double* phi, double* g, double* x);

/* Section 5.4 Steps 3-6 for a batch of global points y [n_pts x n_dim] with
 * weights w [n_pts] (host or device): local index conversion, CG on
 * S^l = sum_i R_i^T Phi_i^{k_i(l)} R_i (Eq. 5.10) from zero until
 * ||r|| <= rtol ||g||, recovery and accumulation of the moments. Outputs
 * (nullable, host or device): lambda_out [n_pts x n_lambda], iters_out
 * [n_pts] (negative: not converged). Returns SFB_ERR_NOT_CONVERGED with all
 * outputs filled if a point did not converge within max_it. An empty batch
 * (n_pts = 0, y and w may be NULL) returns SFB_OK and changes nothing.
 * krylov = SFB_CG_DTN (Method S1) needs the block factors of an SFB_FP64 or
 * SFB_FACTOR_FP64 build, every other solver the flux basis of an SFB_FP64,
 * SFB_MIXED or SFB_FP32_NOREFINE build (SFB_ERR_STATE otherwise). */
sfb_status sfb_interface_solve_batch(sfb_ctx* ctx, const double* y, const double* w, int64_t n_pts,
                                     int32_t krylov, double rtol, int32_t max_it,
                                     double* lambda_out, int32_t* iters_out);

/* Mean and variance (Eq. 2.1; variance sum_l w_l (x_l - mean)^2) of a field
 * over every point solved since the last reset (host buffers of the field's
 * length). SFB_ERR_STATE if nothing was solved. */
sfb_status sfb_moments(sfb_ctx* ctx, int32_t field, double* mean_out, double* var_out);
/* Starts a new accumulation of the moments: the next batches' points are the
 * only ones counted (so one collocation grid can be solved in several
 * batches, or several grids one after another). SFB_ERR_WORKSPACE without a
 * workspace. */
sfb_status sfb_moments_reset(sfb_ctx* ctx);

/* Number of CUDA kernels this context has launched so far (a replayed basis
 * graph counts its kernels). Host memory; no synchronisation. */
sfb_status sfb_launch_count(const sfb_ctx* ctx, int64_t* n);

/* Device time (ms, CUDA events) of the phases of the last
 * sfb_interface_solve_batch: [0] global-to-local index conversion and
 * grouping, [1] the CG iterations, [2] status bookkeeping, [3] Darcy
 * recovery and moments, [4] Stokes moments; cg_iterations (nullable) gets the
 * number of lockstep CG iterations run. Synchronises the stream. */
sfb_status sfb_solve_timings(sfb_ctx* ctx, double* ms_out, int32_t* cg_iterations);

/* SM cycles per CTA of the last interface CG in one cooperative launch
 * ("cg_persistent" 1), by step: [0] tile products of the iterations, [1] the
 * grid barrier after them, [2] point updates, [3] the barrier after them,
 * [4] FP64 products of the mixed CG's checks, [5] the rest of the checks
 * (FP64 residual replacement, iterating-point count, their barriers).
 * cycles_out holds 6 values; all zero after a CG of one launch per step. */
sfb_status sfb_cg_phase_cycles(const sfb_ctx* ctx, double* cycles_out);

/* Builds one stochastic-basis item (Darcy subdomain `sub`, local realization
 * `k`) without allocating device memory; the paper has no counterpart, this
 * is for callers that cannot call cudaMalloc (an application that already
 * holds all device memory in its own pool, or a path that must not allocate).
 * Needs only sfb_kl_setup and sfb_collocation_setup, no workspace. The
 * working memory is a static 8 MiB device array inside the library that a GPU
 * keeps for the rest of the process once sfb_create has run with that device
 * current (or this call first ran on it); items needing more return
 * SFB_ERR_UNSUPPORTED before any copy or launch. Outputs: phi_out [R x R] and g_out
 * [R] (nullable; host or device), x_out [(R+1) x n_cells] device memory, the
 * same values as sfb_build_stochastic_basis + sfb_get_basis. Each call looks
 * up the array's device address on the current device; if the module was not
 * loaded there yet (no sfb_create with that device current), the first call
 * loads it, so make that first call before any stream capture. Calls share
 * the array: calls that overlap on the GPU
 * race and must be serialised by the caller. Synchronises the stream. */
sfb_status sfb_build_basis_item_noalloc(sfb_ctx* ctx, int32_t sub, int32_t k, int32_t prec,
                                         double* phi_out, double* g_out, double* x_out);

/* Tuning knobs (no counterpart in the paper):
 *   "refine_tol"     mixed form: stop refining when the predicted relative
 *                    error of X is below this (default 1e-11: the flux
 *                    responses Phi come from boundary values of X less the
 *                    mortar data, which cancel, so Phi keeps less relative
 *                    accuracy than X);
 *   "refine_max"     mixed form: at most this many FP64 residual passes (8);
 *   "cg_check_every" CG iterations between convergence checks (8);
 *   "cg_persistent"  1: the whole CG in one cooperative launch (grid barriers
 *                    between the product and update steps, convergence checks
 *                    on the device; bit-identical results); 0: one launch per
 *                    step with a host check every cg_check_every iterations.
 *                    The one-launch form falls back to the other when the
 *                    device cannot launch it, and for SFB_CG_MIXED when each
 *                    CTA cannot keep its share of the FP32 bases (three
 *                    tiles) in shared memory (1);
 *   "cg_precond"     interface CG preconditioner: 0 none (CG as the paper
 *                    states it), 1 Jacobi (diag(S^l)), 2 interface blocks
 *                    (the diagonal block of S^l on each mortar interface's
 *                    DOFs, inverted per point, applied in FP32; interfaces of
 *                    more than 32 DOFs fall back to Jacobi), 3 balancing
 *                    Neumann-Neumann (Section 7's suggestion: stiffness-
 *                    weighted Neumann steps on the pseudo-inverses of the
 *                    bases, a coarse space of the floating Darcy subdomains'
 *                    constants, CG from the balanced start; SFB_CG only,
 *                    another solver with it returns SFB_ERR_ARG, more than 16
 *                    floating subdomains SFB_ERR_UNSUPPORTED). The same
 *                    solution and the same stopping test on the
 *                    unpreconditioned residual in every case (2);
 *   "basis_autotune" 1: the next build of each precision first times every
 *                    launch shape of each size class (sfb_basis_launch_shape)
 *                    and keeps the fastest; setting it (0 or 1) forgets
 *                    earlier choices. 0: shape 0 everywhere (1);
 *   "basis_shape"    forces launch shape n for every size class that has it
 *                    (shape 0 for the others) and turns the autotuner off;
 *   "basis_graph"    1: the launches of all size classes are captured once as
 *                    a CUDA graph (on a private stream) and replayed while the
 *                    workspace, refinement options and shapes stay the same;
 *                    plain launches when the context stream is itself being
 *                    captured. 0: plain launches (1);
 *   "basis_persistent"  FP32 builds whose size classes both run a split
 *                    shape: 1 runs every item of both classes in one
 *                    persistent launch (factor tasks, then column-chunk tasks
 *                    that wait, bounded, on their item's factor); 0 one
 *                    launch sequence per class; -1 the autotuner times both
 *                    and keeps the faster (-1);
 *   "basis_pipe_groups"  a split shape's class runs its items in this many
 *                    groups, 1..4: the factor launches of the groups in
 *                    sequence and each group's chunk launch after its factor,
 *                    on a second stream (1);
 *   "cg_test_barrier_timeout"  test hook: 1 makes CTA 0 of the next one-launch
 *                    CG skip its first grid barrier, so that the other CTAs'
 *                    waits run out (1 s). The solve returns SFB_ERR_TIMEOUT and
 *                    the context stays usable. Cleared by that solve (0);
 *   "gmres_restart"  SFB_GMRES: restart length m, 1..30 (30);
 *   "cg_replace_ratio"  SFB_CG_MIXED: a point's residual is replaced by the
 *                    FP64 residual at the next check once the recursive one
 *                    has dropped by this factor since the last replacement,
 *                    and the point pauses at a tenth of it (0.1);
 *   "moments_double_float"  after a mixed-form basis build: 1 runs the
 *                    moment contractions that reuse a field response for four
 *                    or more points (recovery of 4-8 point sub-tiles, the large
 *                    groups' quadratic forms) in double-float, an FP32 hi/lo
 *                    pair with error-free products and sums (about 1e-14
 *                    relative), on the FP32 pipe; 0 keeps them in FP64. The
 *                    FP64 form always uses FP64 (1);
 *   "moments_group_factor"  groups of more than factor * (R+1) points enter
 *                    the moments through their coefficient second moments,
 *                    smaller ones point by point; 0 = always point by point (1).
 * SFB_ERR_ARG for an unknown name or a value out of range. */
sfb_status sfb_set_option(sfb_ctx* ctx, const char* name, double value);

#ifdef __cplusplus
}
#endif
#endif /* SFB_H */
